"""dfr_graph_*: a sort captured once into a CUDA graph and launched again and
again on refilled buffers returns, every time, exactly the oracle's result --
a single array and a key-value batch."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


def test_graph_single_array_relaunched(dfr):
    import torch

    n = 1_000_003
    s = dfr.Sorter(dfr.DFR_U32, n)
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    g = dfr.dfr_graph_create([(dfr.DFR_U32, keys, 0, s.kbuf, 0, n)], s.ws, s.ws_bytes)
    try:
        for r, dist in enumerate(("uniform", "zipf", "sorted", "equal")):
            a = synth.u32(dist, n, synth.BASE_SEED + 1100 + r)
            keys.copy_(dfr.to_device(a))
            assert dfr.dfr_graph_launch(g) == dfr.DFR_OK
            assert s.device_status() == dfr.DFR_OK
            assert np.array_equal(dfr.to_numpy(keys, np.uint32), oracle.sort_u32(a)), dist
    finally:
        dfr.dfr_graph_destroy(g)


def test_graph_kv_batch_relaunched(dfr):
    import torch

    sizes = [5, 4097, 70_001, 300_000]
    keys = [torch.empty(n, dtype=torch.int64, device="cuda") for n in sizes]
    vals = [torch.empty(n, dtype=torch.int32, device="cuda") for n in sizes]
    kbuf = [torch.empty(n, dtype=torch.int64, device="cuda") for n in sizes]
    vbuf = [torch.empty(n, dtype=torch.int32, device="cuda") for n in sizes]
    segs = [(dfr.DFR_U64_KV, keys[i], vals[i], kbuf[i], vbuf[i], n) for i, n in enumerate(sizes)]
    wsb = dfr.dfr_batch_workspace_bytes(segs)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    g = dfr.dfr_graph_create(segs, ws, wsb)
    try:
        for r in range(3):
            arrays = [synth.u64(synth.U64_DISTRIBUTIONS[(i + r) % 3], n, synth.BASE_SEED + 1200 + 10 * r + i)
                      for i, n in enumerate(sizes)]
            for i, a in enumerate(arrays):
                keys[i].copy_(dfr.to_device(a))
                vals[i].copy_(dfr.to_device(synth.index_payload(a.size)))
            assert dfr.dfr_graph_launch(g) == dfr.DFR_OK
            assert dfr.dfr_last_device_status(ws) == dfr.DFR_OK
            for i, a in enumerate(arrays):
                ok, ov = oracle.sort_u64_kv(a, synth.index_payload(a.size))
                assert np.array_equal(dfr.to_numpy(keys[i], np.uint64), ok)
                assert np.array_equal(dfr.to_numpy(vals[i], np.uint32), ov)
    finally:
        dfr.dfr_graph_destroy(g)
