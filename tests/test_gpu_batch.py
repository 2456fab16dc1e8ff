"""dfr_sort_batch: many independent arrays in one launch sequence.  Every
array must come out exactly as the oracle sorts it alone, and exactly as a
plain dfr_sort_* call on that array alone produces it."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_sort, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


def _batch(dfr, key_type, keys_list, vals_list=None):
    import torch

    kb = dfr.KEY_BYTES[key_type]
    kdt = torch.int32 if kb == 4 else torch.int64
    dev_keys, dev_vals, segs, keep = [], [], [], []
    for i, a in enumerate(keys_list):
        n = a.size
        dk = dfr.to_device(a) if n else torch.empty(0, dtype=kdt, device="cuda")
        kbuf = torch.empty(max(1, n), dtype=kdt, device="cuda")
        dv = vb = None
        if vals_list is not None:
            dv = dfr.to_device(vals_list[i]) if n else torch.empty(0, dtype=torch.int32, device="cuda")
            vb = torch.empty(max(1, n), dtype=torch.int32, device="cuda")
        dev_keys.append(dk)
        dev_vals.append(dv)
        keep += [kbuf, vb]
        segs.append((key_type, dk if n else 0, dv if (dv is not None and n) else 0, kbuf, vb if vb is not None else 0, n))
    ws_bytes = dfr.dfr_batch_workspace_bytes(segs)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    rc = dfr.dfr_sort_batch(segs, ws, ws_bytes)
    assert rc == dfr.DFR_OK, dfr.dfr_status_string(rc)
    assert dfr.dfr_last_device_status(ws) == dfr.DFR_OK
    dt = np.uint32 if kb == 4 else np.uint64
    outk = [dfr.to_numpy(k, dt) if k.numel() else np.empty(0, dt) for k in dev_keys]
    outv = None
    if vals_list is not None:
        outv = [dfr.to_numpy(v, np.uint32) if v.numel() else np.empty(0, np.uint32) for v in dev_vals]
    return outk, outv


def test_batch_u32_mixed_sizes(dfr):
    sizes = [0, 1, 2, 17, 32, 33, 1000, 4096, 8192, 8193, 50_000, 300_001, 5, 70_000, 1 << 20]
    arrays = []
    for i, n in enumerate(sizes):
        dist = synth.U32_DISTRIBUTIONS[i % len(synth.U32_DISTRIBUTIONS)]
        arrays.append(synth.u32(dist, n, synth.BASE_SEED + 100 + i))
    out, _ = _batch(dfr, dfr.DFR_U32, arrays)
    for a, o in zip(arrays, out):
        assert np.array_equal(o, oracle.sort_u32(a))
        alone, _, st = gpu_sort(dfr, a)
        assert st == dfr.DFR_OK and np.array_equal(o, alone)


def test_batch_u32_many_small(dfr):
    arrays, _ = synth.batch_u32(300, synth.BASE_SEED + 40, lo=1 << 8, hi=1 << 16)
    out, _ = _batch(dfr, dfr.DFR_U32, arrays)
    for a, o in zip(arrays, out):
        assert np.array_equal(o, oracle.sort_u32(a))


def test_batch_u64_kv(dfr):
    sizes = [3, 33, 4097, 60_000, 250_000, 1]
    keys, vals = [], []
    for i, n in enumerate(sizes):
        dist = synth.U64_DISTRIBUTIONS[i % 3]
        keys.append(synth.u64(dist, n, synth.BASE_SEED + 200 + i))
        vals.append(synth.index_payload(n))
    ok, ov = _batch(dfr, dfr.DFR_U64_KV, keys, vals)
    for k, v, gk, gv in zip(keys, vals, ok, ov):
        ek, ev = oracle.sort_u64_kv(k, v)
        assert np.array_equal(gk, ek) and np.array_equal(gv, ev)


def _segmented(dfr, key_type, a, v, lens, gaps):
    """dfr_sort_batch over slices of one array (a segmented sort): slice i
    holds lens[i] keys and starts gaps[i] keys after the previous slice ends;
    the keys in the gaps are not part of any segment and must not move."""
    import torch

    kb = dfr.KEY_BYTES[key_type]
    dk = dfr.to_device(a)
    dv = dfr.to_device(v) if v is not None else None
    kscratch = torch.empty_like(dk)
    vscratch = torch.empty_like(dv) if dv is not None else None
    segs, spans, o = [], [], 0
    for n, gap in zip(lens, gaps):
        o += gap
        if n:
            segs.append((key_type, dk.data_ptr() + kb * o, dv.data_ptr() + 4 * o if dv is not None else 0,
                         kscratch.data_ptr() + kb * o, vscratch.data_ptr() + 4 * o if dv is not None else 0, n))
        else:
            segs.append((key_type, 0, 0, 0, 0, 0))
        spans.append((o, n))
        o += n
    assert o <= a.size
    ws_bytes = dfr.dfr_batch_workspace_bytes(segs)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dk.device)
    assert dfr.dfr_sort_batch(segs, ws, ws_bytes) == dfr.DFR_OK
    assert dfr.dfr_last_device_status(ws) == dfr.DFR_OK
    got_k = dfr.to_numpy(dk, a.dtype)
    got_v = dfr.to_numpy(dv, np.uint32) if dv is not None else None
    return got_k, got_v, spans


def _segment_plan(seed, count, hi, extra):
    g = np.random.default_rng(seed)
    lens = [int(x) for x in g.integers(0, hi, size=count)] + list(extra)
    g.shuffle(lens)
    gaps = [int(x) for x in g.integers(0, 5, size=len(lens))]
    return lens, gaps, sum(lens) + sum(gaps) + 3


def test_batch_as_segmented_sort_u32(dfr):
    lens, gaps, total = _segment_plan(5100, 300, 40_000, [0, 1, 2, 33, 4097, 200_003])
    a = synth.uniform_u32(total, synth.BASE_SEED + 5100)
    got, _, spans = _segmented(dfr, dfr.DFR_U32, a, None, lens, gaps)
    want = a.copy()
    for o, n in spans:
        want[o:o + n] = oracle.sort_u32(a[o:o + n])
    assert np.array_equal(got, want)


def test_batch_as_segmented_sort_u64_kv(dfr):
    lens, gaps, total = _segment_plan(5200, 60, 30_000, [0, 1, 3, 70_001])
    a = synth.dup90_u64(total, synth.BASE_SEED + 5200)
    v = synth.index_payload(total)
    got_k, got_v, spans = _segmented(dfr, dfr.DFR_U64_KV, a, v, lens, gaps)
    want_k, want_v = a.copy(), v.copy()
    for o, n in spans:
        want_k[o:o + n], want_v[o:o + n] = oracle.sort_u64_kv(a[o:o + n], v[o:o + n])
    assert np.array_equal(got_k, want_k) and np.array_equal(got_v, want_v)
