"""dfr_sort_u32_noalloc: the u32 sort for callers that cannot allocate device
memory (a plug-in whose host application owns all device memory, a process
under a strict memory quota, a latency-critical loop that must not pay
cudaMalloc's implicit synchronisation).  Its scratch buffer and workspace live
in a fixed device array inside the library.

Two calls in a row through the C ABI must each give exactly what the regular
entry point dfr_sort_u32 gives on the same input (the second call runs on the
array the first one left behind), and an oversized request must be refused
before anything is enqueued.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth
from gpu_util import gpu_sort, need_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plain_entry_point_twice_in_a_row():
    dfr = need_gpu()
    import torch

    cases = [("uniform", 1 << 20, synth.BASE_SEED + 61), ("zipf", 777_777, synth.BASE_SEED + 62)]
    inputs = [synth.u32(dist, n, seed) for dist, n, seed in cases]
    expected = []
    for a in inputs:
        k, _, st = gpu_sort(dfr, a)  # dfr_sort_u32 with caller-provided scratch
        assert st == dfr.DFR_OK
        expected.append(k)

    dev = [dfr.to_device(a) for a in inputs]
    torch.cuda.synchronize()
    for d, a in zip(dev, inputs):  # two no-allocation calls back to back
        assert dfr.dfr_sort_u32_noalloc(d, a.size) == dfr.DFR_OK
    torch.cuda.synchronize()
    for d, want in zip(dev, expected):
        assert np.array_equal(dfr.to_numpy(d, np.uint32), want)


def test_noalloc_refuses_oversized_and_accepts_trivial():
    dfr = need_gpu()
    import torch

    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert dfr.dfr_sort_u32_noalloc(d, dfr.DFR_NOALLOC_MAX_N + 1) == dfr.DFR_ERR_TOO_LARGE
    assert dfr.dfr_sort_u32_noalloc(d, 1) == dfr.DFR_OK
    assert dfr.dfr_sort_u32_noalloc(0, 0) == dfr.DFR_OK
