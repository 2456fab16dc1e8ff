"""dfr_sort_u32_noalloc: the u32 sort for callers that cannot allocate device
memory (a plug-in whose host application owns all device memory, a process
under a strict memory quota, a latency-critical loop that must not pay
cudaMalloc's implicit synchronisation).  Its scratch buffer and workspace live
in a fixed device array inside the library.

Calls in a row through the C ABI must each give exactly the oracle's sorted
keys -- and exactly what the regular entry point dfr_sort_u32 gives on the
same input -- even though every call after the first runs on the array the
previous call left behind: a 2^20-key call fills it with its scratch, then an
all-equal array (nothing to deal) and an already-sorted array must still come
out right.  An oversized request must be refused before anything is enqueued.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_sort, need_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_matches_oracle_and_plain_entry_point_in_a_row():
    dfr = need_gpu()
    import torch

    cases = [("uniform", 1 << 20, synth.BASE_SEED + 61), ("zipf", 777_777, synth.BASE_SEED + 62),
             ("equal", 654_321, synth.BASE_SEED + 63), ("sorted", 1 << 20, synth.BASE_SEED + 64)]
    inputs = [synth.u32(dist, n, seed) for dist, n, seed in cases]
    expected = [oracle.sort_u32(a) for a in inputs]
    for a, want in zip(inputs, expected):
        k, _, st = gpu_sort(dfr, a)  # dfr_sort_u32 with caller-provided scratch
        assert st == dfr.DFR_OK
        assert np.array_equal(k, want)

    dev = [dfr.to_device(a) for a in inputs]
    torch.cuda.synchronize()
    for d, a in zip(dev, inputs):  # no-allocation calls back to back on one stream
        assert dfr.dfr_sort_u32_noalloc(d, a.size) == dfr.DFR_OK
    torch.cuda.synchronize()
    for (dist, n, _), d, want in zip(cases, dev, expected):
        assert np.array_equal(dfr.to_numpy(d, np.uint32), want), "%s n=%d" % (dist, n)


def test_noalloc_refuses_oversized_and_accepts_trivial():
    dfr = need_gpu()
    import torch

    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert dfr.dfr_sort_u32_noalloc(d, dfr.DFR_NOALLOC_MAX_N + 1) == dfr.DFR_ERR_TOO_LARGE
    assert dfr.dfr_sort_u32_noalloc(d, 1) == dfr.DFR_OK
    assert dfr.dfr_sort_u32_noalloc(0, 0) == dfr.DFR_OK
