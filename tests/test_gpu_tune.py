"""The launch-plan knobs change how the sort runs, never what it returns:
under extreme and mixed settings of the tuning table every result stays
bit-exact against the oracle (keys, and payloads in stable order)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_sort, need_gpu

pytestmark = pytest.mark.gpu

PLANS = [
    dict(target_log2=6, max_bits=4, warp_max=128, scatter_ctas_per_sm=1, ctasort_ctas_per_sm=1),
    dict(target_log2=13, max_bits=8, warp_max=512, scatter_ctas_per_sm=0, ctasort_ctas_per_sm=0),
    dict(target_log2=9, max_bits=5, warp_max=256, scatter_ctas_per_sm=2, ctasort_ctas_per_sm=2),
]


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


def _all_classes(dfr, plan):
    for kt in (dfr.DFR_U32, dfr.DFR_U64, dfr.DFR_U64_KV, dfr.DFR_U32_KV):
        for c in range(dfr.DFR_TUNE_CLASSES):
            assert dfr.dfr_tune_set(kt, c, plan) == dfr.DFR_OK


@pytest.mark.parametrize("plan", range(len(PLANS)))
def test_results_independent_of_plan(dfr, plan):
    try:
        _all_classes(dfr, PLANS[plan])
        for n, dist in ((5000, "zipf"), (70_001, "normal"), (1_000_003, "uniform"), (300_000, "exponential"),
                        (200_000, "sorted")):
            a = synth.u32(dist, n, synth.BASE_SEED + 900 + n)
            k, _, st = gpu_sort(dfr, a)
            assert st == dfr.DFR_OK and np.array_equal(k, oracle.sort_u32(a)), (plan, n, dist)
        for n, dist in ((4097, "dup90"), (250_001, "uniform64"), (120_000, "uniform16")):
            a = synth.u64(dist, n, synth.BASE_SEED + 950 + n)
            v = synth.index_payload(n)
            k, vv, st = gpu_sort(dfr, a, v)
            ok, ov = oracle.sort_u64_kv(a, v)
            assert st == dfr.DFR_OK and np.array_equal(k, ok) and np.array_equal(vv, ov), (plan, n, dist)
        a = synth.u32("zipf", 150_000, 3)
        v = synth.index_payload(a.size)
        k, vv, st = gpu_sort(dfr, a, v)
        ok, ov = oracle.sort_u32_kv(a, v)
        assert st == dfr.DFR_OK and np.array_equal(k, ok) and np.array_equal(vv, ov)
    finally:
        dfr.dfr_tune_reset()
