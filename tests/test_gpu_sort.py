"""Parity of the CUDA DFR sort (through the C ABI) with the CPU oracle:
bit-exact keys, and bit-exact payloads for key-value sorts (stable order).

Sizes span several tiles and ragged tails around every threshold of the
path: the warp-sort threshold (32), the scatter tile and the CTA-sort
capacity (4096 / 8192), and the full-size workloads the benchmark times.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_sort, need_gpu

pytestmark = pytest.mark.gpu

EDGE_SIZES = [0, 1, 2, 3, 31, 32, 33, 64, 100, 511, 512, 513, 1000, 4095, 4096, 4097, 8191, 8192, 8193, 8194, 16385,
              65537, 300_001, 1_000_000, (1 << 21) + 12345]


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


@pytest.mark.parametrize("n", EDGE_SIZES)
def test_u32_uniform_sizes(dfr, n):
    a = synth.uniform_u32(n, synth.BASE_SEED + n)
    k, _, st = gpu_sort(dfr, a)
    assert st == dfr.DFR_OK
    assert np.array_equal(k, oracle.sort_u32(a))


@pytest.mark.parametrize("dist", synth.U32_DISTRIBUTIONS)
@pytest.mark.parametrize("n", [5000, 70_001, (1 << 22) + 3])
def test_u32_distributions(dfr, dist, n):
    a = synth.u32(dist, n, synth.BASE_SEED + 20)
    k, _, st = gpu_sort(dfr, a)
    assert st == dfr.DFR_OK
    assert np.array_equal(k, oracle.sort_u32(a))


@pytest.mark.parametrize("n", [2, 33, 4097, 100_003, (1 << 20) + 7])
@pytest.mark.parametrize("dist", synth.U64_DISTRIBUTIONS)
def test_u64_keys_and_kv(dfr, dist, n):
    a = synth.u64(dist, n, synth.BASE_SEED + 30)
    k, _, st = gpu_sort(dfr, a)
    assert st == dfr.DFR_OK
    assert np.array_equal(k, oracle.sort_u64(a))
    v = synth.index_payload(n)
    k2, v2, st2 = gpu_sort(dfr, a, v)
    ok, ov = oracle.sort_u64_kv(a, v)
    assert st2 == dfr.DFR_OK
    assert np.array_equal(k2, ok) and np.array_equal(v2, ov)


@pytest.mark.parametrize("dist", ["uniform", "zipf", "equal", "exponential"])
@pytest.mark.parametrize("n", [33, 8193, 200_001])
def test_u32_kv(dfr, dist, n):
    a = synth.u32(dist, n, synth.BASE_SEED + 40)
    v = synth.index_payload(n)
    k, vv, st = gpu_sort(dfr, a, v)
    ok, ov = oracle.sort_u32_kv(a, v)
    assert st == dfr.DFR_OK
    assert np.array_equal(k, ok) and np.array_equal(vv, ov)


def test_adversarial_u32(dfr):
    n = 250_000
    g = np.random.Generator(np.random.PCG64(9))
    cases = {
        "two_values": np.where(g.random(n) < 0.5, 7, 0xFFFFFFF0).astype(np.uint32),
        "one_bit": (g.integers(0, 2, n).astype(np.uint32) << np.uint32(17)),
        "low_bits_only": g.integers(0, 16, n, dtype=np.uint32),
        "sparse_bits": (g.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32) & np.uint32(0x80010001)),
        "top_byte_const": (np.uint32(0xAB000000) | g.integers(0, 1 << 24, n, dtype=np.uint32)),
        "sawtooth": (np.arange(n, dtype=np.uint32) % np.uint32(1000)),
        "max_and_zero": np.where(np.arange(n) % 3 == 0, 0, 0xFFFFFFFF).astype(np.uint32),
    }
    for name, a in cases.items():
        k, _, st = gpu_sort(dfr, a)
        assert st == dfr.DFR_OK, name
        assert np.array_equal(k, oracle.sort_u32(a)), name


def test_kv_stability_equal_keys(dfr):
    n = 123_457
    a = np.full(n, 0x0123456789ABCDEF, dtype=np.uint64)
    v = synth.index_payload(n)
    k, vv, st = gpu_sort(dfr, a, v)
    assert st == dfr.DFR_OK
    assert np.array_equal(k, a) and np.array_equal(vv, v)
    # few distinct keys, many ties: payloads must stay in input order per key
    b = (synth.uniform64_u64(n, 3) % np.uint64(5)) << np.uint64(40)
    k, vv, st = gpu_sort(dfr, b, v)
    ok, ov = oracle.sort_u64_kv(b, v)
    assert np.array_equal(k, ok) and np.array_equal(vv, ov)


def test_repeat_calls_reuse_workspace(dfr):
    for seed in range(3):
        a = synth.zipf_u32(150_000, seed)
        k, _, st = gpu_sort(dfr, a)
        assert st == dfr.DFR_OK
        assert np.array_equal(k, oracle.sort_u32(a))


def test_stats_uniform_plan(dfr):
    import torch

    n = 1 << 22
    a = synth.uniform_u32(n, 77)
    s = dfr.Sorter(dfr.DFR_U32, n)
    d = dfr.to_device(a)
    s.sort_(d)
    st = s.stats()
    assert st["device_status"] == 0
    assert st["n_total"] == n
    # 2^22 uniform keys: one level of 256 buckets of ~16K, a second level of
    # buckets of ~64 keys, which go to the CTA / warp diversion sorts
    assert st["level_keys"][0] == n
    assert st["cta_keys"] + st["wsort_keys"] + st["tiny_keys"] + st["const_keys"] == n
    assert st["model_bytes"] == 4 * n + 8 * sum(st["level_keys"]) + 8 * (st["cta_keys"] + st["wsort_keys"]
                                                                        + st["tiny_keys"] + st["copy_keys"])
    torch.cuda.synchronize()


def test_forced_timeout_reports_and_recovers(dfr):
    """The look-back (used by the stable key-value deal) is pointed at a
    status word nobody sets: every waiting tile must give up after the spin
    limit, record DFR_ERR_TIMEOUT and skip its writes; the next normal call
    must succeed on the same context."""
    n = 200_000
    a = synth.uniform_u32(n, 5)
    v = synth.index_payload(n)
    try:
        dfr.dfr_set_debug(2000, True)
        _, _, st = gpu_sort(dfr, a, v)
    finally:
        dfr.dfr_set_debug(0, False)
    assert st == dfr.DFR_ERR_TIMEOUT
    k, vv, st = gpu_sort(dfr, a, v)
    assert st == dfr.DFR_OK
    ok, ov = oracle.sort_u32_kv(a, v)
    assert np.array_equal(k, ok) and np.array_equal(vv, ov)


def test_cta32_counter_boundaries(dfr):
    """Buckets of ~4000 u32 keys whose keys vary in the low 13..16 bits go to
    the fast CTA sort, which counts each value in a 4-bit counter: a value
    seen 15 times fits, the 16th copy sends the bucket to the general CTA
    sort.  One bucket per top byte, each at one side of that boundary (and
    spans of 13 and 16 bits), in both launch forms, against the oracle."""
    from test_gpu_persist import launch_form

    g = np.random.Generator(np.random.PCG64(1234))

    def bucket(top, nbits, reps):
        hi = (1 << nbits) - 1
        special = [int(x) for x in 1 + g.choice(hi - 1, size=len(reps), replace=False)]
        pool = np.setdiff1d(np.arange(1, hi, dtype=np.uint32), np.array(special, dtype=np.uint32))
        low = [np.array([0, hi], dtype=np.uint32), g.choice(pool, size=4000 - 2 - sum(reps), replace=False)]
        low += [np.full(r, s, dtype=np.uint32) for s, r in zip(special, reps)]
        return (np.uint32(top) << np.uint32(24)) | np.concatenate(low).astype(np.uint32)

    parts = [
        bucket(0x11, 16, [15]),          # 15 copies: the counter is full, not past it
        bucket(0x22, 16, [16]),          # 16 copies: second queue
        bucket(0x33, 16, [15, 15, 15]),  # several full counters in one bucket
        bucket(0x44, 13, [15, 14]),      # 13-bit span (one low bit per group)
        bucket(0x55, 13, [17]),
        bucket(0x66, 16, [40, 15, 2]),
    ]
    a = np.concatenate(parts)
    a = a[g.permutation(a.size)]
    want = oracle.sort_u32(a)
    for launch in (dfr.DFR_LAUNCH_LEVELS, dfr.DFR_LAUNCH_PERSISTENT):
        with launch_form(dfr, launch, (dfr.DFR_U32,)):
            k, _, st = gpu_sort(dfr, a)
        assert st == dfr.DFR_OK
        assert np.array_equal(k, want), launch
