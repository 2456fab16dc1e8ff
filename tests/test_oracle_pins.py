"""Pins for the CPU oracle, against things other than itself (CPU only).

The oracle computes the stable ascending order of unsigned keys (payloads move
with their keys).  That result is unique for a given input, so it is pinned by:
  * brute force: a stable insertion sort (the paper's small-bucket diversion,
    Section "MSD Radix Sorts") on every array up to length 6 over alphabets that
    differ in each byte position and include the extreme values;
  * a library routine: numpy's stable sort / stable argsort on random inputs;
  * the invariants of a sort: output nondecreasing, output a permutation of
    the input (exact multiset histogram), and for key-value input the payload
    (original index) points back at its key and rises inside every run of
    equal keys (stability);
  * special cases with closed-form answers: all-equal, already sorted,
    reverse-sorted distinct keys.
A companion test (test_oracle_mutants.py) checks that plausible mistakes in
oracle.c are caught by these pins.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth

U32_ALPHABET = [0, 0x1, 0x100, 0x10000, 0x1000000, 0xFFFFFFFF]
U64_ALPHABET = [0, 0x1, 0x100, 0x100000000, 0x100000000000000, 0x8000000000000000, 0xFFFFFFFFFFFFFFFF]


def insertion_sort_pairs(keys):
    """Stable insertion sort of (key, original index) pairs, by key only."""
    recs = [(int(k), i) for i, k in enumerate(keys)]
    for i in range(1, len(recs)):
        cur = recs[i]
        j = i - 1
        while j >= 0 and recs[j][0] > cur[0]:
            recs[j + 1] = recs[j]
            j -= 1
        recs[j + 1] = cur
    return [r[0] for r in recs], [r[1] for r in recs]


def check_sorted_permutation(inp, out):
    inp = np.asarray(inp)
    out = np.asarray(out)
    assert out.shape == inp.shape
    if out.size > 1:
        assert np.all(out[1:] >= out[:-1]), "not nondecreasing"
    vi, ci = np.unique(inp, return_counts=True)
    vo, co = np.unique(out, return_counts=True)
    assert np.array_equal(vi, vo) and np.array_equal(ci, co), "not a permutation of the input"


def check_kv_stable(kin, kout, vout):
    kin = np.asarray(kin)
    kout = np.asarray(kout)
    vout = np.asarray(vout).astype(np.int64)
    n = kin.size
    assert np.array_equal(np.sort(vout), np.arange(n)), "payloads are not a permutation"
    assert np.array_equal(kin[vout], kout), "payload does not point back at its key"
    if n > 1:
        same = kout[1:] == kout[:-1]
        assert np.all(vout[1:][same] > vout[:-1][same]), "equal keys out of input order"


@pytest.mark.parametrize("n", range(0, 7))
def test_u32_exhaustive_vs_insertion_sort(n):
    orc = oracle.default()
    for tup in itertools.product(U32_ALPHABET, repeat=n):
        want, _ = insertion_sort_pairs(tup)
        got = orc.sort_u32(np.array(tup, dtype=np.uint32))
        assert got.tolist() == want, tup


@pytest.mark.parametrize("n", range(0, 6))
def test_u64_exhaustive_vs_insertion_sort(n):
    orc = oracle.default()
    for tup in itertools.product(U64_ALPHABET, repeat=n):
        want, _ = insertion_sort_pairs(tup)
        got = orc.sort_u64(np.array(tup, dtype=np.uint64))
        assert got.tolist() == want, tup


@pytest.mark.parametrize("n", range(0, 6))
def test_u64_kv_exhaustive_vs_insertion_sort(n):
    orc = oracle.default()
    alpha = U64_ALPHABET[:5]
    for tup in itertools.product(alpha, repeat=n):
        want_k, want_v = insertion_sort_pairs(tup)
        k, v = orc.sort_u64_kv(np.array(tup, dtype=np.uint64), np.arange(n, dtype=np.uint32))
        assert k.tolist() == want_k and v.tolist() == want_v, tup


@pytest.mark.parametrize("n", range(0, 6))
def test_u32_kv_exhaustive_vs_insertion_sort(n):
    orc = oracle.default()
    alpha = U32_ALPHABET[:5]
    for tup in itertools.product(alpha, repeat=n):
        want_k, want_v = insertion_sort_pairs(tup)
        k, v = orc.sort_u32_kv(np.array(tup, dtype=np.uint32), np.arange(n, dtype=np.uint32))
        assert k.tolist() == want_k and v.tolist() == want_v, tup


def test_random_small_vs_numpy_stable():
    orc = oracle.default()
    g = np.random.Generator(np.random.PCG64(synth.BASE_SEED))
    for trial in range(1500):
        n = int(g.integers(0, 2001))
        bits = int(g.integers(1, 33))
        k32 = g.integers(0, 1 << bits, size=n, dtype=np.uint64).astype(np.uint32)
        assert np.array_equal(orc.sort_u32(k32), np.sort(k32, kind="stable"))
        bits64 = int(g.integers(1, 65))
        k64 = g.bit_generator.random_raw(n).astype(np.uint64) >> np.uint64(64 - bits64)
        assert np.array_equal(orc.sort_u64(k64), np.sort(k64, kind="stable"))
        v = np.arange(n, dtype=np.uint32)
        kk, vv = orc.sort_u64_kv(k64, v)
        order = np.argsort(k64, kind="stable")
        assert np.array_equal(kk, k64[order]) and np.array_equal(vv, v[order])
        kk, vv = orc.sort_u32_kv(k32, v)
        order = np.argsort(k32, kind="stable")
        assert np.array_equal(kk, k32[order]) and np.array_equal(vv, v[order])


@pytest.mark.parametrize("dist", synth.U32_DISTRIBUTIONS)
def test_u32_invariants_medium(dist):
    n = (1 << 20) + 12345
    a = synth.u32(dist, n, synth.BASE_SEED + 20)
    out = oracle.sort_u32(a)
    check_sorted_permutation(a, out)
    assert np.array_equal(out, np.sort(a, kind="stable"))


@pytest.mark.parametrize("dist", synth.U64_DISTRIBUTIONS)
def test_u64_kv_invariants_medium(dist):
    n = (1 << 19) + 777
    k = synth.u64(dist, n, synth.BASE_SEED + 30)
    v = synth.index_payload(n)
    ko, vo = oracle.sort_u64_kv(k, v)
    check_sorted_permutation(k, ko)
    check_kv_stable(k, ko, vo)
    assert np.array_equal(oracle.sort_u64(k), ko)


def test_special_cases():
    n = 100003
    eq = np.full(n, 0xDEADBEEF, dtype=np.uint32)
    assert np.array_equal(oracle.sort_u32(eq), eq)
    srt = synth.sorted_u32(n, 5)
    assert np.array_equal(oracle.sort_u32(srt), srt)
    distinct = np.unique(synth.uniform_u32(n, 6))
    assert np.array_equal(oracle.sort_u32(distinct[::-1].copy()), distinct)
    eq64 = np.full(n, 0xFEDCBA9876543210, dtype=np.uint64)
    k, v = oracle.sort_u64_kv(eq64, np.arange(n, dtype=np.uint32))
    assert np.array_equal(k, eq64) and np.array_equal(v, np.arange(n, dtype=np.uint32))
    d64 = np.unique(synth.uniform64_u64(n, 7))
    k, v = oracle.sort_u64_kv(d64[::-1].copy(), np.arange(d64.size, dtype=np.uint32))
    assert np.array_equal(k, d64)
    assert np.array_equal(v, np.arange(d64.size, dtype=np.uint32)[::-1])


@pytest.mark.parametrize("shift", [0, 3, 8, 13, 16, 24])
def test_counting_pass_is_stable_partition(shift):
    """One counting sort on one digit (Preliminaries): records come out grouped
    by digit in ascending digit order, each group in input order -- exactly a
    stable argsort of the digit (library routine)."""
    a = synth.uniform_u32(50021, 11 + shift)
    out = oracle.counting_pass_u32(a, shift)
    digit = (a >> np.uint32(shift)) & np.uint32(255)
    assert np.array_equal(out, a[np.argsort(digit, kind="stable")])


def test_empty_and_single():
    assert oracle.sort_u32(np.empty(0, np.uint32)).size == 0
    assert oracle.sort_u64(np.array([7], np.uint64)).tolist() == [7]
    k, v = oracle.sort_u64_kv(np.empty(0, np.uint64), np.empty(0, np.uint32))
    assert k.size == 0 and v.size == 0


# ---- key formats (signed, IEEE float total order, descending), pinned to
# numpy's sorts and to hand-written total orders

FMT_SIGNED, FMT_FLOAT, FMT_DESC = 1, 2, 0x100


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("dt,kt", [(np.int32, 0), (np.int64, 1)])
def test_signed_matches_numpy(dt, kt):
    g = _rng(11)
    info = np.iinfo(dt)
    a = g.integers(info.min, info.max, 20000, dtype=dt, endpoint=True)
    a[:6] = [info.min, info.max, -1, 0, 1, info.min + 1]
    got = oracle.sort_format(kt, FMT_SIGNED, a)
    assert got.dtype == dt and np.array_equal(got, np.sort(a))
    desc = oracle.sort_format(kt, FMT_SIGNED | FMT_DESC, a)
    assert np.array_equal(desc, np.sort(a)[::-1])


@pytest.mark.parametrize("dt,kt", [(np.float32, 0), (np.float64, 1)])
def test_float_finite_matches_numpy(dt, kt):
    g = _rng(12)
    a = (g.standard_normal(20000) * 10.0 ** g.integers(-30, 30, 20000)).astype(dt)
    a[:5] = [np.inf, -np.inf, np.finfo(dt).tiny / 4, -np.finfo(dt).tiny / 4, 0.0]  # with subnormals; no -0.0, no NaN
    got = oracle.sort_format(kt, FMT_FLOAT, a)
    assert np.array_equal(got, np.sort(a, kind="stable"))
    assert np.array_equal(oracle.sort_format(kt, FMT_FLOAT | FMT_DESC, a), np.sort(a)[::-1])


@pytest.mark.parametrize("dt,it,kt", [(np.float32, np.uint32, 0), (np.float64, np.uint64, 1)])
def test_float_special_values_total_order(dt, it, kt):
    bits = 8 * np.dtype(dt).itemsize
    sign = 1 << (bits - 1)
    qnan = np.array([np.nan], dtype=dt).view(it)[0]
    order = [int(qnan) | sign | 5,  # a negative NaN with a larger payload sorts first
             int(qnan) | sign,
             int(np.array([-np.inf], dtype=dt).view(it)[0]),
             int(np.array([-1.5], dtype=dt).view(it)[0]),
             sign | 1,  # the negative subnormal closest to zero
             sign,  # -0.0
             0,  # +0.0
             1,  # the smallest positive subnormal
             int(np.array([2.0], dtype=dt).view(it)[0]),
             int(np.array([np.inf], dtype=dt).view(it)[0]),
             int(qnan),
             int(qnan) | 5]
    expected = np.array(order, dtype=it)
    g = _rng(13)
    shuffled = expected[g.permutation(expected.size)]
    assert np.array_equal(oracle.sort_format(kt, FMT_FLOAT, shuffled.view(dt)).view(it), expected)
    assert np.array_equal(oracle.sort_format(kt, FMT_FLOAT | FMT_DESC, shuffled.view(dt)).view(it), expected[::-1])


@pytest.mark.parametrize("kt,dt", [(3, np.int32), (2, np.int64)])
def test_formats_key_value_stability(kt, dt):
    g = _rng(14)
    n = 3000
    a = g.integers(-5, 5, n).astype(dt)  # many ties
    v = np.arange(n, dtype=np.uint32)
    for fmt, key in ((FMT_SIGNED, lambda i: (a[i], i)), (FMT_SIGNED | FMT_DESC, lambda i: (-a[i], i))):
        k, vv = oracle.sort_format(kt, fmt, a, v)
        order = sorted(range(n), key=key)
        assert np.array_equal(vv, np.array(order, dtype=np.uint32))
        assert np.array_equal(k, a[order])


def test_unsigned_descending_and_bad_format():
    g = _rng(15)
    a = g.integers(0, 1 << 32, 5000, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(oracle.sort_format(0, FMT_DESC, a), np.sort(a)[::-1])
    assert np.array_equal(oracle.sort_format(0, 0, a), np.sort(a))
    with pytest.raises(RuntimeError):
        oracle.sort_format(0, 3, a)


def wide_payload(n):
    """64-bit payloads whose high and low halves both vary: the original index
    in the low half, a per-record pattern in the high half, so a payload cut to
    32 bits, or moved as two halves from different records, does not survive."""
    i = np.arange(n, dtype=np.uint64)
    return i | (((i * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)) << np.uint64(32))


@pytest.mark.parametrize("n", range(0, 6))
def test_kv64_exhaustive_vs_insertion_sort(n):
    """64-bit payloads move with their keys, stably, exactly as a stable
    insertion sort of (key, original index) records places them."""
    orc = oracle.default()
    pay = wide_payload(n)
    for tup in itertools.product(U64_ALPHABET[:5], repeat=n):
        want_k, want_i = insertion_sort_pairs(tup)
        k, v = orc.sort_u64_kv64(np.array(tup, dtype=np.uint64), pay)
        assert k.tolist() == want_k and v.tolist() == pay[want_i].tolist(), tup
    for tup in itertools.product(U32_ALPHABET, repeat=n):
        want_k, want_i = insertion_sort_pairs(tup)
        k, v = orc.sort_u32_kv64(np.array(tup, dtype=np.uint32), pay)
        assert k.tolist() == want_k and v.tolist() == pay[want_i].tolist(), tup


def test_kv64_random_vs_numpy_stable_and_special_cases():
    orc = oracle.default()
    g = np.random.Generator(np.random.PCG64(synth.BASE_SEED + 64))
    for trial in range(300):
        n = int(g.integers(0, 3001))
        k64 = g.bit_generator.random_raw(n).astype(np.uint64) >> np.uint64(int(g.integers(0, 64)))
        k32 = (k64 & np.uint64(0xFFFFFFFF)).astype(np.uint32) >> np.uint32(int(g.integers(0, 32)))
        v = g.bit_generator.random_raw(n).astype(np.uint64)
        kk, vv = orc.sort_u64_kv64(k64, v)
        order = np.argsort(k64, kind="stable")
        assert np.array_equal(kk, k64[order]) and np.array_equal(vv, v[order])
        kk, vv = orc.sort_u32_kv64(k32, v)
        order = np.argsort(k32, kind="stable")
        assert np.array_equal(kk, k32[order]) and np.array_equal(vv, v[order])
    # all-equal keys: the payloads keep their order; reverse distinct keys: reversed
    n = 5000
    pay = wide_payload(n)
    k, v = orc.sort_u64_kv64(np.full(n, 0xDEADBEEFCAFEF00D, np.uint64), pay)
    assert np.array_equal(v, pay)
    d = np.arange(n, dtype=np.uint32)[::-1].copy() * np.uint32(97)
    k, v = orc.sort_u32_kv64(d, pay)
    assert np.array_equal(k, d[::-1]) and np.array_equal(v, pay[::-1])
