"""Pins for the oracle's Fast Radix overflow pieces (CPU only).

Two things are pinned here, each against something other than itself:
  * oracle.overflow_count -- the estimated deal of Algorithm 3 played out
    record by record -- against a pure-Python deal of the same records,
    against the per-bucket counting form sum_d max(0, count_d - cap), and
    against closed forms (all keys equal; every digit equally often);
  * oracle.overflow_fraction -- g_o(N, M) of Section "Analysis", read as the
    sum of the Eq. 2 terms over k < ceil(N/M) -- against the paper's own
    recursion (Eq. 1, which it must satisfy exactly), against exhaustive
    enumeration of every way to deal N records into M buckets, against the
    single-record closed form, against the normal limit for large N/M,
    against Monte Carlo, and against the monotonic decrease the paper states.
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def python_deal_overflow(keys, shift, cap):
    """Deal the records one by one into 256 buckets of `cap` slots; count the
    records that find their bucket full."""
    fill = [0] * 256
    over = 0
    for k in keys:
        b = (int(k) >> shift) & 255
        if fill[b] < cap:
            fill[b] += 1
        else:
            over += 1
    return over


# ------------------------------------------------------------ overflow_count --

@pytest.mark.parametrize("dtype,shift", [(np.uint32, 0), (np.uint32, 16), (np.uint32, 24), (np.uint64, 56),
                                         (np.uint64, 8)])
def test_overflow_count_vs_python_deal(dtype, shift):
    g = np.random.default_rng(11 + shift)
    bits = 8 * np.dtype(dtype).itemsize
    for trial in range(6):
        n = int(g.integers(0, 4000))
        keys = g.integers(0, 1 << 63, size=n, dtype=np.uint64)
        if bits == 32:
            keys = (keys >> np.uint64(31)).astype(np.uint32)
        keys = keys.astype(dtype)
        if trial % 2:
            keys = keys & dtype(((1 << bits) - 1) ^ (0x0F << shift))  # skewed digits (low nibble cleared)
        cap = int(g.integers(0, 40))
        want = python_deal_overflow(keys.tolist(), shift, cap)
        assert oracle.overflow_count(keys, shift, cap) == want
        counts = np.bincount(((keys >> dtype(shift)) & dtype(255)).astype(np.int64), minlength=256)
        assert want == int(np.maximum(counts - cap, 0).sum())


def test_overflow_count_closed_forms():
    n = 5000
    eq = np.full(n, 0xDEADBEEF, dtype=np.uint32)
    assert oracle.overflow_count(eq, 16, 100) == n - 100
    assert oracle.overflow_count(eq, 16, n) == 0
    # every digit value exactly c times, in a shuffled order
    c = 37
    k = np.repeat(np.arange(256, dtype=np.uint32) << np.uint32(8), c)
    np.random.default_rng(3).shuffle(k)
    assert oracle.overflow_count(k, 8, c) == 0
    assert oracle.overflow_count(k, 8, c - 1) == 256
    assert oracle.overflow_count(k, 0, c) == k.size - c  # digit 0 of every key is 0
    assert oracle.overflow_count(np.zeros(0, np.uint64), 0, 0) == 0


# ---------------------------------------------------------- overflow model --

def g_o(N, M):
    return oracle.overflow_fraction(N, M)


@pytest.mark.parametrize("M", [2, 3, 16, 256])
def test_eq1_recursion_holds(M):
    # Eq. 1: g_o(N, M) = g_o(N-1, M) - (1/M) g_o(N-1, M, ceil(N/M) - 1)
    Ns = list(range(2, 400)) + list(range(400, 5000, 97))
    for N in Ns:
        lhs = g_o(N, M)
        rhs = g_o(N - 1, M) - oracle.overflow_term(N - 1, M, -(-N // M) - 1) / M
        assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-14), (N, M)


@pytest.mark.parametrize("M", [2, 7, 256])
def test_single_record(M):
    # one record: its bucket of estimated size 1/M is short by 1/M with
    # probability 1 - 1/M (the record went elsewhere), times M/N = M
    assert g_o(1, M) == pytest.approx(1.0 - 1.0 / M, rel=1e-12)


@pytest.mark.parametrize("N,M", [(2, 2), (4, 2), (6, 2), (5, 2), (6, 3), (7, 3), (8, 4), (5, 4), (9, 3)])
def test_exhaustive_deals(N, M):
    # average over all M^N equally likely deals of the total shortfall below
    # N/M (which equals the total excess above it), divided by N
    mean = N / M
    tot_short = 0.0
    tot_excess = 0.0
    for assign in itertools.product(range(M), repeat=N):
        cnt = np.bincount(np.array(assign), minlength=M)
        tot_short += np.maximum(mean - cnt, 0.0).sum()
        tot_excess += np.maximum(cnt - mean, 0.0).sum()
    deals = float(M) ** N
    assert g_o(N, M) == pytest.approx(tot_short / deals / N, rel=1e-12)
    assert g_o(N, M) == pytest.approx(tot_excess / deals / N, rel=1e-12)


def test_normal_limit():
    # large N/M: a bucket's count is close to normal with variance
    # N (1/M)(1 - 1/M); its mean excess above the mean is sigma / sqrt(2 pi)
    for N in (1 << 24, 1 << 28):
        M = 256
        sigma = math.sqrt(N / M * (1.0 - 1.0 / M))
        assert g_o(N, M) == pytest.approx(M / N * sigma / math.sqrt(2 * math.pi), rel=1e-3)


def test_monte_carlo():
    g = np.random.default_rng(20220729)
    N, M = 1 << 16, 256
    trials = 400
    fr = np.empty(trials)
    for t in range(trials):
        cnt = g.multinomial(N, [1.0 / M] * M)
        fr[t] = np.maximum(cnt - N // M, 0).sum() / N
    se = fr.std(ddof=1) / math.sqrt(trials)
    assert abs(fr.mean() - g_o(N, M)) < 4 * se


def test_monte_carlo_with_oracle_deal():
    # the record-by-record deal of the oracle on uniform keys overflows, on
    # average, g_o(N, M) * N records when every bucket holds N/M
    g = np.random.default_rng(5)
    N = 1 << 14
    trials = 200
    fr = np.empty(trials)
    for t in range(trials):
        k = g.integers(0, 1 << 32, size=N, dtype=np.uint64).astype(np.uint32)
        fr[t] = oracle.overflow_count(k, 16, N // 256) / N
    se = fr.std(ddof=1) / math.sqrt(trials)
    assert abs(fr.mean() - g_o(N, 256)) < 4 * se


def test_monotone_decreasing():
    vals = [g_o(N, 256) for N in range(1, 2500)]
    # non-increasing; at N = cM + 1 the step is exactly zero (the Eq. 1 term
    # has the factor N/M - k = 0), so allow fp64 rounding there
    assert all(b <= a * (1 + 1e-11) for a, b in zip(vals, vals[1:]))
    assert vals[-1] < 0.2 * vals[0]
