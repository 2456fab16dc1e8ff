"""Executable checks of two readings of the paper's schedules (CPU only).

* Diverting LSD (Section "Diverting Fast Radix", Algorithm 4): deal the top
  d digits least significant first with stable counting sorts, then sort
  every bucket of the d-digit prefix with a stable small-bucket sort.  The
  reading is that this yields exactly the plain stable sort (so an LSD
  schedule and the MSD recursion may replace each other): checked against
  the oracle's sort, payloads included, for d = 1, 2.
* Fast Radix's estimated deal (Algorithm 3): records go to estimated buckets
  of `cap` slots, a record that finds its bucket full goes to that bucket's
  overflow region, and the next pass reads every bucket's main part and then
  its overflow.  The reading is that this reading order is exactly the order
  of a stable counting pass on the same digit, whatever the overflow, so the
  estimate never costs stability: checked against the oracle's counting pass.

The deals here are played out record by record in plain Python; the oracle
supplies the stable counting pass and the full sort.
"""
import numpy as np
import pytest

import oracle


def stable_insertion_sort(recs):
    """Stable insertion sort of (key, payload) records by key."""
    out = list(recs)
    for i in range(1, len(out)):
        cur = out[i]
        j = i - 1
        while j >= 0 and out[j][0] > cur[0]:
            out[j + 1] = out[j]
            j -= 1
        out[j + 1] = cur
    return out


def counting_deal(recs, shift):
    """One stable counting sort of (key, payload) records on the 8-bit digit at `shift`."""
    buckets = [[] for _ in range(256)]
    for r in recs:
        buckets[(r[0] >> shift) & 255].append(r)
    return [r for b in buckets for r in b]


def diverting_lsd(keys, vals, d):
    """Algorithm 4 on u32 records: LSD over the top d digits, then a stable
    sort of every d-digit-prefix bucket."""
    recs = list(zip((int(k) for k in keys), (int(v) for v in vals)))
    for j in range(d - 1, -1, -1):  # least significant of the top d digits first
        recs = counting_deal(recs, 24 - 8 * j)
    out = []
    i = 0
    pshift = 32 - 8 * d
    while i < len(recs):
        j = i
        while j < len(recs) and (recs[j][0] >> pshift) == (recs[i][0] >> pshift):
            j += 1
        out.extend(stable_insertion_sort(recs[i:j]))
        i = j
    return out


@pytest.mark.parametrize("d", [1, 2])
def test_diverting_lsd_equals_the_stable_sort(d):
    g = np.random.default_rng(300 + d)
    for trial in range(6):
        n = int(g.integers(0, 1500))
        keys = g.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        if trial % 3 == 1:
            keys &= np.uint32(0xFFFF00FF)  # a constant digit inside the dealt range
        if trial % 3 == 2:
            keys = g.choice(keys[: max(1, n // 20)], size=n) if n else keys  # heavy ties
        vals = np.arange(n, dtype=np.uint32)
        got = diverting_lsd(keys, vals, d)
        ok, ov = oracle.sort_u32_kv(keys, vals)
        assert [r[0] for r in got] == ok.tolist()
        assert [r[1] for r in got] == ov.tolist()  # stable: payloads in input order on ties


def estimated_deal(keys, shift, cap):
    """Algorithm 3's estimated deal: bucket b holds `cap` records at b*cap,
    the rest go to its overflow region in arrival order.  Returns the records
    in the order the next pass reads them (bucket b's main part, then its
    overflow, for b = 0..255) and the number that overflowed."""
    main = [[] for _ in range(256)]
    over = [[] for _ in range(256)]
    for k in keys:
        b = (int(k) >> shift) & 255
        (main[b] if len(main[b]) < cap else over[b]).append(int(k))
    order = []
    for b in range(256):
        order.extend(main[b])
        order.extend(over[b])
    return order, sum(len(o) for o in over)


@pytest.mark.parametrize("shift", [0, 16, 24])
def test_estimated_deal_reads_in_stable_order(shift):
    g = np.random.default_rng(400 + shift)
    for trial in range(8):
        n = int(g.integers(0, 4000))
        keys = g.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        if trial % 2:
            keys[: n // 2] &= np.uint32(~(0xFF << shift) & 0xFFFFFFFF)  # half the keys in bucket 0: heavy overflow
        cap = max(0, n // 256 + int(g.integers(-3, 4)))
        order, nover = estimated_deal(keys, shift, cap)
        assert order == oracle.counting_pass_u32(keys, shift).tolist()
        assert nover == oracle.overflow_count(keys, shift, cap)


def test_runs_of_small_buckets_sort_as_each_bucket_alone():
    """Section "Diverting Fast Radix" sorts the small buckets in bulk: after a
    stable deal on the top digit, consecutive small buckets are joined into
    runs and each run is sorted stably as one piece.  Because the buckets of a
    run are adjacent, ordered and never share a key, that equals sorting each
    bucket alone and equals the plain stable sort, payloads included."""
    g = np.random.default_rng(500)
    for trial in range(6):
        n = int(g.integers(1, 3000))
        keys = g.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        if trial % 2:
            keys = g.choice(keys[: max(1, n // 30)], size=n)  # heavy ties inside buckets
        vals = np.arange(n, dtype=np.uint32)
        recs = counting_deal(list(zip((int(k) for k in keys), (int(v) for v in vals))), 24)
        bounds = [0]
        for i in range(1, n):
            if (recs[i][0] >> 24) != (recs[i - 1][0] >> 24):
                bounds.append(i)
        bounds.append(n)
        # join consecutive buckets into runs of random lengths, then sort each run
        out, b = [], 0
        while b < len(bounds) - 1:
            e = min(len(bounds) - 1, b + int(g.integers(1, 6)))
            out.extend(stable_insertion_sort(recs[bounds[b]:bounds[e]]))
            b = e
        ok, ov = oracle.sort_u32_kv(keys, vals)
        assert [r[0] for r in out] == ok.tolist()
        assert [r[1] for r in out] == ov.tolist()
