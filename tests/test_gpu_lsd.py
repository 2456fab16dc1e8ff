"""The LSD top phase on the GPU (paper, Section "Diverting Fast Radix",
Algorithms 3 and 4), forced through the launch-plan table:

  * DFR_SCHED_LSD -- one upfront read counts the two top digits, which are
    dealt least significant first; the 16-bit prefix buckets are then
    diverted or recursed on;
  * DFR_SCHED_DFR -- the same, but the first deal uses estimated buckets of
    N/256 keys with overflow regions and no counting read (Fast Radix); a
    failed estimate falls back to the MSD schedule.

Every result is compared element by element with the oracle (keys, and
payloads in stable order) on each key type and on the paper's distributions,
ragged sizes and the size boundary.  The reported schedule, estimated bucket
size and overflow count are checked against the oracle's record-by-record
deal (exactly) and against the paper's overflow model g_o (statistically).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu, sorter

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


class forced_schedule:
    """Set `schedule` in every entry of the plan table for the duration."""

    def __init__(self, dfr, sched):
        self.dfr, self.sched = dfr, sched

    def __enter__(self):
        d = self.dfr
        for kt in (d.DFR_U32, d.DFR_U64, d.DFR_U64_KV, d.DFR_U32_KV):
            for c in range(d.DFR_TUNE_CLASSES):
                t = d.dfr_tune_get(kt, c)
                t["schedule"] = self.sched
                assert d.dfr_tune_set(kt, c, t) == d.DFR_OK

    def __exit__(self, *exc):
        assert self.dfr.dfr_tune_reset() == self.dfr.DFR_OK


def run(dfr, keys, vals=None):
    """Sort on the GPU; return keys, payloads, device status and the stats."""
    if keys.dtype == np.uint32:
        kt = dfr.DFR_U32 if vals is None else dfr.DFR_U32_KV
    else:
        kt = dfr.DFR_U64 if vals is None else dfr.DFR_U64_KV
    s = sorter(dfr, kt, keys.size)
    dk = dfr.to_device(keys)
    dv = dfr.to_device(vals) if vals is not None else None
    assert s.sort_(dk, dv) == dfr.DFR_OK
    st = s.device_status()
    stats = s.stats()
    k = dfr.to_numpy(dk, keys.dtype)
    v = None if vals is None else dfr.to_numpy(dv, np.uint32)
    return k, v, st, stats


def top_varies(keys):
    w = 8 * keys.dtype.itemsize
    top = keys >> keys.dtype.type(w - 8)
    return top.min() != top.max()


def second_values(keys):
    w = 8 * keys.dtype.itemsize
    return np.unique((keys >> keys.dtype.type(w - 16)) & keys.dtype.type(255)).size


U32_DISTS = synth.U32_DISTRIBUTIONS


@pytest.mark.parametrize("dist", U32_DISTS)
def test_u32_lsd_counted(dfr, dist):
    n = dfr.dfr_lsd_min_keys(dfr.DFR_U32) + 12_345
    a = synth.u32(dist, n, synth.BASE_SEED + 1300 + U32_DISTS.index(dist))
    with forced_schedule(dfr, dfr.DFR_SCHED_LSD):
        k, _, st, stats = run(dfr, a)
    assert st == dfr.DFR_OK
    assert np.array_equal(k, oracle.sort_u32(a)), dist
    eligible = top_varies(a) and second_values(a) >= 2
    assert stats["schedule"] == (dfr.DFR_SCHED_LSD if eligible else dfr.DFR_SCHED_MSD)
    if eligible:
        assert stats["lsd_keys"] == 2 * n and stats["root_read"] == 1
        assert stats["level_keys"][0] == 0  # the top digits were not dealt by an MSD level


@pytest.mark.parametrize("dist", U32_DISTS)
def test_u32_dfr_estimated(dfr, dist):
    n = dfr.dfr_lsd_min_keys(dfr.DFR_U32) + 54_321
    a = synth.u32(dist, n, synth.BASE_SEED + 1400 + U32_DISTS.index(dist))
    with forced_schedule(dfr, dfr.DFR_SCHED_DFR):
        k, _, st, stats = run(dfr, a)
    assert st == dfr.DFR_OK
    assert np.array_equal(k, oracle.sort_u32(a)), dist
    cap = (n // 256) & ~15
    assert stats["est_capacity"] == cap
    if dist in ("uniform", "sorted", "reverse", "normal"):
        # D1 (bits 23..16) is close to uniform: the estimate holds
        assert stats["schedule"] == dfr.DFR_SCHED_DFR and stats["est_aborted"] == 0, stats
        assert stats["root_read"] == 0 and stats["lsd_keys"] == 2 * n
        assert stats["est_overflow"] == oracle.overflow_count(a, 16, cap)
        assert stats["model_bytes"] == 2 * 8 * n + 8 * (stats["cta_keys"] + stats["wsort_keys"]
                                                         + stats["tiny_keys"] + stats["copy_keys"]
                                                         + sum(stats["level_keys"]))
    else:
        # equal keys, Zipf's heavy values and the exponential's skewed D1
        # overflow an estimated bucket's region: the MSD schedule sorts
        assert stats["est_aborted"] == 1 and stats["schedule"] == dfr.DFR_SCHED_MSD, stats
        assert stats["root_read"] == 1


def test_u32_dfr_overflow_matches_the_model(dfr):
    # N = 2^26 uniform keys: buckets of exactly N/256, so the overflow the
    # deal reports is, in expectation, g_o(N, 256) * N (Eq. 1-2); the count
    # itself must equal the oracle's record-by-record deal exactly
    n = 1 << 26
    a = synth.uniform_u32(n, synth.BASE_SEED + 1500)
    with forced_schedule(dfr, dfr.DFR_SCHED_DFR):
        k, _, st, stats = run(dfr, a)
    assert st == dfr.DFR_OK and stats["schedule"] == dfr.DFR_SCHED_DFR
    assert np.array_equal(k, oracle.sort_u32(a))
    cap = n // 256
    assert stats["est_capacity"] == cap
    assert stats["est_overflow"] == oracle.overflow_count(a, 16, cap)
    mean = oracle.overflow_fraction(n, 256) * n
    # one bucket's overflow (X - mu)+ has variance sigma^2 (1/2 - 1/(2 pi));
    # 256 nearly independent buckets
    sigma = math.sqrt(n / 256 * (1 - 1 / 256))
    sd = math.sqrt(256 * sigma ** 2 * (0.5 - 1 / (2 * math.pi)))
    assert abs(stats["est_overflow"] - mean) < 5 * sd, (stats["est_overflow"], mean, sd)


@pytest.mark.parametrize("sched", [1, 2])
@pytest.mark.parametrize("dist", synth.U64_DISTRIBUTIONS)
def test_u64_keys_and_pairs(dfr, sched, dist):
    n = dfr.dfr_lsd_min_keys(dfr.DFR_U64_KV) + 777
    a = synth.u64(dist, n, synth.BASE_SEED + 1600 + synth.U64_DISTRIBUTIONS.index(dist))
    v = synth.index_payload(n)
    with forced_schedule(dfr, sched):
        k, _, st, stats = run(dfr, a)
        kk, vv, st2, stats2 = run(dfr, a, v)
    assert st == dfr.DFR_OK and st2 == dfr.DFR_OK
    assert np.array_equal(k, oracle.sort_u64(a)), dist
    ok, ov = oracle.sort_u64_kv(a, v)
    assert np.array_equal(kk, ok) and np.array_equal(vv, ov), dist
    if dist == "uniform64":
        assert stats["schedule"] == sched and stats2["schedule"] == sched
    if dist == "uniform16":  # top 48 bits zero: nothing for the LSD phase
        assert stats["schedule"] == 0 and stats2["schedule"] == 0


@pytest.mark.parametrize("sched", [1, 2])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "normal", "few"])
def test_u32_pairs_stable(dfr, sched, dist):
    n = dfr.dfr_lsd_min_keys(dfr.DFR_U32_KV) + 4099
    if dist == "few":
        g = np.random.default_rng(77)
        a = g.choice(synth.uniform_u32(300, 78), size=n).astype(np.uint32)  # heavy ties across every digit
    else:
        a = synth.u32(dist, n, synth.BASE_SEED + 1700 + len(dist))
    v = synth.index_payload(n)
    with forced_schedule(dfr, sched):
        k, vv, st, stats = run(dfr, a, v)
    assert st == dfr.DFR_OK
    ok, ov = oracle.sort_u32_kv(a, v)
    assert np.array_equal(k, ok) and np.array_equal(vv, ov), (sched, dist, stats["schedule"])
    if dist == "uniform":
        assert stats["schedule"] == sched


@pytest.mark.parametrize("sched", [1, 2])
def test_size_boundary_and_ragged(dfr, sched):
    m = dfr.dfr_lsd_min_keys(dfr.DFR_U32)
    for n, want in ((m - 1, 0), (m, sched), (m + 1, sched), (m + 15, sched), (3 * m + 7, sched)):
        a = synth.uniform_u32(n, synth.BASE_SEED + 1800 + n)
        with forced_schedule(dfr, sched):
            k, _, st, stats = run(dfr, a)
        assert st == dfr.DFR_OK and np.array_equal(k, oracle.sort_u32(a)), n
        assert stats["schedule"] == want, (n, stats["schedule"])


def test_misaligned_view(dfr):
    # an array that starts 4 bytes past a 16-byte boundary: pass 0 reads it
    # without 128-bit loads; the result is still exact
    import torch

    n = dfr.dfr_lsd_min_keys(dfr.DFR_U32) + 333
    a = synth.uniform_u32(n, synth.BASE_SEED + 1900)
    s = sorter(dfr, dfr.DFR_U32, n + 1)
    base = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    base[1:] = torch.from_numpy(a.view(np.int32)).cuda()
    view = base[1:]
    with forced_schedule(dfr, dfr.DFR_SCHED_DFR):
        assert s.sort_(view) == dfr.DFR_OK
        assert s.device_status() == dfr.DFR_OK
        stats = s.stats()
    assert stats["schedule"] == dfr.DFR_SCHED_DFR
    out = view.cpu().numpy().view(np.uint32)
    assert np.array_equal(out, oracle.sort_u32(a))


def test_graph_with_lsd(dfr):
    n = dfr.dfr_lsd_min_keys(dfr.DFR_U32) + 99
    a = synth.uniform_u32(n, synth.BASE_SEED + 1950)
    import torch

    keys = dfr.to_device(a)
    buf = torch.empty_like(keys)
    ws_bytes = dfr.dfr_workspace_bytes(dfr.DFR_U32, n)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    with forced_schedule(dfr, dfr.DFR_SCHED_DFR):
        g = dfr.dfr_graph_create([(dfr.DFR_U32, keys, None, buf, None, n)], ws, ws_bytes)
    try:
        for rep in range(3):
            keys.copy_(dfr.to_device(a))
            assert dfr.dfr_graph_launch(g) == dfr.DFR_OK
            torch.cuda.synchronize()
            assert dfr.dfr_last_device_status(ws) == dfr.DFR_OK
            assert dfr.dfr_get_stats(ws)["schedule"] == dfr.DFR_SCHED_DFR
            assert np.array_equal(dfr.to_numpy(keys, np.uint32), oracle.sort_u32(a)), rep
    finally:
        dfr.dfr_graph_destroy(g)


def test_forced_timeout_in_lsd_pass(dfr):
    # the second pass chains its tiles with a bounded look-back; a wait on a
    # word nobody sets must end with DFR_ERR_TIMEOUT and leave the context usable
    n = dfr.dfr_lsd_min_keys(dfr.DFR_U32) + 5
    a = synth.uniform_u32(n, 6)
    with forced_schedule(dfr, dfr.DFR_SCHED_LSD):
        try:
            dfr.dfr_set_debug(2000, True)
            _, _, st, _ = run(dfr, a)
        finally:
            dfr.dfr_set_debug(0, False)
        assert st == dfr.DFR_ERR_TIMEOUT
        k, _, st, stats = run(dfr, a)
    assert st == dfr.DFR_OK and stats["schedule"] == dfr.DFR_SCHED_LSD
    assert np.array_equal(k, oracle.sort_u32(a))


@pytest.mark.parametrize("sched", [1, 2])
def test_lsd_with_key_formats(dfr, sched):
    # signed and IEEE-float keys are mapped to their unsigned images in
    # place, sorted (here through the LSD phase) and mapped back
    import torch

    n = dfr.dfr_lsd_min_keys(dfr.DFR_U32) + 1001
    g = np.random.default_rng(3100 + sched)
    a = g.integers(-(1 << 31), (1 << 31) - 1, size=n, dtype=np.int64).astype(np.int32)
    f = (g.standard_normal(n) * 1e6).astype(np.float64)
    v = synth.index_payload(f.size)
    with forced_schedule(dfr, sched):
        s = sorter(dfr, dfr.DFR_U32, n)
        dk = dfr.to_device(a)
        assert s.sort_(dk, key_format=dfr.DFR_FMT_SIGNED) == dfr.DFR_OK
        assert s.device_status() == dfr.DFR_OK
        st = s.stats()
        assert np.array_equal(dk.cpu().numpy(), oracle.sort_format(0, dfr.DFR_FMT_SIGNED, a))
        assert st["schedule"] == sched
        s2 = sorter(dfr, dfr.DFR_U64_KV, f.size)
        dk2 = dfr.to_device(f)
        dv2 = dfr.to_device(v)
        assert s2.sort_(dk2, dv2, key_format=dfr.DFR_FMT_FLOAT | dfr.DFR_FMT_DESCENDING) == dfr.DFR_OK
        assert s2.device_status() == dfr.DFR_OK
        ek, ev = oracle.sort_format(2, dfr.DFR_FMT_FLOAT | dfr.DFR_FMT_DESCENDING, f, v)
        assert np.array_equal(dk2.cpu().numpy().view(np.float64), ek)
        assert np.array_equal(dfr.to_numpy(dv2, np.uint32), ev)
    torch.cuda.synchronize()


@pytest.mark.parametrize("sched", [1, 2])
def test_lsd_through_the_batch_entry(dfr, sched):
    # a batch of one array takes the LSD phase too; its descriptor reaches
    # the device by a copy instead of the first kernel's parameters
    import torch

    n = dfr.dfr_lsd_min_keys(dfr.DFR_U64_KV) + 12_345
    a = synth.uniform64_u64(n, synth.BASE_SEED + 3200 + sched)
    v = synth.index_payload(n)
    keys, vals = dfr.to_device(a), dfr.to_device(v)
    kbuf, vbuf = torch.empty_like(keys), torch.empty_like(vals)
    seg = (dfr.DFR_U64_KV, keys, vals, kbuf, vbuf, n)
    wsb = dfr.dfr_batch_workspace_bytes([seg])
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    with forced_schedule(dfr, sched):
        assert dfr.dfr_sort_batch([seg], ws, wsb) == dfr.DFR_OK
        torch.cuda.synchronize()
        assert dfr.dfr_last_device_status(ws) == dfr.DFR_OK
        assert dfr.dfr_get_stats(ws)["schedule"] == sched
    ok, ov = oracle.sort_u64_kv(a, v)
    assert np.array_equal(dfr.to_numpy(keys, np.uint64), ok)
    assert np.array_equal(dfr.to_numpy(vals, np.uint32), ov)
