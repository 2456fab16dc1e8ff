"""The persistent launch form (DFR_LAUNCH_PERSISTENT): a whole call as one
cooperative kernel whose CTAs pull the count, deal, classification,
diverted-bucket and copy-back items of all arrays from device queues, level
after level until none is left (the recursion of Algorithm 2), with bounded
grid-wide barriers between dependent phases.

Every result is compared element by element with the oracle; the statistics
say which form ran; the level sequence (DFR_LAUNCH_LEVELS) is checked to stay
selectable; the automatic choice follows the call's total key count; the
grid barrier's forced timeout reports DFR_ERR_TIMEOUT and the next call
succeeds; CUDA graphs capture the persistent form.
"""
import contextlib

import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_sort, need_gpu

pytestmark = pytest.mark.gpu

S = synth.BASE_SEED + 3000


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


@contextlib.contextmanager
def launch_form(dfr, launch, key_types=None):
    """Force one launch form for every size class of the given key types."""
    kts = key_types or (dfr.DFR_U32, dfr.DFR_U64, dfr.DFR_U64_KV, dfr.DFR_U32_KV, dfr.DFR_U64_KV64, dfr.DFR_U32_KV64)
    saved = {(kt, c): dfr.dfr_tune_get(kt, c) for kt in kts for c in range(dfr.DFR_TUNE_CLASSES)}
    try:
        for (kt, c), t in saved.items():
            assert dfr.dfr_tune_set(kt, c, dict(t, launch=launch)) == dfr.DFR_OK
        yield
    finally:
        for (kt, c), t in saved.items():
            dfr.dfr_tune_set(kt, c, t)


def sort_with_stats(dfr, keys, vals=None, key_type=None):
    """gpu_sort plus the statistics of the call."""
    from gpu_util import sorter

    k, v, st = gpu_sort(dfr, keys, vals, key_type)
    if key_type is None:
        wide = vals is not None and vals.dtype.itemsize == 8
        if keys.dtype == np.uint32:
            key_type = dfr.DFR_U32 if vals is None else (dfr.DFR_U32_KV64 if wide else dfr.DFR_U32_KV)
        else:
            key_type = dfr.DFR_U64 if vals is None else (dfr.DFR_U64_KV64 if wide else dfr.DFR_U64_KV)
    return k, v, st, sorter(dfr, key_type, keys.size).stats()


def expected(keys, vals):
    if vals is None:
        return (oracle.sort_u32(keys) if keys.dtype == np.uint32 else oracle.sort_u64(keys)), None
    if vals.dtype.itemsize == 8:
        return oracle.sort_u64_kv64(keys, vals) if keys.dtype == np.uint64 else oracle.sort_u32_kv64(keys, vals)
    return oracle.sort_u64_kv(keys, vals) if keys.dtype == np.uint64 else oracle.sort_u32_kv(keys, vals)


@pytest.mark.parametrize("dist", synth.U32_DISTRIBUTIONS)
@pytest.mark.parametrize("n", [33, 4097, 70_001, 1_000_003, (1 << 22) + 12_345])
def test_u32_persistent_matches_oracle(dfr, dist, n):
    a = synth.u32(dist, n, S + n % 1000 + synth.U32_DISTRIBUTIONS.index(dist))
    with launch_form(dfr, dfr.DFR_LAUNCH_PERSISTENT, (dfr.DFR_U32,)):
        k, _, st, stats = sort_with_stats(dfr, a)
    assert st == dfr.DFR_OK
    assert stats["persistent"] == 1
    assert np.array_equal(k, oracle.sort_u32(a))


@pytest.mark.parametrize("kind", ["u64", "u64kv", "u32kv", "u64kv64", "u32kv64"])
@pytest.mark.parametrize("dist", ["uniform64", "uniform16", "dup90"])
@pytest.mark.parametrize("n", [513, 70_001, 1_000_003])
def test_other_key_types_persistent_match_oracle(dfr, kind, dist, n):
    seed = S + 100 + n % 97
    k64 = synth.u64(dist, n, seed)
    keys = k64 if kind.startswith("u64") else (k64 >> np.uint64(32)).astype(np.uint32)
    vals = None
    if kind.endswith("kv"):
        vals = synth.index_payload(n)
    elif kind.endswith("kv64"):
        g = np.random.Generator(np.random.PCG64(seed + 1))
        vals = g.bit_generator.random_raw(n).astype(np.uint64)
    with launch_form(dfr, dfr.DFR_LAUNCH_PERSISTENT):
        k, v, st, stats = sort_with_stats(dfr, keys, vals)
    assert st == dfr.DFR_OK
    assert stats["persistent"] == 1
    wk, wv = expected(keys, vals)
    assert np.array_equal(k, wk)
    if vals is not None:
        assert np.array_equal(v, wv)


def test_deep_recursion_persistent(dfr):
    """64-bit keys varying in their low 40 bits and a heavy-tailed u32 input:
    many levels inside the one launch, each level's segment count read after
    a barrier."""
    n = 1_500_000
    g = np.random.Generator(np.random.PCG64(S + 200))
    a = g.integers(0, 1 << 40, size=n, dtype=np.uint64) | np.uint64(0xABCD << 48)
    z = synth.u32("zipf", n, S + 201)
    with launch_form(dfr, dfr.DFR_LAUNCH_PERSISTENT):
        k, _, st, stats = sort_with_stats(dfr, a)
        assert st == dfr.DFR_OK and stats["persistent"] == 1 and stats["levels"] >= 2
        assert np.array_equal(k, oracle.sort_u64(a))
        kz, _, st, stats = sort_with_stats(dfr, z)
        assert st == dfr.DFR_OK and stats["persistent"] == 1
        assert np.array_equal(kz, oracle.sort_u32(z))


def test_levels_form_and_automatic_choice(dfr):
    """DFR_LAUNCH_LEVELS forces the level sequence; the automatic choice runs
    calls below DFR_PERSIST_AUTO_KEYS keys persistently, larger ones as the
    level sequence; both give the oracle's result."""
    n = 1_000_003
    a = synth.u32("uniform", n, S + 300)
    with launch_form(dfr, dfr.DFR_LAUNCH_LEVELS, (dfr.DFR_U32,)):
        k, _, st, stats = sort_with_stats(dfr, a)
    assert st == dfr.DFR_OK and stats["persistent"] == 0
    assert np.array_equal(k, oracle.sort_u32(a))
    with launch_form(dfr, dfr.DFR_LAUNCH_AUTO, (dfr.DFR_U32,)):
        k, _, st, stats = sort_with_stats(dfr, a)
        assert st == dfr.DFR_OK and stats["persistent"] == 1
        assert np.array_equal(k, oracle.sort_u32(a))
        big = synth.u32("uniform", dfr.DFR_PERSIST_AUTO_KEYS, S + 301)
        kb, _, st, stats = sort_with_stats(dfr, big)
        assert st == dfr.DFR_OK and stats["persistent"] == 0
        assert np.array_equal(kb, oracle.sort_u32(big))


def test_one_launch_per_call(dfr):
    import torch

    n = 1_000_003
    a = synth.u32("uniform", n, S + 310)
    with launch_form(dfr, dfr.DFR_LAUNCH_PERSISTENT, (dfr.DFR_U32,)):
        gpu_sort(dfr, a)  # warm-up: plans and occupancy are cached
        torch.cuda.synchronize()
        before = dfr.dfr_launch_count()
        k, _, st = gpu_sort(dfr, a)
        after = dfr.dfr_launch_count()
    assert st == dfr.DFR_OK and np.array_equal(k, oracle.sort_u32(a))
    assert after - before == 1


def test_batch_persistent(dfr):
    """A batch of arrays of every size class up to 2^20 in one launch, each
    array against the oracle; keys between segmented slices stay put."""
    import torch

    g = np.random.Generator(np.random.PCG64(S + 400))
    sizes = [int(x) for x in np.exp(g.uniform(np.log(2), np.log(1 << 20), size=300))] + [1, 0, 32, 33, 6144, 6145]
    arrays = [synth.u32("zipf" if i % 3 == 0 else "uniform", n, S + 401 + i) for i, n in enumerate(sizes)]
    keys = [dfr.to_device(a) if a.size else torch.empty(0, dtype=torch.int32, device="cuda") for a in arrays]
    bufs = [torch.empty_like(x) for x in keys]
    segs = [(dfr.DFR_U32, keys[i], 0, bufs[i], 0, n) for i, n in enumerate(sizes)]
    wsb = dfr.dfr_batch_workspace_bytes(segs)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    with launch_form(dfr, dfr.DFR_LAUNCH_PERSISTENT, (dfr.DFR_U32,)):
        assert dfr.dfr_sort_batch(segs, ws, wsb) == dfr.DFR_OK
        assert dfr.dfr_last_device_status(ws) == dfr.DFR_OK
        assert dfr.dfr_get_stats(ws)["persistent"] == 1
    for i, a in enumerate(arrays):
        if a.size:
            assert np.array_equal(dfr.to_numpy(keys[i], np.uint32), oracle.sort_u32(a)), i


def test_key_formats_persistent(dfr):
    """Signed keys and descending IEEE floats: the map to unsigned order and
    back are the first and last phases of the launch."""
    import torch

    n = 300_001
    g = np.random.Generator(np.random.PCG64(S + 500))
    s32 = g.integers(-(1 << 31), 1 << 31, size=n, dtype=np.int64).astype(np.int32)
    f64 = g.standard_normal(n) * 1e6
    with launch_form(dfr, dfr.DFR_LAUNCH_PERSISTENT):
        for kt, arr, fmt, want in (
                (dfr.DFR_U32, s32, dfr.DFR_FMT_SIGNED, np.sort(s32, kind="stable")),
                (dfr.DFR_U64, f64, dfr.DFR_FMT_FLOAT | dfr.DFR_FMT_DESCENDING, np.sort(f64)[::-1])):
            s = dfr.Sorter(kt, n)
            d = dfr.to_device(arr)
            assert dfr.dfr_sort_format(kt, fmt, d, 0, s.kbuf, 0, n, s.ws, s.ws_bytes) == dfr.DFR_OK
            assert s.device_status() == dfr.DFR_OK
            assert s.stats()["persistent"] == 1
            got = dfr.to_numpy(d, np.uint32 if arr.itemsize == 4 else np.uint64).view(arr.dtype)
            assert np.array_equal(got, want)
            torch.cuda.synchronize()


def test_grid_barrier_forced_timeout_reports_and_recovers(dfr):
    """The grid barrier's waits are pointed at a word nothing sets: every CTA
    gives up after the spin limit, records DFR_ERR_TIMEOUT and leaves the
    kernel; the next call on the same context sorts correctly."""
    n = 1_000_003
    a = synth.u32("uniform", n, S + 600)
    with launch_form(dfr, dfr.DFR_LAUNCH_PERSISTENT, (dfr.DFR_U32,)):
        try:
            dfr.dfr_set_debug(2000, True)
            _, _, st = gpu_sort(dfr, a)
        finally:
            dfr.dfr_set_debug(0, False)
        assert st == dfr.DFR_ERR_TIMEOUT
        k, _, st, stats = sort_with_stats(dfr, a)
    assert st == dfr.DFR_OK and stats["persistent"] == 1
    assert np.array_equal(k, oracle.sort_u32(a))


def test_graph_of_persistent_launch(dfr):
    import torch

    n = 1_000_003
    s = dfr.Sorter(dfr.DFR_U32, n)
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    with launch_form(dfr, dfr.DFR_LAUNCH_PERSISTENT, (dfr.DFR_U32,)):
        g = dfr.dfr_graph_create([(dfr.DFR_U32, keys, 0, s.kbuf, 0, n)], s.ws, s.ws_bytes)
    try:
        for r, dist in enumerate(("uniform", "zipf", "sorted")):
            a = synth.u32(dist, n, S + 700 + r)
            keys.copy_(dfr.to_device(a))
            assert dfr.dfr_graph_launch(g) == dfr.DFR_OK
            assert s.device_status() == dfr.DFR_OK
            assert np.array_equal(dfr.to_numpy(keys, np.uint32), oracle.sort_u32(a)), dist
        assert s.stats()["persistent"] == 1
    finally:
        dfr.dfr_graph_destroy(g)
