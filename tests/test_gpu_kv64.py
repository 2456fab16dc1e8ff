"""64-bit payloads (DFR_U64_KV64, DFR_U32_KV64) through the C ABI: every
result equals the oracle's stable key-value sort (keys, and payloads whose
high and low halves both vary, so a payload cut to 32 bits or assembled from
two records fails), on every path the narrower payloads take -- the MSD
levels with their CTA and warp sorts, the LSD schedules of large single
arrays, the batch entry, the server, a CUDA graph and the key formats."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_sort, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


def payload(n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return g.bit_generator.random_raw(n).astype(np.uint64)


def expected(keys, vals):
    return oracle.sort_u64_kv64(keys, vals) if keys.dtype == np.uint64 else oracle.sort_u32_kv64(keys, vals)


def keys_of(width, dist, n, seed):
    if width == 8:
        return synth.u64(dist, n, seed)
    return synth.u32(dist, n, seed)


@pytest.mark.parametrize("width,dist", [(8, "uniform64"), (8, "uniform16"), (8, "dup90"), (4, "uniform"),
                                        (4, "zipf"), (4, "equal"), (4, "normal")])
@pytest.mark.parametrize("n", [2, 33, 513, 4097, 70_001, 1_000_003])
def test_kv64_matches_oracle(dfr, width, dist, n):
    seed = synth.BASE_SEED + 900 + n % 97
    k = keys_of(width, dist, n, seed)
    v = payload(n, seed + 1)
    gk, gv, st = gpu_sort(dfr, k, v)
    assert st == dfr.DFR_OK
    wk, wv = expected(k, v)
    assert np.array_equal(gk, wk)
    assert np.array_equal(gv, wv)


@pytest.mark.parametrize("kt_name", ["DFR_U64_KV64", "DFR_U32_KV64"])
@pytest.mark.parametrize("sched", [1, 2])
def test_kv64_lsd_schedules(dfr, kt_name, sched):
    """Single arrays large enough for the LSD top phase, with the counted and
    the estimated first deal forced through the plan table."""
    kt = getattr(dfr, kt_name)
    n = dfr.dfr_lsd_min_keys(kt) + 12_345
    width = 8 if kt == dfr.DFR_U64_KV64 else 4
    k = keys_of(width, "uniform64" if width == 8 else "uniform", n, synth.BASE_SEED + 950 + sched)
    v = payload(n, synth.BASE_SEED + 951)
    c = dfr.dfr_tune_class(n)
    t = dfr.dfr_tune_get(kt, c)
    t["schedule"] = sched
    assert dfr.dfr_tune_set(kt, c, t) == dfr.DFR_OK
    try:
        s = dfr.Sorter(kt, n)
        dk, dv = dfr.to_device(k), dfr.to_device(v)
        s.sort_(dk, dv)
        assert s.device_status() == dfr.DFR_OK
        assert s.stats()["schedule"] == sched
        gk = dfr.to_numpy(dk, k.dtype)
        gv = dfr.to_numpy(dv, np.uint64)
    finally:
        assert dfr.dfr_tune_reset() == dfr.DFR_OK
    wk, wv = expected(k, v)
    assert np.array_equal(gk, wk) and np.array_equal(gv, wv)


def test_kv64_batch_graph_and_formats(dfr):
    import torch

    sizes = [1, 2, 31, 600, 5000, 90_000, 300_001]
    for kt, width in ((dfr.DFR_U64_KV64, 8), (dfr.DFR_U32_KV64, 4)):
        ks = [keys_of(width, "uniform64" if width == 8 else "zipf", n, synth.BASE_SEED + 960 + i)
              for i, n in enumerate(sizes)]
        vs = [payload(n, synth.BASE_SEED + 970 + i) for i, n in enumerate(sizes)]
        dk = [dfr.to_device(a) for a in ks]
        dv = [dfr.to_device(a) for a in vs]
        kdt = torch.int64 if width == 8 else torch.int32
        kb = [torch.empty(max(1, n), dtype=kdt, device="cuda") for n in sizes]
        vb = [torch.empty(max(1, n), dtype=torch.int64, device="cuda") for n in sizes]
        segs = [(kt, dk[i], dv[i], kb[i], vb[i], n) for i, n in enumerate(sizes)]
        wsb = dfr.dfr_batch_workspace_bytes(segs)
        ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
        assert dfr.dfr_sort_batch(segs, ws, wsb) == dfr.DFR_OK
        assert dfr.dfr_last_device_status(ws) == dfr.DFR_OK
        for i in range(len(sizes)):
            wk, wv = expected(ks[i], vs[i])
            assert np.array_equal(dfr.to_numpy(dk[i], ks[i].dtype), wk), (kt, sizes[i])
            assert np.array_equal(dfr.to_numpy(dv[i], np.uint64), wv), (kt, sizes[i])
        # the same buffers as a CUDA graph, relaunched on refilled inputs
        g = dfr.dfr_graph_create(segs, ws, wsb)
        try:
            for rep in range(2):
                for i in range(len(sizes)):
                    dk[i].copy_(dfr.to_device(ks[i]))
                    dv[i].copy_(dfr.to_device(vs[i]))
                assert dfr.dfr_graph_launch(g) == dfr.DFR_OK
                torch.cuda.synchronize()
                for i in range(len(sizes)):
                    wk, wv = expected(ks[i], vs[i])
                    assert np.array_equal(dfr.to_numpy(dv[i], np.uint64), wv), (kt, sizes[i], rep)
        finally:
            dfr.dfr_graph_destroy(g)
    # signed descending keys with 64-bit payloads (stable on ties)
    for kt, dt in ((dfr.DFR_U64_KV64, np.int64), (dfr.DFR_U32_KV64, np.int32)):
        g = np.random.Generator(np.random.PCG64(5))
        a = g.integers(-50, 50, 100_003).astype(dt)
        v = payload(a.size, 77)
        s = dfr.Sorter(kt, a.size)
        da, dv = dfr.to_device(a), dfr.to_device(v)
        s.sort_(da, dv, key_format=dfr.DFR_FMT_SIGNED | dfr.DFR_FMT_DESCENDING)
        assert s.device_status() == dfr.DFR_OK
        wk, wv = oracle.sort_format(int(kt), 0x101, a, v)
        assert np.array_equal(dfr.to_numpy(da, a.dtype), wk) and np.array_equal(dfr.to_numpy(dv, np.uint64), wv)


def test_kv64_served(dfr):
    """Requests of both 64-bit-payload types, some with their own scratch,
    mixed with u32 requests, through the server."""
    import torch

    reqs = []
    g = np.random.Generator(np.random.PCG64(2222))
    for i in range(60):
        kt = [dfr.DFR_U64_KV64, dfr.DFR_U32_KV64, dfr.DFR_U32][i % 3]
        n = int(2 ** g.uniform(4, 17))
        width = dfr.KEY_BYTES[kt]
        k = keys_of(width, "uniform64" if width == 8 else "uniform", n, synth.BASE_SEED + 1000 + i)
        v = payload(n, synth.BASE_SEED + 1100 + i) if dfr.HAS_VALS[kt] else None
        dk = dfr.to_device(k)
        dv = dfr.to_device(v) if v is not None else None
        own = i % 2 == 0
        kb = torch.empty_like(dk) if own else None
        vb = torch.empty_like(dv) if (own and dv is not None) else None
        reqs.append((kt, k, v, dk, dv, kb, vb))
    torch.cuda.synchronize()
    srv = dfr.dfr_server_create(torch.cuda.current_device(), 256 << 20, 3)
    try:
        tickets = []
        for kt, k, v, dk, dv, kb, vb in reqs:
            rc, t = dfr.dfr_submit(srv, (kt, dk, dv if dv is not None else 0, kb if kb is not None else 0,
                                         vb if vb is not None else 0, k.size))
            assert rc == dfr.DFR_OK
            tickets.append(t)
        for t in tickets:
            rc, _ = dfr.dfr_wait(srv, t)
            assert rc == dfr.DFR_OK
    finally:
        assert dfr.dfr_server_destroy(srv) == dfr.DFR_OK
    for kt, k, v, dk, dv, kb, vb in reqs:
        if v is None:
            assert np.array_equal(dfr.to_numpy(dk, np.uint32), oracle.sort_u32(k))
        else:
            wk, wv = expected(k, v)
            assert np.array_equal(dfr.to_numpy(dk, k.dtype), wk) and np.array_equal(dfr.to_numpy(dv, np.uint64), wv)


def test_fill_splitmix64_kv64(dfr):
    import torch

    n = 10_007
    for kt, kdt in ((dfr.DFR_U64_KV64, torch.int64), (dfr.DFR_U32_KV64, torch.int32)):
        k = torch.empty(n, dtype=kdt, device="cuda")
        v = torch.empty(n, dtype=torch.int64, device="cuda")
        assert dfr.dfr_fill_splitmix64(kt, k, v, n, 12345) == dfr.DFR_OK
        torch.cuda.synchronize()
        want = synth.splitmix64(12345, n)
        if kdt == torch.int32:
            want = (want >> np.uint64(32)).astype(np.uint32)
        assert np.array_equal(dfr.to_numpy(k, want.dtype), want)
        assert np.array_equal(dfr.to_numpy(v, np.uint64), np.arange(n, dtype=np.uint64))
