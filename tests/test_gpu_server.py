"""The served form (dfr_server_create / dfr_submit / dfr_poll / dfr_wait):
every request of a mixed stream must come out exactly as the oracle sorts its
array alone and exactly as a plain call on that array alone, whatever batch
it was coalesced into; requests over the memory budget are refused; requests
that do not fit next to the ones in flight wait and then complete."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_sort, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


def _dtype(dfr, kt):
    return np.uint32 if dfr.KEY_BYTES[kt] == 4 else np.uint64


def _make(dfr, kt, n, seed):
    if _dtype(dfr, kt) == np.uint32:
        a = synth.u32(synth.U32_DISTRIBUTIONS[seed % len(synth.U32_DISTRIBUTIONS)], n, seed)
    else:
        a = synth.u64(synth.U64_DISTRIBUTIONS[seed % len(synth.U64_DISTRIBUTIONS)], n, seed)
    v = synth.index_payload(n) if dfr.HAS_VALS[kt] else None
    return a, v


def _expected(kt, a, v):
    if v is None:
        return (oracle.sort_u32(a) if a.dtype == np.uint32 else oracle.sort_u64(a)), None
    return oracle.sort_u32_kv(a, v) if a.dtype == np.uint32 else oracle.sort_u64_kv(a, v)


class _Req:
    """Device buffers of one request; `own_bufs` gives it its own scratch."""

    def __init__(self, dfr, kt, a, v, own_bufs):
        import torch

        self.kt, self.a, self.v, self.n = kt, a, v, a.size
        kdt = torch.int32 if dfr.KEY_BYTES[kt] == 4 else torch.int64
        self.dk = dfr.to_device(a) if self.n else torch.empty(1, dtype=kdt, device="cuda")
        self.dv = None
        if v is not None:
            self.dv = dfr.to_device(v) if self.n else torch.empty(1, dtype=torch.int32, device="cuda")
        self.kb = torch.empty(max(1, self.n), dtype=kdt, device="cuda") if own_bufs else None
        self.vb = torch.empty(max(1, self.n), dtype=torch.int32, device="cuda") if (own_bufs and v is not None) else None

    def seg(self):
        return (self.kt, self.dk, self.dv if self.dv is not None else 0, self.kb if self.kb is not None else 0,
                self.vb if self.vb is not None else 0, self.n)

    def result(self, dfr):
        dt = _dtype(dfr, self.kt)
        k = dfr.to_numpy(self.dk, dt)[: self.n]
        v = None if self.dv is None else dfr.to_numpy(self.dv, np.uint32)[: self.n]
        return k, v


def test_served_mixed_stream_matches_oracle_and_plain(dfr):
    import torch

    g = np.random.Generator(np.random.PCG64(2207))
    kinds = [dfr.DFR_U32, dfr.DFR_U64_KV, dfr.DFR_U32_KV, dfr.DFR_U64]
    sizes = [0, 1, 2, 32, 33, 4097, 8193] + [int(2 ** g.uniform(4, 18)) for _ in range(153)]
    reqs = []
    for i, n in enumerate(sizes):
        kt = kinds[int(g.integers(0, 4))] if i >= 7 else kinds[i % 4]
        a, v = _make(dfr, kt, n, synth.BASE_SEED + 500 + i)
        reqs.append(_Req(dfr, kt, a, v, own_bufs=(i % 3 == 0)))
    torch.cuda.synchronize()
    srv = dfr.dfr_server_create(torch.cuda.current_device(), 256 << 20, 3)
    try:
        tickets = []
        for r in reqs:
            rc, t = dfr.dfr_submit(srv, r.seg())
            assert rc == dfr.DFR_OK, dfr.dfr_status_string(rc)
            tickets.append(t)
        lats = []
        for i, t in enumerate(tickets):
            if i % 2:
                rc, lat = dfr.dfr_wait(srv, t)
            else:
                while True:
                    rc, done, lat = dfr.dfr_poll(srv, t)
                    if done or rc != dfr.DFR_OK:
                        break
            assert rc == dfr.DFR_OK, dfr.dfr_status_string(rc)
            lats.append(lat)
        stats = dfr.dfr_server_stats(srv)
    finally:
        assert dfr.dfr_server_destroy(srv) == dfr.DFR_OK
    assert all(x >= 0.0 for x in lats)
    assert 1 <= stats["batches"] < len(reqs)  # requests were coalesced
    assert stats["pending"] == 0 and stats["inflight"] == 0
    for i, r in enumerate(reqs):
        k, v = r.result(dfr)
        ek, ev = _expected(r.kt, r.a, r.v)
        assert np.array_equal(k, ek), (i, r.kt, r.n)
        if ev is not None:
            assert np.array_equal(v, ev), (i, r.kt, r.n)
        if i % 10 == 0 and r.n > 1:  # the same array sorted alone by a plain call
            ak, av, st = gpu_sort(dfr, r.a, r.v, key_type=r.kt)
            assert st == dfr.DFR_OK and np.array_equal(k, ak)
            if av is not None:
                assert np.array_equal(v, av)


def test_served_tight_budget_queues_then_completes(dfr):
    """A budget that holds one large request at a time: the others wait for
    memory (admission in arrival order) and still all complete correctly."""
    import torch

    n = 1 << 20
    need = dfr.dfr_workspace_bytes(dfr.DFR_U32, n) + 4 * n + 4096
    reqs = [_Req(dfr, dfr.DFR_U32, *_make(dfr, dfr.DFR_U32, n - 17 * i, synth.BASE_SEED + 700 + i), own_bufs=False)
            for i in range(5)]
    torch.cuda.synchronize()
    srv = dfr.dfr_server_create(torch.cuda.current_device(), int(need * 1.5), 2)
    try:
        tickets = []
        for r in reqs:
            rc, t = dfr.dfr_submit(srv, r.seg())
            assert rc == dfr.DFR_OK
            tickets.append(t)
        for t in tickets:
            rc, _ = dfr.dfr_wait(srv, t)
            assert rc == dfr.DFR_OK
        stats = dfr.dfr_server_stats(srv)
    finally:
        dfr.dfr_server_destroy(srv)
    assert stats["batches"] == len(reqs)
    for r in reqs:
        k, _ = r.result(dfr)
        assert np.array_equal(k, oracle.sort_u32(r.a))


def test_served_over_budget_and_bad_requests(dfr):
    import torch

    srv = dfr.dfr_server_create(torch.cuda.current_device(), 1 << 20, 1)
    try:
        big = _Req(dfr, dfr.DFR_U32, *_make(dfr, dfr.DFR_U32, 1 << 20, 3), own_bufs=False)
        small = _Req(dfr, dfr.DFR_U64_KV, *_make(dfr, dfr.DFR_U64_KV, 3000, 4), own_bufs=False)
        torch.cuda.synchronize()
        rc, _ = dfr.dfr_submit(srv, big.seg())
        assert rc == dfr.DFR_ERR_OVER_BUDGET
        rc, _ = dfr.dfr_submit(srv, (7, big.dk, 0, 0, 0, 10))
        assert rc == dfr.DFR_ERR_INVALID_ARG
        rc, _ = dfr.dfr_submit(srv, (dfr.DFR_U64_KV, small.dk, 0, 0, 0, 3000))  # kv without payloads
        assert rc == dfr.DFR_ERR_INVALID_ARG
        rc, t = dfr.dfr_submit(srv, small.seg())
        assert rc == dfr.DFR_OK
        rc, lat = dfr.dfr_wait(srv, t)
        assert rc == dfr.DFR_OK and lat > 0.0
        assert dfr.dfr_poll(srv, t)[0] == dfr.DFR_ERR_INVALID_ARG  # ticket released
    finally:
        dfr.dfr_server_destroy(srv)
    k, v = small.result(dfr)
    ek, ev = oracle.sort_u64_kv(small.a, small.v)
    assert np.array_equal(k, ek) and np.array_equal(v, ev)


def test_served_destroy_finishes_pending(dfr):
    import torch

    reqs = [_Req(dfr, dfr.DFR_U32, *_make(dfr, dfr.DFR_U32, 50_000 + i, synth.BASE_SEED + 800 + i), own_bufs=False)
            for i in range(20)]
    torch.cuda.synchronize()
    srv = dfr.dfr_server_create(torch.cuda.current_device(), 64 << 20, 2)
    for r in reqs:
        assert dfr.dfr_submit(srv, r.seg())[0] == dfr.DFR_OK
    assert dfr.dfr_server_destroy(srv) == dfr.DFR_OK
    for r in reqs:
        k, _ = r.result(dfr)
        assert np.array_equal(k, oracle.sort_u32(r.a))


def test_fill_splitmix64_matches_host_generator(dfr):
    import torch

    for n in (1, 33, 100_003):
        k = torch.empty(n, dtype=torch.int32, device="cuda")
        assert dfr.dfr_fill_splitmix64(dfr.DFR_U32, k, None, n, 0xABCDEF) == dfr.DFR_OK
        assert np.array_equal(dfr.to_numpy(k, np.uint32), synth.splitmix64_u32(0xABCDEF, n))
        k64 = torch.empty(n, dtype=torch.int64, device="cuda")
        v = torch.empty(n, dtype=torch.int32, device="cuda")
        assert dfr.dfr_fill_splitmix64(dfr.DFR_U64_KV, k64, v, n, 99) == dfr.DFR_OK
        assert np.array_equal(dfr.to_numpy(k64, np.uint64), synth.splitmix64(99, n))
        assert np.array_equal(dfr.to_numpy(v, np.uint32), synth.index_payload(n))


def _device_stream(dfr, count, seed, lo, hi, max_batch=None, n_streams=3, inflight=1):
    """Generate each request's keys on a producer stream at submission and
    hand the server an event to wait on; returns the request list."""
    import torch

    sizes, kvs = synth.served_stream(count, seed, lo, hi)
    gen = torch.cuda.Stream()
    srv = dfr.dfr_server_create(torch.cuda.current_device(), 512 << 20, n_streams)
    if max_batch is not None:
        assert dfr.dfr_server_set_limits(srv, max_batch, inflight) == dfr.DFR_OK
    bufs = [(torch.empty(int(n), dtype=torch.int64 if kv else torch.int32, device="cuda"),
             torch.empty(int(n), dtype=torch.int32, device="cuda") if kv else None) for n, kv in zip(sizes, kvs)]
    torch.cuda.synchronize()
    reqs = []
    try:
        for r in range(count):
            n = int(sizes[r])
            kt = dfr.DFR_U64_KV if kvs[r] else dfr.DFR_U32
            keys, vals = bufs[r]
            s = synth.request_seed(seed, r)
            assert dfr.dfr_fill_splitmix64(kt, keys, vals, n, s, stream=gen) == dfr.DFR_OK
            ev = torch.cuda.Event()
            ev.record(gen)
            rc, t = dfr.dfr_submit_after(srv, (kt, keys, vals if vals is not None else 0, 0, 0, n), ev)
            assert rc == dfr.DFR_OK
            reqs.append((t, kt, n, s, keys, vals, ev))
        for t, *_ in reqs:
            rc, lat = dfr.dfr_wait(srv, t)
            assert rc == dfr.DFR_OK and lat > 0.0
        stats = dfr.dfr_server_stats(srv)
    finally:
        dfr.dfr_server_destroy(srv)
    return reqs, stats


def _check_stream(dfr, reqs):
    for t, kt, n, s, keys, vals, _ in reqs:
        if kt == dfr.DFR_U32:
            a = synth.splitmix64_u32(s, n)
            assert np.array_equal(dfr.to_numpy(keys, np.uint32), oracle.sort_u32(a)), (t, n)
        else:
            a = synth.splitmix64(s, n)
            ek, ev = oracle.sort_u64_kv(a, synth.index_payload(n))
            assert np.array_equal(dfr.to_numpy(keys, np.uint64), ek), (t, n)
            assert np.array_equal(dfr.to_numpy(vals, np.uint32), ev), (t, n)


def test_served_device_generated_stream(dfr):
    """1,000 requests whose keys are generated on the device as they arrive
    (70% u32, 30% u64 kv): each result equals the oracle's sort of the same
    keys regenerated on the host."""
    reqs, stats = _device_stream(dfr, 1000, 51, 1 << 4, 1 << 17)
    assert stats["batches"] < len(reqs)
    _check_stream(dfr, reqs)


@pytest.mark.parametrize("inflight", [1, 16])
def test_served_fifo_plain_mode(dfr, inflight):
    """max_batch = 1 on one stream: every request is served alone by the plain
    launch sequence, in arrival order, with the same results (also with many
    plain launches in flight on the stream at once)."""
    reqs, stats = _device_stream(dfr, 120, 52, 1 << 6, 1 << 18, max_batch=1, n_streams=1, inflight=inflight)
    assert stats["batches"] == len(reqs)
    _check_stream(dfr, reqs)


@pytest.mark.parametrize("sched", [1, 2])
def test_served_single_large_request_lsd_schedule(dfr, sched):
    """A request served alone (a batch of one array) takes the plan's schedule
    of the top digits: with the LSD schedules forced, large u64 key-value and
    u32 requests still come out as the oracle sorts them."""
    import torch

    try:
        for kt in (dfr.DFR_U64_KV, dfr.DFR_U32):
            for c in range(dfr.DFR_TUNE_CLASSES):
                t = dfr.dfr_tune_get(kt, c)
                t["schedule"] = sched
                assert dfr.dfr_tune_set(kt, c, t) == dfr.DFR_OK
        reqs = [_Req(dfr, dfr.DFR_U64_KV, *_make(dfr, dfr.DFR_U64_KV, (1 << 21) + 5, synth.BASE_SEED + 810), False),
                _Req(dfr, dfr.DFR_U32, *_make(dfr, dfr.DFR_U32, (1 << 21) + 77, synth.BASE_SEED + 811), True)]
        torch.cuda.synchronize()
        srv = dfr.dfr_server_create(torch.cuda.current_device(), 512 << 20, 1)
        try:
            for r in reqs:  # one at a time: each runs as a batch of one
                rc, t = dfr.dfr_submit(srv, r.seg())
                assert rc == dfr.DFR_OK
                rc, _ = dfr.dfr_wait(srv, t)
                assert rc == dfr.DFR_OK
        finally:
            assert dfr.dfr_server_destroy(srv) == dfr.DFR_OK
    finally:
        assert dfr.dfr_tune_reset() == dfr.DFR_OK
    for r in reqs:
        k, v = r.result(dfr)
        ek, ev = _expected(r.kt, r.a, r.v)
        assert np.array_equal(k, ek)
        if ev is not None:
            assert np.array_equal(v, ev)
