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
