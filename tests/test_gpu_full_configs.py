"""Parity with the oracle at the full sizes of the benchmark workloads, on the
same seeded inputs and in the same launch configuration `bench.py` times.

* 2^28 u32 keys, each of the seven distributions (uniform, normal,
  exponential, Zipf, all-equal, sorted, reverse), through dfr_sort_u32 with
  the built-in launch plan of that size class;
* 2^27 u64 keys with u32 payloads (payload = original index), each of the
  three distributions, through dfr_sort_u64_kv with the built-in plan (which
  picks the diverting-LSD schedule of the top digits where it applies);
* the 4096-array batch (log-uniform sizes over [2^8, 2^20], uniform or Zipf
  per array) through one dfr_sort_batch call, every array checked;
* 2,000 requests of the served stream (sizes log-uniform over [2^10, 2^24],
  70% u32 keys, 30% u64 keys with payloads, keys generated on the device at
  submission) through the server under a 16 GB budget, every request checked.

Every comparison is element by element (keys and payloads) against the CPU
oracle on the same input; the oracle runs in worker threads (its C calls
release the interpreter lock) while the GPU works.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

S = synth.BASE_SEED
N_U32 = 1 << 28
N_KV = 1 << 27


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


@pytest.fixture(scope="module")
def pool():
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        yield ex


def _planned_schedule(dfr, kt, n):
    """The schedule the built-in plan runs for one array of n keys."""
    sched = dfr.dfr_tune_get(kt, dfr.dfr_tune_class(n))["schedule"]
    return sched if n >= dfr.dfr_lsd_min_keys(kt) else dfr.DFR_SCHED_MSD


@pytest.fixture(scope="module")
def u32_inputs():
    """The 2^28 u32 arrays of the default benchmark step (its seeds; reverse =
    the sorted array reversed, as there), generated on first use."""
    cache = {}

    def get(dist):
        if dist not in cache:
            i = synth.U32_DISTRIBUTIONS.index(dist)
            if dist == "reverse":
                cache[dist] = get("sorted")[::-1].copy()
            else:
                cache[dist] = synth.u32(dist, N_U32, S + 20 + i)
            for d in list(cache):  # keep at most the array and the one it derives from
                if d not in (dist, "sorted"):
                    del cache[d]
        return cache[dist]

    return get


@pytest.mark.parametrize("dist", synth.U32_DISTRIBUTIONS)
def test_plain_u32_2p28_matches_oracle(dfr, pool, u32_inputs, dist):
    import torch

    a = u32_inputs(dist)
    want = pool.submit(oracle.sort_u32, a)
    s = dfr.Sorter(dfr.DFR_U32, N_U32)
    d = dfr.to_device(a)
    s.sort_(d)
    assert s.device_status() == dfr.DFR_OK
    st = s.stats()
    assert st["schedule"] == _planned_schedule(dfr, dfr.DFR_U32, N_U32)
    got = dfr.to_numpy(d, np.uint32)
    del d, s
    torch.cuda.empty_cache()
    w = want.result()
    bad = np.flatnonzero(got != w)
    assert bad.size == 0, "%s: %d keys differ, first at %d" % (dist, bad.size, bad[0] if bad.size else -1)


@pytest.mark.parametrize("dist", synth.U64_DISTRIBUTIONS)
def test_kv_u64_2p27_matches_oracle(dfr, pool, dist):
    import torch

    i = synth.U64_DISTRIBUTIONS.index(dist)
    a = synth.u64(dist, N_KV, S + 30 + i)
    v = synth.index_payload(N_KV)
    want = pool.submit(oracle.sort_u64_kv, a, v)
    s = dfr.Sorter(dfr.DFR_U64_KV, N_KV)
    dk, dv = dfr.to_device(a), dfr.to_device(v)
    s.sort_(dk, dv)
    assert s.device_status() == dfr.DFR_OK
    st = s.stats()
    planned = _planned_schedule(dfr, dfr.DFR_U64_KV, N_KV)
    # an array whose top byte is constant has nothing for the LSD phase to deal
    assert st["schedule"] == (planned if dist != "uniform16" else dfr.DFR_SCHED_MSD)
    gk, gv = dfr.to_numpy(dk, np.uint64), dfr.to_numpy(dv, np.uint32)
    del dk, dv, s
    torch.cuda.empty_cache()
    wk, wv = want.result()
    assert np.array_equal(gk, wk), "%s: keys differ" % dist
    assert np.array_equal(gv, wv), "%s: payloads differ (pairing or stability)" % dist


def test_batch_4096_arrays_matches_oracle(dfr, pool):
    """The batched workload: every one of the 4096 arrays against the oracle."""
    import torch

    arrays, kinds = synth.batch_u32(4096, S + 40, 1 << 8, 1 << 20)
    want = [pool.submit(oracle.sort_u32, a) for a in arrays]
    offs, pos = [], 0
    for a in arrays:
        offs.append(pos)
        pos += (a.size + 63) // 64 * 64
    host = np.zeros(pos, dtype=np.uint32)
    for o, a in zip(offs, arrays):
        host[o:o + a.size] = a
    work = dfr.to_device(host)
    kbuf = torch.empty_like(work)
    base, bbase = work.data_ptr(), kbuf.data_ptr()
    segs = [(dfr.DFR_U32, base + 4 * o, 0, bbase + 4 * o, 0, a.size) for o, a in zip(offs, arrays)]
    wsb = dfr.dfr_batch_workspace_bytes(segs)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    assert dfr.dfr_sort_batch(segs, ws, wsb) == dfr.DFR_OK
    assert dfr.dfr_last_device_status(ws) == dfr.DFR_OK
    got = dfr.to_numpy(work, np.uint32)
    del work, kbuf, ws
    torch.cuda.empty_cache()
    bad = [i for i, (o, a, w) in enumerate(zip(offs, arrays, want)) if not np.array_equal(got[o:o + a.size],
                                                                                           w.result())]
    assert not bad, "%d of %d arrays differ from the oracle (first: %d, %s)" % (len(bad), len(arrays), bad[0],
                                                                               kinds[bad[0]])


def _served_expected(kv, seed, n):
    """The oracle's result for one request, its keys regenerated on the host."""
    if kv:
        return oracle.sort_u64_kv(synth.splitmix64(seed, n), synth.index_payload(n))
    return oracle.sort_u32(synth.splitmix64_u32(seed, n)), None


def test_served_stream_2000_requests_matches_oracle(dfr, pool):
    """The first 2,000 requests of the served benchmark stream (its seed and
    size law), submitted as fast as buffers allow with at most 256 in flight;
    each request's keys are written on the device right before it is
    submitted, and every result is compared with the oracle."""
    import collections

    import torch

    R = 2000
    seed = S + 50
    sizes, kvs = synth.served_stream(R, seed, 1 << 10, 1 << 24)
    gen = torch.cuda.Stream()
    srv = dfr.dfr_server_create(torch.cuda.current_device(), 16 << 30, 4)
    inflight = collections.deque()
    checks = []

    def retire_one():
        r, t, keys, vals, ev = inflight.popleft()
        rc, lat = dfr.dfr_wait(srv, t)
        assert rc == dfr.DFR_OK, "request %d: %s" % (r, dfr.dfr_status_string(rc))
        gk = dfr.to_numpy(keys, np.uint64 if kvs[r] else np.uint32)
        gv = dfr.to_numpy(vals, np.uint32) if kvs[r] else None
        checks.append((r, gk, gv, pool.submit(_served_expected, bool(kvs[r]), synth.request_seed(seed, r),
                                               int(sizes[r]))))

    def settle(limit):
        while len(checks) > limit:
            r, gk, gv, fut = checks.pop(0)
            wk, wv = fut.result()
            assert np.array_equal(gk, wk), "request %d (n=%d): keys differ" % (r, sizes[r])
            if wv is not None:
                assert np.array_equal(gv, wv), "request %d (n=%d): payloads differ" % (r, sizes[r])

    try:
        for r in range(R):
            n = int(sizes[r])
            kv = bool(kvs[r])
            kt = dfr.DFR_U64_KV if kv else dfr.DFR_U32
            keys = torch.empty(n, dtype=torch.int64 if kv else torch.int32, device="cuda")
            vals = torch.empty(n, dtype=torch.int32, device="cuda") if kv else None
            assert dfr.dfr_fill_splitmix64(kt, keys, vals, n, synth.request_seed(seed, r), stream=gen) == dfr.DFR_OK
            ev = torch.cuda.Event()
            ev.record(gen)
            rc, t = dfr.dfr_submit_after(srv, (kt, keys, vals if kv else 0, 0, 0, n), ev)
            assert rc == dfr.DFR_OK
            inflight.append((r, t, keys, vals, ev))
            if len(inflight) >= 256:
                retire_one()
                settle(64)
        while inflight:
            retire_one()
            settle(64)
        stats = dfr.dfr_server_stats(srv)
    finally:
        assert dfr.dfr_server_destroy(srv) == dfr.DFR_OK
    settle(0)
    assert stats["batches"] < R  # requests were coalesced
