"""Signed, IEEE-float (total order) and descending keys through the C ABI:
every key type and format against the oracle's format sort, including the
special floating-point values and stability of payloads on ties."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

FMTS = [("signed", 1), ("float", 2), ("unsigned_desc", 0x100), ("signed_desc", 0x101), ("float_desc", 0x102)]


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


def _keys(width, fmt, n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    it = np.uint32 if width == 4 else np.uint64
    if (fmt & 0xFF) == 2:
        ft = np.float32 if width == 4 else np.float64
        f = (g.standard_normal(n) * 10.0 ** g.integers(-30, 30, n)).astype(ft)
        a = f.view(it).copy()
        specials = np.array([np.inf, -np.inf, np.nan, -np.nan, 0.0, -0.0, np.finfo(ft).tiny / 8,
                             -np.finfo(ft).tiny / 8], dtype=ft).view(it)
        a[:min(n, specials.size)] = specials[:min(n, specials.size)]
        a[g.integers(0, n, n // 50)] = specials[g.integers(0, specials.size, n // 50)]  # repeated specials
        return a
    raw = g.integers(0, 1 << 32, n, dtype=np.uint64)
    if width == 8:
        raw = (raw << np.uint64(32)) | g.integers(0, 1 << 32, n, dtype=np.uint64)
    a = raw.astype(it)
    a[g.integers(0, n, n // 10)] = a[0]  # ties
    return a


def _sort(dfr, kt, fmt, a, v=None):
    import torch

    n = a.size
    s = dfr.Sorter(kt, max(2, n))
    dk = dfr.to_device(a)
    dv = dfr.to_device(v) if v is not None else None
    s.sort_(dk, dv, n, key_format=fmt)
    assert s.device_status() == dfr.DFR_OK
    torch.cuda.synchronize()
    k = dfr.to_numpy(dk, a.dtype)
    return k, (dfr.to_numpy(dv, np.uint32) if v is not None else None)


@pytest.mark.parametrize("name,fmt", FMTS)
@pytest.mark.parametrize("n", [7, 4097, 100_003, 1_000_001])
def test_keys_only(dfr, name, fmt, n):
    for kt, width in ((dfr.DFR_U32, 4), (dfr.DFR_U64, 8)):
        a = _keys(width, fmt, n, 1000 + n + fmt)
        k, _ = _sort(dfr, kt, fmt, a)
        assert np.array_equal(k, oracle.sort_format(kt, fmt, a)), (name, n, width)


@pytest.mark.parametrize("name,fmt", FMTS)
@pytest.mark.parametrize("n", [33, 70_001])
def test_key_value_stable(dfr, name, fmt, n):
    for kt, width in ((dfr.DFR_U32_KV, 4), (dfr.DFR_U64_KV, 8)):
        a = _keys(width, fmt, n, 2000 + n + fmt)
        v = synth.index_payload(n)
        k, vv = _sort(dfr, kt, fmt, a, v)
        ok, ov = oracle.sort_format(kt, fmt, a, v)
        assert np.array_equal(k, ok) and np.array_equal(vv, ov), (name, n, width)


def test_batch_formats(dfr):
    import torch

    sizes = [3, 5000, 300_000]
    arrays = [_keys(4, 2, n, 3000 + n) for n in sizes]
    dk = [dfr.to_device(a) for a in arrays]
    kb = [torch.empty(max(1, n), dtype=torch.int32, device="cuda") for n in sizes]
    segs = [(dfr.DFR_U32, dk[i], 0, kb[i], 0, n) for i, n in enumerate(sizes)]
    wsb = dfr.dfr_batch_workspace_bytes(segs)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    assert dfr.dfr_sort_batch_format(segs, dfr.DFR_FMT_FLOAT | dfr.DFR_FMT_DESCENDING, ws, wsb) == dfr.DFR_OK
    assert dfr.dfr_last_device_status(ws) == dfr.DFR_OK
    for a, d in zip(arrays, dk):
        assert np.array_equal(dfr.to_numpy(d, np.uint32), oracle.sort_format(0, 0x102, a))


def test_plain_format_call_ignores_a_stale_descriptor_table(dfr):
    """The key-format pre-pass of a plain call runs before the call's first
    kernel writes the array descriptor into the workspace, so it must take the
    descriptor from its launch parameters.  Here the workspace still holds the
    descriptor of a decoy array, left by a one-array batch call (same table
    slot), and the decoy stays allocated: reading the stale table would map
    the decoy's keys instead of the real ones (a wrong result and a changed
    decoy, no stray access).  Both must come out right."""
    import torch

    decoy = _keys(4, 0, 300_000, 4001)
    real = _keys(4, 1, 100_003, 4002)
    dd = dfr.to_device(decoy)
    db = torch.empty_like(dd)
    s = dfr.Sorter(dfr.DFR_U32, 300_000)
    segs = [(dfr.DFR_U32, dd, 0, db, 0, decoy.size)]
    assert dfr.dfr_sort_batch(segs, s.ws, s.ws_bytes) == dfr.DFR_OK
    assert dfr.dfr_last_device_status(s.ws) == dfr.DFR_OK
    sorted_decoy = dfr.to_numpy(dd, np.uint32)
    assert np.array_equal(sorted_decoy, oracle.sort_u32(decoy))
    dr = dfr.to_device(real)
    s.sort_(dr, None, real.size, key_format=dfr.DFR_FMT_SIGNED)
    assert s.device_status() == dfr.DFR_OK
    assert np.array_equal(dfr.to_numpy(dr, np.uint32), oracle.sort_format(0, 1, real))
    assert np.array_equal(dfr.to_numpy(dd, np.uint32), sorted_decoy)
