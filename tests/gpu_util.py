"""Helpers shared by the GPU tests: run the CUDA path through the C ABI on
numpy inputs and hand back numpy outputs."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2207_14334_gb300 as dfr

    dfr.load()
    return dfr


_sorters = {}


def sorter(dfr, key_type, n):
    cap = max(2, n)
    s = _sorters.get(key_type)
    if s is None or s.capacity < cap:
        s = dfr.Sorter(key_type, max(cap, 1 << 16))
        _sorters[key_type] = s
    return s


def gpu_sort(dfr, keys, vals=None, key_type=None):
    """Sort numpy keys (and payloads) on the GPU; returns numpy results and the
    device status of the call."""
    if key_type is None:
        wide_vals = vals is not None and vals.dtype.itemsize == 8
        if keys.dtype == np.uint32:
            key_type = dfr.DFR_U32 if vals is None else (dfr.DFR_U32_KV64 if wide_vals else dfr.DFR_U32_KV)
        else:
            key_type = dfr.DFR_U64 if vals is None else (dfr.DFR_U64_KV64 if wide_vals else dfr.DFR_U64_KV)
    n = keys.size
    s = sorter(dfr, key_type, n)
    dk = dfr.to_device(keys) if n else None
    dv = dfr.to_device(vals) if (vals is not None and n) else None
    if n <= 1:  # nothing is launched for n <= 1
        rc = s.sort_(dk, dv, n) if n else dfr.DFR_OK
        return keys.copy(), (None if vals is None else vals.copy()), rc
    s.sort_(dk, dv)
    status = s.device_status()
    k = dfr.to_numpy(dk, keys.dtype)
    v = None if vals is None else dfr.to_numpy(dv, np.uint64 if vals.dtype.itemsize == 8 else np.uint32)
    return k, v, status
