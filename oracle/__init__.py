"""CPU oracle for the DFR sort path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  It shares no code with the CUDA path,
and the CUDA path never falls back to it.

The arithmetic lives in ``oracle.c``: a plain least-significant-digit radix
sort made of counting sorts (8-bit digits, every pass run, stable), following
the paper's Preliminaries (count / convert counts to indices / deal) and its
LSD radix sort (Algorithm 1), and the estimated deal of Fast Radix played
out record by record (Algorithm 3: how many records overflow buckets of a
given estimated size).  This module compiles that file with gcc and marshals
numpy arrays to it; it also holds the paper's overflow model (Section
"Analysis", Eq. 1-2) in fp64 numpy, written out as a plain sum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load_library(path: str):
    """Load a compiled oracle library and declare its signatures."""
    lib = ctypes.CDLL(path)
    u64 = ctypes.c_uint64
    p = ctypes.c_void_p
    for name, args in (
        ("oracle_sort_u32", [p, u64]),
        ("oracle_sort_u64", [p, u64]),
        ("oracle_sort_u64_kv", [p, p, u64]),
        ("oracle_sort_u32_kv", [p, p, u64]),
        ("oracle_sort_u64_kv64", [p, p, u64]),
        ("oracle_sort_u32_kv64", [p, p, u64]),
        ("oracle_counting_pass_u32", [p, p, u64, ctypes.c_int]),
        ("oracle_sort_format", [ctypes.c_int, ctypes.c_int, p, p, u64]),
        ("oracle_overflow_count", [p, u64, ctypes.c_int, ctypes.c_int, u64, p]),
    ):
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    return lib


def _get():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int) -> None:
    if rc != 0:
        raise RuntimeError("oracle failed with code %d" % rc)


class Oracle:
    """numpy front end over one compiled oracle library (the real one by
    default; tests may pass a deliberately broken build to check the pins)."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else _get()

    def sort_u32(self, keys) -> np.ndarray:
        k = np.array(keys, dtype=np.uint32, copy=True, order="C")
        _check(self.lib.oracle_sort_u32(_ptr(k), k.size))
        return k

    def sort_u64(self, keys) -> np.ndarray:
        k = np.array(keys, dtype=np.uint64, copy=True, order="C")
        _check(self.lib.oracle_sort_u64(_ptr(k), k.size))
        return k

    def sort_u64_kv(self, keys, vals):
        k = np.array(keys, dtype=np.uint64, copy=True, order="C")
        v = np.array(vals, dtype=np.uint32, copy=True, order="C")
        if k.size != v.size:
            raise ValueError("keys and vals differ in length")
        _check(self.lib.oracle_sort_u64_kv(_ptr(k), _ptr(v), k.size))
        return k, v

    def sort_u32_kv(self, keys, vals):
        k = np.array(keys, dtype=np.uint32, copy=True, order="C")
        v = np.array(vals, dtype=np.uint32, copy=True, order="C")
        if k.size != v.size:
            raise ValueError("keys and vals differ in length")
        _check(self.lib.oracle_sort_u32_kv(_ptr(k), _ptr(v), k.size))
        return k, v

    def sort_u64_kv64(self, keys, vals):
        k = np.array(keys, dtype=np.uint64, copy=True, order="C")
        v = np.array(vals, dtype=np.uint64, copy=True, order="C")
        if k.size != v.size:
            raise ValueError("keys and vals differ in length")
        _check(self.lib.oracle_sort_u64_kv64(_ptr(k), _ptr(v), k.size))
        return k, v

    def sort_u32_kv64(self, keys, vals):
        k = np.array(keys, dtype=np.uint32, copy=True, order="C")
        v = np.array(vals, dtype=np.uint64, copy=True, order="C")
        if k.size != v.size:
            raise ValueError("keys and vals differ in length")
        _check(self.lib.oracle_sort_u32_kv64(_ptr(k), _ptr(v), k.size))
        return k, v

    def sort_format(self, key_type: int, fmt: int, keys, vals=None):
        """Sort in key format `fmt` (0 unsigned, 1 signed, 2 IEEE float total
        order; | 0x100 descending).  `keys` may be any 4- or 8-byte numpy
        array; the result has the same dtype.  Returns keys, or (keys, vals)
        for the key-value types (2: u64 + u32, 3: u32 + u32, 4: u64 + u64,
        5: u32 + u64)."""
        k = np.array(keys, copy=True, order="C")
        width = 8 if key_type in (1, 2, 4) else 4
        if k.dtype.itemsize != width:
            raise ValueError("key width does not match the key type")
        v = None
        if key_type in (2, 3, 4, 5):
            v = np.array(vals, dtype=np.uint64 if key_type in (4, 5) else np.uint32, copy=True, order="C")
            if v.size != k.size:
                raise ValueError("keys and vals differ in length")
        _check(self.lib.oracle_sort_format(int(key_type), int(fmt), _ptr(k), _ptr(v) if v is not None else None,
                                           k.size))
        return k if v is None else (k, v)

    def overflow_count(self, keys, shift: int, cap: int) -> int:
        """Records that overflow when `keys` (u32 or u64) are dealt on the 8-bit
        digit at `shift` into 256 estimated buckets of `cap` records each
        (Fast Radix's estimated deal, Algorithm 3)."""
        k = np.ascontiguousarray(keys)
        if k.dtype not in (np.uint32, np.uint64):
            raise ValueError("u32 or u64 keys")
        out = ctypes.c_uint64(0)
        _check(self.lib.oracle_overflow_count(_ptr(k), k.size, k.dtype.itemsize, int(shift), int(cap),
                                              ctypes.byref(out)))
        return int(out.value)

    def counting_pass_u32(self, keys, shift: int) -> np.ndarray:
        src = np.array(keys, dtype=np.uint32, copy=True, order="C")
        dst = np.empty_like(src)
        _check(self.lib.oracle_counting_pass_u32(_ptr(src), _ptr(dst), src.size, int(shift)))
        return dst


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def sort_u32(keys):
    return default().sort_u32(keys)


def sort_u64(keys):
    return default().sort_u64(keys)


def sort_u64_kv(keys, vals):
    return default().sort_u64_kv(keys, vals)


def sort_u32_kv(keys, vals):
    return default().sort_u32_kv(keys, vals)


def sort_u64_kv64(keys, vals):
    return default().sort_u64_kv64(keys, vals)


def sort_u32_kv64(keys, vals):
    return default().sort_u32_kv64(keys, vals)


def sort_format(key_type, fmt, keys, vals=None):
    return default().sort_format(key_type, fmt, keys, vals)


def counting_pass_u32(keys, shift: int):
    return default().counting_pass_u32(keys, shift)


def overflow_count(keys, shift: int, cap: int) -> int:
    return default().overflow_count(keys, shift, cap)


# ----------------------------------------------------------- overflow model --
#
# Section "Analysis", Eq. 1-2: for N uniformly distributed records dealt into
# M buckets whose size is estimated as N/M, the fraction of records that
# overflow their estimate.  Eq. 2 defines, for k = 0, 1, ..., the term
#     g_o(N, M, k) = (N/M - k) * (M/N) * C(N, k) (1/M)^k (1 - 1/M)^(N-k),
# i.e. (M/N) times the shortfall below N/M of a bucket that received exactly
# k records, weighted by the binomial probability of that.  Eq. 1 (printed
# garbled: its right-hand side uses the three-argument g_o) relates
# consecutive N.  Reading taken here: the two-argument g_o(N, M) is the sum of
# the Eq. 2 terms over the buckets that fall short, k = 0 .. ceil(N/M) - 1.
# Every bucket's shortfall below the mean equals in expectation its excess
# above the mean, so this is the expected overflow fraction for a real-valued
# estimate N/M; when M divides N it is exactly the expected fraction of
# records that overflow buckets of N/M records.  The reading reproduces Eq. 1
# exactly (the tests check the recursion), which the ceiling/floor
# alternatives do not.

def overflow_term(N: int, M: int, k: int) -> float:
    """One term g_o(N, M, k) of Eq. 2, in fp64."""
    from scipy.special import gammaln

    if k < 0 or k > N:
        return 0.0
    lp = (gammaln(N + 1) - gammaln(k + 1) - gammaln(N - k + 1) + k * np.log(1.0 / M)
          + (N - k) * np.log1p(-1.0 / M))
    return float((N / M - k) * (M / N) * np.exp(lp))


def overflow_fraction(N: int, M: int) -> float:
    """g_o(N, M): the sum of the Eq. 2 terms over k = 0 .. ceil(N/M) - 1, in
    fp64 (binomial probabilities through log-gamma)."""
    from scipy.special import gammaln

    if N <= 0 or M <= 0:
        raise ValueError("N and M must be positive")
    kmax = -(-N // M)
    k = np.arange(kmax, dtype=np.float64)
    lp = (gammaln(N + 1) - gammaln(k + 1) - gammaln(N - k + 1) + k * np.log(1.0 / M)
          + (N - k) * np.log1p(-1.0 / M))
    return float(np.sum((N / M - k) * (M / N) * np.exp(lp)))
