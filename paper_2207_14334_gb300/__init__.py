"""Python binding of libdfr.so, the GB300 Diverting Fast Radix sort library.

Argument marshalling only: every function below has the name of the C entry
point it forwards to (include/dfr.h) and passes raw device pointers, lengths
and a CUDA stream.  Pointers may be given as ints or as torch tensors (their
data_ptr() is used); streams as ints, torch.cuda.Stream objects or None (the
current torch stream).  PyTorch is only used for device memory and streams.

There is no fallback: if libdfr.so has not been built, importing works but
the first call raises, naming the build step.

Two environment variables configure the library when it is first loaded
(through the C entry points, as a caller could): DFR_TUNE_FILE names a
launch-plan table in the autotuner's JSON format, whose entries override the
built-in ones (dfr_tune_set); DFR_SPIN_LIMIT sets how many iterations a
device-side wait may spin before it reports DFR_ERR_TIMEOUT (dfr_set_debug).
A file or value the library refuses makes the load raise.
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdfr.so")

DFR_OK = 0
DFR_ERR_INVALID_ARG = 1
DFR_ERR_WORKSPACE = 2
DFR_ERR_CUDA = 3
DFR_ERR_TIMEOUT = 4
DFR_ERR_OVER_BUDGET = 5
DFR_ERR_BUSY = 6
DFR_ERR_BOUNDS = 7
DFR_ERR_TOO_LARGE = 8
DFR_ERR_HOST = 9

DFR_U32 = 0
DFR_U64 = 1
DFR_U64_KV = 2
DFR_U32_KV = 3
DFR_U64_KV64 = 4
DFR_U32_KV64 = 5

DFR_MAX_N = (1 << 30) - 1
DFR_NOALLOC_MAX_N = 1 << 20
DFR_PROFILE_KINDS = 14
DFR_STATS_MAX_LEVELS = 16
DFR_SERVER_MAX_STREAMS = 64
DFR_SERVER_MAX_INFLIGHT = 64
DFR_TUNE_CLASSES = 10
DFR_FMT_UNSIGNED = 0
DFR_FMT_SIGNED = 1
DFR_FMT_FLOAT = 2
DFR_FMT_DESCENDING = 0x100
DFR_TUNE_WARP_MIN = 128
DFR_TUNE_WARP_MAX = 512
DFR_SCHED_MSD = 0
DFR_SCHED_LSD = 1
DFR_SCHED_DFR = 2
DFR_LAUNCH_AUTO = 0
DFR_LAUNCH_LEVELS = 1
DFR_LAUNCH_PERSISTENT = 2
DFR_PERSIST_AUTO_KEYS = 1 << 25

KEY_BYTES = {DFR_U32: 4, DFR_U64: 8, DFR_U64_KV: 8, DFR_U32_KV: 4, DFR_U64_KV64: 8, DFR_U32_KV64: 4}
VAL_BYTES = {DFR_U32: 0, DFR_U64: 0, DFR_U64_KV: 4, DFR_U32_KV: 4, DFR_U64_KV64: 8, DFR_U32_KV64: 8}
HAS_VALS = {kt: vb > 0 for kt, vb in VAL_BYTES.items()}


class DfrError(RuntimeError):
    def __init__(self, code: int, what: str = "", text: str | None = None):
        self.code = code
        super().__init__("%s: %s (code %d)" % (what or "dfr", _status_text(code) if text is None else text, code))


_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t


class dfr_segment_t(ctypes.Structure):
    _fields_ = [("key_type", ctypes.c_int), ("keys", _vp), ("vals", _vp), ("kbuf", _vp), ("vbuf", _vp),
                ("n", _u64)]


class dfr_stats_t(ctypes.Structure):
    _fields_ = [("n_total", _u64), ("key_bytes", _u32), ("val_bytes", _u32), ("levels", _u32),
                ("device_status", _u32),
                ("level_segments", _u64 * DFR_STATS_MAX_LEVELS), ("level_tiles", _u64 * DFR_STATS_MAX_LEVELS),
                ("level_keys", _u64 * DFR_STATS_MAX_LEVELS), ("level_hist_keys", _u64 * DFR_STATS_MAX_LEVELS),
                ("cta_buckets", _u64), ("cta_keys", _u64), ("tiny_buckets", _u64), ("tiny_keys", _u64),
                ("const_buckets", _u64), ("const_keys", _u64), ("copy_keys", _u64), ("model_bytes", _u64),
                ("wsort_buckets", _u64), ("wsort_keys", _u64), ("device_error_site", _u32), ("schedule", _u32),
                ("group_buckets", _u64), ("lsd_keys", _u64), ("est_overflow", _u64), ("est_capacity", _u32),
                ("est_aborted", _u32), ("root_read", _u32), ("persistent", _u32)]


class dfr_tune_t(ctypes.Structure):
    _fields_ = [("target_log2", _u32), ("max_bits", _u32), ("warp_max", _u32), ("scatter_ctas_per_sm", _u32),
                ("ctasort_ctas_per_sm", _u32), ("schedule", _u32), ("launch", _u32), ("reserved", _u32)]


TUNE_FIELDS = ("target_log2", "max_bits", "warp_max", "scatter_ctas_per_sm", "ctasort_ctas_per_sm", "schedule",
               "launch")
_TUNE_OPTIONAL = ("schedule", "launch")  # fields a plan may leave out (0 = DFR_SCHED_MSD, DFR_LAUNCH_AUTO)

_SIGNATURES = {
    "dfr_workspace_bytes": (ctypes.c_int, [ctypes.c_int, _u64, ctypes.POINTER(_sz)]),
    "dfr_sort_u32": (ctypes.c_int, [_vp, _vp, _u64, _vp, _sz, _vp]),
    "dfr_sort_u64": (ctypes.c_int, [_vp, _vp, _u64, _vp, _sz, _vp]),
    "dfr_sort_u64_kv": (ctypes.c_int, [_vp, _vp, _vp, _vp, _u64, _vp, _sz, _vp]),
    "dfr_sort_u32_kv": (ctypes.c_int, [_vp, _vp, _vp, _vp, _u64, _vp, _sz, _vp]),
    "dfr_sort_u64_kv64": (ctypes.c_int, [_vp, _vp, _vp, _vp, _u64, _vp, _sz, _vp]),
    "dfr_sort_u32_kv64": (ctypes.c_int, [_vp, _vp, _vp, _vp, _u64, _vp, _sz, _vp]),
    "dfr_sort_u32_noalloc": (ctypes.c_int, [_vp, _u64, _vp]),
    "dfr_last_device_status": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_int)]),
    "dfr_get_stats": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(dfr_stats_t)]),
    "dfr_batch_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(dfr_segment_t), _u32, ctypes.POINTER(_sz)]),
    "dfr_sort_batch": (ctypes.c_int, [ctypes.POINTER(dfr_segment_t), _u32, _vp, _sz, _vp]),
    "dfr_server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _sz, ctypes.c_int]),
    "dfr_submit": (ctypes.c_int, [_vp, ctypes.POINTER(dfr_segment_t), ctypes.POINTER(_u64)]),
    "dfr_submit_after": (ctypes.c_int, [_vp, ctypes.POINTER(dfr_segment_t), _vp, ctypes.POINTER(_u64)]),
    "dfr_server_set_limits": (ctypes.c_int, [_vp, _u32, _u32]),
    "dfr_fill_splitmix64": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _u64, _u64, _vp]),
    "dfr_poll": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "dfr_wait": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(ctypes.c_double)]),
    "dfr_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "dfr_server_destroy": (ctypes.c_int, [_vp]),
    "dfr_sort_format": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _u64, _vp, _sz, _vp]),
    "dfr_sort_batch_format": (ctypes.c_int, [ctypes.POINTER(dfr_segment_t), _u32, ctypes.c_int, _vp, _sz, _vp]),
    "dfr_graph_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(dfr_segment_t), _u32, _vp, _sz]),
    "dfr_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "dfr_graph_destroy": (ctypes.c_int, [_vp]),
    "dfr_tune_class": (ctypes.c_int, [_u64]),
    "dfr_lsd_min_keys": (_u64, [ctypes.c_int]),
    "dfr_tune_get": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(dfr_tune_t)]),
    "dfr_tune_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(dfr_tune_t)]),
    "dfr_tune_reset": (ctypes.c_int, []),
    "dfr_set_debug": (ctypes.c_int, [_u32, ctypes.c_int]),
    "dfr_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "dfr_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_u64)]),
    "dfr_profile_kind_name": (ctypes.c_char_p, [ctypes.c_int]),
    "dfr_launch_count": (_u64, []),
    "dfr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return LIB_PATH


def load() -> ctypes.CDLL:
    """Load libdfr.so (built by paper_2207_14334_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libdfr.so is not built (run __graft_entry__.build() or "
                                   "python -m paper_2207_14334_gb300.build); there is no CPU fallback")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _apply_env_config(lib)
            _lib = lib
    return _lib


_KEY_TYPE_NAMES = {"DFR_U32": DFR_U32, "DFR_U64": DFR_U64, "DFR_U64_KV": DFR_U64_KV, "DFR_U32_KV": DFR_U32_KV,
                   "DFR_U64_KV64": DFR_U64_KV64, "DFR_U32_KV64": DFR_U32_KV64}


def _apply_env_config(lib) -> None:
    """Apply DFR_TUNE_FILE and DFR_SPIN_LIMIT (see the module docstring); with
    neither set, nothing is called."""
    path = os.environ.get("DFR_TUNE_FILE")
    if path:
        with open(path) as f:
            doc = json.load(f)
        table = doc.get("table", doc)  # the tuner's file, or its bare table
        for name, classes in table.items():
            kt = _KEY_TYPE_NAMES.get(name)
            if kt is None:
                raise ValueError("DFR_TUNE_FILE %s: unknown key type %r" % (path, name))
            for c, entry in classes.items():
                try:
                    t = dfr_tune_t(*(int(entry.get(f, 0) if f in _TUNE_OPTIONAL else entry[f]) for f in TUNE_FIELDS))
                    c = int(c)
                except (KeyError, TypeError, ValueError, AttributeError) as e:
                    raise ValueError("DFR_TUNE_FILE %s: entry %s / class %s: %r" % (path, name, c, e)) from None
                rc = lib.dfr_tune_set(kt, c, ctypes.byref(t))
                if rc != DFR_OK:  # (the text comes from this handle: load() holds its lock)
                    raise DfrError(rc, "DFR_TUNE_FILE %s: entry %s / class %s" % (path, name, c),
                                   lib.dfr_status_string(rc).decode())
    spin = os.environ.get("DFR_SPIN_LIMIT")
    if spin:
        limit = int(spin)
        if not 0 <= limit < (1 << 32):
            raise ValueError("DFR_SPIN_LIMIT must be an integer in [0, 2^32), not %r" % spin)
        rc = lib.dfr_set_debug(limit, 0)
        if rc != DFR_OK:
            raise DfrError(rc, "DFR_SPIN_LIMIT", lib.dfr_status_string(rc).decode())


def _status_text(code: int) -> str:
    try:
        return load().dfr_status_string(int(code)).decode()
    except Exception:  # library missing: still describe the code
        return {0: "ok"}.get(code, "error")


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int:
    if s is None:
        import torch

        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def check(rc: int, what: str = "") -> None:
    """Raise DfrError for a non-zero status."""
    if rc != DFR_OK:
        raise DfrError(rc, what)


# ----------------------------------------------------------- C entry points

def dfr_workspace_bytes(key_type: int, n: int) -> int:
    out = _sz(0)
    check(load().dfr_workspace_bytes(int(key_type), int(n), ctypes.byref(out)), "dfr_workspace_bytes")
    return int(out.value)


def dfr_sort_u32(keys, buf, n, ws, ws_bytes, stream=None) -> int:
    return load().dfr_sort_u32(_ptr(keys), _ptr(buf), int(n), _ptr(ws), int(ws_bytes), _stream(stream))


def dfr_sort_u64(keys, buf, n, ws, ws_bytes, stream=None) -> int:
    return load().dfr_sort_u64(_ptr(keys), _ptr(buf), int(n), _ptr(ws), int(ws_bytes), _stream(stream))


def dfr_sort_u64_kv(keys, vals, kbuf, vbuf, n, ws, ws_bytes, stream=None) -> int:
    return load().dfr_sort_u64_kv(_ptr(keys), _ptr(vals), _ptr(kbuf), _ptr(vbuf), int(n), _ptr(ws),
                                  int(ws_bytes), _stream(stream))


def dfr_sort_u32_kv(keys, vals, kbuf, vbuf, n, ws, ws_bytes, stream=None) -> int:
    return load().dfr_sort_u32_kv(_ptr(keys), _ptr(vals), _ptr(kbuf), _ptr(vbuf), int(n), _ptr(ws),
                                  int(ws_bytes), _stream(stream))


def dfr_sort_u64_kv64(keys, vals, kbuf, vbuf, n, ws, ws_bytes, stream=None) -> int:
    return load().dfr_sort_u64_kv64(_ptr(keys), _ptr(vals), _ptr(kbuf), _ptr(vbuf), int(n), _ptr(ws),
                                    int(ws_bytes), _stream(stream))


def dfr_sort_u32_kv64(keys, vals, kbuf, vbuf, n, ws, ws_bytes, stream=None) -> int:
    return load().dfr_sort_u32_kv64(_ptr(keys), _ptr(vals), _ptr(kbuf), _ptr(vbuf), int(n), _ptr(ws),
                                    int(ws_bytes), _stream(stream))


def dfr_sort_u32_noalloc(keys, n, stream=None) -> int:
    """u32 sort whose scratch lives in the library's fixed device array
    (for callers that cannot allocate device memory; n <= DFR_NOALLOC_MAX_N)."""
    return load().dfr_sort_u32_noalloc(_ptr(keys), int(n), _stream(stream))


def dfr_last_device_status(ws, stream=None) -> int:
    st = ctypes.c_int(0)
    check(load().dfr_last_device_status(_ptr(ws), _stream(stream), ctypes.byref(st)), "dfr_last_device_status")
    return int(st.value)


def dfr_get_stats(ws, stream=None) -> dict:
    s = dfr_stats_t()
    check(load().dfr_get_stats(_ptr(ws), _stream(stream), ctypes.byref(s)), "dfr_get_stats")
    out = {}
    for name, _ in dfr_stats_t._fields_:
        v = getattr(s, name)
        out[name] = list(v) if hasattr(v, "__len__") else int(v)
    return out


def _segments(segs):
    arr = (dfr_segment_t * len(segs))()
    for i, s in enumerate(segs):
        if isinstance(s, dict):
            arr[i] = dfr_segment_t(int(s["key_type"]), _ptr(s.get("keys")), _ptr(s.get("vals")),
                                   _ptr(s.get("kbuf")), _ptr(s.get("vbuf")), int(s["n"]))
        else:
            kt, keys, vals, kbuf, vbuf, n = s
            arr[i] = dfr_segment_t(int(kt), _ptr(keys), _ptr(vals), _ptr(kbuf), _ptr(vbuf), int(n))
    return arr


def dfr_batch_workspace_bytes(segs) -> int:
    arr = _segments(segs)
    out = _sz(0)
    check(load().dfr_batch_workspace_bytes(arr, len(segs), ctypes.byref(out)), "dfr_batch_workspace_bytes")
    return int(out.value)


def dfr_sort_batch(segs, ws, ws_bytes, stream=None) -> int:
    arr = _segments(segs)
    return load().dfr_sort_batch(arr, len(segs), _ptr(ws), int(ws_bytes), _stream(stream))


def dfr_server_create(device: int, mem_budget_bytes: int, n_streams: int) -> int:
    """Returns the server handle (an int); raises DfrError on failure."""
    h = _vp(0)
    check(load().dfr_server_create(ctypes.byref(h), int(device), int(mem_budget_bytes), int(n_streams)),
          "dfr_server_create")
    return int(h.value)


def dfr_submit(server: int, seg) -> tuple:
    """Queue one request (a segment dict or tuple, as for dfr_sort_batch).
    Returns (status, ticket); the ticket is meaningful only for DFR_OK."""
    arr = _segments([seg])
    t = _u64(0)
    rc = load().dfr_submit(_vp(server), arr, ctypes.byref(t))
    return int(rc), int(t.value)


def dfr_submit_after(server: int, seg, ready_event=None) -> tuple:
    """As dfr_submit; the sorting stream first waits on `ready_event` (a
    torch.cuda.Event, a raw cudaEvent_t int, or None)."""
    arr = _segments([seg])
    t = _u64(0)
    ev = 0 if ready_event is None else (ready_event if isinstance(ready_event, int) else int(ready_event.cuda_event))
    rc = load().dfr_submit_after(_vp(server), arr, _vp(ev), ctypes.byref(t))
    return int(rc), int(t.value)


def dfr_server_set_limits(server: int, max_batch: int, max_inflight_per_stream: int = 1) -> int:
    return load().dfr_server_set_limits(_vp(server), int(max_batch), int(max_inflight_per_stream))


def dfr_fill_splitmix64(key_type: int, keys, vals, n: int, seed: int, stream=None) -> int:
    """Seeded SplitMix64 keys on the device (and vals[i] = i for kv types)."""
    return load().dfr_fill_splitmix64(int(key_type), _ptr(keys), _ptr(vals), int(n), int(seed) & (2 ** 64 - 1),
                                      _stream(stream))


def dfr_poll(server: int, ticket: int) -> tuple:
    """Returns (status, done, latency_us)."""
    d = ctypes.c_int(0)
    lat = ctypes.c_double(0.0)
    rc = load().dfr_poll(_vp(server), int(ticket), ctypes.byref(d), ctypes.byref(lat))
    return int(rc), bool(d.value), float(lat.value)


def dfr_wait(server: int, ticket: int) -> tuple:
    """Returns (status, latency_us)."""
    lat = ctypes.c_double(0.0)
    rc = load().dfr_wait(_vp(server), int(ticket), ctypes.byref(lat))
    return int(rc), float(lat.value)


def dfr_server_stats(server: int) -> dict:
    b, p, f = _u64(0), _u64(0), _u64(0)
    check(load().dfr_server_stats(_vp(server), ctypes.byref(b), ctypes.byref(p), ctypes.byref(f)),
          "dfr_server_stats")
    return {"batches": int(b.value), "pending": int(p.value), "inflight": int(f.value)}


def dfr_server_destroy(server: int) -> int:
    return load().dfr_server_destroy(_vp(server))


def dfr_sort_format(key_type, key_format, keys, vals, kbuf, vbuf, n, ws, ws_bytes, stream=None) -> int:
    """Sort signed, IEEE-float or descending keys (DFR_FMT_*): the unsigned
    sort between an in-place order-preserving bit map and its inverse."""
    return load().dfr_sort_format(int(key_type), int(key_format), _ptr(keys), _ptr(vals), _ptr(kbuf), _ptr(vbuf),
                                  int(n), _ptr(ws), int(ws_bytes), _stream(stream))


def dfr_sort_batch_format(segs, key_format, ws, ws_bytes, stream=None) -> int:
    arr = _segments(segs)
    return load().dfr_sort_batch_format(arr, len(segs), int(key_format), _ptr(ws), int(ws_bytes), _stream(stream))


def dfr_graph_create(segs, ws, ws_bytes) -> int:
    """Capture one sort of these segments (as for dfr_sort_batch) into a CUDA
    graph; returns the handle (an int).  Raises DfrError on failure."""
    arr = _segments(segs)
    h = _vp(0)
    check(load().dfr_graph_create(ctypes.byref(h), arr, len(segs), _ptr(ws), int(ws_bytes)), "dfr_graph_create")
    return int(h.value)


def dfr_graph_launch(graph: int, stream=None) -> int:
    return load().dfr_graph_launch(_vp(graph), _stream(stream))


def dfr_graph_destroy(graph: int) -> int:
    return load().dfr_graph_destroy(_vp(graph))


def dfr_tune_class(mean_keys: int) -> int:
    return int(load().dfr_tune_class(int(mean_keys)))


def dfr_tune_get(key_type: int, size_class: int) -> dict:
    t = dfr_tune_t()
    check(load().dfr_tune_get(int(key_type), int(size_class), ctypes.byref(t)), "dfr_tune_get")
    return {f: int(getattr(t, f)) for f in TUNE_FIELDS}


def dfr_tune_set(key_type: int, size_class: int, tune: dict) -> int:
    """Override one entry of the launch-plan table (fields as dfr_tune_get;
    a missing "schedule" means DFR_SCHED_MSD, a missing "launch"
    DFR_LAUNCH_AUTO)."""
    t = dfr_tune_t(*(int(tune.get(f, 0) if f in _TUNE_OPTIONAL else tune[f]) for f in TUNE_FIELDS))
    return load().dfr_tune_set(int(key_type), int(size_class), ctypes.byref(t))


def dfr_tune_reset() -> int:
    return load().dfr_tune_reset()


def dfr_lsd_min_keys(key_type: int) -> int:
    """Smallest single array the LSD schedules (DFR_SCHED_LSD / _DFR) apply to."""
    return int(load().dfr_lsd_min_keys(int(key_type)))


def dfr_set_debug(spin_limit: int = 0, force_timeout: bool = False) -> int:
    return load().dfr_set_debug(int(spin_limit), 1 if force_timeout else 0)


def dfr_profile_enable(on: bool) -> int:
    return load().dfr_profile_enable(1 if on else 0)


def dfr_profile_read() -> dict:
    ms = (ctypes.c_double * DFR_PROFILE_KINDS)()
    n = (_u64 * DFR_PROFILE_KINDS)()
    check(load().dfr_profile_read(ms, n), "dfr_profile_read")
    lib = load()
    return {lib.dfr_profile_kind_name(i).decode(): (float(ms[i]), int(n[i])) for i in range(DFR_PROFILE_KINDS)}


def dfr_launch_count() -> int:
    return int(load().dfr_launch_count())


def dfr_status_string(code: int) -> str:
    return load().dfr_status_string(int(code)).decode()


# ------------------------------------------------------ torch conveniences

class Sorter:
    """Holds a scratch buffer and a workspace (allocated with torch) sized for
    up to `capacity` keys of `key_type`, and sorts device tensors in place
    through the C entry points above."""

    def __init__(self, key_type: int, capacity: int, device="cuda"):
        import torch

        self.key_type = key_type
        self.capacity = int(capacity)
        dev = torch.device(device)
        if dev.type == "cuda" and dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        kb = KEY_BYTES[key_type]
        kdt = torch.int32 if kb == 4 else torch.int64
        self.kbuf = torch.empty(max(1, self.capacity), dtype=kdt, device=self.device)
        vdt = torch.int64 if VAL_BYTES[key_type] == 8 else torch.int32
        self.vbuf = (torch.empty(max(1, self.capacity), dtype=vdt, device=self.device)
                     if HAS_VALS[key_type] else None)
        self.ws_bytes = dfr_workspace_bytes(key_type, max(2, self.capacity))
        # zeroed once so the status word reads DFR_OK before the first call
        self.ws = torch.zeros(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def _arg(self, t, name: str, n: int, item_bytes: int) -> None:
        """The C entry points take a bare pointer and trust it to hold `n`
        contiguous items: check that tensor `t` does, on this sorter's device."""
        if t is None:
            if n:
                raise ValueError("%s is required to sort %d keys" % (name, n))
            return
        if t.element_size() != item_bytes:
            raise ValueError("%s has %d-byte items; this key type needs %d" % (name, t.element_size(), item_bytes))
        if t.numel() < n:
            raise ValueError("%s holds %d items, fewer than n = %d" % (name, t.numel(), n))
        if not t.is_contiguous():
            raise ValueError("%s is not contiguous" % name)
        if t.device != self.device:
            raise ValueError("%s is on %s; this sorter's buffers are on %s" % (name, t.device, self.device))

    def sort_(self, keys, vals=None, n=None, stream=None, key_format=DFR_FMT_UNSIGNED) -> int:
        """Sort the first `n` (default: all) keys of `keys` in place, with their
        payloads `vals` for the kv key types; raises ValueError for a tensor
        that cannot hold them and DfrError for a status other than DFR_OK."""
        n = int(keys.numel() if n is None else n)
        if n < 0 or n > self.capacity:
            raise ValueError("array of %d keys outside this sorter's capacity %d" % (n, self.capacity))
        kt = self.key_type
        self._arg(keys, "keys", n, KEY_BYTES[kt])
        if HAS_VALS[kt]:
            self._arg(vals, "vals", n, VAL_BYTES[kt])
        elif vals is not None:
            raise ValueError("payloads given to a key-only sorter")
        if key_format != DFR_FMT_UNSIGNED:
            rc = dfr_sort_format(kt, key_format, keys, vals, self.kbuf, self.vbuf, n, self.ws, self.ws_bytes, stream)
        elif kt == DFR_U32:
            rc = dfr_sort_u32(keys, self.kbuf, n, self.ws, self.ws_bytes, stream)
        elif kt == DFR_U64:
            rc = dfr_sort_u64(keys, self.kbuf, n, self.ws, self.ws_bytes, stream)
        elif kt == DFR_U64_KV:
            rc = dfr_sort_u64_kv(keys, vals, self.kbuf, self.vbuf, n, self.ws, self.ws_bytes, stream)
        elif kt == DFR_U32_KV:
            rc = dfr_sort_u32_kv(keys, vals, self.kbuf, self.vbuf, n, self.ws, self.ws_bytes, stream)
        elif kt == DFR_U64_KV64:
            rc = dfr_sort_u64_kv64(keys, vals, self.kbuf, self.vbuf, n, self.ws, self.ws_bytes, stream)
        else:
            rc = dfr_sort_u32_kv64(keys, vals, self.kbuf, self.vbuf, n, self.ws, self.ws_bytes, stream)
        check(rc, "sort")
        return rc

    def device_status(self, stream=None) -> int:
        return dfr_last_device_status(self.ws, stream)

    def stats(self, stream=None) -> dict:
        return dfr_get_stats(self.ws, stream)


def to_device(a, device="cuda"):
    """numpy array of 4- or 8-byte items -> torch int32/int64 device tensor
    holding the same bits (torch's unsigned dtypes have patchy op coverage)."""
    import numpy as np
    import torch

    if a.dtype.itemsize == 4 and a.dtype != np.int32:
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.int32))
    elif a.dtype.itemsize == 8 and a.dtype != np.int64:
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.int64))
    else:
        t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to(device)


def to_numpy(t, dtype):
    """Device tensor -> numpy array reinterpreted as `dtype` (np.uint32/uint64)."""
    import numpy as np

    return t.cpu().numpy().view(dtype)
