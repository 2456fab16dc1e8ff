"""The C-ABI library loads, exports every symbol include/dfr.h declares, and its
host-side argument checks behave as documented (no GPU needed: every call
here returns before touching CUDA)."""
import ctypes
import os
import re

import pytest

import paper_2207_14334_gb300 as dfr
from paper_2207_14334_gb300 import build as dfr_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dfr.h")


@pytest.fixture(scope="module")
def lib():
    dfr_build.build()
    return dfr.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(dfr_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dfr_sort_u32", "dfr_sort_u64", "dfr_sort_u64_kv", "dfr_sort_batch",
                     "dfr_workspace_bytes", "dfr_last_device_status", "dfr_get_stats"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_workspace_bytes(lib):
    small = dfr.dfr_workspace_bytes(dfr.DFR_U32, 1000)
    big = dfr.dfr_workspace_bytes(dfr.DFR_U32, 1 << 28)
    assert 0 < small < big
    # the workspace stays a modest fraction of the key array at full size
    assert big < 0.5 * (1 << 28) * 4
    for kt in (dfr.DFR_U64, dfr.DFR_U64_KV, dfr.DFR_U32_KV, dfr.DFR_U64_KV64, dfr.DFR_U32_KV64):
        assert dfr.dfr_workspace_bytes(kt, 1 << 20) > 0
    out = ctypes.c_size_t(0)
    assert lib.dfr_workspace_bytes(99, 10, ctypes.byref(out)) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_workspace_bytes(dfr.DFR_U32, dfr.DFR_MAX_N + 1, ctypes.byref(out)) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_workspace_bytes(dfr.DFR_U32, 10, None) == dfr.DFR_ERR_INVALID_ARG


def test_host_argument_checks(lib):
    # n == 0 and n == 1 are no-ops
    assert dfr.dfr_sort_u32(0, 0, 0, 0, 0, stream=0) == dfr.DFR_OK
    assert dfr.dfr_sort_u32(0x1000, 0x2000, 1, 0, 0, stream=0) == dfr.DFR_OK
    # null pointers
    assert dfr.dfr_sort_u32(0, 0x2000, 10, 0x10000, 1 << 20, stream=0) == dfr.DFR_ERR_INVALID_ARG
    assert dfr.dfr_sort_u64_kv(0x1000, 0, 0x9000, 0xA000, 10, 0x10000, 1 << 20, stream=0) == dfr.DFR_ERR_INVALID_ARG
    # overlapping keys / buf
    assert dfr.dfr_sort_u32(0x1000, 0x1010, 100, 0x100000, 1 << 24, stream=0) == dfr.DFR_ERR_INVALID_ARG
    assert dfr.dfr_sort_u64_kv(0x1000, 0x1100, 0x100000, 0x200000, 100, 0x1000000, 1 << 24,
                               stream=0) == dfr.DFR_ERR_INVALID_ARG
    # n above the maximum
    assert dfr.dfr_sort_u32(0x1000, 0x10000000000, dfr.DFR_MAX_N + 1, 0x100000, 1 << 24,
                            stream=0) == dfr.DFR_ERR_INVALID_ARG
    # misaligned or missing workspace
    ws = dfr.dfr_workspace_bytes(dfr.DFR_U32, 1000)
    assert dfr.dfr_sort_u32(0x100000, 0x200000, 1000, 0x300010, ws, stream=0) == dfr.DFR_ERR_INVALID_ARG
    assert dfr.dfr_sort_u32(0x100000, 0x200000, 1000, 0, ws, stream=0) == dfr.DFR_ERR_INVALID_ARG
    # workspace too small
    assert dfr.dfr_sort_u32(0x100000, 0x200000, 1000, 0x300000, ws - 1, stream=0) == dfr.DFR_ERR_WORKSPACE


def test_batch_host_checks(lib):
    segs = [(dfr.DFR_U32, 0x100000, 0, 0x200000, 0, 1000), (dfr.DFR_U64, 0x300000, 0, 0x400000, 0, 10)]
    with pytest.raises(dfr.DfrError):
        dfr.dfr_batch_workspace_bytes(segs)
    assert dfr.dfr_sort_batch(segs, 0x1000000, 1 << 30, stream=0) == dfr.DFR_ERR_INVALID_ARG
    one = [(dfr.DFR_U32, 0x100000, 0, 0x200000, 0, 1000)]
    assert dfr.dfr_batch_workspace_bytes(one) >= dfr.dfr_workspace_bytes(dfr.DFR_U32, 1000)
    assert dfr.dfr_sort_batch([], 0, 0, stream=0) == dfr.DFR_OK


def test_status_strings_and_counters(lib):
    for code in range(8):
        assert dfr.dfr_status_string(code)
    assert dfr.dfr_launch_count() >= 0
    assert dfr.dfr_set_debug(0, False) == dfr.DFR_OK


def test_server_host_checks(lib):
    """Argument checks of the served form that return before any CUDA call."""
    h = ctypes.c_void_p(0)
    assert lib.dfr_server_create(None, 0, 1 << 20, 1) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_server_create(ctypes.byref(h), 0, 100, 1) == dfr.DFR_ERR_INVALID_ARG  # budget < 4096
    assert lib.dfr_server_create(ctypes.byref(h), 0, 1 << 20, 0) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_server_create(ctypes.byref(h), 0, 1 << 20, dfr.DFR_SERVER_MAX_STREAMS + 1) == dfr.DFR_ERR_INVALID_ARG
    assert h.value is None
    t = ctypes.c_uint64(0)
    seg = dfr.dfr_segment_t(dfr.DFR_U32, 0x1000, 0, 0, 0, 10)
    assert lib.dfr_submit(None, ctypes.byref(seg), ctypes.byref(t)) == dfr.DFR_ERR_INVALID_ARG
    d = ctypes.c_int(0)
    assert lib.dfr_poll(None, 1, ctypes.byref(d), None) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_wait(None, 1, None) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_server_stats(None, None, None, None) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_server_destroy(None) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_server_set_limits(None, 1, 1) == dfr.DFR_ERR_INVALID_ARG


def test_tune_table_api(lib):
    """Size classes, the built-in table, overrides and their validation (no CUDA call)."""
    assert [dfr.dfr_tune_class(n) for n in (0, 1, 4095, 4096, 16383, 16384, 1 << 20, (1 << 28) - 1, 1 << 28,
                                            1 << 40)] == [0, 0, 0, 1, 1, 2, 5, 8, 9, 9]
    for kt in (dfr.DFR_U32, dfr.DFR_U64, dfr.DFR_U64_KV, dfr.DFR_U32_KV, dfr.DFR_U64_KV64, dfr.DFR_U32_KV64):
        for c in range(dfr.DFR_TUNE_CLASSES):
            t = dfr.dfr_tune_get(kt, c)
            assert 6 <= t["target_log2"] <= 13 and 4 <= t["max_bits"] <= 8
            assert dfr.DFR_TUNE_WARP_MIN <= t["warp_max"] <= dfr.DFR_TUNE_WARP_MAX
    base = dfr.dfr_tune_get(dfr.DFR_U32, 3)
    try:
        new = dict(base, target_log2=9, max_bits=6, warp_max=256, scatter_ctas_per_sm=1, ctasort_ctas_per_sm=1,
                   schedule=dfr.DFR_SCHED_DFR, launch=dfr.DFR_LAUNCH_PERSISTENT)
        assert dfr.dfr_tune_set(dfr.DFR_U32, 3, new) == dfr.DFR_OK
        assert dfr.dfr_tune_get(dfr.DFR_U32, 3) == new
        for bad in (dict(base, target_log2=5), dict(base, target_log2=14), dict(base, max_bits=3),
                    dict(base, max_bits=9), dict(base, warp_max=64), dict(base, warp_max=1024),
                    dict(base, scatter_ctas_per_sm=5), dict(base, schedule=3), dict(base, launch=3)):
            assert dfr.dfr_tune_set(dfr.DFR_U32, 3, bad) == dfr.DFR_ERR_INVALID_ARG
        assert dfr.dfr_tune_set(7, 3, base) == dfr.DFR_ERR_INVALID_ARG
        assert dfr.dfr_tune_set(dfr.DFR_U32, dfr.DFR_TUNE_CLASSES, base) == dfr.DFR_ERR_INVALID_ARG
    finally:
        assert dfr.dfr_tune_reset() == dfr.DFR_OK
    assert dfr.dfr_tune_get(dfr.DFR_U32, 3) == base


def test_tuner_writes_a_table_the_library_compiles(tmp_path):
    """tune.write_inc emits the (key types) x DFR_TUNE_CLASSES rows the
    built-in table expects (the checked-in table is such a file)."""
    from paper_2207_14334_gb300 import tune

    table = {"DFR_U32": {"3": dict(target_log2=11, max_bits=7, warp_max=256, scatter_ctas_per_sm=2,
                                   ctasort_ctas_per_sm=1),
                         "9": dict(target_log2=12, max_bits=8, warp_max=512, scatter_ctas_per_sm=0,
                                   ctasort_ctas_per_sm=0, schedule=2),
                         "0": dict(target_log2=11, max_bits=8, warp_max=512, scatter_ctas_per_sm=0,
                                   ctasort_ctas_per_sm=0, launch=1)}}
    p = tmp_path / "t.inc"
    tune.write_inc(table, path=str(p), note="test")
    body = "".join(l for l in p.read_text().splitlines(True) if not l.startswith("//"))
    assert len(tune.KEY_TYPES) == 6
    rows = re.findall(r"\{(\d+), (\d+), (\d+), (\d+), (\d+), (\d+), (\d+), 0\}", body)
    assert len(rows) == len(tune.KEY_TYPES) * dfr.DFR_TUNE_CLASSES  # eight fields per entry, reserved zero
    assert "{11, 7, 256, 2, 1, 0, 0, 0}" in body
    assert "{12, 8, 512, 0, 0, 2, 0, 0}" in body
    assert "{11, 8, 512, 0, 0, 0, 1, 0}" in body
    shipped = "".join(l for l in open(tune.INC).read().splitlines(True) if not l.startswith("//"))
    assert len(re.findall(r"\{(\d+), (\d+), (\d+), (\d+), (\d+), (\d+), (\d+), 0\}", shipped)) == \
        len(tune.KEY_TYPES) * dfr.DFR_TUNE_CLASSES


def test_graph_host_checks(lib):
    h = ctypes.c_void_p(0)
    seg = dfr.dfr_segment_t(dfr.DFR_U32, 0x1000, 0, 0x2000, 0, 10)
    assert lib.dfr_graph_create(None, ctypes.byref(seg), 1, 0x100000, 1 << 20) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_graph_create(ctypes.byref(h), None, 1, 0x100000, 1 << 20) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_graph_create(ctypes.byref(h), ctypes.byref(seg), 0, 0x100000, 1 << 20) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_graph_create(ctypes.byref(h), ctypes.byref(seg), 1, 0x100010, 1 << 20) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_graph_create(ctypes.byref(h), ctypes.byref(seg), 1, 0x100000, 16) == dfr.DFR_ERR_WORKSPACE
    assert h.value is None
    assert lib.dfr_graph_launch(None, None) == dfr.DFR_ERR_INVALID_ARG
    assert lib.dfr_graph_destroy(None) == dfr.DFR_ERR_INVALID_ARG


def test_key_format_host_checks(lib):
    # an unknown format is refused before anything is enqueued
    for bad in (3, 0x200, -1, 0x1FF):
        assert dfr.dfr_sort_format(dfr.DFR_U32, bad, 0x100000, 0, 0x200000, 0, 1000, 0x300000, 1 << 24,
                                   stream=0) == dfr.DFR_ERR_INVALID_ARG
        assert dfr.dfr_sort_batch_format([], bad, 0, 0, stream=0) == dfr.DFR_ERR_INVALID_ARG
    assert dfr.dfr_sort_batch_format([], dfr.DFR_FMT_FLOAT | dfr.DFR_FMT_DESCENDING, 0, 0, stream=0) == dfr.DFR_OK
    # n <= 1 is a no-op in every format
    assert dfr.dfr_sort_format(dfr.DFR_U64, dfr.DFR_FMT_SIGNED, 0x1000, 0, 0x2000, 0, 1, 0, 0, stream=0) == dfr.DFR_OK
    names = [lib.dfr_profile_kind_name(i) for i in range(dfr.DFR_PROFILE_KINDS)]
    assert names[-4:] == [b"keyfmt", b"lsd_pass", b"lsd_plan", b"persist"]


def test_workspace_bytes_never_decrease(lib):
    """A workspace sized for n keys must serve every call of fewer keys, also
    across the sizes where the plan switches the scatter geometry (2^22 keys
    in all) or starts to allow the LSD phase (dfr_lsd_min_keys)."""
    for kt in (dfr.DFR_U32, dfr.DFR_U64, dfr.DFR_U64_KV, dfr.DFR_U32_KV, dfr.DFR_U64_KV64, dfr.DFR_U32_KV64):
        edges = [1 << 22, dfr.dfr_lsd_min_keys(kt)]
        pts = set([1, 2, 3, 31, 33, 4096, 6145, 8193, 12289, 1 << 20, 1 << 24, 1 << 28, dfr.DFR_MAX_N])
        for e in edges:
            pts.update(range(e - 20000, e + 20000, 331))
            pts.update((e - 1, e, e + 1))
        prev = 0
        for n in sorted(pts):
            w = dfr.dfr_workspace_bytes(kt, n)
            assert w >= prev, (kt, n, w, prev)
            prev = w


def test_checked_in_tune_table_is_the_compiled_one(lib):
    """The tuner's JSON record and the table compiled into the library (from
    csrc/dfr_tune_table.inc) hold the same plan for every key type and size
    class."""
    import json

    from paper_2207_14334_gb300 import tune

    with open(os.path.join(os.path.dirname(tune.INC), "..", "tune_table.json")) as f:
        table = json.load(f)["table"]
    assert dfr.dfr_tune_reset() == dfr.DFR_OK
    for name in tune.KEY_TYPES:
        kt = getattr(dfr, name)
        for c in range(dfr.DFR_TUNE_CLASSES):
            rec = table[name][str(c)]
            want = {f: int(rec.get(f, 0)) for f in tune.FIELDS}
            assert dfr.dfr_tune_get(kt, c) == want, (name, c)


def test_lsd_minimum_and_size_classes(lib):
    """The LSD schedules apply from 256 x the CTA sort's capacity (6144 u32
    keys; 4096 u64 keys or key-value records): below that the top digit's
    buckets already fit one CTA sort on average, and dealing a second top
    digit first would not pay.  Size class c covers mean array lengths
    [2^(10+2c), 2^(12+2c)); class 0 everything below 2^12, the last class
    2^28 and up."""
    assert dfr.dfr_lsd_min_keys(dfr.DFR_U32) == 256 * 6144
    for kt in (dfr.DFR_U64, dfr.DFR_U64_KV, dfr.DFR_U32_KV, dfr.DFR_U64_KV64, dfr.DFR_U32_KV64):
        assert dfr.dfr_lsd_min_keys(kt) == 256 * 4096
    for c in range(1, dfr.DFR_TUNE_CLASSES - 1):
        lo, hi = 1 << (10 + 2 * c), 1 << (12 + 2 * c)
        assert dfr.dfr_tune_class(lo) == c and dfr.dfr_tune_class(hi - 1) == c and dfr.dfr_tune_class(hi) == c + 1
    assert dfr.dfr_tune_class((1 << 12) - 1) == 0
    assert dfr.dfr_tune_class(1 << 40) == dfr.DFR_TUNE_CLASSES - 1


def test_tuner_picks_the_plan_balanced_over_launch_forms():
    """tune.pick_plan keeps the plan with the smallest mean of its times
    divided by each launch form's best time: a plan fastest in one form but
    slow in the other loses to one close to the best in both."""
    from paper_2207_14334_gb300 import tune

    times = {
        "fast_levels_only": {1: 1.00, 2: 2.00},  # 1.0 and 2.0 of the bests -> 1.5
        "fast_persistent_only": {1: 1.60, 2: 1.00},  # 1.6 and 1.0 -> 1.3
        "balanced": {1: 1.10, 2: 1.10},  # 1.1 and 1.1 -> 1.1
    }
    assert tune.pick_plan(times) == "balanced"
    # one form only: the fastest plan
    assert tune.pick_plan({"a": {0: 2.0}, "b": {0: 1.5}, "c": {0: 3.0}}) == "b"
