"""Plants plausible mistakes in the oracle (on the CPU) and checks that the
oracle's pins catch every one of them.

Each mutant is oracle.c with one textual edit (a dropped pass, a wrong prefix
index, a wrong digit mask or shift, a payload dealt from the wrong slot, an
unstable deal, a missing buffer swap, an off-by-one bucket capacity in the
estimated deal).  It is compiled into a scratch library
and a battery of the pins from test_oracle_pins.py runs against it in a child
process (so a mutant that writes out of bounds only kills the child).  The
unmodified source must pass the same battery.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

BATTERY = r"""
import itertools, sys
import numpy as np
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import oracle
from test_oracle_pins import (U32_ALPHABET, U64_ALPHABET, insertion_sort_pairs,
                              check_sorted_permutation, check_kv_stable)
orc = oracle.Oracle(oracle.load_library({lib!r}))
for n in range(0, 5):
    for tup in itertools.product(U32_ALPHABET, repeat=n):
        want, _ = insertion_sort_pairs(tup)
        assert orc.sort_u32(np.array(tup, np.uint32)).tolist() == want
        k, v = orc.sort_u32_kv(np.array(tup, np.uint32), np.arange(n, dtype=np.uint32))
        wk, wv = insertion_sort_pairs(tup)
        assert k.tolist() == wk and v.tolist() == wv
    for tup in itertools.product(U64_ALPHABET, repeat=min(n, 4)):
        want, wv = insertion_sort_pairs(tup)
        assert orc.sort_u64(np.array(tup, np.uint64)).tolist() == want
        k, v = orc.sort_u64_kv(np.array(tup, np.uint64), np.arange(len(tup), dtype=np.uint32))
        assert k.tolist() == want and v.tolist() == wv
g = np.random.Generator(np.random.PCG64(7))
for trial in range(50):
    n = int(g.integers(0, 3000))
    k32 = g.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32) >> np.uint32(int(g.integers(0, 28)))
    out = orc.sort_u32(k32)
    check_sorted_permutation(k32, out)
    assert np.array_equal(out, np.sort(k32, kind="stable"))
    k64 = g.bit_generator.random_raw(n).astype(np.uint64) >> np.uint64(int(g.integers(0, 60)))
    assert np.array_equal(orc.sort_u64(k64), np.sort(k64, kind="stable"))
    kk, vv = orc.sort_u64_kv(k64, np.arange(n, dtype=np.uint32))
    check_sorted_permutation(k64, kk)
    check_kv_stable(k64, kk, vv)
    k16 = (k32 & np.uint32(0xF00F))
    kk, vv = orc.sort_u32_kv(k16, np.arange(n, dtype=np.uint32))
    check_kv_stable(k16, kk, vv)
for dt, kt in ((np.int32, 0), (np.int64, 1)):
    info = np.iinfo(dt)
    a = g.integers(info.min, info.max, 2000, dtype=dt, endpoint=True)
    assert np.array_equal(orc.sort_format(kt, 1, a), np.sort(a))
    assert np.array_equal(orc.sort_format(kt, 0x101, a), np.sort(a)[::-1])
for dt, it, kt in ((np.float32, np.uint32, 0), (np.float64, np.uint64, 1)):
    f = (g.standard_normal(2000) * 10.0 ** g.integers(-20, 20, 2000)).astype(dt)
    assert np.array_equal(orc.sort_format(kt, 2, f), np.sort(f, kind="stable"))
    sign = 1 << (8 * np.dtype(dt).itemsize - 1)
    order = np.array([int(np.array([-np.inf], dtype=dt).view(it)[0]), sign | 1, sign, 0, 1,
                      int(np.array([np.inf], dtype=dt).view(it)[0])], dtype=it)
    assert np.array_equal(orc.sort_format(kt, 2, order[::-1].copy().view(dt)).view(it), order)
    assert np.array_equal(orc.sort_format(kt, 0x102, order.view(dt)).view(it), order[::-1])
a = g.integers(-4, 4, 500).astype(np.int32)
k, v = orc.sort_format(3, 0x101, a, np.arange(500, dtype=np.uint32))
assert v.tolist() == sorted(range(500), key=lambda i: (-a[i], i))
for trial in range(8):
    n = int(g.integers(0, 3000))
    k = g.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    if trial % 2:
        k &= np.uint32(0xFF3FFFFF)
    cap = int(g.integers(0, 30))
    cnt = np.bincount(((k >> np.uint32(16)) & np.uint32(255)).astype(np.int64), minlength=256)
    assert orc.overflow_count(k, 16, cap) == int(np.maximum(cnt - cap, 0).sum())
    k64 = k.astype(np.uint64) << np.uint64(32)
    cnt = np.bincount(((k64 >> np.uint64(56)) & np.uint64(255)).astype(np.int64), minlength=256)
    assert orc.overflow_count(k64, 56, cap) == int(np.maximum(cnt - cap, 0).sum())
assert orc.overflow_count(np.full(100, 7, np.uint32), 0, 10) == 90
i64 = np.arange(3000, dtype=np.uint64)
pay = i64 | (((i64 * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)) << np.uint64(32))
for trial in range(20):
    k64 = g.bit_generator.random_raw(3000).astype(np.uint64) >> np.uint64(int(g.integers(0, 60)))
    kk, vv = orc.sort_u64_kv64(k64, pay)
    order = np.argsort(k64, kind="stable")
    assert np.array_equal(kk, k64[order]) and np.array_equal(vv, pay[order])
    k32 = (k64 & np.uint64(0xFFFFFFFF)).astype(np.uint32) >> np.uint32(int(g.integers(0, 28)))
    kk, vv = orc.sort_u32_kv64(k32, pay)
    order = np.argsort(k32, kind="stable")
    assert np.array_equal(kk, k32[order]) and np.array_equal(vv, pay[order])
print("PINS-PASS")
"""

# (function the edit is confined to, text to replace, replacement)
MUTANTS = [
    ("counting_pass_u32(", "index[d] = index[d - 1] + count[d - 1];", "index[d] = index[d - 1] + count[d];"),
    ("counting_pass_u32(", "index[0] = 0;", "index[0] = 1;"),
    ("counting_pass_u32(", "(src[i] >> shift) & 255u] += 1", "(src[i] >> shift) & 127u] += 1"),
    ("counting_pass_u32(", "dst[index[(rec >> shift) & 255u]++] = rec;", "dst[index[(rec >> shift) & 15u]++] = rec;"),
    ("counting_pass_u32(", "const int shift = ORACLE_RADIX_BITS * j;", "const int shift = ORACLE_RADIX_BITS * j + (j == 3);"),
    ("int oracle_sort_u32(", "for (j = 0; j < 4; ++j)", "for (j = 0; j < 2; ++j)"),
    ("int oracle_sort_u32(", "t = src; src = dst; dst = t;", "t = src;"),
    ("int oracle_sort_u64(", "for (j = 0; j < 8; ++j)", "for (j = 0; j < 6; ++j)"),
    ("counting_pass_u64(", "count[(src[i] >> shift) & 255u] += 1", "count[(src[i] >> (shift & 31)) & 255u] += 1"),
    ("counting_pass_u64_kv(", "vdst[at] = vsrc[i];", "vdst[at] = vsrc[at];"),
    ("counting_pass_u64_kv(", "const uint64_t at = index[(key >> shift) & 255u]++;",
     "const uint64_t at = index[(key >> shift) & 255u]++ ; if (i + 1 < n && ksrc[i + 1] == key) { kdst[at] = key; vdst[at] = vsrc[i + 1]; continue; }"),
    ("counting_pass_u32_kv(", "vdst[at] = vsrc[i];", "vdst[at] = vsrc[n - 1 - i];"),
    ("int oracle_sort_u32_kv(", "vt = vs; vs = vd; vd = vt;", "vt = vs;"),
    ("static uint64_t fmt_encode(", "if (x & sign) x = x ^ all;", "if (x & sign) x = x ^ sign;"),
    ("static uint64_t fmt_encode(", "x = x ^ sign;", "x = x ^ (sign >> 1);"),
    ("static uint64_t fmt_decode(", "if (fmt & ORACLE_FMT_DESC) y = y ^ all;", ";"),
    ("static uint64_t fmt_decode(", "if (y & sign) y = y & ~sign;", "if (y & sign) y = y ^ all;"),
    ("counting_pass_u64_kv64(", "vdst[at] = vsrc[i];", "vdst[at] = (uint32_t)vsrc[i];"),
    ("counting_pass_u32_kv64(", "vdst[at] = vsrc[i];", "vdst[at] = vsrc[i] & 0xFFFFFFFF00000000ull | (uint32_t)i;"),
    ("int oracle_sort_u32_kv64(", "vt = vs; vs = vd; vd = vt;", "vt = vs;"),
    ("int oracle_overflow_count(", "if (fill[b] < cap)", "if (fill[b] <= cap)"),
    ("int oracle_overflow_count(", "(unsigned)((key >> shift) & 255u)", "(unsigned)((key >> shift) & 127u)"),
    ("int oracle_overflow_count(", "((const uint32_t*)keys)[i]", "((const uint32_t*)keys)[i] >> 1"),
]


def _compile(src_text: str, out_dir: str, name: str) -> str:
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", c, "-o", so])
    return so


def _battery_passes(lib: str) -> bool:
    code = BATTERY.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    return r.returncode == 0 and "PINS-PASS" in r.stdout


def _mutate(text: str, func: str, old: str, new: str) -> str:
    start = text.index(func)
    at = text.index(old, start)
    return text[:at] + new + text[at + len(old):]


@pytest.fixture(scope="module")
def source_text():
    with open(SRC) as f:
        return f.read()


def test_unmodified_oracle_passes_battery(source_text, tmp_path):
    assert _battery_passes(_compile(source_text, str(tmp_path), "orig"))


@pytest.mark.parametrize("idx", range(len(MUTANTS)))
def test_mutant_is_caught(source_text, tmp_path, idx):
    func, old, new = MUTANTS[idx]
    mutated = _mutate(source_text, func, old, new)
    assert mutated != source_text
    lib = _compile(mutated, str(tmp_path), "mut%d" % idx)
    assert not _battery_passes(lib), "mutant %d (%s: %r) slipped past the pins" % (idx, func, new)
