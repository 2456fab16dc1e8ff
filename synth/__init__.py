"""Seeded synthetic inputs for the DFR sort (shared by the tests, the smoke
check and the benchmark; holds none of the sort's arithmetic).

The paper measures on synthetic distributions only: uniform, a wide and a
narrow normal, and Zipf (Section "Experiments", Figures 1-3).  The workloads
here restate those shapes for 32- and 64-bit unsigned keys, each drawn from a
numpy PCG64 stream seeded by the caller, so the CUDA path and the oracle always
see identical arrays generated in the same process.

u32 workloads (2^28 keys each in the full-size plain-sort workload):
  uniform      i.i.d. uniform over [0, 2^32)
  normal       mean 2^31, sd 2^28, Marsaglia polar method (the paper names it in
               Section "Analysis"), rounded half-to-even and clamped to u32
  exponential  mean 2^24, floored, clamped
  zipf         s = 1.1 over ranks 1..2^20 (bounded inverse CDF), ranks mapped
               through a seeded bijection of u32 (2^20 distinct values)
  equal        every key the same seeded value
  sorted       the order statistics of a uniform sample (exponential spacings),
               i.e. a sorted uniform array, without calling a sort
  reverse      the same array, descending
u64 key-value workloads (payload = original index):
  uniform64    i.i.d. uniform over [0, 2^64)
  uniform16    i.i.d. uniform over [0, 2^16) stored as u64 (few effective bits)
  dup90        90% uniform picks among 1024 seeded distinct u64, 10% uniform
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20220729

U32_DISTRIBUTIONS = ("uniform", "normal", "exponential", "zipf", "equal", "sorted", "reverse")
U64_DISTRIBUTIONS = ("uniform64", "uniform16", "dup90")

_CHUNK = 1 << 22
_U32_MAX = (1 << 32) - 1


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_u32(n: int, seed) -> np.ndarray:
    return _rng(seed).integers(0, 1 << 32, size=n, dtype=np.uint32)


def normal_u32(n: int, seed, mean: float = 2.0 ** 31, sd: float = 2.0 ** 28) -> np.ndarray:
    """Marsaglia polar method: draw (u, v) uniform on the square, keep pairs
    inside the unit disc, and emit u*f and v*f with f = sqrt(-2 ln s / s)."""
    g = _rng(seed)
    out = np.empty(n, dtype=np.uint32)
    filled = 0
    while filled < n:
        m = min(_CHUNK, n - filled) // 2 + 64
        u = g.uniform(-1.0, 1.0, m)
        v = g.uniform(-1.0, 1.0, m)
        s = u * u + v * v
        ok = (s > 0.0) & (s < 1.0)
        u, v, s = u[ok], v[ok], s[ok]
        f = np.sqrt(-2.0 * np.log(s) / s)
        z = np.empty(2 * u.size)
        z[0::2] = u * f
        z[1::2] = v * f
        x = np.rint(mean + sd * z)
        np.clip(x, 0.0, float(_U32_MAX), out=x)
        take = min(z.size, n - filled)
        out[filled:filled + take] = x[:take].astype(np.uint32)
        filled += take
    return out


def exponential_u32(n: int, seed, mean: float = 2.0 ** 24) -> np.ndarray:
    g = _rng(seed)
    out = np.empty(n, dtype=np.uint32)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        u = g.random(hi - lo)
        x = np.floor(-mean * np.log1p(-u))
        np.clip(x, 0.0, float(_U32_MAX), out=x)
        out[lo:hi] = x.astype(np.uint32)
    return out


def mix32(x: np.ndarray) -> np.ndarray:
    """A bijection of u32 (xorshift-multiply steps, each invertible), used to
    map Zipf ranks to distinct scattered key values."""
    x = np.asarray(x, dtype=np.uint32).copy()
    x ^= x >> np.uint32(16)
    x *= np.uint32(0x7FEB352D)
    x ^= x >> np.uint32(15)
    x *= np.uint32(0x846CA68B)
    x ^= x >> np.uint32(16)
    return x


class _ZipfTable:
    """Bounded Zipf(s) over ranks 1..K: cumulative table plus a guide table
    (indexed search) for a fast exact inverse CDF."""

    def __init__(self, s: float, k: int, guide_bits: int = 22):
        w = np.arange(1, k + 1, dtype=np.float64) ** (-s)
        self.h = float(w.sum())
        cdf = np.cumsum(w) / self.h
        cdf[-1] = 1.0
        self.cdf = cdf
        self.k = k
        self.g = 1 << guide_bits
        grid = np.arange(self.g, dtype=np.float64) / self.g
        self.guide = np.searchsorted(cdf, grid, side="right").astype(np.int64)

    def ranks(self, u: np.ndarray) -> np.ndarray:
        """0-based rank r with cdf[r-1] <= u < cdf[r]."""
        r = self.guide[np.minimum((u * self.g).astype(np.int64), self.g - 1)]
        todo = np.nonzero(self.cdf[r] <= u)[0]
        while todo.size:
            r[todo] += 1
            todo = todo[self.cdf[r[todo]] <= u[todo]]
        return r


_zipf_cache: dict = {}


def zipf_table(s: float = 1.1, k: int = 1 << 20) -> _ZipfTable:
    key = (s, k)
    if key not in _zipf_cache:
        _zipf_cache[key] = _ZipfTable(s, k)
    return _zipf_cache[key]


def zipf_u32(n: int, seed, s: float = 1.1, nvalues: int = 1 << 20) -> np.ndarray:
    g = _rng(seed)
    tab = zipf_table(s, nvalues)
    salt = np.uint32(g.integers(0, 1 << 32, dtype=np.uint64))
    out = np.empty(n, dtype=np.uint32)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        r = tab.ranks(g.random(hi - lo)).astype(np.uint32)
        out[lo:hi] = mix32(r ^ salt)
    return out


def equal_u32(n: int, seed) -> np.ndarray:
    v = _rng(seed).integers(0, 1 << 32, dtype=np.uint64)
    return np.full(n, v, dtype=np.uint32)


def sorted_u32(n: int, seed) -> np.ndarray:
    """A sorted uniform sample built from exponential spacings: with E_i i.i.d.
    Exp(1) and S_k their partial sums, S_k / S_{n+1} (k = 1..n) are distributed
    as the order statistics of n uniforms.  Nondecreasing by construction."""
    if n == 0:
        return np.empty(0, dtype=np.uint32)
    nchunks = (n + 1 + _CHUNK - 1) // _CHUNK
    ss = np.random.SeedSequence(seed).spawn(nchunks)
    sizes = [min(_CHUNK, n + 1 - c * _CHUNK) for c in range(nchunks)]
    total = 0.0
    for c in range(nchunks):
        total += float(_rng(ss[c]).standard_exponential(sizes[c]).sum())
    out = np.empty(n, dtype=np.uint32)
    run = 0.0
    pos = 0
    for c in range(nchunks):
        e = _rng(ss[c]).standard_exponential(sizes[c])
        cs = np.cumsum(e) + run
        run = float(cs[-1])
        take = min(sizes[c], n - pos)
        x = np.floor(cs[:take] / total * 4294967296.0)
        np.clip(x, 0.0, float(_U32_MAX), out=x)
        out[pos:pos + take] = x.astype(np.uint32)
        pos += take
    return out


def reverse_u32(n: int, seed) -> np.ndarray:
    return sorted_u32(n, seed)[::-1].copy()


_U32_GEN = {
    "uniform": uniform_u32,
    "normal": normal_u32,
    "exponential": exponential_u32,
    "zipf": zipf_u32,
    "equal": equal_u32,
    "sorted": sorted_u32,
    "reverse": reverse_u32,
}


def u32(dist: str, n: int, seed) -> np.ndarray:
    """One u32 workload array by distribution name."""
    return _U32_GEN[dist](n, seed)


def uniform64_u64(n: int, seed) -> np.ndarray:
    return _rng(seed).bit_generator.random_raw(n).astype(np.uint64)


def uniform16_u64(n: int, seed) -> np.ndarray:
    return _rng(seed).integers(0, 1 << 16, size=n, dtype=np.uint64)


def dup90_u64(n: int, seed, ndistinct: int = 1024, pdup: float = 0.9) -> np.ndarray:
    g = _rng(seed)
    vals = np.unique(g.bit_generator.random_raw(ndistinct).astype(np.uint64))
    while vals.size < ndistinct:
        vals = np.unique(np.concatenate([vals, g.bit_generator.random_raw(ndistinct).astype(np.uint64)]))
    vals = vals[:ndistinct]
    g.shuffle(vals)
    out = np.empty(n, dtype=np.uint64)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        m = hi - lo
        dup = g.random(m) < pdup
        pick = vals[g.integers(0, ndistinct, size=m)]
        fresh = g.bit_generator.random_raw(m).astype(np.uint64)
        out[lo:hi] = np.where(dup, pick, fresh)
    return out


_U64_GEN = {"uniform64": uniform64_u64, "uniform16": uniform16_u64, "dup90": dup90_u64}


def u64(dist: str, n: int, seed) -> np.ndarray:
    """One u64 workload array by distribution name."""
    return _U64_GEN[dist](n, seed)


def index_payload(n: int) -> np.ndarray:
    """u32 payload equal to each record's original index."""
    return np.arange(n, dtype=np.uint32)


def batch_sizes(count: int, seed, lo: int = 1 << 8, hi: int = 1 << 20) -> np.ndarray:
    """Array lengths floor(exp(U(ln lo, ln hi)))."""
    g = _rng(seed)
    x = np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), count)))
    return np.clip(x, lo, hi).astype(np.int64)


def batch_u32(count: int, seed, lo: int = 1 << 8, hi: int = 1 << 20):
    """Many independent u32 arrays of log-uniform lengths; each array is
    uniform or Zipf(1.1) by a per-array coin flip.  Returns (arrays, kinds)."""
    sizes = batch_sizes(count, seed, lo, hi)
    g = _rng((seed, 1))
    coins = g.random(count) < 0.5
    ss = np.random.SeedSequence((seed, 2)).spawn(count)
    arrays = []
    kinds = []
    for i in range(count):
        n = int(sizes[i])
        if coins[i]:
            arrays.append(uniform_u32(n, ss[i]))
            kinds.append("uniform")
        else:
            arrays.append(zipf_u32(n, ss[i]))
            kinds.append("zipf")
    return arrays, kinds


# SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), the counter-based
# generator of the served-form request stream; the device library implements
# the same definition (dfr_fill_splitmix64), so any request can be rebuilt here.
_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_SM_M1 = np.uint64(0xBF58476D1CE4E5B9)
_SM_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+n-1 of the SplitMix64 stream seeded with `seed`:
    z = seed + (i+1)*gamma, then the mixing function (uint64, wrapping)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & (2 ** 64 - 1)) + i * _SM_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _SM_M1
        z = (z ^ (z >> np.uint64(27))) * _SM_M2
        return z ^ (z >> np.uint64(31))


def splitmix64_u32(seed: int, n: int) -> np.ndarray:
    """u32 keys: the high halves of the SplitMix64 outputs."""
    return (splitmix64(seed, n) >> np.uint64(32)).astype(np.uint32)


def request_seed(base: int, r: int) -> int:
    """Seed of request r of a served stream with base seed `base`."""
    return ((base & 0xFFFFFFFF) << 32) | (r & 0xFFFFFFFF)


def served_stream(count: int, seed, lo: int = 1 << 10, hi: int = 1 << 24, p_kv: float = 0.3):
    """Sizes (log-uniform over [lo, hi]) and kinds (True = u64 keys with u32
    payloads, with probability p_kv; else u32 keys only) of a request stream."""
    g = _rng((seed, 5))
    x = np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), count)))
    sizes = np.clip(x, lo, hi).astype(np.int64)
    kv = g.random(count) < p_kv
    return sizes, kv
