// dfr_device.cuh -- device-side data structures and kernels of the DFR sort.
//
// The method (paper, Sections "Preliminaries", "Most Significant Digit (MSD)
// Radix Sorts", "Diverting Fast Radix", "Analysis"): partition the keys on
// their most significant digit with a counting sort (count, convert counts to
// indices, deal into a buffer), then recurse on every bucket with the roles
// of input and buffer swapped; a bucket below the diversion threshold N_d is
// diverted to a stable small-bucket sort, and a bucket whose keys are all
// equal is finished.
//
// GPU mapping (one process, one GPU):
//   * Every array is a root segment.  k_root_count reads each key once and
//     produces, per array, the AND and OR of its keys and the histogram of its
//     top byte.  k_root_classify drops constant arrays, diverts small ones and
//     turns the rest into level-0 segments whose digit window sits at the
//     array's highest varying bit (pass skipping, Section LSD).
//   * One level = k_level_count (histogram of the segment's digit, skipped
//     when the root count already has it) + k_scatter (single-pass decoupled
//     look-back over tiles, shared-memory staging so every run of a digit is
//     written contiguously; it also folds the AND/OR of every destination
//     bucket) + k_classify (per bucket: empty, constant, tiny, CTA-sized or
//     large; large buckets become the next level's segments with their window
//     again at the bucket's highest varying bit).
//   * Diverted buckets: tiny ones (<= T_WARP keys) are sorted by one warp
//     inside k_classify; mid-size ones (<= T_CTA) are queued and sorted by
//     k_ctasort, a stable LSD radix sort in shared memory over the bucket's
//     varying bits only.  Constant buckets that ended in the buffer are
//     copied back (small ones by the same queues, large ones by k_copy).
//   * All kernels are persistent: they pull tiles/segments/items from device
//     counters, so the host never waits on the device between kernels and the
//     number of launches is independent of the data and of the array count.
//
// Stability: the in-tile ranking is in element order, tiles are combined in
// tile order by the look-back, and both diversion sorts are stable, so the
// result is the stable sort by key (payloads keep input order on ties).
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

namespace dfr {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int RB = 8;         // radix bits per partition pass
constexpr int M = 1 << RB;    // buckets per partition pass
constexpr uint32_t FLAG_AGG = 1u << 30;    // look-back: tile aggregate only
constexpr uint32_t FLAG_INC = 2u << 30;    // look-back: inclusive prefix
constexpr uint32_t COUNT_MASK = (1u << 30) - 1u;
constexpr int MAXLV = 9;      // levels of control blocks (>= key bits / RB + 1)
constexpr uint32_t T_WARP = 32;  // tiny-bucket threshold (warp sort)

enum : uint32_t { DERR_TIMEOUT = 1u, DERR_BOUNDS = 2u, DERR_CAPACITY = 4u };
constexpr uint32_t NO_OWNER = 0xffffffffu;  // tile-owner entry of a tile that must be skipped
enum : uint32_t { SEG_NEEDS_HIST = 1u };
enum : uint32_t { ITEM_PARITY = 1u, ITEM_COPY = 2u };

struct NoVal {};

// One array to sort (one per batch entry; a plain call has one).
struct ArrDesc {
  void* keys;
  void* buf;
  void* vals;
  void* vbuf;
  uint32_t n;
  uint32_t root_tile_start;  // first root tile of this array (prefix over arrays)
};

// A large segment being partitioned at some level.
struct Seg {
  uint32_t off;         // first key, index into its array
  uint32_t len;         // keys
  uint32_t arr;         // array index
  uint32_t tile_start;  // first global tile of this segment at its level
  uint32_t shift;       // digit = (key >> shift) & (M-1)
  uint32_t parity;      // 0: data in keys, 1: data in buf
  uint32_t flags;       // SEG_NEEDS_HIST
  uint32_t pad;
};

// A mid-size bucket for k_ctasort (or a mid-size constant bucket to copy back).
struct Item {
  uint32_t off;
  uint32_t len;
  uint32_t arr;
  uint32_t info;  // ITEM_PARITY | ITEM_COPY
};

// A large constant bucket that ended in buf and must be written back.
struct CopyItem {
  uint32_t off;
  uint32_t len;
  uint32_t arr;
  uint32_t tile_start;
  unsigned long long value;
};

struct LevelCtl {
  uint32_t nseg;
  uint32_t ntiles;
  uint32_t hist_claim;
  uint32_t scat_claim;
  unsigned long long keys;       // keys dealt at this level
  unsigned long long hist_keys;  // keys re-read by k_level_count
};

struct Ctl {
  uint32_t err;
  uint32_t never;  // a status word nobody sets (forced-timeout test mode)
  uint32_t root_claim;
  uint32_t cta_count;
  uint32_t cta_claim;
  uint32_t copy_count;
  uint32_t copy_tiles;
  uint32_t copy_claim;
  uint32_t key_bytes;
  uint32_t val_bytes;
  uint32_t pad[2];
  unsigned long long n_total;
  unsigned long long cta_buckets, cta_keys;
  unsigned long long tiny_buckets, tiny_keys;
  unsigned long long const_buckets, const_keys;
  unsigned long long copy_keys;
  LevelCtl lv[MAXLV + 1];
};

template <class K>
struct RootAcc {
  K nand;  // OR of ~key  (AND = ~nand; zero-initialised)
  K orv;   // OR of key
  uint32_t hist[M];  // histogram of the top byte
};

// Device view of the workspace; passed by value to every kernel.
struct Ctx {
  Ctl* ctl;
  ArrDesc* arrs;
  uint32_t narr;
  uint32_t spin_limit;
  void* root;  // RootAcc<K>[narr]
  Seg* segs[2];
  uint32_t* hist[2];  // [segcap][M] per level parity
  void* a_nand;       // K[segcap][M]
  void* a_or;         // K[segcap][M]
  uint32_t* tile_owner;
  uint32_t* status;   // [tilecap][M] look-back words
  Item* cta_q;
  CopyItem* copy_q;
  uint32_t* copy_owner;
  uint32_t segcap, tilecap, ctacap, copycap, copytilecap;
  uint32_t force_timeout;
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <class K>
__device__ __forceinline__ uint32_t digit_of(K k, uint32_t shift) {
  return (uint32_t)(k >> shift) & (uint32_t)(M - 1);
}

template <class K>
__device__ __forceinline__ int top_bit(K x) {
  if constexpr (sizeof(K) == 8)
    return x ? 63 - __clzll((long long)x) : -1;
  else
    return x ? 31 - __clz((int)x) : -1;
}

template <class K>
__device__ __forceinline__ int low_bit(K x) {
  if constexpr (sizeof(K) == 8)
    return __ffsll((long long)x) - 1;
  else
    return __ffs((int)x) - 1;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <class K>
__device__ __forceinline__ K ld_stream(const K* p) {
  return __ldcs(p);
}

template <class K>
__device__ __forceinline__ K warp_or(K x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(FULL, x, o);
  return x;
}

template <class K>
__device__ __forceinline__ K group_or(uint32_t mask, K x) {
  if constexpr (sizeof(K) == 8) {
    const uint32_t lo = __reduce_or_sync(mask, (uint32_t)x);
    const uint32_t hi = __reduce_or_sync(mask, (uint32_t)(x >> 32));
    return ((K)hi << 32) | (K)lo;
  } else {
    return __reduce_or_sync(mask, (uint32_t)x);
  }
}

__device__ __forceinline__ void atomic_or_k(uint32_t* p, uint32_t v) { atomicOr(p, v); }
__device__ __forceinline__ void atomic_or_k(unsigned long long* p, unsigned long long v) {
  atomicOr(p, v);
}

// Exclusive scan of one value per thread for threads [0, 256); every thread
// of the block must call it (it synchronises twice).  `sh` holds 8 words.
__device__ __forceinline__ uint32_t scan256(uint32_t v, uint32_t* sh, uint32_t* total) {
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const uint32_t mine = threadIdx.x < 256 ? v : 0u;
  uint32_t x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31 && w < 8) sh[w] = x;
  __syncthreads();
  uint32_t pre = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t t = sh[i];
    pre += (i < (int)w) ? t : 0u;
    tot += t;
  }
  __syncthreads();
  if (total) *total = tot;
  return pre + x - mine;
}

// Warp-aggregated shared-memory histogram increment: lanes holding the same
// digit elect one lane that adds the group's size.
__device__ __forceinline__ void hist_add(uint32_t* h, uint32_t d, bool valid) {
  const uint32_t active = __ballot_sync(FULL, valid);
  if (valid) {
    const uint32_t peers = __match_any_sync(active, d);
    if (lane_id() == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
}

// Stable in-warp ranking of KPT warp-striped items (element i*32+lane of the
// warp's chunk, `wvalid` of them valid): rank[i] = number of earlier elements
// of the warp with the same digit plus the warp's running count of that digit
// (kept in `wh`, this warp's private M counters).
template <class K, int KPT>
__device__ __forceinline__ void warp_rank(const K (&k)[KPT], uint32_t shift, uint32_t wvalid,
                                          uint32_t* wh, uint32_t (&rank)[KPT]) {
  const uint32_t lane = lane_id();
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    const bool valid = (uint32_t)(i * 32) + lane < wvalid;
    const uint32_t active = __ballot_sync(FULL, valid);
    if (valid) {
      const uint32_t d = digit_of(k[i], shift);
      const uint32_t peers = __match_any_sync(active, d);
      const uint32_t leader = 31u - (uint32_t)__clz((int)peers);
      const uint32_t below = (uint32_t)__popc(peers & lt);
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&wh[d], below + 1u);
      base = __shfl_sync(peers, base, (int)leader);
      rank[i] = base + below;
    }
  }
}

// Visit the keys src[lo, hi) with every thread of the block, using 128-bit
// loads for the 16-byte-aligned body.  f(key, valid) is called with
// warp-uniform control flow (invalid lanes pass valid == false).
template <class K, int NT, class F>
__device__ __forceinline__ void block_visit(const K* src, uint32_t lo, uint32_t hi, F&& f) {
  constexpr uint32_t VK = 16 / sizeof(K);
  const K* p = src + lo;
  const uint32_t n = hi - lo;
  uint32_t head = (uint32_t)(((16u - ((uint32_t)(uintptr_t)p & 15u)) & 15u) / sizeof(K));
  if (head > n) head = n;
  {
    const bool valid = threadIdx.x < head;
    const K k = valid ? p[threadIdx.x] : K(0);
    f(k, valid);
  }
  const uint32_t nv = (n - head) / VK;
  const uint4* pv = reinterpret_cast<const uint4*>(p + head);
  for (uint32_t b = 0; b < nv; b += NT) {
    const uint32_t v = b + threadIdx.x;
    const bool valid = v < nv;
    uint4 x = make_uint4(0u, 0u, 0u, 0u);
    if (valid) x = __ldcs(pv + v);
    if constexpr (sizeof(K) == 4) {
      f((K)x.x, valid);
      f((K)x.y, valid);
      f((K)x.z, valid);
      f((K)x.w, valid);
    } else {
      f((K)(((unsigned long long)x.y << 32) | x.x), valid);
      f((K)(((unsigned long long)x.w << 32) | x.z), valid);
    }
  }
  {
    const uint32_t start = head + nv * VK;
    const uint32_t rem = n - start;
    const bool valid = threadIdx.x < rem;
    const K k = valid ? p[start + threadIdx.x] : K(0);
    f(k, valid);
  }
}

// Stable sort of len <= 32 records by one warp (insertion-sort semantics:
// rank = keys below + equal keys earlier).  src and dst may alias.
template <class K, bool KV>
__device__ __forceinline__ void warp_sort_tiny(const K* src, const uint32_t* vsrc, K* dst,
                                               uint32_t* vdst, uint32_t off, uint32_t len) {
  const uint32_t lane = lane_id();
  const bool valid = lane < len;
  const K k = valid ? src[off + lane] : K(0);
  uint32_t v = 0;
  if constexpr (KV) v = valid ? vsrc[off + lane] : 0u;
  uint32_t rank = 0;
  for (uint32_t j = 0; j < len; ++j) {
    const K kj = __shfl_sync(FULL, k, (int)j);
    rank += (kj < k || (kj == k && j < lane)) ? 1u : 0u;
  }
  __syncwarp();
  if (valid) {
    dst[off + rank] = k;
    if constexpr (KV) vdst[off + rank] = v;
  }
}

// ------------------------------------------------------------------ kernels

// Zero the control block and the per-array root accumulators; for a plain
// call also store the single array descriptor.
template <class K>
__global__ void k_init(Ctx c, ArrDesc a0, int write_a0, uint32_t root_words) {
  const uint32_t ctl_words = sizeof(Ctl) / 4;
  uint32_t* cw = reinterpret_cast<uint32_t*>(c.ctl);
  uint32_t* rw = reinterpret_cast<uint32_t*>(c.root);
  const uint32_t total = ctl_words + root_words;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i < ctl_words)
      cw[i] = 0u;
    else
      rw[i - ctl_words] = 0u;
  }
  if (write_a0 && blockIdx.x == 0 && threadIdx.x == 0) c.arrs[0] = a0;
}

// Root count: one read of every key; per array the OR / NOT-AND of its keys
// and the histogram of its top byte (the initial counting pass, Alg. 1).
template <class K, int NT, int TILE>
__global__ void __launch_bounds__(NT) k_root_count(Ctx c, uint32_t root_tiles) {
  __shared__ uint32_t s_h[M];
  __shared__ uint32_t s_t;
  __shared__ K s_or[NT / 32], s_nand[NT / 32];
  RootAcc<K>* root = reinterpret_cast<RootAcc<K>*>(c.root);
  constexpr uint32_t TOP = 8 * sizeof(K) - RB;
  for (;;) {
    if (threadIdx.x == 0) s_t = atomicAdd(&c.ctl->root_claim, 1u);
    for (uint32_t i = threadIdx.x; i < M; i += NT) s_h[i] = 0;
    __syncthreads();
    const uint32_t t = s_t;
    if (t >= root_tiles) break;
    uint32_t lo = 0, hi = c.narr - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (c.arrs[mid].root_tile_start <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const ArrDesc ad = c.arrs[lo];
    const uint32_t j = t - ad.root_tile_start;
    const uint32_t b = j * (uint32_t)TILE;
    const uint32_t e = min(ad.n, b + (uint32_t)TILE);
    K orv = 0, nandv = 0;
    block_visit<K, NT>(reinterpret_cast<const K*>(ad.keys), b, e, [&](K k, bool valid) {
      if (valid) {
        orv |= k;
        nandv |= ~k;
      }
      hist_add(s_h, (uint32_t)(k >> TOP), valid);
    });
    orv = warp_or(orv);
    nandv = warp_or(nandv);
    if (lane_id() == 0) {
      s_or[threadIdx.x >> 5] = orv;
      s_nand[threadIdx.x >> 5] = nandv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      K o = 0, na = 0;
      for (int w = 0; w < NT / 32; ++w) {
        o |= s_or[w];
        na |= s_nand[w];
      }
      atomic_or_k(reinterpret_cast<std::conditional_t<sizeof(K) == 8, unsigned long long, uint32_t>*>(&root[lo].orv),
                  o);
      atomic_or_k(reinterpret_cast<std::conditional_t<sizeof(K) == 8, unsigned long long, uint32_t>*>(&root[lo].nand),
                  na);
    }
    for (uint32_t i = threadIdx.x; i < M; i += NT)
      if (s_h[i]) atomicAdd(&root[lo].hist[i], s_h[i]);
    __syncthreads();
  }
}

// Root classification, one CTA (256 threads) per array.
template <class K, class V, int TILE, int TCTA>
__global__ void __launch_bounds__(256) k_root_classify(Ctx c, unsigned long long n_total) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr int W = 8 * sizeof(K);
  __shared__ uint32_t s_seg, s_ts, s_ok;
  RootAcc<K>* root = reinterpret_cast<RootAcc<K>*>(c.root);
  Ctl* ctl = c.ctl;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->n_total = n_total;
    ctl->key_bytes = sizeof(K);
    ctl->val_bytes = KV ? 4u : 0u;
  }
  for (uint32_t a = blockIdx.x; a < c.narr; a += gridDim.x) {
    const ArrDesc ad = c.arrs[a];
    const uint32_t n = ad.n;
    if (n <= 1) continue;
    const K orv = root[a].orv;
    const K andv = ~root[a].nand;
    if (orv == andv) {
      if (threadIdx.x == 0) {
        atomicAdd(&ctl->const_buckets, 1ull);
        atomicAdd(&ctl->const_keys, (unsigned long long)n);
      }
      continue;
    }
    if (n <= T_WARP) {
      if (threadIdx.x < 32) {
        warp_sort_tiny<K, KV>(reinterpret_cast<const K*>(ad.keys), reinterpret_cast<const uint32_t*>(ad.vals),
                              reinterpret_cast<K*>(ad.keys), reinterpret_cast<uint32_t*>(ad.vals), 0u, n);
        if (threadIdx.x == 0) {
          atomicAdd(&ctl->tiny_buckets, 1ull);
          atomicAdd(&ctl->tiny_keys, (unsigned long long)n);
        }
      }
      continue;
    }
    if (n <= (uint32_t)TCTA) {
      if (threadIdx.x == 0) {
        const uint32_t q = atomicAdd(&ctl->cta_count, 1u);
        if (q < c.ctacap) {
          c.cta_q[q] = Item{0u, n, a, 0u};
          atomicAdd(&ctl->cta_buckets, 1ull);
          atomicAdd(&ctl->cta_keys, (unsigned long long)n);
        } else {
          atomicOr(&ctl->err, DERR_CAPACITY);
        }
      }
      continue;
    }
    const int hb = top_bit<K>(orv ^ andv);
    const bool use_top = hb >= W - RB;
    const uint32_t shift = use_top ? (uint32_t)(W - RB) : (uint32_t)(hb >= RB - 1 ? hb - (RB - 1) : 0);
    const uint32_t nt = (n + TILE - 1) / TILE;
    if (threadIdx.x == 0) {
      const uint32_t s = atomicAdd(&ctl->lv[0].nseg, 1u);
      const uint32_t ts = atomicAdd(&ctl->lv[0].ntiles, nt);
      s_ok = (s < c.segcap && ts + nt <= c.tilecap) ? 1u : 0u;
      if (s_ok) {
        c.segs[0][s] = Seg{0u, n, a, ts, shift, 0u, use_top ? 0u : SEG_NEEDS_HIST, 0u};
        atomicAdd(&ctl->lv[0].keys, (unsigned long long)n);
      } else {
        // Cannot happen with the workspace bounds; stay consistent anyway.
        atomicOr(&ctl->err, DERR_CAPACITY);
        if (s < c.segcap) c.segs[0][s] = Seg{0u, 0u, a, 0u, 0u, 0u, 0u, 0u};
      }
      s_seg = s;
      s_ts = ts;
    }
    __syncthreads();
    {
      const uint32_t s = s_seg, ts = s_ts;
      if (s < c.segcap) c.hist[0][(size_t)s * M + threadIdx.x] = (s_ok && use_top) ? root[a].hist[threadIdx.x] : 0u;
      const uint32_t owner = s_ok ? s : NO_OWNER;
      const uint32_t ntc = ts < c.tilecap ? min(nt, c.tilecap - ts) : 0u;
      for (uint32_t i = threadIdx.x; i < ntc; i += 256) c.tile_owner[ts + i] = owner;
    }
    __syncthreads();
  }
}

// Level count: histogram of each segment's digit (when the root count does not
// already hold it), plus resetting the look-back words of every tile and the
// AND/OR accumulators of every segment of this level.
template <class K, int NT, int TILE>
__global__ void __launch_bounds__(NT) k_level_count(Ctx c, int L) {
  __shared__ uint32_t s_h[M];
  __shared__ uint32_t s_t;
  LevelCtl* lc = &c.ctl->lv[L];
  const uint32_t ntiles = min(lc->ntiles, c.tilecap);
  const Seg* segs = c.segs[L & 1];
  uint32_t* hist = c.hist[L & 1];
  K* a_or = reinterpret_cast<K*>(c.a_or);
  K* a_nand = reinterpret_cast<K*>(c.a_nand);
  for (;;) {
    if (threadIdx.x == 0) s_t = atomicAdd(&lc->hist_claim, 1u);
    for (uint32_t i = threadIdx.x; i < M; i += NT) s_h[i] = 0;
    __syncthreads();
    const uint32_t t = s_t;
    if (t >= ntiles) break;
    const uint32_t s = c.tile_owner[t];
    for (uint32_t i = threadIdx.x; i < M; i += NT) c.status[(size_t)t * M + i] = 0u;
    if (s >= c.segcap) {
      __syncthreads();
      continue;
    }
    const Seg seg = segs[s];
    const uint32_t j = t - seg.tile_start;
    if (j == 0) {
      for (uint32_t i = threadIdx.x; i < M; i += NT) {
        a_or[(size_t)s * M + i] = K(0);
        a_nand[(size_t)s * M + i] = K(0);
      }
    }
    if (seg.flags & SEG_NEEDS_HIST) {
      const ArrDesc ad = c.arrs[seg.arr];
      const K* src = reinterpret_cast<const K*>(seg.parity ? ad.buf : ad.keys);
      const uint32_t b = seg.off + j * (uint32_t)TILE;
      const uint32_t e = min(seg.off + seg.len, b + (uint32_t)TILE);
      const uint32_t shift = seg.shift;
      block_visit<K, NT>(src, b, e, [&](K k, bool valid) { hist_add(s_h, digit_of(k, shift), valid); });
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < M; i += NT)
        if (s_h[i]) atomicAdd(&hist[(size_t)s * M + i], s_h[i]);
      if (threadIdx.x == 0) atomicAdd(&lc->hist_keys, (unsigned long long)(e - b));
    }
    __syncthreads();
  }
}

template <class K, class V, int NT, int KPT>
constexpr size_t scatter_smem_bytes() {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr size_t TILE = (size_t)NT * KPT;
  return TILE * sizeof(K) + (KV ? TILE * 4 : 0) + (size_t)(NT / 32) * M * 4 + 2 * M * 4 + 2 * M * sizeof(K);
}

// Scatter (deal) of one level: every tile of every segment is ranked in
// shared memory, combined with earlier tiles of its segment by a single-pass
// decoupled look-back per digit, staged in digit order and written to the
// other buffer so that each digit's run is contiguous in HBM.
template <class K, class V, int NT, int KPT>
__global__ void __launch_bounds__(NT, 2) k_scatter(Ctx c, int L) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr uint32_t TILE = (uint32_t)NT * KPT;
  constexpr int NW = NT / 32;
  using KA = std::conditional_t<sizeof(K) == 8, unsigned long long, uint32_t>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* s_keys = reinterpret_cast<K*>(smem_raw);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + TILE);
  uint32_t* s_whist = s_vals + (KV ? TILE : 0);
  uint32_t* s_tstart = s_whist + NW * M;
  uint32_t* s_gstart = s_tstart + M;
  K* s_or = reinterpret_cast<K*>(s_gstart + M);
  K* s_nand = s_or + M;
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_t, s_fail;

  LevelCtl* lc = &c.ctl->lv[L];
  const uint32_t ntiles = min(lc->ntiles, c.tilecap);
  const Seg* segs = c.segs[L & 1];
  const uint32_t* hist = c.hist[L & 1];
  K* a_or = reinterpret_cast<K*>(c.a_or);
  K* a_nand = reinterpret_cast<K*>(c.a_nand);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t* wh = s_whist + warp * M;

  for (;;) {
    if (threadIdx.x == 0) {
      s_t = atomicAdd(&lc->scat_claim, 1u);
      s_fail = 0u;
    }
    for (uint32_t i = threadIdx.x; i < (uint32_t)(NW * M); i += NT) s_whist[i] = 0u;
    for (uint32_t i = threadIdx.x; i < M; i += NT) {
      s_or[i] = K(0);
      s_nand[i] = K(0);
    }
    __syncthreads();
    const uint32_t t = s_t;
    if (t >= ntiles) break;
    const uint32_t s = c.tile_owner[t];
    if (s >= c.segcap) {
      __syncthreads();
      continue;
    }
    const Seg seg = segs[s];
    const ArrDesc ad = c.arrs[seg.arr];
    const K* src = reinterpret_cast<const K*>(seg.parity ? ad.buf : ad.keys);
    K* dst = reinterpret_cast<K*>(seg.parity ? ad.keys : ad.buf);
    const uint32_t* vsrc = reinterpret_cast<const uint32_t*>(seg.parity ? ad.vbuf : ad.vals);
    uint32_t* vdst = reinterpret_cast<uint32_t*>(seg.parity ? ad.vals : ad.vbuf);
    const uint32_t j = t - seg.tile_start;
    const uint32_t tb = seg.off + j * TILE;
    const uint32_t cnt = min(TILE, seg.off + seg.len - tb);
    const uint32_t shift = seg.shift;
    const uint32_t wb = warp * 32u * KPT;
    const uint32_t wvalid = cnt > wb ? min(cnt - wb, 32u * KPT) : 0u;

    K k[KPT];
    uint32_t r[KPT];
    uint32_t v[KV ? KPT : 1];
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const uint32_t e = (uint32_t)(i * 32) + lane;
      if (e < wvalid) {
        k[i] = ld_stream(src + tb + wb + e);
        if constexpr (KV) v[i] = ld_stream(vsrc + tb + wb + e);
      } else {
        k[i] = K(0);
      }
      r[i] = 0u;
    }
    warp_rank<K, KPT>(k, shift, wvalid, wh, r);
    __syncthreads();

    // Per digit: tile count, and per-warp counts turned into exclusive offsets.
    uint32_t tcount = 0;
    if (threadIdx.x < M) {
      for (int w2 = 0; w2 < NW; ++w2) {
        const uint32_t x = s_whist[w2 * M + threadIdx.x];
        s_whist[w2 * M + threadIdx.x] = tcount;
        tcount += x;
      }
    }
    uint32_t* st = c.status + (size_t)t * M;
    if (threadIdx.x < M) st_relaxed(st + threadIdx.x, (j == 0 ? FLAG_INC : FLAG_AGG) | tcount);
    const uint32_t tstart = scan256(tcount, s_scan, nullptr);
    const uint32_t hcount = threadIdx.x < M ? hist[(size_t)s * M + threadIdx.x] : 0u;
    const uint32_t bexcl = scan256(hcount, s_scan, nullptr);

    if (threadIdx.x < M) {
      uint32_t excl = 0;
      if (j > 0) {
        bool ok = true;
        uint32_t tp = t - 1;
        for (;;) {
          const uint32_t* p = c.force_timeout ? &c.ctl->never : c.status + (size_t)tp * M + threadIdx.x;
          uint32_t x = ld_relaxed(p);
          uint32_t spins = 0;
          while ((x >> 30) == 0u) {
            if (++spins > c.spin_limit) break;
            if (spins > 64) __nanosleep(64);
            x = ld_relaxed(p);
          }
          if ((x >> 30) == 0u) {
            ok = false;
            break;
          }
          excl += x & COUNT_MASK;
          if ((x & FLAG_INC) || tp == seg.tile_start) break;
          --tp;
        }
        if (!ok) {
          atomicOr(&c.ctl->err, DERR_TIMEOUT);
          s_fail = 1u;
        }
        st_relaxed(st + threadIdx.x, FLAG_INC | ((excl + tcount) & COUNT_MASK));
      }
      s_tstart[threadIdx.x] = tstart;
      s_gstart[threadIdx.x] = seg.off + bexcl + excl;
    }
    __syncthreads();

    // Stage the tile in shared memory in stable digit order.
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      if ((uint32_t)(i * 32) + lane < wvalid) {
        const uint32_t d = digit_of(k[i], shift);
        const uint32_t pos = s_tstart[d] + wh[d] + r[i];
        if (pos < cnt) {
          s_keys[pos] = k[i];
          if constexpr (KV) s_vals[pos] = v[i];
        } else {
          atomicOr(&c.ctl->err, DERR_BOUNDS);
        }
      }
    }
    __syncthreads();

    // Coalesced write-out; fold the AND/OR of every destination bucket.
    const bool fail = s_fail != 0u;
    const uint32_t seg_end = seg.off + seg.len;
    for (uint32_t b0 = 0; b0 < cnt; b0 += NT) {
      const uint32_t e = b0 + threadIdx.x;
      const bool valid = e < cnt;
      const K kk = valid ? s_keys[e] : K(0);
      const uint32_t d = digit_of(kk, shift);
      if (valid && !fail) {
        const uint32_t g = s_gstart[d] + (e - s_tstart[d]);
        if (g >= seg.off && g < seg_end) {
          dst[g] = kk;
          if constexpr (KV) vdst[g] = s_vals[e];
        } else {
          atomicOr(&c.ctl->err, DERR_BOUNDS);
        }
      }
      const uint32_t active = __ballot_sync(FULL, valid);
      if (valid) {
        const uint32_t peers = __match_any_sync(active, d);
        const K o = group_or<K>(peers, kk);
        const K na = group_or<K>(peers, ~kk);
        if (lane == (uint32_t)(__ffs(peers) - 1)) {
          atomic_or_k(reinterpret_cast<KA*>(&s_or[d]), (KA)o);
          atomic_or_k(reinterpret_cast<KA*>(&s_nand[d]), (KA)na);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < M && tcount > 0) {
      atomic_or_k(reinterpret_cast<KA*>(&a_or[(size_t)s * M + threadIdx.x]), (KA)s_or[threadIdx.x]);
      atomic_or_k(reinterpret_cast<KA*>(&a_nand[(size_t)s * M + threadIdx.x]), (KA)s_nand[threadIdx.x]);
    }
    __syncthreads();
  }
}

enum : uint32_t { CLS_NONE = 0, CLS_DONE, CLS_TINY_SORT, CLS_TINY_COPY, CLS_CTA_SORT, CLS_CTA_COPY, CLS_BIG, CLS_BIG_COPY };

// Classification of the buckets of one level, one CTA (256 threads = one per
// digit) per segment: diversion decision by bucket size (threshold N_d,
// Section "Analysis"), constant buckets finished (Section MSD), tiny buckets
// sorted here by warps, large buckets turned into next-level segments.
template <class K, class V, int TILE, int TCTA>
__global__ void __launch_bounds__(256) k_classify(Ctx c, int L) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_tiny_n, s_new_n;
  __shared__ uint32_t s_tiny_off[M], s_tiny_len[M];
  // New next-level segments / large copy items of this segment: owner value
  // for their tile range, histogram slot to clear, first tile, tile count.
  __shared__ uint32_t s_new_owner[M], s_new_zero[M], s_new_ts[M], s_new_nt[M], s_new_copy[M];
  __shared__ unsigned long long s_stat[8];
  Ctl* ctl = c.ctl;
  const uint32_t nseg = min(ctl->lv[L].nseg, c.segcap);
  const Seg* segs = c.segs[L & 1];
  const uint32_t* hist = c.hist[L & 1];
  const K* a_or = reinterpret_cast<const K*>(c.a_or);
  const K* a_nand = reinterpret_cast<const K*>(c.a_nand);
  LevelCtl* ln = &ctl->lv[L + 1];
  Seg* segs_n = c.segs[(L + 1) & 1];
  uint32_t* hist_n = c.hist[(L + 1) & 1];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t d = threadIdx.x;

  for (uint32_t s = blockIdx.x; s < nseg; s += gridDim.x) {
    const Seg seg = segs[s];
    const uint32_t cnt = hist[(size_t)s * M + d];
    const uint32_t excl = scan256(cnt, s_scan, nullptr);
    if (threadIdx.x == 0) {
      s_tiny_n = 0;
      s_new_n = 0;
    }
    if (threadIdx.x < 8) s_stat[threadIdx.x] = 0ull;
    __syncthreads();
    const uint32_t off = seg.off + excl;
    const uint32_t pout = seg.parity ^ 1u;
    const K orv = a_or[(size_t)s * M + d];
    const K andv = ~a_nand[(size_t)s * M + d];
    uint32_t cls = CLS_NONE;
    if (cnt == 0)
      cls = CLS_NONE;
    else if (cnt == 1 || orv == andv)
      cls = !pout ? CLS_DONE : (cnt <= T_WARP ? CLS_TINY_COPY : (cnt <= (uint32_t)TCTA ? CLS_CTA_COPY : CLS_BIG_COPY));
    else if (cnt <= T_WARP)
      cls = CLS_TINY_SORT;
    else if (cnt <= (uint32_t)TCTA)
      cls = CLS_CTA_SORT;
    else
      cls = CLS_BIG;

    // Mid-size buckets: warp-aggregated append to the CTA-sort queue.
    const bool want = cls == CLS_CTA_SORT || cls == CLS_CTA_COPY;
    const uint32_t wm = __ballot_sync(FULL, want);
    if (wm) {
      const uint32_t first = (uint32_t)(__ffs(wm) - 1);
      uint32_t qb = 0;
      if (lane == first) qb = atomicAdd(&ctl->cta_count, (uint32_t)__popc(wm));
      qb = __shfl_sync(FULL, qb, (int)first);
      if (want) {
        const uint32_t q = qb + (uint32_t)__popc(wm & lanemask_lt());
        if (q < c.ctacap)
          c.cta_q[q] = Item{off, cnt, seg.arr, pout | (cls == CLS_CTA_COPY ? ITEM_COPY : 0u)};
        else
          atomicOr(&ctl->err, DERR_CAPACITY);
      }
    }
    if (cls == CLS_TINY_SORT || cls == CLS_TINY_COPY) {
      const uint32_t i = atomicAdd(&s_tiny_n, 1u);
      s_tiny_off[i] = off;
      s_tiny_len[i] = cnt | (cls == CLS_TINY_COPY ? 0x80000000u : 0u);
    }
    if (cls == CLS_BIG) {
      const uint32_t nt = (cnt + (uint32_t)TILE - 1) / (uint32_t)TILE;
      const uint32_t s2 = atomicAdd(&ln->nseg, 1u);
      const uint32_t ts = atomicAdd(&ln->ntiles, nt);
      const bool ok = L + 1 < MAXLV && s2 < c.segcap && ts + nt <= c.tilecap;
      if (ok) {
        const int hb = top_bit<K>(orv ^ andv);
        const uint32_t shift = (uint32_t)(hb >= RB - 1 ? hb - (RB - 1) : 0);
        segs_n[s2] = Seg{off, cnt, seg.arr, ts, shift, pout, SEG_NEEDS_HIST, 0u};
        atomicAdd(&ln->keys, (unsigned long long)cnt);
      } else {
        // Cannot happen with the workspace bounds; keep every slot consistent
        // anyway: an empty segment and tiles nobody processes.
        atomicOr(&ctl->err, DERR_CAPACITY);
        if (s2 < c.segcap) segs_n[s2] = Seg{0u, 0u, seg.arr, 0u, 0u, 0u, 0u, 0u};
      }
      const uint32_t i = atomicAdd(&s_new_n, 1u);
      s_new_owner[i] = ok ? s2 : NO_OWNER;
      s_new_zero[i] = s2 < c.segcap ? s2 : NO_OWNER;
      s_new_ts[i] = ts;
      s_new_nt[i] = ts < c.tilecap ? min(nt, c.tilecap - ts) : 0u;
      s_new_copy[i] = 0u;
    }
    if (cls == CLS_BIG_COPY) {
      const uint32_t nt = (cnt + (uint32_t)TILE - 1) / (uint32_t)TILE;
      const uint32_t q = atomicAdd(&ctl->copy_count, 1u);
      const uint32_t ts = atomicAdd(&ctl->copy_tiles, nt);
      const bool ok = q < c.copycap && ts + nt <= c.copytilecap;
      if (ok)
        c.copy_q[q] = CopyItem{off, cnt, seg.arr, ts, (unsigned long long)andv};
      else
        atomicOr(&ctl->err, DERR_CAPACITY);
      const uint32_t i = atomicAdd(&s_new_n, 1u);
      s_new_owner[i] = ok ? q : NO_OWNER;
      s_new_zero[i] = NO_OWNER;
      s_new_ts[i] = ts;
      s_new_nt[i] = ts < c.copytilecap ? min(nt, c.copytilecap - ts) : 0u;
      s_new_copy[i] = 1u;
    }
    // statistics
    if (cls == CLS_DONE || cls == CLS_TINY_COPY || cls == CLS_CTA_COPY || cls == CLS_BIG_COPY) {
      atomicAdd(&s_stat[0], 1ull);
      atomicAdd(&s_stat[1], (unsigned long long)cnt);
      if (cls != CLS_DONE) atomicAdd(&s_stat[2], (unsigned long long)cnt);
    } else if (cls == CLS_TINY_SORT) {
      atomicAdd(&s_stat[3], 1ull);
      atomicAdd(&s_stat[4], (unsigned long long)cnt);
    } else if (cls == CLS_CTA_SORT) {
      atomicAdd(&s_stat[5], 1ull);
      atomicAdd(&s_stat[6], (unsigned long long)cnt);
    }
    __syncthreads();

    // New segments: clear their histogram slots and fill the tile-owner map.
    const uint32_t nn = s_new_n;
    for (uint32_t i = 0; i < nn; ++i) {
      if (s_new_zero[i] != NO_OWNER) hist_n[(size_t)s_new_zero[i] * M + threadIdx.x] = 0u;
      uint32_t* owner = s_new_copy[i] ? c.copy_owner : c.tile_owner;
      const uint32_t id = s_new_owner[i];
      for (uint32_t x = threadIdx.x; x < s_new_nt[i]; x += 256) owner[s_new_ts[i] + x] = id;
    }
    // Tiny buckets: one warp each.
    const uint32_t tn = s_tiny_n;
    const ArrDesc ad = c.arrs[seg.arr];
    const K* psrc = reinterpret_cast<const K*>(pout ? ad.buf : ad.keys);
    const uint32_t* pvsrc = reinterpret_cast<const uint32_t*>(pout ? ad.vbuf : ad.vals);
    for (uint32_t i = warp; i < tn; i += 8) {
      const uint32_t o = s_tiny_off[i];
      const uint32_t len = s_tiny_len[i] & 0x7fffffffu;
      if (s_tiny_len[i] & 0x80000000u) {
        if (lane < len) {
          reinterpret_cast<K*>(ad.keys)[o + lane] = psrc[o + lane];
          if constexpr (KV) reinterpret_cast<uint32_t*>(ad.vals)[o + lane] = pvsrc[o + lane];
        }
      } else {
        warp_sort_tiny<K, KV>(psrc, pvsrc, reinterpret_cast<K*>(ad.keys), reinterpret_cast<uint32_t*>(ad.vals), o,
                              len);
      }
    }
    if (threadIdx.x == 0) {
      if (s_stat[0]) {
        atomicAdd(&ctl->const_buckets, s_stat[0]);
        atomicAdd(&ctl->const_keys, s_stat[1]);
      }
      if (s_stat[2]) atomicAdd(&ctl->copy_keys, s_stat[2]);
      if (s_stat[3]) {
        atomicAdd(&ctl->tiny_buckets, s_stat[3]);
        atomicAdd(&ctl->tiny_keys, s_stat[4]);
      }
      if (s_stat[5]) {
        atomicAdd(&ctl->cta_buckets, s_stat[5]);
        atomicAdd(&ctl->cta_keys, s_stat[6]);
      }
    }
    __syncthreads();
  }
}

template <class K, class V, int NT, int KPT>
constexpr size_t ctasort_smem_bytes() {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr size_t CAP = (size_t)NT * KPT;
  return CAP * sizeof(K) + (KV ? CAP * 4 : 0) + (size_t)(NT / 32) * M * 4 + M * 4;
}

// Diversion sort of mid-size buckets: one CTA per bucket, a stable LSD radix
// sort in shared memory over the bucket's varying bits only (windows of RB
// bits, constant bits skipped), writing the final order into `keys`.
template <class K, class V, int NT, int KPT>
__global__ void __launch_bounds__(NT, 2) k_ctasort(Ctx c) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr uint32_t CAP = (uint32_t)NT * KPT;
  constexpr int NW = NT / 32;
  constexpr int W = 8 * sizeof(K);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* s_keys = reinterpret_cast<K*>(smem_raw);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + CAP);
  uint32_t* s_whist = s_vals + (KV ? CAP : 0);
  uint32_t* s_dstart = s_whist + NW * M;
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_q;
  __shared__ K s_or[NW], s_nand[NW];
  Ctl* ctl = c.ctl;
  const uint32_t count = min(ctl->cta_count, c.ctacap);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t* wh = s_whist + warp * M;

  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(&ctl->cta_claim, 1u);
    __syncthreads();
    const uint32_t q = s_q;
    if (q >= count) break;
    const Item it = c.cta_q[q];
    const ArrDesc ad = c.arrs[it.arr];
    const bool par = (it.info & ITEM_PARITY) != 0u;
    const K* src = reinterpret_cast<const K*>(par ? ad.buf : ad.keys);
    const uint32_t* vsrc = reinterpret_cast<const uint32_t*>(par ? ad.vbuf : ad.vals);
    K* dst = reinterpret_cast<K*>(ad.keys);
    uint32_t* vdst = reinterpret_cast<uint32_t*>(ad.vals);
    const uint32_t off = it.off, len = min(it.len, CAP);
    if (it.info & ITEM_COPY) {
      for (uint32_t e = threadIdx.x; e < len; e += NT) {
        dst[off + e] = src[off + e];
        if constexpr (KV) vdst[off + e] = vsrc[off + e];
      }
      __syncthreads();
      continue;
    }
    const uint32_t wb = warp * 32u * KPT;
    const uint32_t wvalid = len > wb ? min(len - wb, 32u * KPT) : 0u;
    K k[KPT];
    uint32_t r[KPT];
    uint32_t v[KV ? KPT : 1];
    K orv = 0, nandv = 0;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const uint32_t e = (uint32_t)(i * 32) + lane;
      if (e < wvalid) {
        k[i] = src[off + wb + e];
        if constexpr (KV) v[i] = vsrc[off + wb + e];
        orv |= k[i];
        nandv |= ~k[i];
      } else {
        k[i] = K(0);
      }
      r[i] = 0u;
    }
    orv = warp_or(orv);
    nandv = warp_or(nandv);
    if (lane == 0) {
      s_or[warp] = orv;
      s_nand[warp] = nandv;
    }
    __syncthreads();
    K vm = 0;
    {
      K o = 0, na = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        o |= s_or[w];
        na |= s_nand[w];
      }
      vm = o & na;  // bits that are 1 in some key and 0 in another
    }
    if (vm == K(0)) {
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        const uint32_t e = (uint32_t)(i * 32) + lane;
        if (e < wvalid) {
          dst[off + wb + e] = k[i];
          if constexpr (KV) vdst[off + wb + e] = v[i];
        }
      }
      __syncthreads();
      continue;
    }
    uint32_t sh = (uint32_t)low_bit<K>(vm);
    for (;;) {
      for (uint32_t i = threadIdx.x; i < (uint32_t)(NW * M); i += NT) s_whist[i] = 0u;
      __syncthreads();
      warp_rank<K, KPT>(k, sh, wvalid, wh, r);
      __syncthreads();
      uint32_t tcount = 0;
      if (threadIdx.x < M) {
        for (int w2 = 0; w2 < NW; ++w2) {
          const uint32_t x = s_whist[w2 * M + threadIdx.x];
          s_whist[w2 * M + threadIdx.x] = tcount;
          tcount += x;
        }
      }
      const uint32_t ds = scan256(tcount, s_scan, nullptr);
      if (threadIdx.x < M) s_dstart[threadIdx.x] = ds;
      __syncthreads();
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        if ((uint32_t)(i * 32) + lane < wvalid) {
          const uint32_t d = digit_of(k[i], sh);
          const uint32_t pos = s_dstart[d] + wh[d] + r[i];
          if (pos < len) {
            s_keys[pos] = k[i];
            if constexpr (KV) s_vals[pos] = v[i];
          } else {
            atomicOr(&ctl->err, DERR_BOUNDS);
          }
        }
      }
      __syncthreads();
      const uint32_t nsh = sh + RB;
      const K rest = nsh < (uint32_t)W ? (K)(vm >> nsh) : K(0);
      if (rest == K(0)) break;
      sh = nsh + (uint32_t)low_bit<K>(rest);
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        const uint32_t e = (uint32_t)(i * 32) + lane;
        if (e < wvalid) {
          k[i] = s_keys[wb + e];
          if constexpr (KV) v[i] = s_vals[wb + e];
        }
      }
      __syncthreads();
    }
    for (uint32_t e = threadIdx.x; e < len; e += NT) {
      dst[off + e] = s_keys[e];
      if constexpr (KV) vdst[off + e] = s_vals[e];
    }
    __syncthreads();
  }
}

// Write-back of large constant buckets that ended in buf: the keys are a fill
// of the bucket's single value, the payloads are copied.
template <class K, class V, int NT, int TILE>
__global__ void __launch_bounds__(NT) k_copy(Ctx c) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  __shared__ uint32_t s_t;
  Ctl* ctl = c.ctl;
  const uint32_t ntiles = min(ctl->copy_tiles, c.copytilecap);
  for (;;) {
    if (threadIdx.x == 0) s_t = atomicAdd(&ctl->copy_claim, 1u);
    __syncthreads();
    const uint32_t t = s_t;
    if (t >= ntiles) break;
    const uint32_t q = c.copy_owner[t];
    if (q >= c.copycap) {
      __syncthreads();
      continue;
    }
    const CopyItem it = c.copy_q[q];
    const ArrDesc ad = c.arrs[it.arr];
    const uint32_t j = t - it.tile_start;
    const uint32_t b = it.off + j * (uint32_t)TILE;
    const uint32_t e = min(it.off + it.len, b + (uint32_t)TILE);
    K* dst = reinterpret_cast<K*>(ad.keys);
    const K val = (K)it.value;
    for (uint32_t i = b + threadIdx.x; i < e; i += NT) {
      dst[i] = val;
      if constexpr (KV) reinterpret_cast<uint32_t*>(ad.vals)[i] = reinterpret_cast<const uint32_t*>(ad.vbuf)[i];
    }
    __syncthreads();
  }
}

}  // namespace dfr
