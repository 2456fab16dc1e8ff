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
//     turns the rest into level-0 segments whose 8-bit digit window sits at
//     the array's highest varying bit (pass skipping, Section LSD).
//   * One level = k_level_count (histogram of each segment's window and the
//     AND/OR of its keys) + k_scatter (single-pass decoupled look-back over
//     tiles, shared-memory staging so every run of a digit is written
//     contiguously) + k_classify (per segment: constant -> finished; window
//     without varying bits -> re-windowed at the highest varying bit without
//     moving data; else per bucket: empty, tiny, CTA-sized or large -> next
//     level).  Every level lowers the window top by at least 8 bits, so a
//     W-bit key needs at most W/8 levels.
//   * Diverted buckets: tiny ones (<= T_WARP keys) are sorted by one warp
//     inside k_classify; mid-size ones (<= T_CTA) are queued and sorted by
//     k_ctasort, an LSD radix sort in shared memory over the bucket's varying
//     bits only.  Constant buckets that ended in the buffer are copied back
//     (small ones through the same queues, large ones by k_copy).
//   * All kernels are persistent: they pull tiles/segments/items from device
//     counters, so the host never waits on the device between kernels and the
//     number of launches is independent of the data and of the array count.
//
// Ranking inside a tile: key-only sorts rank with warp-private shared-memory
// counters (count, then cursor) in whatever order the atomics resolve -- the
// order of equal digits inside a bucket cannot change the output, because
// every bucket is later sorted by its remaining bits and equal keys are
// indistinguishable.  Key-value sorts rank stably (element order, full-warp
// ballot peer matching), tiles are chained in tile order by the look-back and
// the diversion sorts are stable, so payloads keep input order on ties.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "dfr.h"

namespace dfr {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int RB = 8;         // radix bits per partition pass
constexpr int M = 1 << RB;    // buckets per partition pass
constexpr uint32_t FLAG_AGG = 1u << 30;    // look-back: tile aggregate only
constexpr uint32_t FLAG_INC = 2u << 30;    // look-back: inclusive prefix
constexpr uint32_t COUNT_MASK = (1u << 30) - 1u;
constexpr int MAXLV = 12;     // control blocks per level (>= launched levels + 1)
constexpr int EXTRA_LEVELS = 2;  // levels launched beyond key bits / RB (room for narrow windows)
constexpr uint32_t T_WARP = 32;  // tiny-bucket threshold (warp sort)

struct NoVal {};

// The payload type of a sort: V itself (uint32_t or uint64_t), and a
// placeholder for key-only sorts.
template <class V>
struct ValT {
  using type = V;
};
template <>
struct ValT<NoVal> {
  using type = uint32_t;
};
// u32 key-only sorts have two CTA sorts: k_ctasort32 for buckets whose keys
// vary in at most CTA32_SPAN bits (the usual case), the general k_ctasort
// (second queue) for the rest; the classifiers route by a bound on the span.
constexpr uint32_t CTA32_SPAN = 16;
template <class K, class V>
constexpr bool two_cta_queues() {
  return std::is_same<K, uint32_t>::value && std::is_same<V, NoVal>::value;
}

enum : uint32_t { DERR_TIMEOUT = 1u, DERR_BOUNDS = 2u, DERR_CAPACITY = 4u };
enum : uint32_t {
  ERR_SITE_SCATTER_STAGE = 1u, ERR_SITE_SCATTER_WRITE, ERR_SITE_CTASORT_STAGE, ERR_SITE_WARPSORT_STAGE,
  ERR_SITE_LOOKBACK, ERR_SITE_LSD_STAGE, ERR_SITE_LSD_WRITE, ERR_SITE_CLASSIFY, ERR_SITE_GRID_SYNC
};
constexpr uint32_t NO_OWNER = 0xffffffffu;  // tile-owner entry of a tile that must be skipped
// SEG_PREDEALT: a level-0 segment made by the LSD top phase, whose keys are
// already dealt on its window (k_classify only classifies its buckets).
enum : uint32_t { SEG_NEEDS_HIST = 1u, SEG_NEEDS_ANDOR = 2u, SEG_PREDEALT = 4u };
enum : uint32_t { ITEM_PARITY = 1u, ITEM_COPY = 2u };

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
  uint32_t flags;       // SEG_NEEDS_HIST | SEG_NEEDS_ANDOR
  uint32_t bits;        // varying bits the window covers (window = [shift, shift + bits))
  unsigned long long nand;  // OR of ~key over the segment (AND = ~nand)
  unsigned long long orv;   // OR of key over the segment
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
  uint32_t ncnt;  // segments that need the level count (histogram or AND/OR)
  uint32_t pad;
  unsigned long long keys;       // keys dealt at this level
  unsigned long long hist_keys;  // keys read by k_level_count
};

struct Ctl {
  uint32_t err;
  uint32_t never;     // a status word nobody sets (forced-timeout test mode)
  uint32_t err_site;  // first place a device check failed (ERR_SITE_*), 0 if none
  uint32_t pad0;
  uint32_t root_claim;
  uint32_t cta_count;
  uint32_t cta_claim;
  uint32_t copy_count;
  uint32_t copy_tiles;
  uint32_t copy_claim;
  uint32_t key_bytes;
  uint32_t val_bytes;
  uint32_t wq_count;
  uint32_t wq_claim;
  uint32_t cta2_count;  // u32 key-only: buckets the fast CTA sort handed to the general one
  uint32_t cta2_claim;
  unsigned long long n_total;
  unsigned long long cta_buckets, cta_keys;
  unsigned long long wsort_buckets, wsort_keys;
  unsigned long long group_buckets;  // diverted buckets finished by the key-only group pass
  unsigned long long tiny_buckets, tiny_keys;
  unsigned long long const_buckets, const_keys;
  unsigned long long copy_keys;
  // LSD top phase (single-array calls whose plan asks for it)
  uint32_t sched;         // schedule that sorted the top digits: 0 MSD, 1 LSD, 2 LSD with estimated deal
  uint32_t est_abort;     // the estimated deal gave up (an overflow region filled up)
  uint32_t root_skipped;  // the root count did not read the keys (the estimated deal counted them)
  uint32_t est_cap;       // estimated bucket size of the estimated deal
  unsigned long long lsd_keys;      // keys dealt by the LSD passes (both passes)
  unsigned long long est_overflow;  // keys the estimated deal sent to an overflow region
  // one persistent launch (k_persist): grid-barrier arrivals (only grow) and
  // the number of barriers completed; 1 once the kernel ran
  uint32_t gbar_count, gbar_gen, persist, pad1;
  LevelCtl lv[MAXLV + 1];
};

template <class K>
struct RootAcc {
  K nand;  // OR of ~key  (AND = ~nand; zero-initialised)
  K orv;   // OR of key
  uint32_t hist[M];  // histogram of the top byte
};

// State of the LSD top phase of one single-array call (Section "Diverting
// Fast Radix", Algorithms 3-4): the two top digits D0 = bits [W-8, W) and
// D1 = bits [W-16, W-8) are dealt least significant first -- D1 into the
// buffer, then D0 back into the array -- after which the buckets of the
// 16-bit prefix are diverted or recursed on by the MSD levels.  Zeroed by
// k_init.
struct LsdCtl {
  uint32_t on;        // 1: the LSD phase sorts the top digits (else the MSD schedule runs alone)
  uint32_t abort;     // mode 2: an overflow region filled up; the estimated deal is discarded
  uint32_t claim[2];  // tile claims of the two passes
  uint32_t tiles_b;   // tiles of the second pass
  uint32_t pad[3];
  unsigned long long orv, nand;  // mode 2: OR / NOT-AND of the keys, gathered by the estimated deal
  unsigned long long overflow;   // mode 2: keys sent to an overflow region
  uint32_t cur1[M];   // key-only first pass: keys of each D1 digit placed so far (fill cursors)
  uint32_t h0[M];     // D0 histogram (mode 2: counted by the estimated deal)
  uint32_t h1[M];     // mode 1: D1 histogram, counted by the root count
  uint32_t base0[M];  // exclusive scan of h0
  uint32_t base1[M];  // mode 1: exclusive scan of h1
  uint32_t pstart[2 * M + 1];         // first second-pass tile of each piece (and the total)
  uint32_t poff[2 * M], plen[2 * M];  // piece 2d: D1 bucket d in buf; 2d+1: its overflow region
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
  uint32_t* cur[2];   // key-only sorts: [segcap][M] fill cursors per level parity
  uint32_t* tile_owner;
  uint32_t* status;   // key-value sorts: [tilecap][M] look-back words
  Item* cta_q;
  Item* cta_q2;       // u32 key-only: buckets for the general CTA sort (capacity ctacap)
  Item* w_q;          // buckets for the warp sort
  CopyItem* copy_q;
  uint32_t* copy_owner;
  uint32_t segcap, tilecap, ctacap, wqcap, copycap, copytilecap;
  uint32_t force_timeout;
  uint32_t nlev;      // partition levels launched
  // launch plan of this call (none of it changes the result)
  uint32_t target;    // buckets of about this many keys per radix window
  uint32_t max_bits;  // radix bits per level (<= RB)
  uint32_t warp_max;  // runs of at most this many keys go to the warp sort (<= its capacity)
  // LSD top phase of a single-array call (lsd_mode 0 = MSD schedule only)
  uint32_t lsd_mode;      // 0 off, 1 LSD with counted digits, 2 LSD with the estimated first deal
  uint32_t est_cap;       // mode 2: keys per estimated bucket (multiple of 16, M * est_cap <= n)
  uint32_t est_ocap;      // mode 2: overflow slots per bucket (multiple of 16)
  uint32_t lsd_tiles_a;   // tiles of the first pass (the array in TILE-key tiles)
  uint32_t lsd_tiles_b_cap;  // look-back words (per digit) reserved for the second pass
  LsdCtl* lsd;
  uint32_t* lsd_st[2];    // look-back words of the two passes ([tiles][M]; pass 0 only for key-value)
  void* pool_k;           // mode 2: overflow regions, M x est_ocap keys
  void* pool_v;           //          and payloads
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

__device__ __forceinline__ uint32_t warp_max(uint32_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(FULL, x, o));
  return x;
}

__device__ __forceinline__ void atomic_or_u64(unsigned long long* p, unsigned long long v) { atomicOr(p, v); }

// Record a failed device-side check: the error bit and, if it is the first,
// where it happened.
__device__ __forceinline__ void record_error(Ctl* ctl, uint32_t bit, uint32_t site) {
  atomicOr(&ctl->err, bit);
  atomicCAS(&ctl->err_site, 0u, site);
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

// Two exclusive scans at once over threads [0, 256) (one synchronisation
// pair instead of two); every thread of the block must call it.  `sh` holds
// 16 words.
__device__ __forceinline__ void scan256x2(uint32_t a, uint32_t b, uint32_t* sh, uint32_t& ea, uint32_t& eb) {
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const uint32_t ma = threadIdx.x < 256 ? a : 0u, mb = threadIdx.x < 256 ? b : 0u;
  uint32_t x = ma, y = mb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t xa = __shfl_up_sync(FULL, x, o);
    const uint32_t yb = __shfl_up_sync(FULL, y, o);
    if (lane >= (uint32_t)o) {
      x += xa;
      y += yb;
    }
  }
  if (lane == 31 && w < 8) {
    sh[w] = x;
    sh[8 + w] = y;
  }
  __syncthreads();
  uint32_t pa = 0, pb = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i < (int)w) {
      pa += sh[i];
      pb += sh[8 + i];
    }
  }
  __syncthreads();
  ea = pa + x - ma;
  eb = pb + y - mb;
}

// Exclusive scan of one value per thread over the whole block of NT threads
// (NT <= 1024); every thread must call it (it synchronises twice).  `sh`
// holds NT/32 words.  Warp totals are scanned by warp 0.
template <int NT>
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t* sh) {
  constexpr int NW = NT / 32;
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    const uint32_t t = lane < (uint32_t)NW ? sh[lane] : 0u;
    uint32_t u = t;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, u, o);
      if (lane >= (uint32_t)o) u += y;
    }
    if (lane < (uint32_t)NW) sh[lane] = u - t;
  }
  __syncthreads();
  return sh[w] + x - v;
}

// Turn per-warp digit counts cnt[w][d] (NW x M words) into the shared-memory
// position of the first element of digit d from warp w: the exclusive scan of
// the counts taken in (digit, warp) order.  Each of the NT threads scans
// NW * M / NT consecutive entries of that order.
template <int NT, int NW>
__device__ __forceinline__ void scan_digit_warp(uint32_t* cnt, uint32_t* sh) {
  constexpr int E = NW * M / NT;
  static_assert(E >= 1 && NW % E == 0, "entries per thread must split the warps of a digit");
  const uint32_t first = threadIdx.x * E;
  const uint32_t d = first / NW, w0 = first % NW;
  uint32_t x[E];
  uint32_t tot = 0;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const uint32_t c = cnt[(w0 + q) * M + d];
    x[q] = tot;
    tot += c;
  }
  const uint32_t base = block_scan<NT>(tot, sh);
#pragma unroll
  for (int q = 0; q < E; ++q) cnt[(w0 + q) * M + d] = base + x[q];
}

// Add 1 to wh[d] for every valid lane; with RET, return each lane's distinct
// pre-increment value (no particular order among lanes of equal digit).  A
// warp whose valid lanes all hold one digit issues a single atomic.  Every
// lane of the warp must call it.
template <bool RET>
__device__ __forceinline__ uint32_t warp_inc(uint32_t* wh, uint32_t d, bool valid) {
  const uint32_t vmask = __ballot_sync(FULL, valid);
  if (vmask == 0u) return 0u;
  const int src = __ffs((int)vmask) - 1;
  const uint32_t d0 = __shfl_sync(FULL, d, src);
  if (__all_sync(FULL, !valid || d == d0)) {
    uint32_t base = 0;
    if ((int)lane_id() == src) base = atomicAdd(&wh[d0], (uint32_t)__popc(vmask));
    if constexpr (RET) {
      base = __shfl_sync(FULL, base, src);
      return base + (uint32_t)__popc(vmask & lanemask_lt());
    }
    return 0u;
  }
  if (!valid) return 0u;
  if constexpr (RET)
    return atomicAdd(&wh[d], 1u);
  atomicAdd(&wh[d], 1u);
  return 0u;
}

// Peer mask of an RB-bit digit: the lanes holding the same digit as this lane
// (every lane of the warp takes part).  RB ballots, a fixed cost; or, with
// NATIVE, the warp match instruction, which measured 1.4x slower on digits
// spread over the whole range (uniform keys) and faster on few repeated
// digits (the skewed buckets of the CTA sort's LSD passes).
template <bool NATIVE = false>
__device__ __forceinline__ uint32_t match_digit(uint32_t d) {
  if constexpr (NATIVE) {
    return __match_any_sync(FULL, d);
  } else {
    uint32_t m = FULL;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      const bool bit = (d >> b) & 1u;
      const uint32_t bal = __ballot_sync(FULL, bit);
      m &= bit ? bal : ~bal;
    }
    return m;
  }
}

// Stable in-warp ranking of the warp-striped items of one warp (item i of
// lane l is element i*32 + l of the warp's chunk, elements [vlo, vhi) are
// valid, items i >= kpt are absent): rank[i] = the warp's running count of
// the digit (kept in `wh`, this warp's private M counters) plus the number of
// earlier lanes of the same item holding the same digit.  Full-warp
// operations only.  FULLW: every item is valid (no bounds are checked);
// NATIVE: peers by the warp match instruction (see match_digit).
template <class K, int KPT, bool FULLW = false, bool NATIVE = false>
__device__ __forceinline__ void warp_rank_stable(const K (&k)[KPT], uint32_t shift, uint32_t vlo, uint32_t vhi,
                                                 uint32_t kpt, uint32_t* wh, uint32_t (&rank)[KPT]) {
  const uint32_t lane = lane_id();
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    if (FULLW || (uint32_t)i < kpt) {
      const uint32_t e = (uint32_t)(i * 32) + lane;
      const bool valid = FULLW || (e >= vlo && e < vhi);
      const uint32_t vmask = FULLW ? FULL : __ballot_sync(FULL, valid);
      const uint32_t d = digit_of(k[i], shift);
      const uint32_t peers = match_digit<NATIVE>(d) & vmask;
      const uint32_t before = valid ? wh[d] : 0u;
      __syncwarp();
      const uint32_t below = (uint32_t)__popc(peers & lt);
      if (valid && below == 0u) wh[d] = before + (uint32_t)__popc(peers);
      __syncwarp();
      rank[i] = before + below;
    }
  }
}

// Block-wide OR of two values; the result is valid in every thread.  `sh`
// holds 2 * (NT / 32) values of K.  Synchronises twice.
template <class K, int NT>
__device__ __forceinline__ void block_or2(K& a, K& b, K* sh) {
  a = warp_or(a);
  b = warp_or(b);
  if (lane_id() == 0) {
    sh[threadIdx.x >> 5] = a;
    sh[NT / 32 + (threadIdx.x >> 5)] = b;
  }
  __syncthreads();
  K x = 0, y = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    x |= sh[w];
    y |= sh[NT / 32 + w];
  }
  __syncthreads();
  a = x;
  b = y;
}

// Stable sort of len <= 32 records by one warp (insertion-sort semantics:
// rank = keys below + equal keys earlier).  src and dst may alias.
template <class K, bool KV, class VT = uint32_t>
__device__ __forceinline__ void warp_sort_tiny(const K* src, const VT* vsrc, K* dst, VT* vdst, uint32_t off,
                                               uint32_t len) {
  const uint32_t lane = lane_id();
  const bool valid = lane < len;
  const K k = valid ? src[off + lane] : K(0);
  VT v = 0;
  if constexpr (KV) v = valid ? vsrc[off + lane] : VT(0);
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

// Tiles of a segment start at its first key rounded down to a 16-byte
// boundary, so that full tiles can be read with 128-bit loads; the first and
// the last tile are partial.
template <class K>
__device__ __forceinline__ uint32_t tile_base(uint32_t off) {
  return off & ~(uint32_t)(16 / sizeof(K) - 1);
}
template <class K, int TILE>
__device__ __forceinline__ uint32_t seg_tiles(uint32_t off, uint32_t len) {
  return (off + len - tile_base<K>(off) + (uint32_t)TILE - 1) / (uint32_t)TILE;
}

// Digit width for a segment of `len` keys whose varying bits all lie below
// bit `top1`, partitioned at level L of the c.nlev launched levels: wide
// enough that its buckets come out near c.target keys (the radix adapts to
// the segment size; at most c.max_bits), and at least ceil(top1 / levels
// left) so the remaining levels always consume every bit; at most RB.
__device__ __forceinline__ uint32_t window_bits(const Ctx& c, uint32_t len, uint32_t top1, int L) {
  uint32_t b = 1;
  while (b < c.max_bits && (len >> b) > c.target) ++b;
  const uint32_t left = c.nlev > (uint32_t)L ? c.nlev - (uint32_t)L : 1u;
  const uint32_t bmin = (top1 + left - 1) / left;
  if (b < bmin) b = bmin;
  return b > (uint32_t)RB ? (uint32_t)RB : b;
}

// ------------------------------------------------------------------ kernels

// Zero the control block and the per-array root accumulators (and, when
// `z16` > 0, the LSD top phase's control block and look-back words: z16
// 16-byte words from `z`); for a plain call also store the single array
// descriptor.
template <class K>
__global__ void k_init(Ctx c, ArrDesc a0, int write_a0, uint32_t root_words, uint4* z, uint32_t z16) {
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
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < z16; i += gridDim.x * blockDim.x)
    z[i] = make_uint4(0u, 0u, 0u, 0u);
  if (write_a0 && blockIdx.x == 0 && threadIdx.x == 0) c.arrs[0] = a0;
}

// Warp-level streaming count over keys src[lo, hi): 128-bit loads (batches
// of 8 vectors per lane in flight), one shared atomic per key on the warp's
// private counters `wh` at digit (key >> shift) & (M-1) when HIST (lanes
// that hit one counter are serialised by the hardware, which measured faster
// than aggregating them in software on every input, skewed or sorted ones
// included), and OR / NOT-AND of the keys into orv / nandv.
template <class K, bool TWO = false, bool HIST = true>
__device__ __forceinline__ void warp_count_range(const K* src, uint32_t lo, uint32_t hi, uint32_t shift,
                                                 uint32_t* wh, K& orv, K& nandv,
                                                 uint32_t* wh2 = nullptr, uint32_t shift2 = 0) {
  constexpr uint32_t VK = 16 / sizeof(K);
  constexpr int BATCH = 8;
  const uint32_t lane = lane_id();
  const K* p = src + lo;
  const uint32_t n = hi - lo;
  uint32_t head = (uint32_t)(((16u - ((uint32_t)(uintptr_t)p & 15u)) & 15u) / sizeof(K));
  if (head > n) head = n;
  auto one = [&](K k, bool valid) {
    if (valid) {
      orv |= k;
      nandv |= ~k;
    }
    if (HIST && valid) atomicAdd(&wh[digit_of(k, shift)], 1u);
    if constexpr (TWO) {
      if (valid) atomicAdd(&wh2[digit_of(k, shift2)], 1u);
    }
  };
  {
    const bool valid = lane < head;
    one(valid ? p[lane] : K(0), valid);
  }
  const uint32_t nv = (n - head) / VK;
  const uint4* pv = reinterpret_cast<const uint4*>(p + head);
  // whole batches first, with no per-vector bound (the common case), then
  // the last partial batch
  const uint32_t nfull = nv / (32u * BATCH) * (32u * BATCH);
  for (uint32_t b = 0; b < nfull; b += 32u * BATCH) {
    uint4 x[BATCH];
#pragma unroll
    for (int q = 0; q < BATCH; ++q) x[q] = __ldcs(pv + b + (uint32_t)q * 32u + lane);
#pragma unroll
    for (int q = 0; q < BATCH; ++q) {
      if constexpr (sizeof(K) == 4) {
        one((K)x[q].x, true);
        one((K)x[q].y, true);
        one((K)x[q].z, true);
        one((K)x[q].w, true);
      } else {
        one((K)(((unsigned long long)x[q].y << 32) | x[q].x), true);
        one((K)(((unsigned long long)x[q].w << 32) | x[q].z), true);
      }
    }
  }
  for (uint32_t b = nfull; b < nv; b += 32u * BATCH) {
    uint4 x[BATCH];
#pragma unroll
    for (int q = 0; q < BATCH; ++q) {
      const uint32_t v = b + (uint32_t)q * 32u + lane;
      x[q] = v < nv ? __ldcs(pv + v) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int q = 0; q < BATCH; ++q) {
      const bool valid = b + (uint32_t)q * 32u + lane < nv;
      if constexpr (sizeof(K) == 4) {
        one((K)x[q].x, valid);
        one((K)x[q].y, valid);
        one((K)x[q].z, valid);
        one((K)x[q].w, valid);
      } else {
        one((K)(((unsigned long long)x[q].y << 32) | x[q].x), valid);
        one((K)(((unsigned long long)x[q].w << 32) | x[q].z), valid);
      }
    }
  }
  {
    const uint32_t start = head + nv * VK;
    const uint32_t rem = n - start;
    const bool valid = lane < rem;
    one(valid ? p[start + lane] : K(0), valid);
  }
}

// Add a warp's private counters into a global histogram and clear them.
__device__ __forceinline__ void warp_flush_hist(uint32_t* wh, uint32_t* gh) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int i = 0; i < M / 32; ++i) {
    const uint32_t x = wh[i * 32 + lane];
    if (x) {
      atomicAdd(&gh[i * 32 + lane], x);
      wh[i * 32 + lane] = 0u;
    }
  }
  __syncwarp();
}

template <class K>
__device__ __forceinline__ void atomic_or_key(K* p, K v) {
  if constexpr (sizeof(K) == 8)
    atomicOr(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
  else
    atomicOr(reinterpret_cast<uint32_t*>(p), (uint32_t)v);
}

// End of a warp-granular count (root and level counts): the warps of the CTA
// that ended on the same target (an array or a segment) merge their private
// counters and OR / NOT-AND registers, and one warp per target adds the sums
// to the target -- one global atomic per bin and CTA instead of per warp.
// add_hist(target, bin, count), add_ornand(target, or, not_and).  Every
// thread of the block calls it; s_h holds the NW warps' M counters each.
template <class K, int NW, class AddHist, class AddOrNand>
__device__ __forceinline__ void cta_merge_counts(const uint32_t* s_h, uint32_t cur, K orv, K nandv,
                                                 AddHist&& add_hist, AddOrNand&& add_ornand) {
  __shared__ uint32_t s_wcur[NW];
  __shared__ K s_wor[NW], s_wnand[NW];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const K o = warp_or(orv), na = warp_or(nandv);
  if (lane == 0) {
    s_wcur[warp] = cur;
    s_wor[warp] = o;
    s_wnand[warp] = na;
  }
  __syncthreads();
  if (cur == 0xffffffffu) return;
  for (uint32_t w = 0; w < warp; ++w)
    if (s_wcur[w] == cur) return;  // an earlier warp leads this target
  K mo = 0, mna = 0;
  for (uint32_t w = warp; w < (uint32_t)NW; ++w)
    if (s_wcur[w] == cur) {
      mo |= s_wor[w];
      mna |= s_wnand[w];
    }
#pragma unroll
  for (int i = 0; i < M / 32; ++i) {
    const uint32_t bin = (uint32_t)i * 32u + lane;
    uint32_t sum = 0;
    for (uint32_t w = warp; w < (uint32_t)NW; ++w)
      if (s_wcur[w] == cur) sum += s_h[w * M + bin];
    if (sum) add_hist(cur, bin, sum);
  }
  if (lane == 0) add_ornand(cur, mo, mna);
}

// Root count: one read of every key; per array the OR / NOT-AND of its keys
// and the histogram of its top byte (the initial counting pass, Alg. 1).
// Every warp claims whole tiles on its own and keeps private counters and
// OR/NOT-AND registers, flushed only when its next tile belongs to another
// array -- no block-wide barrier.  With TWO (the LSD schedule of a
// single-array call) the same read also counts the second byte into h2: all
// the digit histograms the LSD passes need come from one upfront read (Alg. 4).
// When the estimated deal already counted the keys (LSD mode 2), it does
// nothing.
template <class K, int NT, int TILE, bool TWO>
__device__ __forceinline__ void root_count_body(const Ctx& c, uint32_t root_tiles, uint32_t* h2, uint32_t* s_h,
                                                uint32_t* s_h2, uint32_t sub = 1u) {
  constexpr uint32_t TOP = 8 * sizeof(K) - RB;
  if (c.lsd_mode == 2u && ld_relaxed(&c.lsd->on) != 0u) {
    if (blockIdx.x == 0 && threadIdx.x == 0) c.ctl->root_skipped = 1u;
    return;
  }
  RootAcc<K>* root = reinterpret_cast<RootAcc<K>*>(c.root);
  const uint32_t lane = lane_id();
  uint32_t* wh = s_h + (threadIdx.x >> 5) * M;
  uint32_t* wh2 = s_h2 + (TWO ? (threadIdx.x >> 5) * M : 0u);
#pragma unroll
  for (int i = 0; i < M / 32; ++i) {
    wh[i * 32 + lane] = 0u;
    if constexpr (TWO) wh2[i * 32 + lane] = 0u;
  }
  __syncwarp();
  uint32_t cur = 0xffffffffu;
  K orv = 0, nandv = 0;
  auto flush = [&]() {
    if (cur == 0xffffffffu) return;
    warp_flush_hist(wh, root[cur].hist);
    if constexpr (TWO) warp_flush_hist(wh2, h2);
    const K o = warp_or(orv), na = warp_or(nandv);
    if (lane == 0) {
      atomic_or_key(&root[cur].orv, o);
      atomic_or_key(&root[cur].nand, na);
    }
    orv = 0;
    nandv = 0;
  };
  // a warp claims 1/sub of a tile at a time (sub > 1 spreads a small call's
  // few tiles over more warps)
  const uint32_t part_keys = (uint32_t)TILE / sub;
  for (;;) {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(&c.ctl->root_claim, 1u);
    u = __shfl_sync(FULL, u, 0);
    if (u >= root_tiles * sub) break;
    const uint32_t t = u / sub, part = u - t * sub;
    uint32_t lo = 0, hi = c.narr - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (c.arrs[mid].root_tile_start <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    if (lo != cur) {
      flush();
      cur = lo;
    }
    const ArrDesc ad = c.arrs[lo];
    const uint32_t j = t - ad.root_tile_start;
    const uint32_t b = j * (uint32_t)TILE + part * part_keys;
    const uint32_t e = min(ad.n, b + part_keys);
    if (b < e)
      warp_count_range<K, TWO, true>(reinterpret_cast<const K*>(ad.keys), b, e, TOP, wh, orv, nandv, wh2, TOP - RB);
  }
  if constexpr (TWO) {
    flush();
  } else {
    cta_merge_counts<K, NT / 32>(
        s_h, cur, orv, nandv, [&](uint32_t a, uint32_t bin, uint32_t v) { atomicAdd(&root[a].hist[bin], v); },
        [&](uint32_t a, K o, K na) {
          atomic_or_key(&root[a].orv, o);
          atomic_or_key(&root[a].nand, na);
        });
  }
}

template <class K, int NT, int TILE, bool TWO>
__global__ void __launch_bounds__(NT) k_root_count(Ctx c, uint32_t root_tiles, uint32_t* h2) {
  __shared__ uint32_t s_h[(NT / 32) * M];
  __shared__ uint32_t s_h2[TWO ? (NT / 32) * M : 1];
  root_count_body<K, NT, TILE, TWO>(c, root_tiles, h2, s_h, s_h2);
}

// Key formats: the order-preserving bijection between a key's bits and the
// unsigned value the sort orders by -- two's complement: flip the sign bit;
// IEEE 754 totalOrder: flip every bit of a negative value, set the sign bit
// of a positive one; descending: complement the image.
template <class K>
__device__ __forceinline__ K fmt_to_order(K x, uint32_t fmt) {
  constexpr K SIGN = K(1) << (8 * sizeof(K) - 1);
  const uint32_t base = fmt & 0xFFu;
  if (base == DFR_FMT_SIGNED)
    x ^= SIGN;
  else if (base == DFR_FMT_FLOAT)
    x = (x & SIGN) ? ~x : (x | SIGN);
  return (fmt & DFR_FMT_DESCENDING) ? ~x : x;
}
template <class K>
__device__ __forceinline__ K fmt_from_order(K y, uint32_t fmt) {
  constexpr K SIGN = K(1) << (8 * sizeof(K) - 1);
  const uint32_t base = fmt & 0xFFu;
  if (fmt & DFR_FMT_DESCENDING) y = ~y;
  if (base == DFR_FMT_SIGNED)
    y ^= SIGN;
  else if (base == DFR_FMT_FLOAT)
    y = (y & SIGN) ? (y & ~SIGN) : ~y;
  return y;
}

// Map every key of every array of the call to its image (encode) or back, in
// place: one persistent pass over the root tiles (the arrays of 2+ keys).
// `single`: the one array is a0 (the descriptor table is not in the
// workspace yet); else the arrays are the workspace's descriptor table.
template <class K, int NT, int TILE>
__device__ __forceinline__ void keyfmt_body(const Ctx& c, const ArrDesc& a0, uint32_t single, uint32_t root_tiles,
                                            uint32_t fmt, uint32_t encode) {
  for (uint32_t t = blockIdx.x; t < root_tiles; t += gridDim.x) {
    uint32_t lo = 0;
    if (!single) {
      uint32_t hi = c.narr - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (c.arrs[mid].root_tile_start <= t)
          lo = mid;
        else
          hi = mid - 1;
      }
    }
    const ArrDesc ad = single ? a0 : c.arrs[lo];
    const uint32_t b = (t - ad.root_tile_start) * (uint32_t)TILE;
    const uint32_t e = min(ad.n, b + (uint32_t)TILE);
    K* keys = reinterpret_cast<K*>(ad.keys);
    for (uint32_t i = b + threadIdx.x; i < e; i += NT) keys[i] = encode ? fmt_to_order(keys[i], fmt) : fmt_from_order(keys[i], fmt);
  }
}

template <class K, int NT, int TILE>
__global__ void __launch_bounds__(NT) k_keyfmt(Ctx c, ArrDesc a0, uint32_t single, uint32_t root_tiles, uint32_t fmt,
                                               uint32_t encode) {
  keyfmt_body<K, NT, TILE>(c, a0, single, root_tiles, fmt, encode);
}

// Root classification, one CTA per array (NTB >= 256 threads: one per top
// digit for the histogram copy).
template <class K, class V, int TILE, int TCTA, int WCAP, int NTB>
__device__ __forceinline__ void root_classify_body(const Ctx& c, unsigned long long n_total) {
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
    if (c.lsd_mode != 0u && a == 0u && c.lsd->on != 0u) continue;  // the LSD top phase sorts it
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
        using VT = typename ValT<V>::type;
        warp_sort_tiny<K, KV, VT>(reinterpret_cast<const K*>(ad.keys), reinterpret_cast<const VT*>(ad.vals),
                                  reinterpret_cast<K*>(ad.keys), reinterpret_cast<VT*>(ad.vals), 0u, n);
        if (threadIdx.x == 0) {
          atomicAdd(&ctl->tiny_buckets, 1ull);
          atomicAdd(&ctl->tiny_keys, (unsigned long long)n);
        }
      }
      continue;
    }
    if (n <= (uint32_t)TCTA) {
      if (threadIdx.x == 0) {
        const bool small = n <= c.warp_max;
        // keys varying in more bits than k_ctasort32 sorts go to the general CTA sort
        const K vmk = orv ^ andv;
        const bool wide =
            two_cta_queues<K, V>() && (uint32_t)(top_bit<K>(vmk) - low_bit<K>(vmk) + 1) > CTA32_SPAN;
        uint32_t* qc = small ? &ctl->wq_count : (wide ? &ctl->cta2_count : &ctl->cta_count);
        const uint32_t q = atomicAdd(qc, 1u);
        if (q < (small ? c.wqcap : c.ctacap)) {
          (small ? c.w_q : (wide ? c.cta_q2 : c.cta_q))[q] = Item{0u, n, a, 0u};
          atomicAdd(small ? &ctl->wsort_buckets : &ctl->cta_buckets, 1ull);
          atomicAdd(small ? &ctl->wsort_keys : &ctl->cta_keys, (unsigned long long)n);
        } else {
          atomicOr(&ctl->err, DERR_CAPACITY);
        }
      }
      continue;
    }
    const int hb = top_bit<K>(orv ^ andv);
    const uint32_t b = window_bits(c, n, (uint32_t)hb + 1u, 0);
    const uint32_t shift0 = (uint32_t)hb + 1u > b ? (uint32_t)hb + 1u - b : 0u;
    // a window inside the top byte reuses the root histogram (coarsened)
    const bool use_top = hb >= W - RB;
    const uint32_t shift = use_top ? max(shift0, (uint32_t)(W - RB)) : shift0;
    const uint32_t bits = (uint32_t)hb + 1u - shift;
    const uint32_t nt = (n + TILE - 1) / TILE;
    if (threadIdx.x == 0) {
      const uint32_t s = atomicAdd(&ctl->lv[0].nseg, 1u);
      const uint32_t ts = atomicAdd(&ctl->lv[0].ntiles, nt);
      s_ok = (s < c.segcap && ts + nt <= c.tilecap) ? 1u : 0u;
      if (s_ok) {
        c.segs[0][s] = Seg{0u, n, a, ts, shift, 0u, use_top ? 0u : SEG_NEEDS_HIST, bits,
                           (unsigned long long)root[a].nand, (unsigned long long)orv};
        if (!use_top) atomicAdd(&ctl->lv[0].ncnt, 1u);
      } else {
        // Cannot happen with the workspace bounds; stay consistent anyway.
        atomicOr(&ctl->err, DERR_CAPACITY);
        if (s < c.segcap) c.segs[0][s] = Seg{0u, 0u, a, 0u, 0u, 0u, 0u, 0u, 0ull, 0ull};
      }
      s_seg = s;
      s_ts = ts;
    }
    __syncthreads();
    {
      const uint32_t s = s_seg, ts = s_ts;
      if (s < c.segcap) {
        uint32_t h = 0;
        if (s_ok && use_top) {
          // digit (key >> shift) & 255 = top byte >> (shift - (W - RB))
          const uint32_t sd = shift - (uint32_t)(W - RB);
          const uint32_t x = threadIdx.x;
          if ((x << sd) < (uint32_t)M)
            for (uint32_t y = x << sd; y < ((x + 1) << sd); ++y) h += root[a].hist[y];
        }
        if (threadIdx.x < (uint32_t)M) {
          c.hist[0][(size_t)s * M + threadIdx.x] = h;
          if constexpr (!KV) c.cur[0][(size_t)s * M + threadIdx.x] = 0u;
        }
      }
      const uint32_t owner = s_ok ? s : NO_OWNER;
      const uint32_t ntc = ts < c.tilecap ? min(nt, c.tilecap - ts) : 0u;
      for (uint32_t i = threadIdx.x; i < ntc; i += NTB) c.tile_owner[ts + i] = owner;
    }
    __syncthreads();
  }
}

template <class K, class V, int TILE, int TCTA, int WCAP>
__global__ void __launch_bounds__(256) k_root_classify(Ctx c, unsigned long long n_total) {
  root_classify_body<K, V, TILE, TCTA, WCAP, 256>(c, n_total);
}

// Level count: per segment of this level, the histogram of its digit window
// (unless the root count already holds it) and the AND/OR of its keys (unless
// known); for key-value sorts it also resets the look-back words of every tile
// of the level.  Warp-granular like k_root_count: private counters flushed per
// segment.
template <class K, bool KV, int NT, int TILE>
__device__ __forceinline__ void level_count_body(const Ctx& c, int L, uint32_t* s_h, uint32_t sub = 1u) {
  LevelCtl* lc = &c.ctl->lv[L];
  const uint32_t ntiles = min(lc->ntiles, c.tilecap);
  Seg* segs = ((L & 1) ? c.segs[1] : c.segs[0]);
  uint32_t* hist = ((L & 1) ? c.hist[1] : c.hist[0]);
  const uint32_t lane = lane_id();
  uint32_t* wh = s_h + (threadIdx.x >> 5) * M;
#pragma unroll
  for (int i = 0; i < M / 32; ++i) wh[i * 32 + lane] = 0u;
  __syncwarp();
  uint32_t cur = 0xffffffffu, cur_flags = 0u;
  unsigned long long keys_read = 0;
  K orv = 0, nandv = 0;
  auto flush = [&]() {
    if (cur == 0xffffffffu) return;
    if (cur_flags & SEG_NEEDS_HIST) warp_flush_hist(wh, hist + (size_t)cur * M);
    if (cur_flags & SEG_NEEDS_ANDOR) {
      const K o = warp_or(orv), na = warp_or(nandv);
      if (lane == 0) {
        atomic_or_u64(&segs[cur].orv, (unsigned long long)o);
        atomic_or_u64(&segs[cur].nand, (unsigned long long)na);
      }
    }
    orv = 0;
    nandv = 0;
  };
  // A warp claims 1/sub of a tile at a time (as in the root count).  Claims
  // map to units column by column -- claim q is unit (q mod W) * rows + q / W
  // for W warps -- so that a warp's successive claims, about W apart, take
  // adjacent units, mostly of one segment: its counters then go to the
  // segment's histogram once per run of units, not once per unit.
  const uint32_t part_keys = (uint32_t)TILE / sub;
  const uint32_t units = ntiles * sub;
  const uint32_t nwarps = gridDim.x * (uint32_t)(NT / 32);
  const uint32_t rows = (units + nwarps - 1u) / nwarps;
  for (;;) {
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(&lc->hist_claim, 1u);
    q = __shfl_sync(FULL, q, 0);
    if (q >= nwarps * rows) break;
    const uint32_t u = (q % nwarps) * rows + q / nwarps;
    if (u >= units) continue;
    const uint32_t t = u / sub, part = u - t * sub;
    if constexpr (KV) {
      if (part == 0u) {
#pragma unroll
        for (int i = 0; i < M / 32; ++i) c.status[(size_t)t * M + i * 32 + lane] = 0u;
      }
    }
    const uint32_t s = c.tile_owner[t];
    if (s >= c.segcap) continue;
    const Seg seg = segs[s];
    const uint32_t flags = seg.flags & (SEG_NEEDS_HIST | SEG_NEEDS_ANDOR);
    if (!flags) continue;
    if (s != cur) {
      flush();
      cur = s;
      cur_flags = flags;
    }
    const uint32_t j = t - seg.tile_start;
    const ArrDesc ad = c.arrs[seg.arr];
    const K* src = reinterpret_cast<const K*>(seg.parity ? ad.buf : ad.keys);
    const uint32_t pb = tile_base<K>(seg.off) + j * (uint32_t)TILE + part * part_keys;
    const uint32_t b = max(pb, seg.off);
    const uint32_t e = min(seg.off + seg.len, pb + part_keys);
    if (b >= e) continue;
    if (flags & SEG_NEEDS_HIST)
      warp_count_range<K, false, true>(src, b, e, seg.shift, wh, orv, nandv);
    else
      warp_count_range<K, false, false>(src, b, e, seg.shift, wh, orv, nandv);
    keys_read += e - b;
  }
  cta_merge_counts<K, NT / 32>(
      s_h, cur, orv, nandv,
      [&](uint32_t sg, uint32_t bin, uint32_t v) {
        if (cur_flags & SEG_NEEDS_HIST) atomicAdd(&hist[(size_t)sg * M + bin], v);
      },
      [&](uint32_t sg, K o, K na) {
        if (cur_flags & SEG_NEEDS_ANDOR) {
          atomic_or_u64(&segs[sg].orv, (unsigned long long)o);
          atomic_or_u64(&segs[sg].nand, (unsigned long long)na);
        }
      });
  if (lane == 0 && keys_read) atomicAdd(&lc->hist_keys, keys_read);
}

template <class K, bool KV, int NT, int TILE>
__global__ void __launch_bounds__(NT) k_level_count(Ctx c, int L) {
  __shared__ uint32_t s_h[(NT / 32) * M];
  level_count_body<K, KV, NT, TILE>(c, L, s_h);
}

template <class K, class V, int NT, int KPT>
constexpr size_t scatter_smem_bytes() {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr size_t TILE = (size_t)NT * KPT;
  // staging area; counters (per warp for the stable key-value ranking, one
  // block-wide set otherwise); tile digit starts; global offsets
  return TILE * sizeof(K) + (KV ? TILE * sizeof(typename ValT<V>::type) : 0) +
         (KV ? (size_t)(NT / 32) * M * 4 : (size_t)M * 4) + 2 * M * 4;
}

// CTAs per SM the scatter-shaped kernels are compiled for: key-only tiles of
// up to 16 keys per thread fit three (40 registers); larger key-only tiles,
// key-value tiles and the estimated LSD pass (EST) take two (64 registers);
// blocks of 256 threads take twice as many.
template <class V, int KPT, bool EST, int NT = 512>
constexpr int scatter_min_blocks() {
  return ((std::is_same<V, NoVal>::value && !EST && KPT <= 16) ? 3 : 2) * (NT <= 256 ? 2 : 1);
}

// A segment is dealt at its level unless all its keys are equal or its digit
// window holds no varying bit (then k_classify finishes or re-windows it).
template <class K>
__device__ __forceinline__ bool seg_is_dealt(const Seg& seg) {
  const K vm = (K)seg.orv & (K)seg.nand;
  return vm != K(0) && ((vm >> seg.shift) & (K)(M - 1)) != K(0);
}

// Adaptive key-only ranking (k_scatter and the LSD passes).  One returning
// shared atomic per key on block-wide counters gives each key a distinct slot
// of its digit (the order among equal digits is free); lanes that hit one
// counter are serialised by the hardware.  Two tile kinds are cheaper to rank
// otherwise, and a CTA recognises them from the tile it dealt last:
//  * run mode, after a tile of at most RUN_DIGITS distinct digits (runs of
//    equal digits: sorted or reverse-sorted input, heavy values): each warp's
//    32 x VK consecutive keys are checked first, and a chunk whose keys all
//    share a digit takes its slots with a single atomic;
//  * dominant-digit mode, after a tile whose most frequent digit held at
//    least half its keys (a digit scattered at random, as the exponential's
//    top byte or a heavy Zipf value's bucket): keys of that digit are ranked
//    by one ballot and one atomic per warp item.
// Other tiles skip both checks, which cost more than they save on random
// digits.  The state lives in shared memory; thread 0 updates the modes at
// the top of each tile, the first M threads note the tile's digit counts.
constexpr uint32_t RUN_DIGITS = 8;
constexpr uint32_t NO_DIGIT = 0xffffffffu;

struct TileDigits {
  uint32_t run;    // run mode for this tile
  uint32_t dom;    // dominant digit for this tile, or NO_DIGIT
  uint32_t nd;     // distinct digits of the tile being ranked
  uint32_t dompk;  // max over digits of (count << 8 | digit) of the tile being ranked
  uint32_t nvl;    // keys of the tile being ranked
};

// Thread 0, before the first tile.
__device__ __forceinline__ void adapt_init(TileDigits& a) {
  a.nd = M;
  a.dompk = 0u;
  a.nvl = 1u;
}

// Thread 0, at the top of every tile (after the previous tile's last barrier).
__device__ __forceinline__ void adapt_next(TileDigits& a) {
  a.run = a.nd <= RUN_DIGITS ? 1u : 0u;
  a.dom = ((a.dompk >> 8) * 2u >= a.nvl) ? (a.dompk & 255u) : NO_DIGIT;
  a.nd = 0u;
  a.dompk = 0u;
}

// Threads [0, M) (whole warps), with thread d holding the tile's count of
// digit d; read by thread 0 after the tile's last barrier.
__device__ __forceinline__ void adapt_note(TileDigits& a, uint32_t tcount, uint32_t nvalid) {
  const uint32_t nd = __reduce_add_sync(FULL, tcount ? 1u : 0u);
  if (lane_id() == 0 && nd) atomicAdd(&a.nd, nd);
  const uint32_t pk = __reduce_max_sync(FULL, (tcount << 8) | threadIdx.x);
  if (lane_id() == 0) atomicMax(&a.dompk, pk);
  if (threadIdx.x == 0) a.nvl = nvalid;
}

// Rank the key-only items of one tile: item i = VK*q + u of thread x is
// element VK*(q*NT + x) + u, elements [vlo, vhi) are valid (FULL: the whole
// tile is, and no item is checked); put(i, rank) receives a distinct slot of
// the key's digit on the counters cnt (0 for an invalid item).  Every thread
// of the block calls it.
template <class K, int NT, int KPT, bool FULL = false, class Put>
__device__ __forceinline__ void rank_keys_to(const K (&k)[KPT], Put&& put, uint32_t shift, uint32_t vlo,
                                             uint32_t vhi, uint32_t* cnt, const TileDigits& a) {
  constexpr uint32_t VK = 16 / sizeof(K);
  const uint32_t lane = lane_id();
  if (a.run) {
    // chunk q of a warp = its lanes' items VK*q .. VK*q+VK-1: 32 x VK
    // consecutive keys, lane 0 holding the first and lane 31 the last
#pragma unroll
    for (int q = 0; q < KPT / (int)VK; ++q) {
      const uint32_t e0 = VK * ((uint32_t)q * NT + threadIdx.x);
      const uint32_t dfirst = __shfl_sync(FULL, digit_of(k[q * VK], shift), 0);
      const uint32_t dlast = __shfl_sync(FULL, digit_of(k[q * VK + VK - 1], shift), 31);
      bool one = false;
      if (dfirst == dlast) {
        bool mine = FULL || (e0 >= vlo && e0 + VK <= vhi);
#pragma unroll
        for (int u = 0; u < (int)VK; ++u) mine = mine && digit_of(k[q * VK + u], shift) == dfirst;
        one = __all_sync(FULL, mine);
      }
      if (one) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&cnt[dfirst], 32u * VK);
        base = __shfl_sync(FULL, base, 0) + lane * VK;
#pragma unroll
        for (int u = 0; u < (int)VK; ++u) put(q * VK + u, base + (uint32_t)u);
      } else {
#pragma unroll
        for (int u = 0; u < (int)VK; ++u) {
          const uint32_t e = e0 + (uint32_t)u;
          put(q * VK + u, (e >= vlo && e < vhi) ? atomicAdd(&cnt[digit_of(k[q * VK + u], shift)], 1u) : 0u);
        }
      }
    }
  } else if (a.dom != NO_DIGIT) {
    const uint32_t dom = a.dom;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const uint32_t e = VK * ((uint32_t)(i / VK) * NT + threadIdx.x) + (uint32_t)(i % VK);
      const bool valid = FULL || (e >= vlo && e < vhi);
      const uint32_t d = digit_of(k[i], shift);
      const bool isdom = valid && d == dom;
      const uint32_t m = __ballot_sync(FULL, isdom);
      uint32_t base = 0;
      if (m) {
        const int leader = __ffs((int)m) - 1;
        if ((int)lane == leader) base = atomicAdd(&cnt[dom], (uint32_t)__popc(m));
        base = __shfl_sync(FULL, base, leader);
      }
      put(i, isdom ? base + (uint32_t)__popc(m & lt) : (valid ? atomicAdd(&cnt[d], 1u) : 0u));
    }
  } else if constexpr (FULL) {
#pragma unroll
    for (int i = 0; i < KPT; ++i) put(i, atomicAdd(&cnt[digit_of(k[i], shift)], 1u));
  } else {
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
      const uint32_t e = VK * ((uint32_t)(i / VK) * NT + threadIdx.x) + (uint32_t)(i % VK);
      put(i, (e >= vlo && e < vhi) ? atomicAdd(&cnt[digit_of(k[i], shift)], 1u) : 0u);
    }
  }
}

// As rank_keys_to, with the ranks in r[].
template <class K, int NT, int KPT, bool FULL = false>
__device__ __forceinline__ void rank_keys(const K (&k)[KPT], uint32_t (&r)[KPT], uint32_t shift, uint32_t vlo,
                                          uint32_t vhi, uint32_t* cnt, const TileDigits& a) {
  rank_keys_to<K, NT, KPT, FULL>(k, [&](int i, uint32_t v) { r[i] = v; }, shift, vlo, vhi, cnt, a);
}

// Decoupled look-back for digit d of tile t (one thread per digit): sums the
// counts of the earlier tiles of the segment back to the first inclusive
// prefix, then publishes this tile's inclusive prefix.  Every wait is bounded
// by c.spin_limit; a wait that runs out records DERR_TIMEOUT and sets *fail.
__device__ __forceinline__ uint32_t look_back(const Ctx& c, uint32_t* status, uint32_t t, uint32_t tile_start,
                                              uint32_t d, uint32_t tcount, uint32_t* fail) {
  uint32_t* st = status + (size_t)t * M;
  uint32_t excl = 0;
  if (t > tile_start) {
    bool ok = true;
    uint32_t tp = t - 1;
    for (;;) {
      const uint32_t* p = c.force_timeout ? &c.ctl->never : status + (size_t)tp * M + d;
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
      if ((x & FLAG_INC) || tp == tile_start) break;
      --tp;
    }
    if (!ok) {
      record_error(c.ctl, DERR_TIMEOUT, ERR_SITE_LOOKBACK);
      *fail = 1u;
    }
    st_relaxed(st + d, FLAG_INC | ((excl + tcount) & COUNT_MASK));
  }
  return excl;
}

// Scatter (deal) of one level: every tile of every dealt segment is ranked in
// shared memory, placed inside each bucket of its segment, staged in digit
// order and written to the other buffer, so each digit's run is contiguous in
// HBM.
// Key-only: adaptive ranking (rank_keys: one shared atomic per key, one per
// warp run of a digit, or one ballot per warp item for a dominant digit);
// the tile claims its run of every bucket with one atomic on the bucket's
// fill cursor; full tiles of 16-byte-aligned arrays are read with 128-bit
// loads.
// Key-value: stable per-warp ranking in element order, tiles placed in tile
// order by a single-pass decoupled look-back per digit.
template <class K, class V, int NT, int KPT>
__device__ __forceinline__ void scatter_body(const Ctx& c, int L) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr uint32_t TILE = (uint32_t)NT * KPT;
  constexpr int NW = NT / 32;
  constexpr uint32_t VK = 16 / sizeof(K);
  static_assert(KV || KPT % VK == 0, "vector loads cover whole items");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* s_keys = reinterpret_cast<K*>(smem_raw);
  using VT = typename ValT<V>::type;
  VT* s_vals = reinterpret_cast<VT*>(s_keys + TILE);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_vals + (KV ? TILE : 0));  // KV: [NW][M] per warp; else [M]
  uint32_t* s_tstart = s_cnt + (KV ? NW * M : M);
  uint32_t* s_goff = s_tstart + M;  // global destination of staged element e of digit d = s_goff[d] + e
  __shared__ uint32_t s_scan[16];
  __shared__ uint32_t s_t, s_fail;
  __shared__ TileDigits s_ad;  // key-only adaptive ranking state

  LevelCtl* lc = &c.ctl->lv[L];
  const uint32_t ntiles = min(lc->ntiles, c.tilecap);
  const Seg* segs = ((L & 1) ? c.segs[1] : c.segs[0]);
  const uint32_t* hist = ((L & 1) ? c.hist[1] : c.hist[0]);
  uint32_t* cur = ((L & 1) ? c.cur[1] : c.cur[0]);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) adapt_init(s_ad);
  // Tiles are claimed in increasing order by running CTAs only, so the tile a
  // look-back waits for is always being processed by some resident CTA.
  for (;;) {
    if (threadIdx.x == 0) {
      s_t = atomicAdd(&lc->scat_claim, 1u);
      s_fail = 0u;
      adapt_next(s_ad);
    }
    for (uint32_t i = threadIdx.x; i < (uint32_t)(KV ? NW * M : M); i += NT) s_cnt[i] = 0u;
    __syncthreads();
    const uint32_t t = s_t;
    if (t >= ntiles) break;
    const uint32_t s = c.tile_owner[t];
    if (s >= c.segcap) {
      __syncthreads();
      continue;
    }
    const Seg seg = segs[s];
    if (!seg_is_dealt<K>(seg)) {
      __syncthreads();
      continue;
    }
    const ArrDesc ad = c.arrs[seg.arr];
    const K* src = reinterpret_cast<const K*>(seg.parity ? ad.buf : ad.keys);
    K* dst = reinterpret_cast<K*>(seg.parity ? ad.keys : ad.buf);
    const VT* vsrc = reinterpret_cast<const VT*>(seg.parity ? ad.vbuf : ad.vals);
    VT* vdst = reinterpret_cast<VT*>(seg.parity ? ad.vals : ad.vbuf);
    const uint32_t j = t - seg.tile_start;
    const uint32_t tb = tile_base<K>(seg.off) + j * TILE;         // first element of the tile
    const uint32_t seg_end = seg.off + seg.len;
    const uint32_t vlo = seg.off > tb ? seg.off - tb : 0u;         // valid elements: [vlo, vhi)
    const uint32_t vhi = min(TILE, seg_end - tb);
    const uint32_t nvalid = vhi - vlo;
    const uint32_t shift = seg.shift;

    K k[KPT];
    uint32_t r[KPT];
    VT v[KV ? KPT : 1];
    // a tile the segment covers whole is loaded, ranked and staged without
    // per-item bounds (only a segment's first and last tiles are partial)
    const bool full = vlo == 0u && vhi == TILE;
    auto load_rank = [&](auto full_tag) {
      constexpr bool FL = decltype(full_tag)::value;
      if constexpr (KV) {
        // warp-striped: item i of lane l is element wb + i*32 + l
        const uint32_t wb = warp * 32u * KPT;
#pragma unroll
        for (int i = 0; i < KPT; ++i) {
          const uint32_t e = wb + (uint32_t)(i * 32) + lane;
          k[i] = K(0);
          if (FL || (e >= vlo && e < vhi)) {
            k[i] = ld_stream(src + tb + e);
            v[i] = ld_stream(vsrc + tb + e);
          }
        }
        uint32_t* wh = s_cnt + warp * M;
        const uint32_t wlo = vlo > wb ? vlo - wb : 0u;
        const uint32_t whi = vhi > wb ? min(vhi - wb, 32u * KPT) : 0u;
        warp_rank_stable<K, KPT, FL>(k, shift, wlo, whi, KPT, wh, r);
      } else {
        // item i = VK * q + u of thread x is element VK * (q * NT + x) + u
        const bool vec = ((((uintptr_t)src) & 15u) == 0u) && tb + TILE <= ad.n;
        if (vec) {
          const uint4* pv = reinterpret_cast<const uint4*>(src + tb);
#pragma unroll
          for (int q = 0; q < KPT / (int)VK; ++q) {
            const uint4 x = __ldcs(pv + q * NT + threadIdx.x);
            if constexpr (sizeof(K) == 4) {
              k[q * 4 + 0] = (K)x.x;
              k[q * 4 + 1] = (K)x.y;
              k[q * 4 + 2] = (K)x.z;
              k[q * 4 + 3] = (K)x.w;
            } else {
              k[q * 2 + 0] = (K)(((unsigned long long)x.y << 32) | x.x);
              k[q * 2 + 1] = (K)(((unsigned long long)x.w << 32) | x.z);
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < KPT; ++i) {
            const uint32_t e = VK * ((uint32_t)(i / VK) * NT + threadIdx.x) + (uint32_t)(i % VK);
            k[i] = (e >= vlo && e < vhi) ? src[tb + e] : K(0);
          }
        }
        rank_keys<K, NT, KPT, FL>(k, r, shift, vlo, vhi, s_cnt, s_ad);
      }
    };
    if (full)
      load_rank(std::true_type{});
    else
      load_rank(std::false_type{});
    __syncthreads();

    // Per digit: tile count (KV: per-warp counts become exclusive offsets).
    uint32_t tcount = 0;
    if (threadIdx.x < M) {
      if constexpr (KV) {
        for (int w2 = 0; w2 < NW; ++w2) {
          const uint32_t x = s_cnt[w2 * M + threadIdx.x];
          s_cnt[w2 * M + threadIdx.x] = tcount;
          tcount += x;
        }
      } else {
        tcount = s_cnt[threadIdx.x];
      }
      if constexpr (KV) st_relaxed(c.status + (size_t)t * M + threadIdx.x, (j == 0 ? FLAG_INC : FLAG_AGG) | tcount);
      if constexpr (!KV) adapt_note(s_ad, tcount, nvalid);
    }
    const uint32_t hcount = threadIdx.x < M ? hist[(size_t)s * M + threadIdx.x] : 0u;
    uint32_t tstart, bexcl;
    scan256x2(tcount, hcount, s_scan, tstart, bexcl);
    if (threadIdx.x < M) {
      // Key-value: the tile's place among the segment's tiles in tile order
      // (decoupled look-back), which keeps the deal stable.  Key-only: any
      // order of tiles inside a bucket is fine, so the tile claims its run of
      // each bucket with one atomic on the bucket's fill cursor.
      uint32_t excl;
      if constexpr (KV)
        excl = look_back(c, c.status, t, seg.tile_start, threadIdx.x, tcount, &s_fail);
      else
        excl = tcount ? atomicAdd(&cur[(size_t)s * M + threadIdx.x], tcount) : 0u;
      s_tstart[threadIdx.x] = tstart;
      s_goff[threadIdx.x] = seg.off + bexcl + excl - tstart;
    }
    __syncthreads();

    // Stage the tile in shared memory in digit order (a slot past the tile
    // is skipped and reported once).
    bool bad = false;
    auto stage = [&](auto full_tag) {
      constexpr bool FL = decltype(full_tag)::value;
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        bool valid;
        uint32_t pos;
        const uint32_t d = digit_of(k[i], shift);
        if constexpr (KV) {
          const uint32_t e = warp * 32u * KPT + (uint32_t)(i * 32) + lane;
          valid = FL || (e >= vlo && e < vhi);
          pos = s_tstart[d] + s_cnt[warp * M + d] + r[i];
        } else {
          const uint32_t e = VK * ((uint32_t)(i / VK) * NT + threadIdx.x) + (uint32_t)(i % VK);
          valid = FL || (e >= vlo && e < vhi);
          pos = s_tstart[d] + r[i];
        }
        if (valid) {
          if (pos < nvalid) {
            s_keys[pos] = k[i];
            if constexpr (KV) s_vals[pos] = v[i];
          } else {
            bad = true;
          }
        }
      }
    };
    if (full)
      stage(std::true_type{});
    else
      stage(std::false_type{});
    if (bad) record_error(c.ctl, DERR_BOUNDS, ERR_SITE_SCATTER_STAGE);
    __syncthreads();

    // Coalesced write-out of the staged runs.
    if (s_fail == 0u) {
#pragma unroll 4
      for (uint32_t e = threadIdx.x; e < nvalid; e += NT) {
        const K kk = s_keys[e];
        const uint32_t g = s_goff[digit_of(kk, shift)] + e;
        if (g - seg.off < seg.len) {
          dst[g] = kk;
          if constexpr (KV) vdst[g] = s_vals[e];
        } else {
          record_error(c.ctl, DERR_BOUNDS, ERR_SITE_SCATTER_WRITE);
        }
      }
    }
    __syncthreads();
  }
}

template <class K, class V, int NT, int KPT>
__global__ void __launch_bounds__(NT, (scatter_min_blocks<V, KPT, false, NT>())) k_scatter(Ctx c, int L) {
  scatter_body<K, V, NT, KPT>(c, L);
}

// Inclusive scan with an associative `op` over threads [0, 256), forward
// (thread x gets op(v_0 .. v_x)) or, with REV, backward (op(v_x .. v_255));
// threads >= 256 contribute `ident`.  Every thread of the block calls it (two
// barriers); `sh` holds 8 words.
template <bool REV, class Op>
__device__ __forceinline__ uint32_t scan256_op(uint32_t v, uint32_t ident, Op op, uint32_t* sh) {
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t x = threadIdx.x < 256 ? v : ident;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = REV ? __shfl_down_sync(FULL, x, o) : __shfl_up_sync(FULL, x, o);
    if (REV ? lane + (uint32_t)o < 32u : lane >= (uint32_t)o) x = op(x, y);
  }
  if (w < 8 && lane == (REV ? 0u : 31u)) sh[w] = x;
  __syncthreads();
  uint32_t acc = ident;
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (REV ? i > (int)w : i < (int)w) acc = op(acc, sh[i]);
  __syncthreads();
  return op(acc, x);
}

// Bulk diversion of the small buckets of one segment (Section "Diverting
// Fast Radix": small buckets are sorted together): consecutive small buckets,
// in digit order, are packed greedily into runs of at most T keys -- a run
// starts at a non-empty small bucket and takes the following buckets while
// they fit, ends before a bucket that does not fit (which starts the next
// run) or at a large bucket (the next run starts at the first non-empty small
// bucket after it).  Computed in parallel with one thread per digit: f(x),
// the start of the run after a run that starts at x, comes from prefix sums
// (a binary search for the first bucket that does not fit) and two suffix
// scans; the run starts are the chain x0, f(x0), f(f(x0)), ..., found by
// pointer jumping (8 doublings for 256 digits).  The runs are the ones a
// serial greedy walk gives, written in digit order: offset, length and the
// bound on the run's highest varying bit + 1 (digits of the run that differ
// vary in the window).  cnt[x] = bucket size, LARGE for a large bucket.
// Every thread of the block calls it; `tmp` holds 4 x 256 words.
template <uint32_t T>
__device__ __forceinline__ uint32_t pack_runs(const uint32_t* cnt, const uint32_t* boff, uint32_t shift,
                                              uint32_t* run_off, uint32_t* run_len, uint32_t* run_top,
                                              uint32_t* tmp, uint32_t* sh) {
  constexpr uint32_t LARGE = 0xffffffffu, END = 256u;
  const uint32_t x = threadIdx.x;
  const bool dig = x < 256u;
  const uint32_t cx = dig ? cnt[x] : 0u;
  const bool large = dig && cx == LARGE, start_ok = dig && cx != LARGE && cx != 0u;
  const uint32_t v = (dig && !large) ? cx : 0u;
  uint32_t* P = tmp;          // inclusive prefix sums of the small buckets
  uint32_t* NL = tmp + 256;   // first large bucket >= x (END if none)
  uint32_t* NS = tmp + 512;   // first non-empty small bucket >= x
  uint32_t* PS = tmp + 768;   // last non-empty small bucket <= x, plus one (0 if none)
  auto plus = [](uint32_t a, uint32_t b) { return a + b; };
  auto mn = [](uint32_t a, uint32_t b) { return a < b ? a : b; };
  auto mx = [](uint32_t a, uint32_t b) { return a > b ? a : b; };
  const uint32_t pin = scan256_op<false>(v, 0u, plus, sh);
  const uint32_t nl = scan256_op<true>(large ? x : END, END, mn, sh);
  const uint32_t ns = scan256_op<true>(start_ok ? x : END, END, mn, sh);
  const uint32_t ps = scan256_op<false>(start_ok ? x + 1u : 0u, 0u, mx, sh);
  if (dig) {
    P[x] = pin;
    NL[x] = nl;
    NS[x] = ns;
    PS[x] = ps;
  }
  __syncthreads();
  // a run starting at x: it stops at y (the first bucket after x that is
  // large or no longer fits), and the next run starts at nxt
  uint32_t y = END, nxt = END, rlen = 0, last = 0;
  if (start_ok) {
    const uint32_t lim = pin - v + T;  // prefix sum up to which the run's buckets fit
    uint32_t lo = x + 1u, hi = END;    // first z in [x+1, END) with P[z] > lim, else END
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (P[mid] > lim)
        hi = mid;
      else
        lo = mid + 1u;
    }
    const uint32_t lg = x + 1u < END ? NL[x + 1u] : END;
    y = lo < lg ? lo : lg;
    nxt = y == END ? END : (y == lg ? (y + 1u < END ? NS[y + 1u] : END) : y);
    rlen = P[y - 1u] - (pin - v);  // the small buckets in [x, y)
    last = PS[y - 1u] - 1u;        // the run's last non-empty bucket
  }
  // pointer jumping: after round k every run start within 2^(k+1) steps of
  // the first one is marked
  uint32_t* J = tmp;         // (reuses P: read above, before this barrier)
  uint32_t* MK = tmp + 512;  // (reuses NS)
  const uint32_t x0 = NS[0];
  __syncthreads();
  if (dig) {
    J[x] = nxt;
    MK[x] = (x == x0) ? 1u : 0u;
  }
  __syncthreads();
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    uint32_t j = dig ? J[x] : END;
    if (dig && MK[x] && j < END) MK[j] = 1u;
    const uint32_t jj = (dig && j < END) ? J[j] : END;
    __syncthreads();
    if (dig) J[x] = jj;
    __syncthreads();
  }
  const bool is_start = dig && MK[x] != 0u;
  uint32_t nrun = 0;
  const uint32_t idx = scan256(is_start ? 1u : 0u, sh, &nrun);
  if (is_start) {
    run_off[idx] = boff[x];
    run_len[idx] = rlen;
    run_top[idx] = shift + (x == last ? 0u : 32u - (uint32_t)__clz((int)(x ^ last)));
  }
  __syncthreads();
  return nrun;
}

// Classification of one level, one CTA (256 threads = one per digit) per
// segment.  A constant segment is finished (copied back if it sits in the
// buffer); a segment whose window held no varying bit is passed to the next
// level with its window at the highest varying bit, without moving data; for
// a dealt segment every bucket is classified by size against the diversion
// thresholds (Section "Analysis", N_d): tiny buckets are sorted here by warps,
// mid-size ones queued for k_ctasort, large ones become next-level segments.
template <class K, class V, int TILE, int TCTA, int WCAP, int NTB>
__device__ __forceinline__ void classify_body(const Ctx& c, int L) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_tiny_n, s_new_n;
  __shared__ uint32_t s_tiny_off[M], s_tiny_len[M];
  // New next-level segments / large copy items of this segment: owner value
  // for their tile range, histogram slot to clear, first tile, tile count.
  __shared__ uint32_t s_new_owner[M], s_new_zero[M], s_new_ts[M], s_new_nt[M], s_new_copy[M];
  // per-segment statistics (every count fits 32 bits: a segment holds < 2^30
  // keys); native 32-bit shared atomics, added to the 64-bit totals once
  __shared__ uint32_t s_stat[10];
  __shared__ __align__(16) uint32_t s_bcnt[M];
  __shared__ uint32_t s_boff[M], s_run_off[M], s_run_len[M];
  __shared__ uint32_t s_nrun, s_qn[3], s_qbase[3];
  __shared__ uint32_t s_run_top[M];  // bound on each run's highest varying bit + 1
  __shared__ uint32_t s_pack[4 * M];  // pack_runs' prefix sums, suffix scans and jump pointers
  Ctl* ctl = c.ctl;
  const uint32_t nseg = min(ctl->lv[L].nseg, c.segcap);
  const Seg* segs = ((L & 1) ? c.segs[1] : c.segs[0]);
  const uint32_t* hist = ((L & 1) ? c.hist[1] : c.hist[0]);
  LevelCtl* ln = &ctl->lv[L + 1];
  Seg* segs_n = ((L & 1) ? c.segs[0] : c.segs[1]);
  uint32_t* hist_n = ((L & 1) ? c.hist[0] : c.hist[1]);
  uint32_t* cur_n = ((L & 1) ? c.cur[0] : c.cur[1]);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t d = threadIdx.x;
  const bool dig = d < (uint32_t)M;  // one thread per digit

  // Append one next-level segment and record its tile range for the owner
  // fill.  Called by one thread.
  auto add_big = [&](uint32_t off, uint32_t cnt, uint32_t arr, uint32_t shift, uint32_t bits, uint32_t parity,
                     uint32_t flags, unsigned long long nand, unsigned long long orv) {
    const uint32_t nt = seg_tiles<K, TILE>(off, cnt);
    const uint32_t s2 = atomicAdd(&ln->nseg, 1u);
    const uint32_t ts = atomicAdd(&ln->ntiles, nt);
    const bool ok = L + 1 < MAXLV && s2 < c.segcap && ts + nt <= c.tilecap;
    if (ok) {
      segs_n[s2] = Seg{off, cnt, arr, ts, shift, parity, flags, bits, nand, orv};
      if (flags & (SEG_NEEDS_HIST | SEG_NEEDS_ANDOR)) atomicAdd(&ln->ncnt, 1u);
    } else {
      // Cannot happen with the workspace bounds; keep every slot consistent
      // anyway: an empty segment and tiles nobody processes.
      atomicOr(&ctl->err, DERR_CAPACITY);
      if (s2 < c.segcap) segs_n[s2] = Seg{0u, 0u, arr, 0u, 0u, 0u, 0u, 0u, 0ull, 0ull};
    }
    const uint32_t i = atomicAdd(&s_new_n, 1u);
    s_new_owner[i] = ok ? s2 : NO_OWNER;
    s_new_zero[i] = s2 < c.segcap ? s2 : NO_OWNER;
    s_new_ts[i] = ts;
    s_new_nt[i] = ts < c.tilecap ? min(nt, c.tilecap - ts) : 0u;
    s_new_copy[i] = 0u;
  };
  // Append one large copy item (constant keys in buf) and its tile range.
  auto add_copy = [&](uint32_t off, uint32_t cnt, uint32_t arr, unsigned long long value) {
    const uint32_t nt = (cnt + (uint32_t)TILE - 1) / (uint32_t)TILE;
    const uint32_t q = atomicAdd(&ctl->copy_count, 1u);
    const uint32_t ts = atomicAdd(&ctl->copy_tiles, nt);
    const bool ok = q < c.copycap && ts + nt <= c.copytilecap;
    if (ok)
      c.copy_q[q] = CopyItem{off, cnt, arr, ts, value};
    else
      atomicOr(&ctl->err, DERR_CAPACITY);
    const uint32_t i = atomicAdd(&s_new_n, 1u);
    s_new_owner[i] = ok ? q : NO_OWNER;
    s_new_zero[i] = NO_OWNER;
    s_new_ts[i] = ts;
    s_new_nt[i] = ts < c.copytilecap ? min(nt, c.copytilecap - ts) : 0u;
    s_new_copy[i] = 1u;
  };

  for (uint32_t s = blockIdx.x; s < nseg; s += gridDim.x) {
    const Seg seg = segs[s];
    if (threadIdx.x == 0) {
      s_tiny_n = 0;
      s_new_n = 0;
    }
    if (threadIdx.x < 10) s_stat[threadIdx.x] = 0u;
    __syncthreads();
    const K vm = (K)seg.orv & (K)seg.nand;
    const bool dealt = vm != K(0) && ((vm >> seg.shift) & (K)(M - 1)) != K(0);
    if (!dealt) {
      if (threadIdx.x == 0 && seg.len > 0) {
        if (vm == K(0)) {
          // every key of the segment is equal: finished where it lies
          s_stat[0] = 1u;
          s_stat[1] = seg.len;
          if (seg.parity) {
            s_stat[2] = seg.len;
            if (seg.len <= (uint32_t)TCTA) {
              const uint32_t q = atomicAdd(&ctl->cta_count, 1u);
              if (q < c.ctacap)
                c.cta_q[q] = Item{seg.off, seg.len, seg.arr, ITEM_PARITY | ITEM_COPY};
              else
                atomicOr(&ctl->err, DERR_CAPACITY);
            } else {
              add_copy(seg.off, seg.len, seg.arr, (unsigned long long)(K)seg.orv);
            }
          }
        } else {
          // the window held no varying bit: move it down to the highest one
          const uint32_t top1 = (uint32_t)top_bit<K>(vm) + 1u;
          const uint32_t b = window_bits(c, seg.len, top1, L + 1);
          const uint32_t shift = top1 > b ? top1 - b : 0u;
          add_big(seg.off, seg.len, seg.arr, shift, top1 - shift, seg.parity, SEG_NEEDS_HIST, seg.nand, seg.orv);
        }
      }
    } else {
      const uint32_t cnt = dig ? hist[(size_t)s * M + d] : 0u;
      uint32_t tot = 0;
      const uint32_t excl = scan256(cnt, s_scan, &tot);
      // A histogram that does not add up to the segment (only after a failed
      // device check upstream) must not become buckets: skip the segment.
      if (tot != seg.len) {
        if (threadIdx.x == 0) record_error(ctl, DERR_BOUNDS, ERR_SITE_CLASSIFY);
      } else {
        if (threadIdx.x == 0 && !(seg.flags & SEG_PREDEALT)) atomicAdd(&ctl->lv[L].keys, (unsigned long long)seg.len);
        const uint32_t off = seg.off + excl;
        const uint32_t pout = seg.parity ^ 1u;
        // Large buckets go to the next level (or, when every bit is consumed,
        // they are constant and only move back if they sit in the buffer).
        if (cnt > (uint32_t)TCTA) {
          if (seg.shift == 0u) {
            atomicAdd(&s_stat[0], 1u);
            atomicAdd(&s_stat[1], cnt);
            if (pout) {
              atomicAdd(&s_stat[2], cnt);
              // the bucket's keys are the segment prefix with this digit
              const K val = (K)(((K)seg.orv & ~(((K)(M - 1)) << seg.shift)) | ((K)d << seg.shift));
              add_copy(off, cnt, seg.arr, (unsigned long long)val);
            }
          } else {
            // the bucket's varying bits all lie below the parent's window
            const uint32_t b = window_bits(c, cnt, seg.shift, L + 1);
            const uint32_t shift = seg.shift > b ? seg.shift - b : 0u;
            add_big(off, cnt, seg.arr, shift, seg.shift - shift, pout, SEG_NEEDS_HIST | SEG_NEEDS_ANDOR, 0ull, 0ull);
          }
        }
        // Small buckets are diverted in bulk: consecutive ones (in digit order,
        // hence adjacent in memory and ordered) are joined into runs of at
        // most TCTA keys and each run is sorted as one item -- sorting the run
        // sorts every bucket in it, and equal keys never span two buckets.
        if (dig) {
          s_bcnt[d] = cnt > (uint32_t)TCTA ? 0xffffffffu : cnt;
          s_boff[d] = off;
        }
        __syncthreads();
        {
          const uint32_t nr = pack_runs<(uint32_t)TCTA>(s_bcnt, s_boff, seg.shift, s_run_off, s_run_len, s_run_top,
                                                        s_pack, s_scan);
          if (threadIdx.x == 0) {
            s_nrun = nr;
            s_qn[0] = 0;
            s_qn[1] = 0;
            s_qn[2] = 0;
          }
        }
        __syncthreads();
        const uint32_t nr = s_nrun;
        // run classes: single key, tiny (warp sort here), warp-sort queue, CTA queue
        uint32_t rcls = 0, rloc = 0, rlen = 0, roff = 0;
        bool rcopy = false;
        if (threadIdx.x < nr) {
          roff = s_run_off[threadIdx.x];
          rlen = s_run_len[threadIdx.x];
          if (seg.shift == 0u) {
            // The window reached bit 0: every bucket of the run holds one
            // repeated key (§MSD).  The run is final where it lies, or only
            // moves back from the buffer: the tiny pass copies up to a warp of
            // keys, a CTA-queue copy item the rest.
            atomicAdd(&s_stat[0], 1u);
            atomicAdd(&s_stat[1], rlen);
            if (pout) {
              atomicAdd(&s_stat[2], rlen);
              if (rlen <= T_WARP) {
                rcls = 1;
              } else {
                rcls = 4;
                rcopy = true;
                rloc = atomicAdd(&s_qn[1], 1u);
              }
            }
          } else if (rlen == 1u) {
            atomicAdd(&s_stat[0], 1u);
            atomicAdd(&s_stat[1], 1u);
            if (pout) {
              atomicAdd(&s_stat[2], 1u);
              rcls = 1;  // a single key in the buffer: copied by the tiny pass
            }
          } else if (rlen <= T_WARP) {
            rcls = 2;
            atomicAdd(&s_stat[3], 1u);
            atomicAdd(&s_stat[4], rlen);
          } else if (rlen <= c.warp_max) {
            rcls = 3;
            rloc = atomicAdd(&s_qn[0], 1u);
            atomicAdd(&s_stat[8], 1u);
            atomicAdd(&s_stat[7], rlen);
          } else {
            // a run whose keys may vary in more bits than k_ctasort32 sorts
            // goes to the general CTA sort's queue
            rcls = (two_cta_queues<K, V>() && s_run_top[threadIdx.x] > CTA32_SPAN) ? 5 : 4;
            rloc = atomicAdd(&s_qn[rcls - 3], 1u);
            atomicAdd(&s_stat[5], 1u);
            atomicAdd(&s_stat[6], rlen);
          }
          if (rcls == 1 || rcls == 2) {
            const uint32_t i = atomicAdd(&s_tiny_n, 1u);
            s_tiny_off[i] = roff;
            s_tiny_len[i] = rlen | (rcls == 1 ? 0x80000000u : 0u);
          }
        }
        __syncthreads();
        if (threadIdx.x < 3u) {  // the three queues' slots, claimed side by side
          const uint32_t qn = s_qn[threadIdx.x];
          uint32_t* qc = threadIdx.x == 0u ? &ctl->wq_count : (threadIdx.x == 1u ? &ctl->cta_count : &ctl->cta2_count);
          s_qbase[threadIdx.x] = qn ? atomicAdd(qc, qn) : 0u;
        }
        __syncthreads();
        if (rcls >= 3) {
          const uint32_t q = s_qbase[rcls - 3] + rloc;
          Item* qa = rcls == 3 ? c.w_q : (rcls == 4 ? c.cta_q : c.cta_q2);
          if (q < (rcls == 3 ? c.wqcap : c.ctacap))
            qa[q] = Item{roff, rlen, seg.arr, pout | (rcopy ? ITEM_COPY : 0u)};
          else
            atomicOr(&ctl->err, DERR_CAPACITY);
        }
      }
    }
    __syncthreads();

    // New segments / copy items: clear histogram slots, fill tile-owner maps.
    const uint32_t nn = s_new_n;
    for (uint32_t i = 0; i < nn; ++i) {
      if (dig && s_new_zero[i] != NO_OWNER) {
        hist_n[(size_t)s_new_zero[i] * M + threadIdx.x] = 0u;
        if constexpr (!KV) cur_n[(size_t)s_new_zero[i] * M + threadIdx.x] = 0u;
      }
      uint32_t* owner = s_new_copy[i] ? c.copy_owner : c.tile_owner;
      const uint32_t id = s_new_owner[i];
      for (uint32_t x = threadIdx.x; x < s_new_nt[i]; x += NTB) owner[s_new_ts[i] + x] = id;
    }
    // Tiny buckets: one warp each.
    const uint32_t tn = s_tiny_n;
    if (tn) {
      const ArrDesc ad = c.arrs[seg.arr];
      const uint32_t pout = seg.parity ^ 1u;
      const K* psrc = reinterpret_cast<const K*>(pout ? ad.buf : ad.keys);
      using VT = typename ValT<V>::type;
      const VT* pvsrc = reinterpret_cast<const VT*>(pout ? ad.vbuf : ad.vals);
      for (uint32_t i = warp; i < tn; i += NTB / 32) {
        const uint32_t o = s_tiny_off[i];
        const uint32_t len = s_tiny_len[i] & 0x7fffffffu;
        if (s_tiny_len[i] & 0x80000000u) {
          if (lane < len) {
            reinterpret_cast<K*>(ad.keys)[o + lane] = psrc[o + lane];
            if constexpr (KV) reinterpret_cast<VT*>(ad.vals)[o + lane] = pvsrc[o + lane];
          }
        } else {
          warp_sort_tiny<K, KV, VT>(psrc, pvsrc, reinterpret_cast<K*>(ad.keys), reinterpret_cast<VT*>(ad.vals),
                                o, len);
        }
      }
    }
    if (threadIdx.x == 0) {
      if (s_stat[0]) {
        atomicAdd(&ctl->const_buckets, (unsigned long long)s_stat[0]);
        atomicAdd(&ctl->const_keys, (unsigned long long)s_stat[1]);
      }
      if (s_stat[2]) atomicAdd(&ctl->copy_keys, (unsigned long long)s_stat[2]);
      if (s_stat[3]) {
        atomicAdd(&ctl->tiny_buckets, (unsigned long long)s_stat[3]);
        atomicAdd(&ctl->tiny_keys, (unsigned long long)s_stat[4]);
      }
      if (s_stat[5]) {
        atomicAdd(&ctl->cta_buckets, (unsigned long long)s_stat[5]);
        atomicAdd(&ctl->cta_keys, (unsigned long long)s_stat[6]);
      }
      if (s_stat[7]) {
        atomicAdd(&ctl->wsort_keys, (unsigned long long)s_stat[7]);
        atomicAdd(&ctl->wsort_buckets, (unsigned long long)s_stat[8]);
      }
    }
    __syncthreads();
  }
}

template <class K, class V, int TILE, int TCTA, int WCAP>
__global__ void __launch_bounds__(256) k_classify(Ctx c, int L) {
  classify_body<K, V, TILE, TCTA, WCAP, 256>(c, L);
}

// Diversion sort of mid-size buckets: one CTA per bucket, writing the final
// order into `keys`.  Every warp holds KPTA keys per lane (KPTA = the bucket
// size over the block rounded up to a power of two, so the item loops are
// fully unrolled).
//  * Key-only buckets: one counting pass on the top (at most GB) varying bits
//    groups the keys by those bits; if that covered every varying bit the
//    groups hold equal keys and the bucket is sorted, otherwise each key is
//    placed inside its (small) group by the rank an insertion sort would give
//    it (keys below it, plus equal keys stored before it).  A group of more
//    than GMAX keys (skewed bucket) keeps its staged order if it holds one
//    repeated key; a bucket with a larger group of mixed keys falls back to
//    the LSD passes.
//  * Otherwise: an LSD radix sort in shared memory over the bucket's varying
//    bits only (windows of RB bits, constant bits skipped); every pass is
//    stable except the first of a key-only sort.
//
// Shared memory: s_keys (the staging buffer) and, for key-only sorts, s_out
// (the ranked output) hold CAP keys plus one 16-byte granule, so that a
// bucket can be laid out with the same alignment as its destination and
// leave the SM as 16-byte vector stores.
template <class K, class V, int NT, int KPT>
constexpr size_t ctasort_smem_bytes() {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr size_t CAPX = (size_t)NT * KPT + 16 / sizeof(K);
  // key-value sorts add u16 staged positions and a u16 output permutation
  return CAPX * sizeof(K) * (KV ? 1 : 2) + (KV ? (size_t)NT * KPT * (sizeof(typename ValT<V>::type) + 2 + 2) : 0) +
         (size_t)(NT / 32) * M * 4 +
         M * 4;
}

// Write elements [0, len) of a staged bucket to g, where element e sits at
// b[sh + e] and sh = the element offset of g inside its 16-byte granule (so
// b + sh + e and g + e share their alignment): 16-byte vector stores for the
// aligned interior, single stores for the ragged ends.  b is 16-byte aligned.
template <class K, int NT>
__device__ __forceinline__ void store_staged(const K* b, uint32_t sh, K* g, uint32_t len) {
  constexpr uint32_t VE = 16u / sizeof(K);
  const uint32_t lo = min(len, (VE - sh) % VE);
  const uint32_t nv = (len - lo) / VE;
  const uint32_t hi = lo + nv * VE;
  for (uint32_t v = threadIdx.x; v < nv; v += NT)
    *reinterpret_cast<uint4*>(g + lo + v * VE) = *reinterpret_cast<const uint4*>(b + sh + lo + v * VE);
  if (threadIdx.x < lo) g[threadIdx.x] = b[sh + threadIdx.x];
  if (threadIdx.x < len - hi) g[hi + threadIdx.x] = b[sh + hi + threadIdx.x];
}

template <class K>
__device__ __forceinline__ uint32_t granule_shift(const K* g) {
  return (uint32_t)((reinterpret_cast<uintptr_t>(g) & 15u) / sizeof(K));
}

template <class K, class V, int NT, int KPT, int KPTA>
__device__ __forceinline__ void cta_sort_bucket(Ctl* ctl, const K* src, const typename ValT<V>::type* vsrc, K* dst,
                                                typename ValT<V>::type* vdst, uint32_t off, uint32_t len, bool par,
                                                K* s_keys, typename ValT<V>::type* s_vals,
                                                uint32_t* s_whist, uint32_t* s_dstart, uint32_t* s_scan,
                                                uint32_t* s_scan16, uint32_t* s_maxc, uint32_t* s_mixed,
                                                unsigned long long* s_orv, K* s_out, uint16_t* s_pos,
                                                uint16_t* s_perm) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr int NW = NT / 32;
  constexpr int W = 8 * sizeof(K);
  constexpr int GB = (NW * M >= 8192) ? 13 : (NW * M >= 4096) ? 12 : (NW * M >= 2048 ? 11 : 10);
  constexpr uint32_t GMAX = 64;  // largest group ranked by the in-group insertion rank (measured: 32 or 48 slower on Zipf)
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t* wh = s_whist + warp * M;
  const uint32_t wb = warp * 32u * KPTA;
  const uint32_t wvalid = len > wb ? min(len - wb, 32u * KPTA) : 0u;
  K k[KPTA];
  uint32_t r[KPTA];
  typename ValT<V>::type v[KV ? KPTA : 1];
  K orv = 0, nandv = 0;
#pragma unroll
  for (int i = 0; i < KPTA; ++i) {
    const uint32_t e = (uint32_t)(i * 32) + lane;
    k[i] = K(0);
    r[i] = 0u;
    if (e < wvalid) {
      k[i] = src[off + wb + e];
      if constexpr (KV) v[i] = vsrc[off + wb + e];
      orv |= k[i];
      nandv |= ~k[i];
    }
  }
  orv = warp_or(orv);
  nandv = warp_or(nandv);
  if (lane == 0) {
    atomicOr(&s_orv[0], (unsigned long long)orv);
    atomicOr(&s_orv[1], (unsigned long long)nandv);
  }
  __syncthreads();
  const K vm = (K)s_orv[0] & (K)s_orv[1];  // bits that are 1 in some key and 0 in another
  if (vm == K(0)) {
    if (par) {
#pragma unroll
      for (int i = 0; i < KPTA; ++i) {
        const uint32_t e = (uint32_t)(i * 32) + lane;
        if (e < wvalid) {
          dst[off + wb + e] = k[i];
          if constexpr (KV) vdst[off + wb + e] = v[i];
        }
      }
    }
    return;
  }
  {
    const int hb = top_bit<K>(vm), lb = low_bit<K>(vm);
    const uint32_t span = (uint32_t)(hb - lb + 1);
    const uint32_t wbits = span < (uint32_t)GB ? span : (uint32_t)GB;
    const uint32_t gshift = (uint32_t)hb + 1u - wbits;
    const uint32_t nb = 1u << wbits;
    uint32_t* cnt = s_whist;  // nb <= NW * M counters
    // all NW * M counters in use and 8 per thread: vector zeroing and scan
    constexpr bool VEC_OK = (NW * M == NT * 8);
    const bool vec = VEC_OK && nb == (uint32_t)(NW * M);
    if (vec) {
      uint4* c4 = reinterpret_cast<uint4*>(cnt) + threadIdx.x * 2u;
      c4[0] = make_uint4(0u, 0u, 0u, 0u);
      c4[1] = make_uint4(0u, 0u, 0u, 0u);
    } else {
      for (uint32_t x = threadIdx.x; x < nb; x += NT) cnt[x] = 0u;
    }
    if (threadIdx.x == 0) *s_maxc = 0u;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KPTA; ++i) {
      const uint32_t ri = ((uint32_t)(i * 32) + lane < wvalid) ? atomicAdd(&cnt[(uint32_t)(k[i] >> gshift) & (nb - 1u)], 1u) : 0u;
      if constexpr (KV)
        r[i] = ri;
      else
        s_out[(uint32_t)i * NT + threadIdx.x] = (K)ri;  // parked in the idle output buffer until staging (fewer live registers)
    }
    __syncthreads();
    if (vec) {
      // thread t owns counters 8t .. 8t+7
      uint4* c4 = reinterpret_cast<uint4*>(cnt) + threadIdx.x * 2u;
      const uint4 a = c4[0], b4 = c4[1];
      const uint32_t p1 = a.x, p2 = p1 + a.y, p3 = p2 + a.z, p4 = p3 + a.w, p5 = p4 + b4.x, p6 = p5 + b4.y,
                     p7 = p6 + b4.z, tot = p7 + b4.w;
      uint32_t mx = max(max(max(a.x, a.y), max(a.z, a.w)), max(max(b4.x, b4.y), max(b4.z, b4.w)));
      mx = warp_max(mx);
      if (lane == 0 && mx) atomicMax(s_maxc, mx);
      const uint32_t run = block_scan<NT>(tot, s_scan16);
      c4[0] = make_uint4(run, run + p1, run + p2, run + p3);
      c4[1] = make_uint4(run + p4, run + p5, run + p6, run + p7);
    } else {
      // exclusive scan of the nb counters, EMAX consecutive ones per thread
      constexpr uint32_t EMAX = (uint32_t)(NW * M) / NT;
      const uint32_t e_per = nb >= (uint32_t)NT ? nb / NT : 1u;
      const uint32_t first_c = threadIdx.x * e_per;
      uint32_t tot = 0, mx = 0;
#pragma unroll
      for (uint32_t x = 0; x < EMAX; ++x) {
        const uint32_t c0 = (x < e_per && first_c + x < nb) ? cnt[first_c + x] : 0u;
        tot += c0;
        mx = max(mx, c0);
      }
      mx = warp_max(mx);
      if (lane == 0 && mx) atomicMax(s_maxc, mx);
      uint32_t run = block_scan<NT>(tot, s_scan16);
#pragma unroll
      for (uint32_t x = 0; x < EMAX; ++x) {
        if (x < e_per && first_c + x < nb) {
          const uint32_t c0 = cnt[first_c + x];
          cnt[first_c + x] = run;
          run += c0;
        }
      }
    }
    __syncthreads();
    if (KV && *s_maxc <= GMAX) {
      // Stable: rank by (key, input position).  Keys and positions are staged
      // in group order, payloads by input position; s_perm[final slot] =
      // staged index; then keys and payloads leave in final order, coalesced.
      if (threadIdx.x == 0) atomicAdd(&ctl->group_buckets, 1ull);
#pragma unroll
      for (int i = 0; i < KPTA; ++i) {
        const uint32_t x = (uint32_t)(i * 32) + lane;
        if (x < wvalid) {
          const uint32_t pos = cnt[(uint32_t)(k[i] >> gshift) & (nb - 1u)] + r[i];
          if (pos < len) {
            s_keys[pos] = k[i];
            s_pos[pos] = (uint16_t)(wb + x);
            if constexpr (KV) s_vals[wb + x] = v[i];
          } else {
            record_error(ctl, DERR_BOUNDS, ERR_SITE_CTASORT_STAGE);
          }
        }
      }
      __syncthreads();
      for (uint32_t e = threadIdx.x; e < len; e += NT) {
        const K key = s_keys[e];
        const uint32_t pe = s_pos[e];
        const uint32_t h = (uint32_t)(key >> gshift) & (nb - 1u);
        const uint32_t gs = cnt[h];
        const uint32_t ge = h + 1u < nb ? cnt[h + 1u] : len;
        uint32_t rank = 0;
        for (uint32_t jj = gs; jj < ge; ++jj) {
          const K kj = s_keys[jj];
          rank += (kj < key || (kj == key && (uint32_t)s_pos[jj] < pe)) ? 1u : 0u;
        }
        s_perm[gs + rank] = (uint16_t)e;
      }
      __syncthreads();
      for (uint32_t o = threadIdx.x; o < len; o += NT) {
        const uint32_t e = s_perm[o];
        dst[off + o] = s_keys[e];
        if constexpr (KV) vdst[off + o] = s_vals[s_pos[e]];
      }
      return;
    }
    if (!KV && (span <= wbits || *s_maxc <= GMAX)) {
      if (threadIdx.x == 0) atomicAdd(&ctl->group_buckets, 1ull);
      const uint32_t osh = granule_shift(dst + off);
      // one counting pass covered every varying bit: the staged order is final
      const uint32_t ssh = span <= wbits ? osh : 0u;
#pragma unroll
      for (int i = 0; i < KPTA; ++i) {
        if ((uint32_t)(i * 32) + lane < wvalid) {
          const uint32_t pos = cnt[(uint32_t)(k[i] >> gshift) & (nb - 1u)] + (uint32_t)s_out[(uint32_t)i * NT + threadIdx.x];
          if (pos < len)
            s_keys[ssh + pos] = k[i];
          else
            record_error(ctl, DERR_BOUNDS, ERR_SITE_CTASORT_STAGE);
        }
      }
      __syncthreads();
      if (span <= wbits) {
        store_staged<K, NT>(s_keys, osh, dst + off, len);
      } else {
        for (uint32_t e = threadIdx.x; e < len; e += NT) {
          const K key = s_keys[e];
          const uint32_t h = (uint32_t)(key >> gshift) & (nb - 1u);
          const uint32_t gs = cnt[h];
          const uint32_t ge = h + 1u < nb ? cnt[h + 1u] : len;
          uint32_t rank = 0;
          for (uint32_t jj = gs; jj < ge; ++jj) {
            const K kj = s_keys[jj];
            rank += (kj < key || (kj == key && jj < e)) ? 1u : 0u;
          }
          s_out[osh + gs + rank] = key;
        }
        __syncthreads();
        store_staged<K, NT>(s_out, osh, dst + off, len);
      }
      return;
    }
    if (!KV && span > wbits) {
      // Some group holds more than GMAX keys.  If every such group holds one
      // repeated key (a heavy value, as in Zipf buckets), its keys need no
      // order and keep their staged slots, and the other groups take the
      // insertion rank; if one of them mixes keys, fall back to LSD.
      if (threadIdx.x == 0) *s_mixed = 0u;
#pragma unroll
      for (int i = 0; i < KPTA; ++i) {
        if ((uint32_t)(i * 32) + lane < wvalid) {
          const uint32_t pos = cnt[(uint32_t)(k[i] >> gshift) & (nb - 1u)] + (uint32_t)s_out[(uint32_t)i * NT + threadIdx.x];
          if (pos < len)
            s_keys[pos] = k[i];
          else
            record_error(ctl, DERR_BOUNDS, ERR_SITE_CTASORT_STAGE);
        }
      }
      __syncthreads();
      for (uint32_t e = threadIdx.x; e < len; e += NT) {
        const K key = s_keys[e];
        const uint32_t h = (uint32_t)(key >> gshift) & (nb - 1u);
        const uint32_t gs = cnt[h];
        const uint32_t ge = h + 1u < nb ? cnt[h + 1u] : len;
        if (ge - gs > GMAX && key != s_keys[gs]) *s_mixed = 1u;
      }
      __syncthreads();
      if (*s_mixed == 0u) {
        if (threadIdx.x == 0) atomicAdd(&ctl->group_buckets, 1ull);
        const uint32_t osh = granule_shift(dst + off);
        for (uint32_t e = threadIdx.x; e < len; e += NT) {
          const K key = s_keys[e];
          const uint32_t h = (uint32_t)(key >> gshift) & (nb - 1u);
          const uint32_t gs = cnt[h];
          const uint32_t ge = h + 1u < nb ? cnt[h + 1u] : len;
          uint32_t slot = e;
          if (ge - gs <= GMAX) {
            uint32_t rank = 0;
            for (uint32_t jj = gs; jj < ge; ++jj) {
              const K kj = s_keys[jj];
              rank += (kj < key || (kj == key && jj < e)) ? 1u : 0u;
            }
            slot = gs + rank;
          }
          s_out[osh + slot] = key;
        }
        __syncthreads();
        store_staged<K, NT>(s_out, osh, dst + off, len);
        return;
      }
    }
    // skewed bucket: LSD passes from the registers (r[] is recomputed)
  }
  uint32_t sh = (uint32_t)low_bit<K>(vm);
  bool first = true;
  for (;;) {
    const bool unstable = !KV && first;
    if (unstable) {
      if (threadIdx.x < M) s_dstart[threadIdx.x] = 0u;
      __syncthreads();
#pragma unroll
      for (int i = 0; i < KPTA; ++i)
        r[i] = warp_inc<true>(s_dstart, digit_of(k[i], sh), (uint32_t)(i * 32) + lane < wvalid);
      __syncthreads();
      const uint32_t cnt = threadIdx.x < M ? s_dstart[threadIdx.x] : 0u;
      const uint32_t ds = scan256(cnt, s_scan, nullptr);
      if (threadIdx.x < M) s_dstart[threadIdx.x] = ds;
    } else {
      for (uint32_t i = threadIdx.x; i < (uint32_t)(NW * M); i += NT) s_whist[i] = 0u;
      __syncthreads();
      // (a bucket gets here when its keys are skewed: few distinct digits)
      warp_rank_stable<K, KPTA, false, true>(k, sh, 0u, wvalid, (uint32_t)KPTA, wh, r);
      __syncthreads();
      scan_digit_warp<NT, NW>(s_whist, s_scan16);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KPTA; ++i) {
      if ((uint32_t)(i * 32) + lane < wvalid) {
        const uint32_t d = digit_of(k[i], sh);
        const uint32_t pos = (unstable ? s_dstart[d] : wh[d]) + r[i];
        if (pos < len) {
          s_keys[pos] = k[i];
          if constexpr (KV) s_vals[pos] = v[i];
        } else {
          record_error(ctl, DERR_BOUNDS, ERR_SITE_CTASORT_STAGE);
        }
      }
    }
    __syncthreads();
    first = false;
    const uint32_t nsh = sh + RB;
    const K rest = nsh < (uint32_t)W ? (K)(vm >> nsh) : K(0);
    if (rest == K(0)) break;
    sh = nsh + (uint32_t)low_bit<K>(rest);
#pragma unroll
    for (int i = 0; i < KPTA; ++i) {
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
}

// Two CTAs per SM, three for u32 key-only buckets (12 keys per lane, 66 KB of
// shared memory), where a third bucket in flight measured faster.
template <class K, class V, int NT>
constexpr int ctasort_min_blocks() {
  return NT >= 1024 ? 1 : ((std::is_same<V, NoVal>::value && sizeof(K) == 4) ? 3 : 2);
}

// `second`: sort the second queue (buckets the u32 key-only fast CTA sort
// handed over) instead of the classifier's queue.
template <class K, class V, int NT, int KPT>
__device__ __forceinline__ void ctasort_body(const Ctx& c, int second) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr uint32_t CAP = (uint32_t)NT * KPT;
  constexpr int NW = NT / 32;
  constexpr uint32_t CAPX = CAP + 16u / sizeof(K);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* s_keys = reinterpret_cast<K*>(smem_raw);
  K* s_out = s_keys + CAPX;  // key-only sorts only
  using VT = typename ValT<V>::type;
  VT* s_vals = reinterpret_cast<VT*>(s_keys + (KV ? CAPX : 2 * CAPX));
  uint32_t* s_whist = reinterpret_cast<uint32_t*>(s_vals + (KV ? CAP : 0));
  uint32_t* s_dstart = s_whist + NW * M;
  uint16_t* s_pos = reinterpret_cast<uint16_t*>(s_dstart + M);  // key-value sorts only
  uint16_t* s_perm = s_pos + (KV ? CAP : 0);
  static_assert(!KV || CAP <= 65536u, "u16 positions");
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_scan16[NW];
  __shared__ uint32_t s_q, s_maxc, s_mixed;
  __shared__ unsigned long long s_orv[2];
  Ctl* ctl = c.ctl;
  const uint32_t count = min(second ? ctl->cta2_count : ctl->cta_count, c.ctacap);
  if (count == 0u) return;  // (the same value for every thread)
  uint32_t* claim = second ? &ctl->cta2_claim : &ctl->cta_claim;
  const Item* queue = second ? c.cta_q2 : c.cta_q;

  for (;;) {
    if (threadIdx.x == 0) {
      s_q = atomicAdd(claim, 1u);
      s_orv[0] = 0ull;
      s_orv[1] = 0ull;
    }
    __syncthreads();
    const uint32_t q = s_q;
    if (q >= count) break;
    const Item it = queue[q];
    const ArrDesc ad = c.arrs[it.arr];
    const bool par = (it.info & ITEM_PARITY) != 0u;
    const K* src = reinterpret_cast<const K*>(par ? ad.buf : ad.keys);
    const VT* vsrc = reinterpret_cast<const VT*>(par ? ad.vbuf : ad.vals);
    K* dst = reinterpret_cast<K*>(ad.keys);
    VT* vdst = reinterpret_cast<VT*>(ad.vals);
    const uint32_t off = it.off, len = min(it.len, CAP);
    if (it.info & ITEM_COPY) {
      for (uint32_t e = threadIdx.x; e < len; e += NT) {
        dst[off + e] = src[off + e];
        if constexpr (KV) vdst[off + e] = vsrc[off + e];
      }
    } else {
      const uint32_t kpt = (len + NT - 1) / NT;  // 1..KPT keys per lane
#define DFR_CTA_BODY(A)                                                                                      \
  cta_sort_bucket<K, V, NT, KPT, A>(ctl, src, vsrc, dst, vdst, off, len, par, s_keys, s_vals, s_whist, s_dstart, \
                                    s_scan, s_scan16, &s_maxc, &s_mixed, s_orv, s_out, s_pos, s_perm)
      if (kpt <= 1)
        DFR_CTA_BODY(1);
      else if (kpt <= 2)
        DFR_CTA_BODY(KPT >= 2 ? 2 : KPT);
      else if (kpt <= 4)
        DFR_CTA_BODY(KPT >= 4 ? 4 : KPT);
      else if (kpt <= 8)
        DFR_CTA_BODY(KPT >= 8 ? 8 : KPT);
      else
        DFR_CTA_BODY(KPT);
#undef DFR_CTA_BODY
    }
    __syncthreads();
  }
}

template <class K, class V, int NT, int KPT>
__global__ void __launch_bounds__(NT, (ctasort_min_blocks<K, V, NT>())) k_ctasort(Ctx c, int second) {
  ctasort_body<K, V, NT, KPT>(c, second);
}

// Exclusive scan, in place, of a warp's M = 256 counters (lane l owns
// counters 8l..8l+7); returns the largest counter.  Call with the whole warp.
__device__ __forceinline__ uint32_t warp_scan_counters(uint32_t* wh) {
  static_assert(M == 256, "the counter scan assumes 8 counters per lane");
  const uint32_t lane = lane_id();
  uint4* w4 = reinterpret_cast<uint4*>(wh) + lane * 2;
  const uint4 a = w4[0], b4 = w4[1];
  const uint32_t x0 = 0, x1 = a.x, x2 = x1 + a.y, x3 = x2 + a.z, x4 = x3 + a.w, x5 = x4 + b4.x, x6 = x5 + b4.y,
                 x7 = x6 + b4.z, run = x7 + b4.w;
  uint32_t mx = max(max(max(a.x, a.y), max(a.z, a.w)), max(max(b4.x, b4.y), max(b4.z, b4.w)));
  uint32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, inc, o);
    if (lane >= (uint32_t)o) inc += y;
    mx = max(mx, __shfl_xor_sync(FULL, mx, o));
  }
  const uint32_t bv = inc - run;
  w4[0] = make_uint4(bv + x0, bv + x1, bv + x2, bv + x3);
  w4[1] = make_uint4(bv + x4, bv + x5, bv + x6, bv + x7);
  return mx;
}

template <class K, class V, int WKPT>
constexpr size_t warpsort_warp_bytes() {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr size_t WCAP = (size_t)32 * WKPT;
  return WCAP * sizeof(K) + (KV ? WCAP * sizeof(typename ValT<V>::type) : 0) + M * 4;
}

// Diversion sort of small buckets (T_WARP < len <= 32 * WKPT): every warp
// sorts its own buckets, pulled from the warp-sort queue, with an LSD radix
// sort over the bucket's varying bits in its own slice of shared memory
// (staging area + M counters) -- no block-wide barrier, so the many small
// buckets of skewed inputs do not pay a whole CTA each.  Ranking as in
// k_ctasort (stable except the first pass of a key-only sort).
template <class K, class V, int WPB, int WKPT>
__device__ __forceinline__ void warpsort_body(const Ctx& c) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr uint32_t WCAP = 32u * WKPT;
  constexpr int W = 8 * sizeof(K);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  unsigned char* base = smem_raw + (size_t)warp * warpsort_warp_bytes<K, V, WKPT>();
  using VT = typename ValT<V>::type;
  K* sk = reinterpret_cast<K*>(base);
  VT* sv = reinterpret_cast<VT*>(sk + WCAP);
  uint32_t* wh = reinterpret_cast<uint32_t*>(sv + (KV ? WCAP : 0));
  Ctl* ctl = c.ctl;
  const uint32_t count = min(ctl->wq_count, c.wqcap);
  if (count == 0u) return;
  for (;;) {
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(&ctl->wq_claim, 1u);
    q = __shfl_sync(FULL, q, 0);
    if (q >= count) break;
    const Item it = c.w_q[q];
    const ArrDesc ad = c.arrs[it.arr];
    const bool par = (it.info & ITEM_PARITY) != 0u;
    const K* src = reinterpret_cast<const K*>(par ? ad.buf : ad.keys);
    const VT* vsrc = reinterpret_cast<const VT*>(par ? ad.vbuf : ad.vals);
    K* dst = reinterpret_cast<K*>(ad.keys);
    VT* vdst = reinterpret_cast<VT*>(ad.vals);
    const uint32_t off = it.off, len = min(it.len, WCAP);
    const uint32_t kpt = (len + 31u) / 32u;
    K k[WKPT];
    uint32_t r[WKPT];
    VT v[KV ? WKPT : 1];
    K orv = 0, nandv = 0;
#pragma unroll
    for (int i = 0; i < WKPT; ++i) {
      const uint32_t e = (uint32_t)(i * 32) + lane;
      k[i] = K(0);
      r[i] = 0u;
      if ((uint32_t)i < kpt && e < len) {
        k[i] = src[off + e];
        if constexpr (KV) v[i] = vsrc[off + e];
        orv |= k[i];
        nandv |= ~k[i];
      }
    }
    const K vm = warp_or(orv) & warp_or(nandv);
    if (vm == K(0)) {
      if (par) {
#pragma unroll
        for (int i = 0; i < WKPT; ++i) {
          const uint32_t e = (uint32_t)(i * 32) + lane;
          if ((uint32_t)i < kpt && e < len) {
            dst[off + e] = k[i];
            if constexpr (KV) vdst[off + e] = v[i];
          }
        }
      }
      continue;
    }
    if constexpr (!KV) {
      // Key-only: count on the top (at most RB) varying bits, then the
      // insertion-sort rank inside each small group (as in k_ctasort); a group
      // of more than GMAX keys falls back to the LSD passes below.
      constexpr uint32_t GMAX = 32;
      const int hb = top_bit<K>(vm), lb = low_bit<K>(vm);
      const uint32_t span = (uint32_t)(hb - lb + 1);
      const uint32_t wbits = span < (uint32_t)RB ? span : (uint32_t)RB;
      const uint32_t gshift = (uint32_t)hb + 1u - wbits;
#pragma unroll
      for (int i = 0; i < M / 32; ++i) wh[i * 32 + lane] = 0u;
      __syncwarp();
#pragma unroll
      for (int i = 0; i < WKPT; ++i)
        if ((uint32_t)i < kpt) r[i] = warp_inc<true>(wh, digit_of(k[i], gshift), (uint32_t)(i * 32) + lane < len);
      __syncwarp();
      const uint32_t maxc = warp_scan_counters(wh);
      __syncwarp();
      if (span <= wbits || maxc <= GMAX) {
        if (lane == 0) atomicAdd(&ctl->group_buckets, 1ull);
#pragma unroll
        for (int i = 0; i < WKPT; ++i) {
          if ((uint32_t)i < kpt && (uint32_t)(i * 32) + lane < len) {
            const uint32_t pos = wh[digit_of(k[i], gshift)] + r[i];
            if (pos < len)
              sk[pos] = k[i];
            else
              record_error(ctl, DERR_BOUNDS, ERR_SITE_WARPSORT_STAGE);
          }
        }
        __syncwarp();
        if (span <= wbits) {
          for (uint32_t e = lane; e < len; e += 32) dst[off + e] = sk[e];
        } else {
          for (uint32_t e = lane; e < len; e += 32) {
            const K key = sk[e];
            const uint32_t h = digit_of(key, gshift);  // the same 8-bit index the counters used
            const uint32_t gs = wh[h];
            const uint32_t ge = h + 1u < (uint32_t)M ? wh[h + 1u] : len;
            uint32_t rank = 0;
            for (uint32_t jj = gs; jj < ge; ++jj) {
              const K kj = sk[jj];
              rank += (kj < key || (kj == key && jj < e)) ? 1u : 0u;
            }
            dst[off + gs + rank] = key;
          }
        }
        __syncwarp();
        continue;
      }
    }
    uint32_t sh = (uint32_t)low_bit<K>(vm);
    bool first = true;
    for (;;) {
#pragma unroll
      for (int i = 0; i < M / 32; ++i) wh[i * 32 + lane] = 0u;
      __syncwarp();
      const bool unstable = !KV && first;
      if (unstable) {
#pragma unroll
        for (int i = 0; i < WKPT; ++i)
          if ((uint32_t)i < kpt) warp_inc<false>(wh, digit_of(k[i], sh), (uint32_t)(i * 32) + lane < len);
      } else {
        warp_rank_stable<K, WKPT>(k, sh, 0u, len, kpt, wh, r);
      }
      __syncwarp();
      warp_scan_counters(wh);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < WKPT; ++i) {
        if ((uint32_t)i < kpt) {
          const bool valid = (uint32_t)(i * 32) + lane < len;
          const uint32_t d = digit_of(k[i], sh);
          const uint32_t pos = unstable ? warp_inc<true>(wh, d, valid) : wh[d] + r[i];
          if (valid) {
            if (pos < len) {
              sk[pos] = k[i];
              if constexpr (KV) sv[pos] = v[i];
            } else {
              record_error(ctl, DERR_BOUNDS, ERR_SITE_WARPSORT_STAGE);
            }
          }
        }
      }
      __syncwarp();
      first = false;
      const uint32_t nsh = sh + RB;
      const K rest = nsh < (uint32_t)W ? (K)(vm >> nsh) : K(0);
      if (rest == K(0)) break;
      sh = nsh + (uint32_t)low_bit<K>(rest);
#pragma unroll
      for (int i = 0; i < WKPT; ++i) {
        const uint32_t e = (uint32_t)(i * 32) + lane;
        if ((uint32_t)i < kpt && e < len) {
          k[i] = sk[e];
          if constexpr (KV) v[i] = sv[e];
        }
      }
      __syncwarp();
    }
    for (uint32_t e = lane; e < len; e += 32) {
      dst[off + e] = sk[e];
      if constexpr (KV) vdst[off + e] = sv[e];
    }
    __syncwarp();
  }
}

template <class K, class V, int WPB, int WKPT>
__global__ void __launch_bounds__(WPB * 32) k_warpsort(Ctx c) {
  warpsort_body<K, V, WPB, WKPT>(c);
}

// Write-back of large constant buckets that ended in buf: the keys are a fill
// of the bucket's single value, the payloads are copied.
template <class K, class V, int NT, int TILE>
__device__ __forceinline__ void copy_body(const Ctx& c) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  __shared__ uint32_t s_t;
  Ctl* ctl = c.ctl;
  const uint32_t ntiles = min(ctl->copy_tiles, c.copytilecap);
  if (ntiles == 0u) return;  // (the same value for every thread)
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
      if constexpr (KV) {
        using VT = typename ValT<V>::type;
        reinterpret_cast<VT*>(ad.vals)[i] = reinterpret_cast<const VT*>(ad.vbuf)[i];
      }
    }
    __syncthreads();
  }
}

template <class K, class V, int NT, int TILE>
__global__ void __launch_bounds__(NT) k_copy(Ctx c) {
  copy_body<K, V, NT, TILE>(c);
}

}  // namespace dfr
