// dfr_persist.cuh -- a whole call (one array or a batch) as one persistent,
// cooperative launch.
//
// The recursion of the diverting MSD sort (Section "Most Significant Digit
// (MSD) Radix Sorts", Algorithm 2: partition, divert the small buckets,
// recurse on the large ones) runs inside the kernel: the root count, the root
// classification, then level after level the count, the deal and the
// classification of every large segment of every array -- until a level has
// no segment left -- and finally the diverted buckets (CTA sort, warp sort)
// and the copy-back of constant buckets.  Every CTA pulls its work items --
// count tiles, deal tiles, segments, queued buckets, copy tiles -- from the
// same device counters and queues the level-sequence kernels use (the phase
// bodies are those kernels' bodies), so the result is the same; phases that
// depend on each other are separated by a grid-wide barrier instead of a
// kernel boundary.  For calls of a few million keys the level sequence is
// bound by its ~24 launches; this form pays one launch and ~3 barriers per
// level that did work.
#pragma once

#include "dfr_device.cuh"

namespace dfr {

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier between two phases.  The launch is cooperative, so every
// CTA of the grid is resident and each one that has not given up arrives.
// The arrival count only grows (zeroed before the launch): barrier g, counted
// from 1, is complete once gridDim.x * g CTAs have arrived, and the last one
// to arrive publishes g in the generation word.  The wait is bounded by
// c.spin_limit polls; one that runs out records DFR_ERR_TIMEOUT and returns
// false, after which the CTA leaves the kernel (the CTAs still waiting for it
// time out in turn, so the launch always ends).  In the forced-timeout test
// mode the waiters poll a word nobody sets.
__device__ __forceinline__ bool grid_sync(const Ctx& c, uint32_t& gen, uint32_t* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t target = gen + 1u;
    uint32_t ok = 1u;
    __threadfence();
    const uint32_t arrived = atomicAdd(&c.ctl->gbar_count, 1u) + 1u;
    if (arrived == gridDim.x * target) {
      st_release_gpu(&c.ctl->gbar_gen, target);
    } else {
      const uint32_t* p = c.force_timeout ? &c.ctl->never : &c.ctl->gbar_gen;
      uint32_t spins = 0;
      while (ld_acquire_gpu(p) < target) {
        if (++spins > c.spin_limit) {
          ok = 0u;
          break;
        }
        if (spins > 32) __nanosleep(100);
      }
      if (!ok) record_error(c.ctl, DERR_TIMEOUT, ERR_SITE_GRID_SYNC);
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  ++gen;
  return *s_ok != 0u;
}

// The persistent form's geometry: the level-sequence geometry of the key
// type (NT threads x SKPT keys per deal tile, NT x CKPT keys per CTA-sort
// bucket, 32 x WKPT keys per warp-sort bucket), so the workspace layout is
// the same; every phase runs in blocks of NT threads.
template <class K, class V, int NT_, int SKPT_, int CKPT_, int WKPT_>
struct PersistCfg {
  static constexpr int NT = NT_, SKPT = SKPT_, CKPT = CKPT_, WKPT = WKPT_;
  static_assert(NT >= M, "one thread per digit");
  static constexpr int TILE = NT * SKPT, TCTA = NT * CKPT, WCAP = 32 * WKPT;
  static constexpr size_t sc_smem = scatter_smem_bytes<K, V, NT, SKPT>();
  static constexpr size_t cs_smem = ctasort_smem_bytes<K, V, NT, CKPT>();
  static constexpr size_t count_smem = (size_t)(NT / 32) * M * 4;  // warp-private counters
  static constexpr size_t warp_bytes = warpsort_warp_bytes<K, V, WKPT>();
  static constexpr size_t base_smem =
      sc_smem > cs_smem ? (sc_smem > count_smem ? sc_smem : count_smem) : (cs_smem > count_smem ? cs_smem : count_smem);
  // warps that run the warp sort: as many as fit the other phases' shared memory
  static constexpr int WPB = (int)(base_smem / warp_bytes) < NT / 32 ? (int)(base_smem / warp_bytes) : NT / 32;
  static_assert(WPB >= 1, "at least one warp-sort warp");
  static constexpr size_t smem = base_smem;
};

// fmt: the key format (DFR_FMT_*); signed, float and descending keys are
// mapped to their unsigned images in the first phase and back in the last.
template <class K, class V, int NT, int SKPT, int CKPT, int WKPT>
__global__ void __launch_bounds__(NT, 2)
    k_persist(Ctx c, ArrDesc a0, uint32_t write_a0, uint32_t root_tiles, unsigned long long n_total, uint32_t fmt) {
  using P = PersistCfg<K, V, NT, SKPT, CKPT, WKPT>;
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* s_h = reinterpret_cast<uint32_t*>(smem_raw);
  __shared__ uint32_t s_ok, s_ntiles, s_ncnt;
  uint32_t gen = 0;
  // Count phases: a warp claims 1/sub of a tile, sub (1..8, a power of two)
  // chosen so that a call's tiles spread over the grid's warps.
  auto sub_of = [&](uint32_t tiles) {
    const uint32_t warps = gridDim.x * (uint32_t)(NT / 32);
    uint32_t sub = 1u;
    while (sub < 8u && tiles * sub * 2u <= warps) sub <<= 1;
    return sub;
  };

  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (write_a0) c.arrs[0] = a0;
    c.ctl->persist = 1u;
  }
  if (fmt != DFR_FMT_UNSIGNED) keyfmt_body<K, P::NT, P::TILE>(c, a0, write_a0, root_tiles, fmt, 1u);
  if (!grid_sync(c, gen, &s_ok)) return;
  root_count_body<K, P::NT, P::TILE, false>(c, root_tiles, nullptr, s_h, nullptr, sub_of(root_tiles));
  if (!grid_sync(c, gen, &s_ok)) return;
  root_classify_body<K, V, P::TILE, P::TCTA, P::WCAP, P::NT>(c, n_total);
  if (!grid_sync(c, gen, &s_ok)) return;
  for (int L = 0; L < (int)c.nlev; ++L) {
    // the previous classification's last barrier published this level's
    // segment and tile counts; every CTA reads the same values
    if (threadIdx.x == 0) {
      s_ntiles = ld_acquire_gpu(&c.ctl->lv[L].nseg) ? ld_acquire_gpu(&c.ctl->lv[L].ntiles) : 0u;
      s_ncnt = ld_acquire_gpu(&c.ctl->lv[L].ncnt);
    }
    __syncthreads();
    const uint32_t ntiles = s_ntiles;
    if (ntiles == 0u) break;
    // the count (and its barrier) only where a segment needs it: level 0
    // segments whose window is the top byte already have the root count's
    // histogram and AND/OR (key-value sorts always run it: it also clears
    // the level's look-back words)
    if (KV || s_ncnt != 0u) {
      level_count_body<K, KV, P::NT, P::TILE>(c, L, s_h, sub_of(ntiles));
      if (!grid_sync(c, gen, &s_ok)) return;
    }
    scatter_body<K, V, NT, SKPT>(c, L);
    if (!grid_sync(c, gen, &s_ok)) return;
    classify_body<K, V, P::TILE, P::TCTA, P::WCAP, P::NT>(c, L);
    if (!grid_sync(c, gen, &s_ok)) return;
  }
  // Diverted buckets and copy-back: independent items, no barrier between.
  ctasort_body<K, V, NT, CKPT>(c, 0);
  if constexpr (two_cta_queues<K, V>()) ctasort_body<K, V, NT, CKPT>(c, 1);
  __syncthreads();
  if ((threadIdx.x >> 5) < (uint32_t)P::WPB) warpsort_body<K, V, P::WPB, WKPT>(c);
  copy_body<K, V, P::NT, P::TILE>(c);
  if (fmt != DFR_FMT_UNSIGNED) {
    if (!grid_sync(c, gen, &s_ok)) return;
    keyfmt_body<K, P::NT, P::TILE>(c, a0, write_a0, root_tiles, fmt, 0u);
  }
}

}  // namespace dfr
