// dfr_lsd.cuh -- the LSD top phase of the DFR sort (paper, Section "Diverting
// Fast Radix", Algorithms 3 and 4).
//
// For a single large array the paper's schedule differs from the MSD one: it
// estimates how many top digits d must be dealt before the buckets of the
// d-digit prefix fall under the diversion threshold, deals those d digits
// least significant first (an LSD radix sort restricted to the top digits),
// then sorts the small buckets in bulk with a stable small-bucket sort and
// recurses on the large ones.  Here d = 2 (8-bit digits): D1 = bits
// [W-16, W-8), then D0 = bits [W-8, W).  Every launched size of this phase
// has N / 256 above the CTA-sort capacity and N / 65536 below it for keys up
// to 2^28, so two digits are the estimate; larger buckets recurse through the
// MSD levels.
//
//   mode 1 (LSD):  the root count reads the keys once and counts both digits
//                  (one upfront read for all the histograms); pass 0 deals D1
//                  into the buffer at exact bucket bases, pass 1 deals D0
//                  back into the array.
//   mode 2 (DFR):  Fast Radix -- pass 0 deals D1 with no count at all, into
//                  estimated buckets of est_cap keys (N/256 rounded down to
//                  16); keys past a full bucket go to that bucket's overflow
//                  region (est_ocap slots).  The same pass counts D0 for the
//                  exact last pass.  If an overflow region fills up, the
//                  estimate has failed: the pass is discarded (the array is
//                  untouched) and the MSD schedule sorts the array, so the
//                  failed pass cost about one counting pass, as the paper
//                  notes for a wrong estimate.
//
// Pass 1 reads the first pass's output bucket by bucket -- bucket d's main
// part, then its overflow ("pieces" 2d and 2d+1) -- in tiles that never span
// two pieces, chained in piece order by a decoupled look-back per D0 digit.
// All keys of a piece share their D1 digit, so the look-back's inclusive
// prefix at the last tile of each D1 bucket gives the exact (D0, D1)
// histogram for free; k_lsd_fin turns it into level-0 segments for the MSD
// machinery (one per D0 digit, already dealt on D1), which classifies the
// 65,536 prefix buckets: diversion, merging of small neighbours, recursion.
//
// Ordering: key-value sorts rank stably inside a tile and chain tiles in
// tile order in both passes (payloads keep input order on ties).  Key-only
// sorts rank with the scatter's adaptive ranking (rank_keys); pass 0 claims its bucket space
// with fill-cursor atomics (the order inside a D1 bucket is free: every
// prefix bucket is sorted afterwards), pass 1 keeps the look-back because the
// D1 buckets must stay in order inside every D0 bucket.
#pragma once

#include "dfr_device.cuh"

namespace dfr {

template <class K, class V, int NT, int KPT>
constexpr size_t lsd_smem_bytes() {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr size_t TILE = (size_t)NT * KPT;
  // staging area; counters (per warp for key-value, block-wide otherwise);
  // per digit: tile start, main destination base, main-part length, overflow
  // base, and the estimated pass's D0 counts
  return TILE * sizeof(K) + (KV ? TILE * sizeof(typename ValT<V>::type) : 0) +
         (KV ? (size_t)(NT / 32) * M * 4 : (size_t)M * 4) + 5 * M * 4;
}

// One LSD pass (pass 0 deals D1 into buf / the overflow regions, pass 1 deals
// D0 back into the array).  Persistent: CTAs claim tiles in increasing order.
// EST: the estimated first pass of mode 2 (also counts D0 and the OR/AND).
template <class K, class V, int NT, int KPT, int PASS, bool EST>
__global__ void __launch_bounds__(NT, (scatter_min_blocks<V, KPT, EST, NT>())) k_lsd_pass(Ctx c) {
  static_assert(PASS == 0 || !EST, "only the first pass is estimated");
  constexpr int pass = PASS;
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr uint32_t TILE = (uint32_t)NT * KPT;
  constexpr int NW = NT / 32;
  constexpr uint32_t VK = 16 / sizeof(K);
  constexpr uint32_t W = 8 * sizeof(K);
  static_assert(KV || KPT % VK == 0, "vector loads cover whole items");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* s_keys = reinterpret_cast<K*>(smem_raw);
  using VT = typename ValT<V>::type;
  VT* s_vals = reinterpret_cast<VT*>(s_keys + TILE);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_vals + (KV ? TILE : 0));  // KV: [NW][M] per warp; else [M]
  uint32_t* s_tstart = s_cnt + (KV ? NW * M : M);
  uint32_t* s_dst = s_tstart + M;  // main destination of staged element e of digit d: s_dst[d] + e
  uint32_t* s_lim = s_dst + M;     // staged elements [tstart, tstart + lim) of digit d go to the main bucket
  uint32_t* s_ovf = s_lim + M;     // the rest: overflow slot s_ovf[d] + e (arithmetic mod 2^32)
  uint32_t* s_h0 = s_ovf + M;      // estimated pass: D0 counts of this CTA's tiles
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_t, s_fail, s_p;
  __shared__ TileDigits s_ad;  // key-only adaptive ranking state

  LsdCtl* lsd = c.lsd;
  constexpr bool est = EST;
  if (!est && lsd->on == 0u) return;
  const uint32_t shift = pass == 0 ? W - 2 * RB : W - RB;
  const uint32_t ntiles = pass == 0 ? c.lsd_tiles_a : min(lsd->tiles_b, c.lsd_tiles_b_cap);
  const ArrDesc ad = c.arrs[0];
  uint32_t* status = c.lsd_st[pass];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t pool_n = (uint32_t)M * c.est_ocap;
  if (est)
    for (uint32_t i = threadIdx.x; i < (uint32_t)M; i += NT) s_h0[i] = 0u;
  K orv = 0, nandv = 0;
  unsigned long long dealt = 0;
  if (threadIdx.x == 0) adapt_init(s_ad);

  for (;;) {
    if (threadIdx.x == 0) {
      adapt_next(s_ad);
      uint32_t t = ntiles;
      // after a failed estimate no new tile is claimed (tiles already claimed
      // finish, so no look-back waits on a tile nobody processes)
      if (!est || ld_relaxed(&lsd->abort) == 0u) t = atomicAdd(&lsd->claim[pass], 1u);
      s_t = t;
      s_fail = 0u;
      uint32_t p = 0;
      if (PASS == 1 && t < ntiles) {
        // the piece holding tile t: the last piece starting at or before it
        uint32_t lo = 0, hi = 2 * M - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (lsd->pstart[mid] <= t)
            lo = mid;
          else
            hi = mid - 1;
        }
        p = lo;
      }
      s_p = p;
    }
    for (uint32_t i = threadIdx.x; i < (uint32_t)(KV ? NW * M : M); i += NT) s_cnt[i] = 0u;
    __syncthreads();
    const uint32_t t = s_t;
    if (t >= ntiles) break;

    const K* src;
    const VT* vsrc;
    uint32_t tb, vlo, vhi;
    if constexpr (PASS == 0) {
      src = reinterpret_cast<const K*>(ad.keys);
      vsrc = reinterpret_cast<const VT*>(ad.vals);
      tb = t * TILE;
      vlo = 0u;
      vhi = min(TILE, ad.n - tb);
    } else {
      const uint32_t p = s_p;
      src = reinterpret_cast<const K*>((p & 1u) ? c.pool_k : ad.buf);
      vsrc = reinterpret_cast<const VT*>((p & 1u) ? (void*)c.pool_v : ad.vbuf);
      const uint32_t poff = lsd->poff[p], plen = lsd->plen[p];
      tb = tile_base<K>(poff) + (t - lsd->pstart[p]) * TILE;
      vlo = poff > tb ? poff - tb : 0u;
      vhi = min(TILE, poff + plen - tb);
    }
    const uint32_t nvalid = vhi - vlo;

    K k[KPT];
    uint32_t r[KPT];
    VT v[KV ? KPT : 1];
    // a tile the piece covers whole is loaded, ranked and staged without
    // per-item bounds
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
        if (est) {
#pragma unroll
          for (int i = 0; i < KPT; ++i) {
            const uint32_t e = wb + (uint32_t)(i * 32) + lane;
            if (FL || (e >= vlo && e < vhi)) {
              atomicAdd(&s_h0[digit_of(k[i], W - RB)], 1u);
              orv |= k[i];
              nandv |= ~k[i];
            }
          }
        }
      } else {
        // item i = VK * q + u of thread x is element VK * (q * NT + x) + u
        const bool vec = ((((uintptr_t)src) & 15u) == 0u) && vlo == 0u && vhi == TILE;
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
        if (est) {
#pragma unroll
          for (int i = 0; i < KPT; ++i) {
            const uint32_t e = VK * ((uint32_t)(i / VK) * NT + threadIdx.x) + (uint32_t)(i % VK);
            if (FL || (e >= vlo && e < vhi)) {
              atomicAdd(&s_h0[digit_of(k[i], W - RB)], 1u);
              orv |= k[i];
              nandv |= ~k[i];
            }
          }
        }
      }
    };
    if (full)
      load_rank(std::true_type{});
    else
      load_rank(std::false_type{});
    __syncthreads();

    // Per digit: tile count (key-value: per-warp counts become exclusive
    // offsets) and, where tiles are chained, this tile's aggregate.
    constexpr bool chained = KV || PASS == 1;
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
      if (chained) st_relaxed(status + (size_t)t * M + threadIdx.x, (t == 0 ? FLAG_INC : FLAG_AGG) | tcount);
      if constexpr (!KV) adapt_note(s_ad, tcount, nvalid);
    }
    const uint32_t tstart = scan256(tcount, s_scan, nullptr);
    if (threadIdx.x < M) {
      const uint32_t d = threadIdx.x;
      const uint32_t excl = chained ? look_back(c, status, t, 0u, d, tcount, &s_fail)
                                    : (tcount ? atomicAdd(&lsd->cur1[d], tcount) : 0u);
      uint32_t lim = tcount, dst, ovf = 0u;
      if constexpr (PASS == 1) {
        dst = lsd->base0[d] + excl - tstart;
      } else if constexpr (!EST) {
        dst = lsd->base1[d] + excl - tstart;
      } else {
        // this tile's keys of digit d take places [excl, excl + tcount) of
        // bucket d; places from est_cap on are the bucket's overflow
        const uint32_t cap = c.est_cap;
        lim = excl >= cap ? 0u : min(tcount, cap - excl);
        dst = d * cap + excl - tstart;
        ovf = d * c.est_ocap + excl - cap - tstart;
        if (lim < tcount) {
          atomicAdd(&lsd->overflow, (unsigned long long)(tcount - lim));
          if (excl + tcount - cap > c.est_ocap) {
            atomicExch(&lsd->abort, 1u);
            s_fail = 1u;
          }
        }
      }
      s_tstart[d] = tstart;
      s_dst[d] = dst;
      s_lim[d] = lim;
      s_ovf[d] = ovf;
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
    if (bad) record_error(c.ctl, DERR_BOUNDS, ERR_SITE_LSD_STAGE);
    __syncthreads();

    // Coalesced write-out of the staged runs.
    if (s_fail == 0u) {
      K* dk = reinterpret_cast<K*>(pass == 0 ? ad.buf : ad.keys);
      VT* dv = reinterpret_cast<VT*>(pass == 0 ? ad.vbuf : ad.vals);
      K* pk = reinterpret_cast<K*>(c.pool_k);
#pragma unroll 4
      for (uint32_t e = threadIdx.x; e < nvalid; e += NT) {
        const K kk = s_keys[e];
        const uint32_t d = digit_of(kk, shift);
        if (!EST || e - s_tstart[d] < s_lim[d]) {
          const uint32_t g = s_dst[d] + e;
          if (g < ad.n) {
            dk[g] = kk;
            if constexpr (KV) dv[g] = s_vals[e];
          } else {
            record_error(c.ctl, DERR_BOUNDS, ERR_SITE_LSD_WRITE);
          }
        } else {
          const uint32_t q = s_ovf[d] + e;
          if (q < pool_n) {
            pk[q] = kk;
            if constexpr (KV) reinterpret_cast<VT*>(c.pool_v)[q] = s_vals[e];
          } else {
            record_error(c.ctl, DERR_BOUNDS, ERR_SITE_LSD_WRITE);
          }
        }
      }
    }
    if (threadIdx.x == 0) dealt += nvalid;
    __syncthreads();
  }

  if (est) {
    for (uint32_t i = threadIdx.x; i < (uint32_t)M; i += NT)
      if (s_h0[i]) atomicAdd(&lsd->h0[i], s_h0[i]);
    block_or2<K, NT>(orv, nandv, s_keys);
    if (threadIdx.x == 0) {
      atomic_or_u64(&lsd->orv, (unsigned long long)orv);
      atomic_or_u64(&lsd->nand, (unsigned long long)nandv);
    }
  }
  if (threadIdx.x == 0 && dealt) atomicAdd(&c.ctl->lsd_keys, dealt);
}

// Between the passes (one CTA, 256 threads = one per digit): decide whether
// the LSD phase sorts this array -- the top byte must vary, D1 must take at
// least two values and, for the estimated deal, no overflow region may have
// filled up -- and if so lay out the second pass (pieces, their tiles, the D0
// bucket bases) and write the level-0 segments (one per D0 digit, window D1,
// data in the array after the second pass).  Otherwise nothing is written
// and the MSD schedule sorts the array.
template <class K, class V, int TILE>
__global__ void __launch_bounds__(256) k_lsd_mid(Ctx c) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr uint32_t W = 8 * sizeof(K);
  __shared__ uint32_t s_scan[8];
  LsdCtl* lsd = c.lsd;
  Ctl* ctl = c.ctl;
  const uint32_t d = threadIdx.x;
  K orv, andv;
  uint32_t h0, t1, abort = 0u;
  if (c.lsd_mode == 1u) {
    const RootAcc<K>* root = reinterpret_cast<const RootAcc<K>*>(c.root);
    orv = root[0].orv;
    andv = ~root[0].nand;
    h0 = root[0].hist[d];
    t1 = lsd->h1[d];
  } else {
    orv = (K)lsd->orv;
    andv = ~(K)lsd->nand;
    abort = lsd->abort;
    h0 = lsd->h0[d];
    if constexpr (KV)
      t1 = c.lsd_tiles_a ? (c.lsd_st[0][(size_t)(c.lsd_tiles_a - 1) * M + d] & COUNT_MASK) : 0u;
    else
      t1 = lsd->cur1[d];
  }
  const int nz1 = __syncthreads_count(t1 != 0u);
  const bool top_varies = ((orv ^ andv) >> (W - RB)) != K(0);

  uint32_t moff, mlen, ooff = 0u, olen = 0u;
  uint32_t sum1 = 0, sum0 = 0;
  const uint32_t base1 = scan256(t1, s_scan, &sum1);
  if (c.lsd_mode == 1u) {
    moff = base1;
    mlen = t1;
  } else {
    moff = d * c.est_cap;
    mlen = min(t1, c.est_cap);
    ooff = d * c.est_ocap;
    olen = t1 > c.est_cap ? t1 - c.est_cap : 0u;
  }
  const uint32_t mt = mlen ? seg_tiles<K, TILE>(moff, mlen) : 0u;
  const uint32_t ot = olen ? seg_tiles<K, TILE>(ooff, olen) : 0u;
  uint32_t total = 0;
  const uint32_t ts = scan256(mt + ot, s_scan, &total);
  const uint32_t base0 = scan256(h0, s_scan, &sum0);
  const int fits = __syncthreads_and(olen <= c.est_ocap);
  if (d == 0) {
    ctl->est_cap = c.lsd_mode == 2u ? c.est_cap : 0u;
    ctl->est_abort = abort;
    ctl->est_overflow = c.lsd_mode == 2u ? lsd->overflow : 0ull;
  }
  // The counts must describe exactly the array's keys (they might not only
  // after a failed device check, e.g. a timed-out look-back); otherwise the
  // MSD schedule sorts the array.
  const uint32_t n = c.arrs[0].n;
  const bool ok = abort == 0u && ld_relaxed(&ctl->err) == 0u && top_varies && nz1 >= 2 && sum1 == n &&
                  sum0 == n && fits && total <= c.lsd_tiles_b_cap;
  if (!ok) return;  // uniform over the block
  lsd->pstart[2 * d] = ts;
  lsd->pstart[2 * d + 1] = ts + mt;
  if (d == M - 1) lsd->pstart[2 * M] = total;
  lsd->poff[2 * d] = moff;
  lsd->plen[2 * d] = mlen;
  lsd->poff[2 * d + 1] = ooff;
  lsd->plen[2 * d + 1] = olen;
  lsd->base0[d] = base0;
  lsd->base1[d] = base1;
  c.segs[0][d] = Seg{base0, h0, 0u, 0u, W - 2 * RB, 1u, SEG_PREDEALT, (uint32_t)RB, ~0ull, ~0ull};
  if (d == 0) {
    lsd->tiles_b = total;
    ctl->lv[0].nseg = M;
    ctl->lv[0].ntiles = 0u;
    ctl->sched = c.lsd_mode;
    lsd->on = 1u;
  }
}

// After the second pass (M blocks of M threads; block g = D1 digit, thread
// d = D0 digit): the (D0, D1) histogram from the second pass's look-back
// words.  The inclusive prefix at the last tile of D1 bucket g counts the
// keys of digit d in D1 buckets 0..g, so the difference of two such prefixes
// is the count of prefix (d, g); it becomes entry g of level-0 segment d.
template <class K>
__global__ void __launch_bounds__(256) k_lsd_fin(Ctx c) {
  const LsdCtl* lsd = c.lsd;
  if (lsd->on == 0u) return;
  const uint32_t g = blockIdx.x, d = threadIdx.x;
  const uint32_t* st = c.lsd_st[1];
  const uint32_t e1 = lsd->pstart[2 * g + 2], e0 = lsd->pstart[2 * g];
  const uint32_t inc1 = e1 ? (st[(size_t)(e1 - 1) * M + d] & COUNT_MASK) : 0u;
  const uint32_t inc0 = e0 ? (st[(size_t)(e0 - 1) * M + d] & COUNT_MASK) : 0u;
  c.hist[0][(size_t)d * M + g] = inc1 >= inc0 ? inc1 - inc0 : 0u;  // (a negative difference only after a failed check)
}

}  // namespace dfr
