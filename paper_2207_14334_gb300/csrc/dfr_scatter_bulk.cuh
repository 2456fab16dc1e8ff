// dfr_scatter_bulk.cuh -- the key-only deal of one level with bulk-copy
// write-out (Preliminaries: convert the counts into indices and deal every
// key to buf[index[digit]++]; Section "Most Significant Digit (MSD) Radix
// Sorts": recurse per bucket with input and buffer swapped).
//
// As k_scatter for key-only sorts -- rank every key of a tile in shared
// memory, claim the tile's run of every bucket with one atomic on the
// bucket's fill cursor, stage the tile in digit order -- but each digit's run
// is staged at a shared-memory address with the same 16-byte phase as its
// destination in HBM (runs are padded by up to three keys), so that the run's
// aligned body leaves the SM as one asynchronous bulk copy (cp.async.bulk,
// shared -> global) issued by the digit's thread, and only its ragged ends
// (at most three keys each) are plain stores.  The bulk copies take the
// per-key store instructions off the issue slots; a tile waits for its
// copies to have read the staging buffer before the next tile overwrites it.
#pragma once

#include "dfr_async.cuh"
#include "dfr_device.cuh"

namespace dfr {

template <class K, int NT, int KPT>
constexpr size_t scatter_bulk_smem_bytes() {
  constexpr size_t TILE = (size_t)NT * KPT;
  constexpr size_t VK = 16 / sizeof(K);
  // staging area with up to VK-1 keys of padding before every run; digit
  // counters; padded run starts; global run starts
  return (TILE + (VK - 1) * (M + 1)) * sizeof(K) + (size_t)M * 4 * 3;
}

template <class K, int NT, int KPT>
__global__ void __launch_bounds__(NT, (scatter_min_blocks<NoVal, KPT, false>())) k_scatter_bulk(Ctx c, int L) {
  constexpr uint32_t TILE = (uint32_t)NT * KPT;
  constexpr uint32_t VK = 16 / sizeof(K);
  constexpr uint32_t STAGE = TILE + (VK - 1) * (M + 1);
  static_assert(KPT % VK == 0, "vector loads cover whole items");
  static_assert(NT >= M, "one thread per digit");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* s_keys = reinterpret_cast<K*>(smem_raw);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_keys + STAGE);  // [M]
  uint32_t* s_pst = s_cnt + M;    // padded staging start of each digit's run
  uint32_t* s_goff = s_pst + M;   // global index of each digit's first key
  __shared__ uint32_t s_scan[16];
  __shared__ uint32_t s_t;
  __shared__ TileDigits s_ad;

  LevelCtl* lc = &c.ctl->lv[L];
  const uint32_t ntiles = min(lc->ntiles, c.tilecap);
  const Seg* segs = ((L & 1) ? c.segs[1] : c.segs[0]);
  const uint32_t* hist = ((L & 1) ? c.hist[1] : c.hist[0]);
  uint32_t* cur = ((L & 1) ? c.cur[1] : c.cur[0]);
  const uint32_t tid = threadIdx.x;

  if (tid == 0) adapt_init(s_ad);
  for (;;) {
    if (tid == 0) {
      s_t = atomicAdd(&lc->scat_claim, 1u);
      adapt_next(s_ad);
    }
    for (uint32_t i = tid; i < (uint32_t)M; i += NT) s_cnt[i] = 0u;
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
    const uint32_t j = t - seg.tile_start;
    const uint32_t tb = tile_base<K>(seg.off) + j * TILE;
    const uint32_t seg_end = seg.off + seg.len;
    const uint32_t vlo = seg.off > tb ? seg.off - tb : 0u;
    const uint32_t vhi = min(TILE, seg_end - tb);
    const uint32_t nvalid = vhi - vlo;
    const uint32_t shift = seg.shift;

    K k[KPT];
    uint32_t r[KPT];
    const bool vec = ((((uintptr_t)src) & 15u) == 0u) && tb + TILE <= ad.n;
    if (vec) {
      const uint4* pv = reinterpret_cast<const uint4*>(src + tb);
#pragma unroll
      for (int q = 0; q < KPT / (int)VK; ++q) {
        const uint4 x = __ldcs(pv + q * NT + tid);
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
        const uint32_t e = VK * ((uint32_t)(i / VK) * NT + tid) + (uint32_t)(i % VK);
        k[i] = (e >= vlo && e < vhi) ? src[tb + e] : K(0);
      }
    }
    // a tile the segment covers whole is ranked and staged without the
    // per-item bounds (the common case: only a segment's first and last
    // tiles are partial)
    const bool full = vlo == 0u && vhi == TILE;
    if (full)
      rank_keys<K, NT, KPT, true>(k, r, shift, vlo, vhi, s_cnt, s_ad);
    else
      rank_keys<K, NT, KPT, false>(k, r, shift, vlo, vhi, s_cnt, s_ad);
    __syncthreads();

    const uint32_t tcount = tid < (uint32_t)M ? s_cnt[tid] : 0u;
    if (tid < (uint32_t)M) adapt_note(s_ad, tcount, nvalid);
    const uint32_t hcount = tid < (uint32_t)M ? hist[(size_t)s * M + tid] : 0u;
    uint32_t tstart, bexcl;
    scan256x2(tcount, hcount, s_scan, tstart, bexcl);
    if (tid < (uint32_t)M) {
      // the tile's run of bucket `tid`: claimed with one atomic on the
      // bucket's fill cursor (any order of tiles inside a bucket is fine:
      // equal digits are sorted again later)
      const uint32_t excl = tcount ? atomicAdd(&cur[(size_t)s * M + tid], tcount) : 0u;
      const uint32_t g0 = seg.off + bexcl + excl;
      const uint32_t gph = (uint32_t)(((uintptr_t)(dst + g0) & 15u) / sizeof(K));
      const uint32_t base = tstart + (VK - 1u) * tid;
      s_pst[tid] = base + ((gph + VK - (base & (VK - 1u))) & (VK - 1u));
      s_goff[tid] = g0;
      // the previous tile's bulk copies must have read the staging area
      bulk_wait_read();
    }
    __syncthreads();

    // Stage the tile in digit order, each run at its padded start (a slot
    // past the staging area is skipped and reported once).
    bool bad = false;
    if (full) {
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        const uint32_t pos = s_pst[digit_of(k[i], shift)] + r[i];
        if (pos < STAGE)
          s_keys[pos] = k[i];
        else
          bad = true;
      }
    } else {
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        const uint32_t e = VK * ((uint32_t)(i / VK) * NT + tid) + (uint32_t)(i % VK);
        if (e >= vlo && e < vhi) {
          const uint32_t pos = s_pst[digit_of(k[i], shift)] + r[i];
          if (pos < STAGE)
            s_keys[pos] = k[i];
          else
            bad = true;
        }
      }
    }
    if (bad) record_error(c.ctl, DERR_BOUNDS, ERR_SITE_SCATTER_STAGE);
    fence_async_shared();
    __syncthreads();

    // Write-out: the digit's thread copies its run -- ragged ends with plain
    // stores, the aligned body with one bulk copy.
    if (tid < (uint32_t)M && tcount) {
      const uint32_t g0 = s_goff[tid];
      if (g0 < seg.off || g0 - seg.off + tcount > seg.len) {
        record_error(c.ctl, DERR_BOUNDS, ERR_SITE_SCATTER_WRITE);
      } else {
        const K* run = s_keys + s_pst[tid];
        K* out = dst + g0;
        const uint32_t gph = (uint32_t)(((uintptr_t)out & 15u) / sizeof(K));
        const uint32_t h = min(tcount, (VK - gph) & (VK - 1u));
        const uint32_t nb = (tcount - h) / VK;
        const uint32_t te = h + nb * VK;
        for (uint32_t x = 0; x < h; ++x) out[x] = run[x];
        for (uint32_t x = te; x < tcount; ++x) out[x] = run[x];
        if (nb) {
          bulk_store(out + h, run + h, nb * 16u);
          bulk_commit();
        }
      }
    }
    // No barrier here: the next tile overwrites the digit counters only after
    // its claim barrier (every thread has read this tile's counts by now),
    // the run starts only after its ranking barrier (each digit's thread
    // reads its own), and the staging area only after every digit thread has
    // waited for its bulk copies.
  }
  if (tid < (uint32_t)M) bulk_wait_read();
}

}  // namespace dfr
