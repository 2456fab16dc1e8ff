// dfr_ctasort32.cuh -- the diversion sort of mid-size u32 key-only buckets
// (Section "Most Significant Digit (MSD) Radix Sorts": a bucket below the
// diversion threshold N_d goes to a different sort; Section "Diverting Fast
// Radix": a simple, stable sort for the small buckets).
//
// One CTA sorts one queued bucket (or run of adjacent buckets) at a time, in
// shared memory, and writes it in final position into the array's `keys`.
//
// Warp roles.  One producer warp runs ahead of the sort: it claims the next
// bucket from the queue, reads its descriptor and starts an asynchronous bulk
// copy (cp.async.bulk, global -> shared, completing on an mbarrier) of the
// bucket's 16-byte-aligned interior into a free slot of a STAGES-deep ring,
// and reads its unaligned head and tail (at most three keys each) into the
// slot's descriptor.  The NC consumer threads sort the bucket of the oldest
// full slot and hand the slot back.  So the claim, descriptor and key latencies of a
// bucket overlap the sort of the previous one.  Consumer phases synchronise
// on a named barrier that the producer warp does not join.
//
// The sort works on the bucket's varying bits [lb, hb] only (from its AND /
// OR of the keys):
//   * span <= 12 bits: one counting pass on all of them -- one shared atomic
//     per key ranks it inside its digit, and the staged order is final;
//   * span of 13..16 bits: keys are grouped by their top 12 varying bits and,
//     inside a group, ordered by the L = span - 12 low bits, whose 2^L <= 16
//     values each get a 4-bit counter (two 32-bit words per group).  One
//     shared atomic per key adds it to its (group, low bits) counter and
//     returns how many equal keys came before it; after a scan of the group
//     totals, a key's final position is its group's start + the keys of its
//     group with smaller low bits + that count -- one pass, no second sort;
//   * a wider span, or more than 15 equal keys in one bucket (a counter would
//     overflow), goes to the general CTA sort (k_ctasort, second queue),
//     which groups by the top bits and ranks inside the small groups.  The
//     classifiers already send runs whose span may exceed 16 bits there.
// The keys are staged in the bucket's own slot (they are all in registers by
// then), laid out with the destination's 16-byte alignment so that the
// bucket leaves with 16-byte stores.
//
// Waits.  Every mbarrier wait is bounded (c.spin_limit polls); one that runs
// out records DFR_ERR_TIMEOUT and ends the waiting role.  Before it exits the
// producer waits, bounded again, for the bulk copies it started.
#pragma once

#include "dfr_async.cuh"
#include "dfr_device.cuh"

namespace dfr {

template <int NC, int NV, int STAGES>
struct Cta32 {
  static constexpr int NW = NC / 32;                      // consumer warps
  static constexpr int NT = NC + 32;                      // + the producer warp
  static constexpr uint32_t CAP = (uint32_t)NC * NV * 4;  // keys per bucket (the diversion threshold)
  static constexpr uint32_t B1MAX = 12;                   // bits of the first counting pass
  static constexpr uint32_t SPANMAX = B1MAX + 4;          // widest span sorted here
  static_assert(SPANMAX == CTA32_SPAN, "the classifiers route by the same span");
  static constexpr size_t slot_bytes = ((size_t)CAP + 8) * 4;
  // Nibble-pass layout: block b holds the counter words of the 12-bit groups
  // [8b, 8b + 8) (two per group) and then their 16-bit starts, 20 words in
  // all.  In the scan a thread owns one block; at the 80-byte block stride
  // the 16-byte accesses of eight consecutive threads fall in distinct banks.
  static constexpr uint32_t GPB = 8;                                  // groups per block
  static constexpr uint32_t BLKW = 2 * GPB + GPB / 2;                 // words per block
  static constexpr uint32_t NIBW = BLKW * ((1u << B1MAX) / GPB);      // 10,240
  static constexpr size_t cnt1_bytes = ((size_t)NIBW + 4) * 4;  // first-pass counters or nibble blocks
  static constexpr size_t smem_bytes = STAGES * slot_bytes + cnt1_bytes;
};

// Word of the nibble-counter block layout where 12-bit group g's counters start.
__device__ __forceinline__ uint32_t nib_word(uint32_t g) { return (g >> 3) * 20u + (g & 7u) * 2u; }

template <int NC, int NV, int STAGES>
constexpr size_t ctasort32_smem_bytes() {
  return Cta32<NC, NV, STAGES>::smem_bytes;
}

// Sum of wsum[w] over the warps w < warp (wsum: one total per warp of the
// NW <= 32 warps): one shared load per lane and a warp scan, the same value
// in every lane of the warp.
template <int NW>
__device__ __forceinline__ uint32_t warps_before(const uint32_t* wsum, uint32_t warp, uint32_t lane) {
  static_assert(NW <= 32, "one warp total per lane");
  const uint32_t x = lane < (uint32_t)NW ? wsum[lane] : 0u;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < NW; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  return __shfl_sync(FULL, inc - x, warp);
}

// Exclusive scan of the n counters c[0, n) in place (n a power of two; each
// of the NC consumer threads owns n / NC consecutive counters, or one when
// n <= NC); every consumer thread calls it.  `wsum` holds NC/32 words that no
// other phase of the bucket uses.  One consumer barrier inside; the caller
// synchronises again before reading the result.
template <int NC>
__device__ __forceinline__ void scan_counters(uint32_t* c, uint32_t n, uint32_t* wsum) {
  constexpr int NW = NC / 32;
  const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  const uint32_t E = n >= (uint32_t)NC ? n / NC : 1u;
  const uint32_t c0 = tid * E;
  const bool owns = c0 < n;
  uint32_t tot = 0u;
  if (owns) {
    if (E >= 4u) {
      for (uint32_t k = 0; k < E; k += 4u) {
        const uint4 w = *reinterpret_cast<const uint4*>(c + c0 + k);
        tot += w.x + w.y + w.z + w.w;
      }
    } else {
      for (uint32_t k = 0; k < E; ++k) tot += c[c0 + k];
    }
  }
  uint32_t inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  named_sync(1, NC);
  uint32_t base = inc - tot + warps_before<NW>(wsum, warp, lane);
  if (owns) {
    if (E >= 4u) {
      for (uint32_t k = 0; k < E; k += 4u) {
        uint4* pw = reinterpret_cast<uint4*>(c + c0 + k);
        const uint4 w = *pw;
        uint4 o4;
        o4.x = base;
        o4.y = base + w.x;
        o4.z = o4.y + w.y;
        o4.w = o4.z + w.z;
        base = o4.w + w.w;
        *pw = o4;
      }
    } else {
      for (uint32_t k = 0; k < E; ++k) {
        const uint32_t w = c[c0 + k];
        c[c0 + k] = base;
        base += w;
      }
    }
  }
}

// Sum of the sixteen 4-bit fields of x and y (at most 16 x 15).
__device__ __forceinline__ uint32_t nib_sum2(uint32_t x, uint32_t y) {
  const uint32_t b = (x & 0x0F0F0F0Fu) + ((x >> 4) & 0x0F0F0F0Fu) + (y & 0x0F0F0F0Fu) +
                     ((y >> 4) & 0x0F0F0F0Fu);  // four byte sums <= 60
  return (b * 0x01010101u) >> 24;              // no byte of the partial sums passes 240
}

// What the producer hands the consumers with each slot.
struct SlotMeta {
  Item item;       // the queue item (item.arr = NO_OWNER: no more buckets)
  const uint32_t* src;
  uint32_t head;     // keys before the first 16-byte boundary
  uint32_t nvec;     // 16-byte vectors copied into the slot
  uint32_t edge[6];  // the head keys, then the tail keys past the last vector (at most 3 each)
};

template <int NC, int NV, int STAGES, int MINB>
__global__ void __launch_bounds__(NC + 32, MINB) k_ctasort32(Ctx c) {
  using P = Cta32<NC, NV, STAGES>;
  static_assert(NC >= 256 && (NC & (NC - 1)) == 0, "threads [0, 256) take one digit each in the (digit, warp) scan");
  constexpr uint32_t CAP = P::CAP;
  constexpr int NW = P::NW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint32_t* s_cnt1 = reinterpret_cast<uint32_t*>(smem_raw + STAGES * P::slot_bytes);
  static_assert(P::BLKW == 20u && P::GPB == 8u, "nib_word's block layout");
  static_assert(P::slot_bytes % 16 == 0, "16-byte aligned counter blocks");
  __shared__ __align__(8) uint64_t s_full[STAGES], s_empty[STAGES];
  __shared__ SlotMeta s_meta[STAGES];
  __shared__ uint32_t s_or[2], s_and[2], s_ovf[2];
  __shared__ uint32_t s_wsum[2][2][NW > 8 ? NW : 8];  // [bucket parity][first pass | stable passes][warp]
  Ctl* ctl = c.ctl;
  const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&s_full[s], 1u);
      mbar_init(&s_empty[s], 1u);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_or[0] = s_or[1] = 0u;
    s_and[0] = s_and[1] = 0xffffffffu;
    s_ovf[0] = s_ovf[1] = 0u;
  }
  for (uint32_t i = tid; i < P::NIBW + 4u; i += P::NT) s_cnt1[i] = 0u;
  __syncthreads();

  if (warp == (uint32_t)NW) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      const uint32_t count = min(ctl->cta_count, c.ctacap);
      uint32_t issued = 0u;  // bit s: the last use of slot s started a bulk copy
      uint32_t it = 0;
      for (;; ++it) {
        const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
        if (!mbar_wait(&s_empty[s], ph ^ 1u, c.spin_limit)) {
          record_error(ctl, DERR_TIMEOUT, ERR_SITE_CTASORT_STAGE);
          break;
        }
        const uint32_t q = atomicAdd(&ctl->cta_claim, 1u);
        SlotMeta m;
        m.item = Item{0u, 0u, NO_OWNER, 0u};
        m.src = nullptr;
        m.head = 0u;
        m.nvec = 0u;
        if (q < count) {
          m.item = c.cta_q[q];
          const ArrDesc ad = c.arrs[m.item.arr];
          const bool par = (m.item.info & ITEM_PARITY) != 0u;
          m.src = reinterpret_cast<const uint32_t*>(par ? ad.buf : ad.keys) + m.item.off;
          const uint32_t len = min(m.item.len, CAP);
          if (!(m.item.info & ITEM_COPY)) {
            m.head = min(len, (uint32_t)((16u - ((uint32_t)(uintptr_t)m.src & 15u)) & 15u) / 4u);
            m.nvec = (len - m.head) / 4u;
            // the ragged ends, read here so that the sort does not wait for them
            const uint32_t tb = m.head + m.nvec * 4u;
            for (uint32_t e = 0; e < m.head; ++e) m.edge[e] = m.src[e];
            for (uint32_t e = tb; e < len; ++e) m.edge[m.head + (e - tb)] = m.src[e];
          }
        }
        s_meta[s] = m;
        issued &= ~(1u << s);
        if (m.nvec) {
          mbar_arrive_tx(&s_full[s], m.nvec * 16u);
          bulk_load(smem_raw + (size_t)s * P::slot_bytes, m.src + m.head, m.nvec * 16u, &s_full[s]);
          issued |= 1u << s;
        } else {
          mbar_arrive(&s_full[s]);
        }
        if (q >= count) break;
      }
      // the bulk copies of the last STAGES slots must have landed before the
      // CTA's shared memory goes away
      for (uint32_t back = 0; back < (uint32_t)STAGES && back <= it; ++back) {
        const uint32_t j = it - back, s = j % STAGES;
        if ((issued >> s) & 1u) {
          if (!mbar_wait(&s_full[s], (j / STAGES) & 1u, c.spin_limit))
            record_error(ctl, DERR_TIMEOUT, ERR_SITE_CTASORT_STAGE);
        }
      }
    }
    return;
  }

  // ------------------------------------------------------------ consumers
  for (uint32_t it = 0;; ++it) {
    const uint32_t slot = it % STAGES, ph = (it / STAGES) & 1u, p = it & 1u;
    // every consumer waits (its own acquire of the slot); they agree on the
    // outcome so that a wait running out ends all of them together
    if (!named_sync_and(1, NC, mbar_wait(&s_full[slot], ph, c.spin_limit))) {
      if (tid == 0) record_error(ctl, DERR_TIMEOUT, ERR_SITE_CTASORT_STAGE);
      break;
    }
    const SlotMeta m = s_meta[slot];
    if (m.item.arr == NO_OWNER) break;
    uint32_t* s_keys = reinterpret_cast<uint32_t*>(smem_raw + (size_t)slot * P::slot_bytes);
    const Item item = m.item;
    const uint32_t* src = m.src;
    uint32_t* dst = reinterpret_cast<uint32_t*>(c.arrs[item.arr].keys) + item.off;
    const uint32_t len = min(item.len, CAP);
    if (tid == 0) {  // the next bucket's scalars (their slots were last read two buckets ago)
      s_or[p ^ 1u] = 0u;
      s_and[p ^ 1u] = 0xffffffffu;
      s_ovf[p ^ 1u] = 0u;
    }
    if (item.info & ITEM_COPY) {
      for (uint32_t e = tid; e < len; e += NC) dst[e] = src[e];
    } else {
      // Keys: the interior from the slot, the head and tail from global memory.
      const uint32_t head = m.head, nvec = m.nvec;
      const uint32_t tail = len - head - nvec * 4u;
      uint4 x[NV];
      uint32_t xe = 0u;
      uint32_t orv = 0u, andv = 0xffffffffu;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const uint32_t v = tid + (uint32_t)j * NC;
        if (v < nvec) {
          x[j] = reinterpret_cast<const uint4*>(s_keys)[v];
          orv |= x[j].x | x[j].y | x[j].z | x[j].w;
          andv &= x[j].x & x[j].y & x[j].z & x[j].w;
        }
      }
      const bool has_e = tid < head + tail;
      if (has_e) {
        xe = s_meta[slot].edge[tid];
        orv |= xe;
        andv &= xe;
      }
      orv = __reduce_or_sync(FULL, orv);
      andv = __reduce_and_sync(FULL, andv);
      if (lane == 0) {
        atomicOr(&s_or[p], orv);
        atomicAnd(&s_and[p], andv);
      }
      named_sync(1, NC);
      const uint32_t vm = s_or[p] & ~s_and[p];
      const uint32_t hb = vm ? 31u - (uint32_t)__clz((int)vm) : 0u;
      const uint32_t lb = vm ? (uint32_t)__ffs((int)vm) - 1u : 0u;
      const uint32_t span = vm ? hb - lb + 1u : 0u;
      if (vm == 0u) {  // one repeated key: finished, or written back from the buffer
        if (item.info & ITEM_PARITY) {
          const uint32_t key = s_or[p];  // (dst need not share src's 16-byte alignment)
          for (uint32_t e = tid; e < len; e += NC) dst[e] = key;
        }
      } else if (span > P::SPANMAX) {  // too spread for this sort: the general CTA sort takes it
        if (tid == 0) {
          const uint32_t q2 = atomicAdd(&ctl->cta2_count, 1u);
          if (q2 < c.ctacap)
            c.cta_q2[q2] = item;
          else
            record_error(ctl, DERR_CAPACITY, ERR_SITE_CTASORT_STAGE);
        }
      } else {
        const uint32_t osh = (uint32_t)(((uintptr_t)dst & 15u) / 4u);
        bool done = false;
        if (span > P::B1MAX && span <= P::B1MAX + 4u) {
          // Spans of 13..16 bits: one pass.  Keys are grouped by their top 12
          // varying bits; inside a group by the L = span - 12 low bits, whose
          // 2^L <= 16 values each get a 4-bit counter (two 32-bit words per
          // group).  One shared atomic per key adds it to its (group, low
          // bits) counter and returns how many equal keys came first; the
          // final position is the group's start + the keys of the group with
          // smaller low bits + that count.  A counter that would pass 15
          // (more than 15 equal keys) sends the bucket to the general CTA
          // sort (second queue).
          const uint32_t L = span - P::B1MAX;
          const uint32_t gshift = lb + L, lmask = (1u << L) - 1u;
          uint32_t dupw[(NV * 4 + 1 + 7) / 8];  // 4-bit counts of earlier equal keys, eight to a register
#pragma unroll
          for (int i = 0; i < (NV * 4 + 1 + 7) / 8; ++i) dupw[i] = 0u;
          auto nib_add = [&](uint32_t k, int slot) {
            const uint32_t g = (k >> gshift) & 4095u, lo = (k >> lb) & lmask;
            const uint32_t shf = 4u * (lo & 7u);
            const uint32_t old = atomicAdd(&s_cnt1[nib_word(g) + (lo >> 3)], 1u << shf);
            const uint32_t dup = (old >> shf) & 15u;
            dupw[slot / 8] |= dup << (4 * (slot % 8));
          };
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            const uint32_t v = tid + (uint32_t)j * NC;
            if (v < nvec) {
              nib_add(x[j].x, 4 * j + 0);
              nib_add(x[j].y, 4 * j + 1);
              nib_add(x[j].z, 4 * j + 2);
              nib_add(x[j].w, 4 * j + 3);
            }
          }
          if (has_e) nib_add(xe, NV * 4);
          {  // a count of 15 earlier equal keys: the counter is full
            uint32_t full = 0u;
#pragma unroll
            for (int i = 0; i < (NV * 4 + 1 + 7) / 8; ++i) {
              const uint32_t t = dupw[i] & (dupw[i] >> 1);
              full |= t & (t >> 2);
            }
            if (full & 0x11111111u) s_ovf[p] = 1u;
          }
          named_sync(1, NC);
          if (!s_ovf[p]) {
            // Group totals and their exclusive scan: thread t owns block t,
            // groups [8t, 8t + 8); their starts go to the block's last four
            // words, two 16-bit starts to a word.
            static_assert(NC * P::GPB == 4096u, "one counter block per thread");
            constexpr uint32_t GPT = P::GPB;
            uint4* blk = reinterpret_cast<uint4*>(s_cnt1 + tid * P::BLKW);
            uint32_t gt[GPT];
            uint32_t tot = 0u;
#pragma unroll
            for (uint32_t q = 0; q < GPT; q += 2u) {
              const uint4 w = blk[q / 2u];
              gt[q] = nib_sum2(w.x, w.y);
              gt[q + 1] = nib_sum2(w.z, w.w);
              tot += gt[q] + gt[q + 1];
            }
            uint32_t inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const uint32_t y = __shfl_up_sync(FULL, inc, o);
              if (lane >= (uint32_t)o) inc += y;
            }
            if (lane == 31) s_wsum[p][0][warp] = inc;
            named_sync(1, NC);
            uint32_t base = inc - tot + warps_before<NW>(s_wsum[p][0], warp, lane);
            uint32_t st[GPT / 2];  // starts < CAP <= 65536
#pragma unroll
            for (uint32_t q = 0; q < GPT; q += 2u) {
              st[q / 2u] = base | ((base + gt[q]) << 16);
              base += gt[q] + gt[q + 1];
            }
            blk[GPT / 2u] = make_uint4(st[0], st[1], st[2], st[3]);
            named_sync(1, NC);
            auto place = [&](uint32_t k, int slot) {
              const uint32_t g = (k >> gshift) & 4095u, lo = (k >> lb) & lmask;
              const uint32_t bw = (g >> 3) * P::BLKW;
              const uint2 w = *reinterpret_cast<const uint2*>(s_cnt1 + bw + (g & 7u) * 2u);
              const uint32_t gs = reinterpret_cast<const uint16_t*>(s_cnt1)[2u * (bw + 2u * P::GPB) + (g & 7u)];
              const unsigned long long m = (1ull << (4u * lo)) - 1ull;  // the counters of lower values
              const uint32_t below = nib_sum2(w.x & (uint32_t)m, w.y & (uint32_t)(m >> 32));
              const uint32_t pos = gs + below + ((dupw[slot / 8] >> (4 * (slot % 8))) & 15u);
              if (pos < len)
                s_keys[osh + pos] = k;
              else
                record_error(ctl, DERR_BOUNDS, ERR_SITE_CTASORT_STAGE);
            };
#pragma unroll
            for (int j = 0; j < NV; ++j) {
              const uint32_t v = tid + (uint32_t)j * NC;
              if (v < nvec) {
                place(x[j].x, 4 * j + 0);
                place(x[j].y, 4 * j + 1);
                place(x[j].z, 4 * j + 2);
                place(x[j].w, 4 * j + 3);
              }
            }
            if (has_e) place(xe, NV * 4);
            done = true;
          }
          named_sync(1, NC);
          {  // for the next bucket: counters and starts (the 12-bit pass counts in the same words)
            static_assert(NC * P::BLKW == P::NIBW, "one block per thread");
            uint4* blk = reinterpret_cast<uint4*>(s_cnt1 + tid * P::BLKW);
#pragma unroll
            for (uint32_t j = 0; j < P::BLKW / 4u; ++j) blk[j] = make_uint4(0u, 0u, 0u, 0u);
          }
        }
        if (!done && span <= P::B1MAX) {
          // One counting pass on every varying bit: the staged order is final.
          const uint32_t m1 = (1u << span) - 1u;
          static_assert(CAP <= 65536u, "16-bit ranks");
          uint2 r[NV];
          uint32_t re = 0u;
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            const uint32_t v = tid + (uint32_t)j * NC;
            if (v < nvec) {
              r[j].x = atomicAdd(&s_cnt1[(x[j].x >> lb) & m1], 1u) | (atomicAdd(&s_cnt1[(x[j].y >> lb) & m1], 1u) << 16);
              r[j].y = atomicAdd(&s_cnt1[(x[j].z >> lb) & m1], 1u) | (atomicAdd(&s_cnt1[(x[j].w >> lb) & m1], 1u) << 16);
            }
          }
          if (has_e) re = atomicAdd(&s_cnt1[(xe >> lb) & m1], 1u);
          named_sync(1, NC);
          scan_counters<NC>(s_cnt1, m1 + 1u, s_wsum[p][0]);
          named_sync(1, NC);
          auto stage1 = [&](uint32_t k, uint32_t rk) {
            const uint32_t pos = s_cnt1[(k >> lb) & m1] + rk;
            if (pos < len)
              s_keys[osh + pos] = k;
            else
              record_error(ctl, DERR_BOUNDS, ERR_SITE_CTASORT_STAGE);
          };
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            const uint32_t v = tid + (uint32_t)j * NC;
            if (v < nvec) {
              stage1(x[j].x, r[j].x & 0xffffu);
              stage1(x[j].y, r[j].x >> 16);
              stage1(x[j].z, r[j].y & 0xffffu);
              stage1(x[j].w, r[j].y >> 16);
            }
          }
          if (has_e) stage1(xe, re);
          named_sync(1, NC);
          for (uint32_t i = tid; i <= m1; i += NC) s_cnt1[i] = 0u;  // for the next bucket (read no more)
          done = true;
        }
        if (done) {
          if (tid == 0) atomicAdd(&ctl->group_buckets, 1ull);
          store_staged<uint32_t, NC>(s_keys, osh, dst, len);
        } else if (tid == 0) {
          // more than 15 equal keys (a heavy value): the general CTA sort
          const uint32_t q2 = atomicAdd(&ctl->cta2_count, 1u);
          if (q2 < c.ctacap)
            c.cta_q2[q2] = item;
          else
            record_error(ctl, DERR_CAPACITY, ERR_SITE_CTASORT_STAGE);
        }
      }
    }
    named_sync(1, NC);  // every consumer is done with the slot
    if (tid == 0) mbar_arrive(&s_empty[slot]);
  }
}

}  // namespace dfr
