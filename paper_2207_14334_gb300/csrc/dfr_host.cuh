// dfr_host.cuh -- host driver of the DFR sort: workspace layout, argument
// checks and the launch sequence (one per key type, instantiated in
// dfr_<type>.cu).  The host never reads device state during a call: every
// kernel is persistent and takes its work counts from the workspace, so a
// call is a fixed sequence of launches (graph-capturable for plain sorts).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "dfr.h"
#include "dfr_ctasort32.cuh"
#include "dfr_device.cuh"
#include "dfr_lsd.cuh"
#include "dfr_persist.cuh"
#include "dfr_scatter_bulk.cuh"

namespace dfr {

struct HostArr {
  void* keys;
  void* buf;
  void* vals;
  void* vbuf;
  uint64_t n;
};

// Process-wide knobs and counters (defined in dfr_api.cu).
uint32_t rt_spin_limit();
int rt_force_timeout();
void rt_prof_begin(int kind, cudaStream_t st);
void rt_prof_end(int kind, cudaStream_t st);
void rt_count_launch();
int rt_grid(const void* kern, int threads, size_t smem);
int rt_sms();
// The launch plan for a call of `key_type` whose arrays hold `mean_keys` keys
// on average (the tuning table; dfr_api.cu).
dfr_tune_t rt_tune(int key_type, uint64_t mean_keys);

enum ProfKind { PK_INIT = 0, PK_ROOT_COUNT, PK_ROOT_CLASSIFY, PK_LEVEL_COUNT, PK_SCATTER, PK_CLASSIFY, PK_CTASORT,
                PK_COPY, PK_H2D, PK_WARPSORT, PK_KEYFMT, PK_LSD_PASS, PK_LSD_PLAN, PK_PERSIST };

// Properties of the key types of the C interface (enum dfr_key_type).
inline bool key_type_valid(int kt) { return kt >= DFR_U32 && kt <= DFR_U32_KV64; }
inline size_t key_bytes_of(int kt) { return (kt == DFR_U64 || kt == DFR_U64_KV || kt == DFR_U64_KV64) ? 8u : 4u; }
inline size_t val_bytes_of(int kt) {  // 0 for key-only types
  return (kt == DFR_U64_KV || kt == DFR_U32_KV) ? 4u : (kt == DFR_U64_KV64 || kt == DFR_U32_KV64) ? 8u : 0u;
}
inline bool has_vals(int kt) { return val_bytes_of(kt) != 0u; }

inline bool fmt_valid(int fmt) {
  return (fmt & ~(0xFF | DFR_FMT_DESCENDING)) == 0 && (fmt & 0xFF) <= DFR_FMT_FLOAT;
}

// Per key type: scatter tile (threads x keys per thread), CTA-sort capacity
// (threads x keys per thread) = the diversion threshold T_CTA, and the warp
// sort (warps per block, keys per lane; 32 x WKPT = its threshold).  u32 keys
// cap the CTA sort at 12 keys per lane (6144): buckets near 4096 keys are then
// never joined into runs of ~8192 (which sort slower) and three CTAs fit an SM.
// The u32 key-only scatter deals tiles of 512 x 24 keys at two CTAs per SM
// (measured against 16, 20, 28 and 32 keys per thread: 24 is the fastest at
// 2^28 keys).  Geometry G = 1 serves calls of fewer than SMALL_TOTAL keys in
// all: a wave of the large tiles (152 SMs x 2 CTAs x 12,288 keys) is about
// 3.7M keys, and fewer tiles than CTA slots would leave SMs idle, so such u32
// key-only calls take tiles of 512 x 16 keys at three CTAs per SM (measured:
// 10^6 keys 0.201 -> 0.193 ms; a batch of 4096 arrays of 126K keys on average
// is faster with the large tiles, 48.2 against 46.6 Gkeys/s).  The other key
// types have one geometry (Cfg<K, V, 1> = Cfg<K, V, 0>).
template <class K, class V, int G = 0>
struct Cfg;
template <>
struct Cfg<uint32_t, NoVal> {
  static constexpr int SNT = 512, SKPT = 24, CNT = 512, CKPT = 12, WPB = 8, WKPT = 16;
};
template <>
struct Cfg<uint32_t, uint32_t> {
  static constexpr int SNT = 512, SKPT = 8, CNT = 512, CKPT = 8, WPB = 8, WKPT = 16;
};
template <>
struct Cfg<uint64_t, NoVal> {
  static constexpr int SNT = 512, SKPT = 8, CNT = 512, CKPT = 8, WPB = 8, WKPT = 16;
};
template <>
struct Cfg<uint64_t, uint32_t> {
  static constexpr int SNT = 512, SKPT = 8, CNT = 512, CKPT = 8, WPB = 8, WKPT = 16;
};
// 64-bit payloads: the same tiles and capacities (16-byte records for u64
// keys: the CTA sort's staging grows to 4096 x (8 + 8 + 2 + 2) bytes)
template <>
struct Cfg<uint64_t, uint64_t> {
  static constexpr int SNT = 512, SKPT = 8, CNT = 512, CKPT = 8, WPB = 8, WKPT = 16;
};
template <>
struct Cfg<uint32_t, uint64_t> {
  static constexpr int SNT = 512, SKPT = 8, CNT = 512, CKPT = 8, WPB = 8, WKPT = 16;
};
template <class K, class V>
struct Cfg<K, V, 1> : Cfg<K, V, 0> {};
template <>
struct Cfg<uint32_t, NoVal, 1> {
  static constexpr int SNT = 512, SKPT = 16, CNT = 512, CKPT = 12, WPB = 8, WKPT = 16;
};

constexpr uint64_t SMALL_TOTAL = 1ull << 22;

template <class K, class V>
constexpr bool has_small_geometry() {
  return std::is_same<K, uint32_t>::value && std::is_same<V, NoVal>::value;
}

// The geometry of a call of `narr` arrays holding `ntot` keys in all (the
// workspace size follows the same rule, so it always matches the call).
template <class K, class V>
inline int geometry_of(uint64_t ntot, uint32_t narr) {
  return (has_small_geometry<K, V>() && narr > 0u && ntot < SMALL_TOTAL) ? 1 : 0;
}

struct Layout {
  size_t ctl, arrs, root, segs0, segs1, hist0, hist1, cur0, cur1, owner, status, ctaq, ctaq2, wq, copyq, copyowner,
      total;
  uint32_t segcap, tilecap, ctacap, wqcap, copycap, copytilecap;
  // LSD top phase (single arrays of at least lsd_min_n keys)
  bool has_lsd;
  size_t lsd, lsd_st0, lsd_st1, pool_k, pool_v;
  uint32_t lsd_zero16;  // 16-byte words zeroed by k_init from `lsd` (control block + look-back words)
  uint32_t lsd_tiles_a, lsd_tiles_b_cap, est_cap, est_ocap;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Smallest single array the LSD top phase takes: below M x T_CTA keys one
// digit already brings buckets under the CTA-sort capacity (d = 1), where the
// LSD and MSD schedules coincide.
template <class K, class V>
constexpr uint64_t lsd_min_n() {
  return (uint64_t)M * Cfg<K, V>::CNT * Cfg<K, V>::CKPT;
}

template <class K, class V, int G = 0>
Layout make_layout(uint64_t ntot, uint32_t narr) {
  using C = Cfg<K, V, G>;
  constexpr uint64_t TILE = (uint64_t)C::SNT * C::SKPT;
  constexpr uint64_t TCTA = (uint64_t)C::CNT * C::CKPT;
  Layout l{};
  l.segcap = (uint32_t)(ntot / (TCTA + 1) + narr + 1);
  l.tilecap = (uint32_t)(ntot / TILE + l.segcap + 1);
  constexpr uint64_t WCAP = 32ull * C::WKPT;
  // runs of more than the smallest allowed warp-sort limit (DFR_TUNE_WARP_MIN)
  l.ctacap = (uint32_t)(ntot / (DFR_TUNE_WARP_MIN + 1) + narr + 1);
  static_assert(DFR_TUNE_WARP_MIN <= WCAP, "warp-sort limits");
  l.wqcap = (uint32_t)(ntot / (T_WARP + 1) + narr + 1);  // buckets of more than T_WARP keys
  l.copycap = (uint32_t)(ntot / (TCTA + 1) + 1);
  l.copytilecap = (uint32_t)(ntot / TILE + l.copycap + 1);
  size_t o = 0;
  l.ctl = o;
  o = align256(o + sizeof(Ctl));
  l.root = o;  // right after ctl: k_init zeroes [ctl, root end)
  o = align256(o + (size_t)narr * sizeof(RootAcc<K>));
  l.arrs = o;
  o = align256(o + (size_t)narr * sizeof(ArrDesc));
  l.segs0 = o;
  o = align256(o + (size_t)l.segcap * sizeof(Seg));
  l.segs1 = o;
  o = align256(o + (size_t)l.segcap * sizeof(Seg));
  l.hist0 = o;
  o = align256(o + (size_t)l.segcap * M * 4);
  l.hist1 = o;
  o = align256(o + (size_t)l.segcap * M * 4);
  // key-only sorts: per (segment, digit) fill cursors of the scatter
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  l.cur0 = o;
  o = align256(o + (KV ? 0 : (size_t)l.segcap * M * 4));
  l.cur1 = o;
  o = align256(o + (KV ? 0 : (size_t)l.segcap * M * 4));
  l.owner = o;
  o = align256(o + (size_t)l.tilecap * 4);
  l.status = o;  // key-value sorts: look-back words
  o = align256(o + (KV ? (size_t)l.tilecap * M * 4 : 0));
  l.ctaq = o;
  o = align256(o + (size_t)l.ctacap * sizeof(Item));
  l.ctaq2 = o;  // u32 key-only: buckets the fast CTA sort hands to the general one
  o = align256(o + (has_small_geometry<K, V>() ? (size_t)l.ctacap * sizeof(Item) : 0));
  l.wq = o;
  o = align256(o + (size_t)l.wqcap * sizeof(Item));
  l.copyq = o;
  o = align256(o + (size_t)l.copycap * sizeof(CopyItem));
  l.copyowner = o;
  o = align256(o + (size_t)l.copytilecap * 4);
  l.has_lsd = narr == 1u && ntot >= lsd_min_n<K, V>();
  if (l.has_lsd) {
    l.lsd_tiles_a = (uint32_t)((ntot + TILE - 1) / TILE);
    // second-pass tiles: every one of the 2M pieces adds at most two partial tiles
    l.lsd_tiles_b_cap = (uint32_t)(ntot / TILE) + 4u * M + 1u;
    l.est_cap = (uint32_t)(ntot / M) & ~15u;
    // overflow slots per bucket: 8 standard deviations of a uniform bucket's
    // count (binomial, about sqrt(N/M)) plus a margin, at least N/(32 M)
    const uint64_t sd8 = 8ull * (uint64_t)std::ceil(std::sqrt((double)ntot / M)) + 64ull;
    l.est_ocap = (uint32_t)((std::max<uint64_t>(ntot / (32ull * M), sd8) + 15ull) & ~15ull);
    l.lsd = o;
    o = align256(o + sizeof(LsdCtl));
    l.lsd_st0 = o;
    o = align256(o + (KV ? (size_t)l.lsd_tiles_a * M * 4 : 0));
    l.lsd_st1 = o;
    o = align256(o + (size_t)l.lsd_tiles_b_cap * M * 4);
    l.lsd_zero16 = (uint32_t)((o - l.lsd) / 16);
    l.pool_k = o;
    o = align256(o + (size_t)M * l.est_ocap * sizeof(K));
    l.pool_v = o;
    o = align256(o + (KV ? (size_t)M * l.est_ocap * sizeof(typename ValT<V>::type) : 0));
  }
  l.total = o;
  return l;
}

inline Ctx make_ctx(void* ws, const Layout& l, uint32_t narr) {
  char* b = static_cast<char*>(ws);
  Ctx c{};
  c.ctl = reinterpret_cast<Ctl*>(b + l.ctl);
  c.arrs = reinterpret_cast<ArrDesc*>(b + l.arrs);
  c.narr = narr;
  c.root = b + l.root;
  c.segs[0] = reinterpret_cast<Seg*>(b + l.segs0);
  c.segs[1] = reinterpret_cast<Seg*>(b + l.segs1);
  c.hist[0] = reinterpret_cast<uint32_t*>(b + l.hist0);
  c.hist[1] = reinterpret_cast<uint32_t*>(b + l.hist1);
  c.cur[0] = reinterpret_cast<uint32_t*>(b + l.cur0);
  c.cur[1] = reinterpret_cast<uint32_t*>(b + l.cur1);
  c.tile_owner = reinterpret_cast<uint32_t*>(b + l.owner);
  c.status = reinterpret_cast<uint32_t*>(b + l.status);
  c.cta_q = reinterpret_cast<Item*>(b + l.ctaq);
  c.cta_q2 = reinterpret_cast<Item*>(b + l.ctaq2);
  c.w_q = reinterpret_cast<Item*>(b + l.wq);
  c.copy_q = reinterpret_cast<CopyItem*>(b + l.copyq);
  c.copy_owner = reinterpret_cast<uint32_t*>(b + l.copyowner);
  c.segcap = l.segcap;
  c.tilecap = l.tilecap;
  c.ctacap = l.ctacap;
  c.wqcap = l.wqcap;
  c.copycap = l.copycap;
  c.copytilecap = l.copytilecap;
  if (l.has_lsd) {
    c.lsd = reinterpret_cast<LsdCtl*>(b + l.lsd);
    c.lsd_st[0] = reinterpret_cast<uint32_t*>(b + l.lsd_st0);
    c.lsd_st[1] = reinterpret_cast<uint32_t*>(b + l.lsd_st1);
    c.pool_k = b + l.pool_k;
    c.pool_v = b + l.pool_v;
    c.lsd_tiles_a = l.lsd_tiles_a;
    c.lsd_tiles_b_cap = l.lsd_tiles_b_cap;
    c.est_cap = l.est_cap;
    c.est_ocap = l.est_ocap;
  }
  return c;
}

inline bool ranges_overlap(const void* a, uint64_t abytes, const void* b, uint64_t bbytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bbytes && y < x + abytes;
}

template <class K, class V>
int check_arrays(const HostArr* arrs, uint32_t narr, uint64_t* ntot_out) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  constexpr uint64_t VB = sizeof(typename ValT<V>::type);  // payload bytes
  uint64_t ntot = 0;
  for (uint32_t a = 0; a < narr; ++a) {
    const HostArr& h = arrs[a];
    if (h.n > DFR_MAX_N) return DFR_ERR_INVALID_ARG;
    if (h.n == 0) continue;
    if (!h.keys || !h.buf) return DFR_ERR_INVALID_ARG;
    if (KV && (!h.vals || !h.vbuf)) return DFR_ERR_INVALID_ARG;
    // element alignment (the 16-byte vector body of every load starts from it)
    if (((uintptr_t)h.keys % sizeof(K)) || ((uintptr_t)h.buf % sizeof(K))) return DFR_ERR_INVALID_ARG;
    if (KV && (((uintptr_t)h.vals % VB) || ((uintptr_t)h.vbuf % VB))) return DFR_ERR_INVALID_ARG;
    if (ranges_overlap(h.keys, h.n * sizeof(K), h.buf, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
    if (KV) {
      if (ranges_overlap(h.vals, h.n * VB, h.vbuf, h.n * VB)) return DFR_ERR_INVALID_ARG;
      if (ranges_overlap(h.vals, h.n * VB, h.keys, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
      if (ranges_overlap(h.vals, h.n * VB, h.buf, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
      if (ranges_overlap(h.vbuf, h.n * VB, h.keys, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
      if (ranges_overlap(h.vbuf, h.n * VB, h.buf, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
    }
    ntot += h.n;
  }
  *ntot_out = ntot;
  return DFR_OK;
}

// The workspace a call of ntot keys in narr arrays needs: the larger of the
// two geometries' layouts, so that the size never decreases with ntot (a
// workspace sized for n keys serves every call of fewer keys, whichever
// geometry that call selects).
template <class K, class V>
size_t workspace_bytes(uint64_t ntot, uint32_t narr) {
  if constexpr (has_small_geometry<K, V>())
    return std::max(make_layout<K, V, 0>(ntot, narr).total, make_layout<K, V, 1>(ntot, narr).total);
  else
    return make_layout<K, V, 0>(ntot, narr).total;
}

// Persistent grid sizes of every kernel of one key type on one device.
struct Grids {
  int rc, rcl, lc, sc, cl, cs, ws, cp, kf, lp, le, rc2, lp1, cs32, ps;
};

// The tuning entry's CTAs-per-SM caps applied to the persistent grids.
inline void apply_tune(const dfr_tune_t& t, int sms, Grids* g) {
  if (t.scatter_ctas_per_sm && sms > 0) {
    g->sc = std::min(g->sc, (int)t.scatter_ctas_per_sm * sms);
    g->lp = std::min(g->lp, (int)t.scatter_ctas_per_sm * sms);
    g->le = std::min(g->le, (int)t.scatter_ctas_per_sm * sms);
    g->lp1 = std::min(g->lp1, (int)t.scatter_ctas_per_sm * sms);
  }
  if (t.ctasort_ctas_per_sm && sms > 0) g->cs = std::min(g->cs, (int)t.ctasort_ctas_per_sm * sms);
}

// Fill the launch-plan fields of a context from a tuning entry.
template <class K, class V>
void ctx_plan(Ctx* c, const dfr_tune_t& t) {
  constexpr uint32_t WCAP = 32u * Cfg<K, V>::WKPT;
  c->target = 1u << t.target_log2;
  c->max_bits = t.max_bits;
  c->warp_max = std::min(t.warp_max, WCAP);
}

template <class K, class V>
constexpr int key_type_of() {
  return std::is_same<V, NoVal>::value     ? (sizeof(K) == 8 ? DFR_U64 : DFR_U32)
         : std::is_same<V, uint32_t>::value ? (sizeof(K) == 8 ? DFR_U64_KV : DFR_U32_KV)
                                            : (sizeof(K) == 8 ? DFR_U64_KV64 : DFR_U32_KV64);
}

template <class K, class V, int G = 0>
struct Kernels {
  using C = Cfg<K, V, G>;
  static constexpr int SNT = C::SNT, SKPT = C::SKPT, TILE = SNT * SKPT;
  static constexpr int CNT = C::CNT, CKPT = C::CKPT, TCTA = CNT * CKPT;
  static constexpr int WPB = C::WPB, WKPT = C::WKPT, WCAP = 32 * WKPT;
  static constexpr size_t sc_smem = scatter_smem_bytes<K, V, SNT, SKPT>();
  static constexpr size_t cs_smem = ctasort_smem_bytes<K, V, CNT, CKPT>();
  static constexpr size_t ws_smem = (size_t)WPB * warpsort_warp_bytes<K, V, WKPT>();
  static constexpr size_t lp_smem = lsd_smem_bytes<K, V, SNT, SKPT>();
  static constexpr int nlev = (int)sizeof(K) + EXTRA_LEVELS;
  static_assert(nlev + 1 <= MAXLV, "control blocks for every launched level");
  static constexpr auto root_count = k_root_count<K, SNT, TILE, false>;
  static constexpr auto root_count2 = k_root_count<K, SNT, TILE, true>;
  static constexpr auto root_classify = k_root_classify<K, V, TILE, TCTA, WCAP>;
  static constexpr auto level_count = k_level_count<K, !std::is_same<V, NoVal>::value, SNT, TILE>;
  // key-only deals write each digit run's 16-byte-aligned body with one bulk
  // copy (measured against plain stores: uniform keys alike, sorted and
  // reverse runs 1.42 -> 1.21 ms at 2^28)
  static constexpr bool BULK = std::is_same<V, NoVal>::value;
  static constexpr size_t sb_smem = scatter_bulk_smem_bytes<K, SNT, SKPT>();
  static constexpr auto scatter = k_scatter<K, V, SNT, SKPT>;
  static constexpr auto scatter_bulk = k_scatter_bulk<K, SNT, SKPT>;
  static constexpr auto classify = k_classify<K, V, TILE, TCTA, WCAP>;
  static constexpr auto ctasort = k_ctasort<K, V, CNT, CKPT>;
  static constexpr auto warpsort = k_warpsort<K, V, WPB, WKPT>;
  static constexpr auto copy = k_copy<K, V, SNT, TILE>;
  static constexpr auto keyfmt = k_keyfmt<K, SNT, TILE>;
  static constexpr auto lsd_pass0 = k_lsd_pass<K, V, SNT, SKPT, 0, false>;
  static constexpr auto lsd_est = k_lsd_pass<K, V, SNT, SKPT, 0, true>;
  static constexpr auto lsd_pass1 = k_lsd_pass<K, V, SNT, SKPT, 1, false>;
  static constexpr auto lsd_mid = k_lsd_mid<K, V, TILE>;
  static constexpr auto lsd_fin = k_lsd_fin<K>;
  // u32 key-only buckets: k_ctasort32 (CS32_NC threads x 4 * CS32_NV keys)
  // for spans up to CTA32_SPAN bits; wider ones and heavy duplicates go to
  // the general CTA sort through the second queue
  static constexpr bool FAST32 = has_small_geometry<K, V>();
  // 512 sorting threads + one producer warp, a two-bucket ring, two CTAs per
  // SM (measured: three stages 2-3% slower)
  static constexpr int CS32_NC = 512, CS32_NV = 3, CS32_MINB = 2, CS32_STAGES = 2;
  static constexpr int CS32_NT = CS32_NC + 32;
  using C32 = Cta32<CS32_NC, CS32_NV, CS32_STAGES>;
  static_assert(!FAST32 || C32::CAP == (uint32_t)TCTA, "both CTA sorts take buckets up to the diversion threshold");
  static constexpr size_t cs32_smem = ctasort32_smem_bytes<CS32_NC, CS32_NV, CS32_STAGES>();
  static constexpr auto ctasort32 = k_ctasort32<CS32_NC, CS32_NV, CS32_STAGES, CS32_MINB>;
  // the whole call as one persistent, cooperative launch (dfr_persist.cuh)
  static_assert(SNT == CNT, "the persistent form runs every phase in one block size");
  using PC = PersistCfg<K, V, SNT, SKPT, CKPT, WKPT>;
  static constexpr auto persist = k_persist<K, V, SNT, SKPT, CKPT, WKPT>;

  // grid_of(kernel, threads, dynamic smem) -> persistent grid (or < 0 on error)
  template <class GridOf>
  static bool grids(GridOf&& grid_of, Grids* g) {
    g->rc = grid_of((const void*)root_count, SNT, (size_t)0);
    g->rcl = grid_of((const void*)root_classify, 256, (size_t)0);
    g->lc = grid_of((const void*)level_count, SNT, (size_t)0);
    g->sc = BULK ? grid_of((const void*)scatter_bulk, SNT, sb_smem) : grid_of((const void*)scatter, SNT, sc_smem);
    g->cl = grid_of((const void*)classify, 256, (size_t)0);
    g->cs = grid_of((const void*)ctasort, CNT, cs_smem);
    g->ws = grid_of((const void*)warpsort, WPB * 32, ws_smem);
    g->cp = grid_of((const void*)copy, SNT, (size_t)0);
    g->kf = grid_of((const void*)keyfmt, SNT, (size_t)0);
    g->lp = grid_of((const void*)lsd_pass0, SNT, lp_smem);
    g->lp1 = grid_of((const void*)lsd_pass1, SNT, lp_smem);
    g->le = grid_of((const void*)lsd_est, SNT, lp_smem);
    g->rc2 = grid_of((const void*)root_count2, SNT, (size_t)0);
    g->cs32 = FAST32 ? grid_of((const void*)ctasort32, CS32_NT, cs32_smem) : 1;
    g->ps = grid_of((const void*)persist, PC::NT, PC::smem);
    return g->ps > 0 && g->cs32 > 0 && g->rc > 0 && g->rcl > 0 && g->lc > 0 && g->sc > 0 && g->cl > 0 && g->cs > 0 && g->ws > 0 && g->cp > 0 &&
           g->kf > 0 && g->lp > 0 && g->le > 0 && g->rc2 > 0 && g->lp1 > 0;
  }
};

inline uint32_t min_u32(uint32_t a, uint32_t b) { return a < b ? a : b; }

// The schedule of a call: the plan's LSD mode for a single array large
// enough to have the LSD workspace, the MSD schedule (0) otherwise.
inline uint32_t lsd_mode_of(const dfr_tune_t& t, const Layout& lay, uint32_t narr) {
  return (narr == 1u && lay.has_lsd && t.schedule <= 2u) ? t.schedule : 0u;
}

// The whole device launch sequence of one call (no host synchronisation, no
// allocation).  `hook(kind, stream, launch_fn)` wraps every launch (profiling
// and launch counting in the regular path, counting only in the no-allocation
// path).  `a0` rides in k_init's parameters when `write_a0`.  With c.lsd_mode
// set the top two digits go through the LSD phase (dfr_lsd.cuh): mode 1 =
// root count (both digits) -> plan -> root classify -> pass 0 -> pass 1;
// mode 2 = estimated pass 0 -> plan -> root count (skipped when the estimate
// held) -> root classify -> pass 1.  The MSD levels follow either way.
template <class K, class V, int G, class Hook>
void enqueue_sort(const Ctx& c, const Layout& lay, const Grids& g, uint32_t narr, uint32_t root_tiles,
                  unsigned long long ntot, const ArrDesc& a0, bool write_a0, cudaStream_t st, Hook&& hook) {
  using T = Kernels<K, V, G>;
  const uint32_t mode = c.lsd_mode;
  const uint32_t root_words = (uint32_t)((size_t)narr * sizeof(RootAcc<K>) / 4);
  const uint32_t words = (uint32_t)(sizeof(Ctl) / 4) + root_words;
  const uint32_t z16 = mode ? lay.lsd_zero16 : 0u;
  const uint32_t gi = min_u32((std::max(words, z16) + 255) / 256, 1024u);
  uint4* z = mode ? reinterpret_cast<uint4*>(c.lsd) : nullptr;
  hook(PK_INIT, st, [&] { k_init<K><<<gi, 256, 0, st>>>(c, a0, write_a0 ? 1 : 0, root_words, z, z16); });
  const uint32_t lp_grid = min_u32(lay.lsd_tiles_a, (uint32_t)g.lp);
  if (mode == 2u) {
    const uint32_t le_grid = min_u32(lay.lsd_tiles_a, (uint32_t)g.le);
    hook(PK_LSD_PASS, st, [&] { T::lsd_est<<<le_grid, T::SNT, T::lp_smem, st>>>(c); });
    hook(PK_LSD_PLAN, st, [&] { T::lsd_mid<<<1, 256, 0, st>>>(c); });
  }
  if (mode == 1u) {
    uint32_t* h2 = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(c.lsd) + offsetof(LsdCtl, h1));
    hook(PK_ROOT_COUNT, st,
         [&] { T::root_count2<<<min_u32(root_tiles, (uint32_t)g.rc2), T::SNT, 0, st>>>(c, root_tiles, h2); });
  } else {
    hook(PK_ROOT_COUNT, st,
         [&] { T::root_count<<<min_u32(root_tiles, (uint32_t)g.rc), T::SNT, 0, st>>>(c, root_tiles, nullptr); });
  }
  if (mode == 1u) hook(PK_LSD_PLAN, st, [&] { T::lsd_mid<<<1, 256, 0, st>>>(c); });
  hook(PK_ROOT_CLASSIFY, st, [&] { T::root_classify<<<min_u32(narr, (uint32_t)g.rcl), 256, 0, st>>>(c, ntot); });
  if (mode == 1u) hook(PK_LSD_PASS, st, [&] { T::lsd_pass0<<<lp_grid, T::SNT, T::lp_smem, st>>>(c); });
  if (mode) {
    const uint32_t lp1_grid = min_u32(lay.lsd_tiles_b_cap, (uint32_t)g.lp1);
    hook(PK_LSD_PASS, st, [&] { T::lsd_pass1<<<lp1_grid, T::SNT, T::lp_smem, st>>>(c); });
    hook(PK_LSD_PLAN, st, [&] { T::lsd_fin<<<M, M, 0, st>>>(c); });
  }
  const uint32_t lc_grid = min_u32(lay.tilecap, (uint32_t)g.lc);
  const uint32_t sc_grid = min_u32(lay.tilecap, (uint32_t)g.sc);
  const uint32_t cl_grid = min_u32(lay.segcap, (uint32_t)g.cl);
  for (int L = 0; L < T::nlev; ++L) {
    hook(PK_LEVEL_COUNT, st, [&] { T::level_count<<<lc_grid, T::SNT, 0, st>>>(c, L); });
    if constexpr (T::BULK)
      hook(PK_SCATTER, st, [&] { T::scatter_bulk<<<sc_grid, T::SNT, T::sb_smem, st>>>(c, L); });
    else
      hook(PK_SCATTER, st, [&] { T::scatter<<<sc_grid, T::SNT, T::sc_smem, st>>>(c, L); });
    hook(PK_CLASSIFY, st, [&] { T::classify<<<cl_grid, 256, 0, st>>>(c, L); });
  }
  if constexpr (T::FAST32) {
    hook(PK_CTASORT, st,
         [&] { T::ctasort32<<<min_u32(lay.ctacap, (uint32_t)g.cs32), T::CS32_NT, T::cs32_smem, st>>>(c); });
    hook(PK_CTASORT, st, [&] { T::ctasort<<<min_u32(lay.ctacap, (uint32_t)g.cs), T::CNT, T::cs_smem, st>>>(c, 1); });
  } else {
    hook(PK_CTASORT, st, [&] { T::ctasort<<<min_u32(lay.ctacap, (uint32_t)g.cs), T::CNT, T::cs_smem, st>>>(c, 0); });
  }
  hook(PK_WARPSORT, st, [&] {
    T::warpsort<<<min_u32((lay.wqcap + T::WPB - 1) / T::WPB, (uint32_t)g.ws), T::WPB * 32, T::ws_smem, st>>>(c);
  });
  hook(PK_COPY, st, [&] { T::copy<<<min_u32(lay.copytilecap, (uint32_t)g.cp), T::SNT, 0, st>>>(c); });
}

// Whether a call runs as one persistent launch (dfr_persist.cuh): the plan's
// launch form (DFR_LAUNCH_*), the MSD schedule only, and a device on which
// the persistent kernel fits (g.ps > 0).
inline bool use_persist(const dfr_tune_t& t, uint64_t ntot, uint32_t lsd_mode, const Grids& g, bool persist_ok) {
  if (!persist_ok || lsd_mode != 0u || g.ps <= 0 || t.launch == DFR_LAUNCH_LEVELS) return false;
  return t.launch == DFR_LAUNCH_PERSISTENT || ntot < DFR_PERSIST_AUTO_KEYS;
}

// The persistent launch of one call: the control block and the per-array
// root accumulators are zeroed by a memset (the grid barrier's counters live
// in the control block), then one cooperative launch runs every phase.  Its
// grid: one CTA per 2048 keys and per array, at most what is resident at
// once (g.ps).  Returns the first CUDA error.
template <class K, class V, int G, class Hook>
cudaError_t enqueue_persist(const Ctx& c, const Layout& lay, const Grids& g, uint32_t narr, uint32_t root_tiles,
                            unsigned long long ntot, const ArrDesc& a0, bool write_a0, int fmt, cudaStream_t st,
                            Hook&& hook) {
  using T = Kernels<K, V, G>;
  const size_t zero_bytes = lay.root + (size_t)narr * sizeof(RootAcc<K>) - lay.ctl;
  const uint64_t want = ntot / 2048u + narr;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1u, std::min<uint64_t>(want, (uint64_t)g.ps));
  cudaError_t e = cudaSuccess;
  hook(PK_PERSIST, st, [&] {
    e = cudaMemsetAsync(c.ctl, 0, zero_bytes, st);
    if (e != cudaSuccess) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(T::PC::NT);
    cfg.dynamicSmemBytes = T::PC::smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, T::persist, c, a0, write_a0 ? 1u : 0u, root_tiles, ntot, (uint32_t)fmt);
  });
  return e;
}

// Regular entry: checks, layout, descriptor table, then enqueue_sort with
// profiling hooks.  `batch` = the descriptor table is uploaded with one copy
// (else the single descriptor rides in k_init's parameters, keeping the call
// a pure kernel sequence).
template <class K, class V, int G>
int run_sort_g(const HostArr* arrs, uint32_t narr, bool batch, void* ws, size_t ws_bytes, cudaStream_t st,
               int fmt, bool persist_ok) {
  using T = Kernels<K, V, G>;
  if (!fmt_valid(fmt)) return DFR_ERR_INVALID_ARG;
  if (narr == 0) return DFR_OK;
  uint64_t ntot = 0;
  int rc = check_arrays<K, V>(arrs, narr, &ntot);
  if (rc != DFR_OK) return rc;
  bool any = false;
  for (uint32_t a = 0; a < narr; ++a) any = any || arrs[a].n > 1;
  if (!any) return DFR_OK;
  const Layout lay = make_layout<K, V, G>(ntot, narr);
  if (!ws || ((uintptr_t)ws & 255u)) return DFR_ERR_INVALID_ARG;
  if (ws_bytes < lay.total) return DFR_ERR_WORKSPACE;
  Ctx c = make_ctx(ws, lay, narr);
  c.spin_limit = rt_spin_limit();
  c.force_timeout = rt_force_timeout() ? 1u : 0u;
  c.nlev = (uint32_t)T::nlev;
  const dfr_tune_t tune = rt_tune(key_type_of<K, V>(), ntot / narr);
  ctx_plan<K, V>(&c, tune);
  c.lsd_mode = lsd_mode_of(tune, lay, narr);

  Grids g;
  if (!T::grids([](const void* k, int t, size_t sm) { return rt_grid(k, t, sm); }, &g)) return DFR_ERR_CUDA;
  apply_tune(tune, rt_sms(), &g);

  std::vector<ArrDesc> tab(narr);
  uint32_t rt = 0;
  for (uint32_t a = 0; a < narr; ++a) {
    const HostArr& h = arrs[a];
    tab[a] = ArrDesc{h.keys, h.buf, h.vals, h.vbuf, (uint32_t)h.n, rt};
    if (h.n > 1) rt += (uint32_t)((h.n + T::TILE - 1) / T::TILE);
  }
  auto hook = [](int kind, cudaStream_t s, auto&& fn) {
    rt_prof_begin(kind, s);
    fn();
    rt_count_launch();
    rt_prof_end(kind, s);
  };
  if (batch) {
    cudaError_t e = cudaSuccess;
    rt_prof_begin(PK_H2D, st);
    e = cudaMemcpyAsync(c.arrs, tab.data(), narr * sizeof(ArrDesc), cudaMemcpyHostToDevice, st);
    rt_prof_end(PK_H2D, st);
    if (e != cudaSuccess) return DFR_ERR_CUDA;
  }
  if (use_persist(tune, ntot, c.lsd_mode, g, persist_ok)) {
    if (enqueue_persist<K, V, G>(c, lay, g, narr, rt, (unsigned long long)ntot, tab[0], !batch, fmt, st, hook) !=
        cudaSuccess)
      return DFR_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? DFR_OK : DFR_ERR_CUDA;
  }
  // Signed, float or descending keys: map every key to its unsigned image in
  // place, sort the images, map them back (two extra read+write passes).
  const uint32_t kf_grid = min_u32(rt, (uint32_t)g.kf);
  if (fmt != DFR_FMT_UNSIGNED)
    hook(PK_KEYFMT, st, [&] { T::keyfmt<<<kf_grid, T::SNT, 0, st>>>(c, tab[0], batch ? 0u : 1u, rt, (uint32_t)fmt, 1u); });
  enqueue_sort<K, V, G>(c, lay, g, narr, rt, (unsigned long long)ntot, tab[0], !batch, st, hook);
  if (fmt != DFR_FMT_UNSIGNED)
    hook(PK_KEYFMT, st, [&] { T::keyfmt<<<kf_grid, T::SNT, 0, st>>>(c, tab[0], batch ? 0u : 1u, rt, (uint32_t)fmt, 0u); });
  return cudaGetLastError() == cudaSuccess ? DFR_OK : DFR_ERR_CUDA;
}

// A call in the geometry its array sizes select (geometry_of).
template <class K, class V>
int run_sort(const HostArr* arrs, uint32_t narr, bool batch, void* ws, size_t ws_bytes, cudaStream_t st,
             int fmt = DFR_FMT_UNSIGNED, bool persist_ok = true) {
  uint64_t ntot = 0;  // (each n is validated by run_sort_g)
  for (uint32_t a = 0; a < narr; ++a) ntot += arrs[a].n;
  return geometry_of<K, V>(ntot, narr) ? run_sort_g<K, V, 1>(arrs, narr, batch, ws, ws_bytes, st, fmt, persist_ok)
                                       : run_sort_g<K, V, 0>(arrs, narr, batch, ws, ws_bytes, st, fmt, persist_ok);
}

// Capture one call's launch sequence into an executable CUDA graph bound to
// these buffers and this workspace.  The descriptor table is uploaded now
// (synchronously), so the captured sequence is kernels only.
template <class K, class V, int G>
int build_graph_g(const HostArr* arrs, uint32_t narr, void* ws, size_t ws_bytes, cudaGraphExec_t* out,
                  uint32_t* nodes) {
  using T = Kernels<K, V, G>;
  *out = nullptr;
  *nodes = 0;
  if (narr == 0) return DFR_ERR_INVALID_ARG;
  uint64_t ntot = 0;
  int rc = check_arrays<K, V>(arrs, narr, &ntot);
  if (rc != DFR_OK) return rc;
  const Layout lay = make_layout<K, V, G>(ntot, narr);
  if (!ws || ((uintptr_t)ws & 255u)) return DFR_ERR_INVALID_ARG;
  if (ws_bytes < lay.total) return DFR_ERR_WORKSPACE;
  Ctx c = make_ctx(ws, lay, narr);
  c.spin_limit = rt_spin_limit();
  c.force_timeout = 0u;
  c.nlev = (uint32_t)T::nlev;
  const dfr_tune_t tune = rt_tune(key_type_of<K, V>(), ntot / narr);
  ctx_plan<K, V>(&c, tune);
  c.lsd_mode = lsd_mode_of(tune, lay, narr);
  Grids g;
  if (!T::grids([](const void* k, int t, size_t sm) { return rt_grid(k, t, sm); }, &g)) return DFR_ERR_CUDA;
  apply_tune(tune, rt_sms(), &g);
  std::vector<ArrDesc> tab(narr);
  uint32_t rt = 0;
  for (uint32_t a = 0; a < narr; ++a) {
    const HostArr& h = arrs[a];
    tab[a] = ArrDesc{h.keys, h.buf, h.vals, h.vbuf, (uint32_t)h.n, rt};
    if (h.n > 1) rt += (uint32_t)((h.n + T::TILE - 1) / T::TILE);
  }
  if (cudaMemcpy(c.arrs, tab.data(), narr * sizeof(ArrDesc), cudaMemcpyHostToDevice) != cudaSuccess)
    return DFR_ERR_CUDA;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return DFR_ERR_CUDA;
  // Capture the persistent launch where the plan picks it; should that
  // capture fail, capture the level sequence instead.
  auto capture = [&](bool persist) -> int {
    cudaGraph_t graph = nullptr;
    int r = DFR_OK;
    uint32_t n = 0;
    auto count = [&n](int, cudaStream_t, auto&& fn) {
      fn();
      ++n;
    };
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DFR_ERR_CUDA;
    if (persist) {
      if (enqueue_persist<K, V, G>(c, lay, g, narr, rt, (unsigned long long)ntot, tab[0], false, DFR_FMT_UNSIGNED,
                                   cs, count) != cudaSuccess)
        r = DFR_ERR_CUDA;
    } else {
      enqueue_sort<K, V, G>(c, lay, g, narr, rt, (unsigned long long)ntot, tab[0], false, cs, count);
    }
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !graph) r = DFR_ERR_CUDA;
    if (r == DFR_OK && cudaGraphInstantiate(out, graph, 0) != cudaSuccess) r = DFR_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    if (r != DFR_OK) {
      *out = nullptr;
      cudaGetLastError();  // clear the failed capture's error before a retry
    }
    *nodes = n;
    return r;
  };
  const bool persist = use_persist(tune, ntot, c.lsd_mode, g, true);
  rc = capture(persist);
  if (rc != DFR_OK && persist) rc = capture(false);
  cudaStreamDestroy(cs);
  if (rc != DFR_OK) *out = nullptr;
  return rc;
}

template <class K, class V>
int build_graph(const HostArr* arrs, uint32_t narr, void* ws, size_t ws_bytes, cudaGraphExec_t* out,
                uint32_t* nodes) {
  uint64_t ntot = 0;  // (each n is validated by build_graph_g)
  for (uint32_t a = 0; a < narr; ++a) ntot += arrs[a].n;
  return geometry_of<K, V>(ntot, narr) ? build_graph_g<K, V, 1>(arrs, narr, ws, ws_bytes, out, nodes)
                                       : build_graph_g<K, V, 0>(arrs, narr, ws, ws_bytes, out, nodes);
}

// Entry points instantiated per key type (dfr_u32.cu, ...).
int run_u32(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st, int fmt,
            bool persist_ok);
int run_u32_kv(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st, int fmt,
            bool persist_ok);
int run_u64(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st, int fmt,
            bool persist_ok);
int run_u64_kv(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st, int fmt,
            bool persist_ok);
int run_u64_kv64(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st, int fmt,
            bool persist_ok);
int run_u32_kv64(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st, int fmt,
            bool persist_ok);
size_t ws_u32(uint64_t ntot, uint32_t narr);
size_t ws_u32_kv(uint64_t ntot, uint32_t narr);
size_t ws_u64(uint64_t ntot, uint32_t narr);
size_t ws_u64_kv(uint64_t ntot, uint32_t narr);
size_t ws_u64_kv64(uint64_t ntot, uint32_t narr);
size_t ws_u32_kv64(uint64_t ntot, uint32_t narr);
int graph_u32(const HostArr* a, uint32_t n, void* ws, size_t wsb, cudaGraphExec_t* out, uint32_t* nodes);
int graph_u32_kv(const HostArr* a, uint32_t n, void* ws, size_t wsb, cudaGraphExec_t* out, uint32_t* nodes);
int graph_u64(const HostArr* a, uint32_t n, void* ws, size_t wsb, cudaGraphExec_t* out, uint32_t* nodes);
int graph_u64_kv(const HostArr* a, uint32_t n, void* ws, size_t wsb, cudaGraphExec_t* out, uint32_t* nodes);
int graph_u64_kv64(const HostArr* a, uint32_t n, void* ws, size_t wsb, cudaGraphExec_t* out, uint32_t* nodes);
int graph_u32_kv64(const HostArr* a, uint32_t n, void* ws, size_t wsb, cudaGraphExec_t* out, uint32_t* nodes);
// Dispatch by key type, and the device error word as a DFR status (dfr_api.cu).
int run_typed(int key_type, const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st,
              int fmt = DFR_FMT_UNSIGNED, bool persist_ok = true);
int graph_typed(int key_type, const HostArr* a, uint32_t n, void* ws, size_t wsb, cudaGraphExec_t* out,
                uint32_t* nodes);
int ws_typed(int key_type, uint64_t ntot, uint32_t narr, size_t* bytes);
int map_device_status(uint32_t err);

}  // namespace dfr
