// dfr_host.cuh -- host driver of the DFR sort: workspace layout, argument
// checks and the launch sequence (one per key type, instantiated in
// dfr_<type>.cu).  The host never reads device state during a call: every
// kernel is persistent and takes its work counts from the workspace, so a
// call is a fixed sequence of launches (graph-capturable for plain sorts).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "dfr.h"
#include "dfr_device.cuh"

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

enum ProfKind { PK_INIT = 0, PK_ROOT_COUNT, PK_ROOT_CLASSIFY, PK_LEVEL_COUNT, PK_SCATTER, PK_CLASSIFY, PK_CTASORT,
                PK_COPY, PK_H2D, PK_OTHER };

// Per key type: scatter tile (threads x keys per thread) and CTA-sort
// capacity (threads x keys per thread) = the diversion threshold T_CTA.
template <class K, class V>
struct Cfg;
template <>
struct Cfg<uint32_t, NoVal> {
  static constexpr int SNT = 512, SKPT = 16, CNT = 512, CKPT = 16;
};
template <>
struct Cfg<uint32_t, uint32_t> {
  static constexpr int SNT = 512, SKPT = 8, CNT = 512, CKPT = 8;
};
template <>
struct Cfg<uint64_t, NoVal> {
  static constexpr int SNT = 512, SKPT = 8, CNT = 512, CKPT = 8;
};
template <>
struct Cfg<uint64_t, uint32_t> {
  static constexpr int SNT = 512, SKPT = 8, CNT = 512, CKPT = 8;
};

struct Layout {
  size_t ctl, arrs, root, segs0, segs1, hist0, hist1, a_nand, a_or, owner, status, ctaq, copyq, copyowner, total;
  uint32_t segcap, tilecap, ctacap, copycap, copytilecap;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class K, class V>
Layout make_layout(uint64_t ntot, uint32_t narr) {
  using C = Cfg<K, V>;
  constexpr uint64_t TILE = (uint64_t)C::SNT * C::SKPT;
  constexpr uint64_t TCTA = (uint64_t)C::CNT * C::CKPT;
  Layout l{};
  l.segcap = (uint32_t)(ntot / (TCTA + 1) + narr + 1);
  l.tilecap = (uint32_t)(ntot / TILE + l.segcap + 1);
  l.ctacap = (uint32_t)(ntot / (T_WARP + 1) + narr + 1);
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
  l.a_nand = o;
  o = align256(o + (size_t)l.segcap * M * sizeof(K));
  l.a_or = o;
  o = align256(o + (size_t)l.segcap * M * sizeof(K));
  l.owner = o;
  o = align256(o + (size_t)l.tilecap * 4);
  l.status = o;
  o = align256(o + (size_t)l.tilecap * M * 4);
  l.ctaq = o;
  o = align256(o + (size_t)l.ctacap * sizeof(Item));
  l.copyq = o;
  o = align256(o + (size_t)l.copycap * sizeof(CopyItem));
  l.copyowner = o;
  o = align256(o + (size_t)l.copytilecap * 4);
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
  c.a_nand = b + l.a_nand;
  c.a_or = b + l.a_or;
  c.tile_owner = reinterpret_cast<uint32_t*>(b + l.owner);
  c.status = reinterpret_cast<uint32_t*>(b + l.status);
  c.cta_q = reinterpret_cast<Item*>(b + l.ctaq);
  c.copy_q = reinterpret_cast<CopyItem*>(b + l.copyq);
  c.copy_owner = reinterpret_cast<uint32_t*>(b + l.copyowner);
  c.segcap = l.segcap;
  c.tilecap = l.tilecap;
  c.ctacap = l.ctacap;
  c.copycap = l.copycap;
  c.copytilecap = l.copytilecap;
  return c;
}

inline bool ranges_overlap(const void* a, uint64_t abytes, const void* b, uint64_t bbytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bbytes && y < x + abytes;
}

template <class K, class V>
int check_arrays(const HostArr* arrs, uint32_t narr, uint64_t* ntot_out) {
  constexpr bool KV = !std::is_same<V, NoVal>::value;
  uint64_t ntot = 0;
  for (uint32_t a = 0; a < narr; ++a) {
    const HostArr& h = arrs[a];
    if (h.n > DFR_MAX_N) return DFR_ERR_INVALID_ARG;
    if (h.n == 0) continue;
    if (!h.keys || !h.buf) return DFR_ERR_INVALID_ARG;
    if (KV && (!h.vals || !h.vbuf)) return DFR_ERR_INVALID_ARG;
    // element alignment (the 16-byte vector body of every load starts from it)
    if (((uintptr_t)h.keys % sizeof(K)) || ((uintptr_t)h.buf % sizeof(K))) return DFR_ERR_INVALID_ARG;
    if (KV && (((uintptr_t)h.vals % 4) || ((uintptr_t)h.vbuf % 4))) return DFR_ERR_INVALID_ARG;
    if (ranges_overlap(h.keys, h.n * sizeof(K), h.buf, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
    if (KV) {
      if (ranges_overlap(h.vals, h.n * 4, h.vbuf, h.n * 4)) return DFR_ERR_INVALID_ARG;
      if (ranges_overlap(h.vals, h.n * 4, h.keys, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
      if (ranges_overlap(h.vals, h.n * 4, h.buf, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
      if (ranges_overlap(h.vbuf, h.n * 4, h.keys, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
      if (ranges_overlap(h.vbuf, h.n * 4, h.buf, h.n * sizeof(K))) return DFR_ERR_INVALID_ARG;
    }
    ntot += h.n;
  }
  *ntot_out = ntot;
  return DFR_OK;
}

template <class K, class V>
size_t workspace_bytes(uint64_t ntot, uint32_t narr) {
  return make_layout<K, V>(ntot, narr).total;
}

template <class F>
inline void launch(int kind, cudaStream_t st, F&& f) {
  rt_prof_begin(kind, st);
  f();
  rt_count_launch();
  rt_prof_end(kind, st);
}

// Enqueue the whole sort of `narr` arrays.  `batch` = the descriptor table is
// uploaded with one copy (else the single descriptor rides in k_init's
// parameters, keeping the call a pure kernel sequence).
template <class K, class V>
int run_sort(const HostArr* arrs, uint32_t narr, bool batch, void* ws, size_t ws_bytes, cudaStream_t st) {
  using C = Cfg<K, V>;
  constexpr int SNT = C::SNT, SKPT = C::SKPT, TILE = SNT * SKPT;
  constexpr int CNT = C::CNT, CKPT = C::CKPT, TCTA = CNT * CKPT;
  if (narr == 0) return DFR_OK;
  uint64_t ntot = 0;
  int rc = check_arrays<K, V>(arrs, narr, &ntot);
  if (rc != DFR_OK) return rc;
  bool any = false;
  for (uint32_t a = 0; a < narr; ++a) any = any || arrs[a].n > 1;
  if (!any) return DFR_OK;
  const Layout lay = make_layout<K, V>(ntot, narr);
  if (!ws || ((uintptr_t)ws & 255u)) return DFR_ERR_INVALID_ARG;
  if (ws_bytes < lay.total) return DFR_ERR_WORKSPACE;
  Ctx c = make_ctx(ws, lay, narr);
  c.spin_limit = rt_spin_limit();
  c.force_timeout = rt_force_timeout() ? 1u : 0u;

  std::vector<ArrDesc> tab(narr);
  uint32_t rt = 0;
  for (uint32_t a = 0; a < narr; ++a) {
    const HostArr& h = arrs[a];
    tab[a] = ArrDesc{h.keys, h.buf, h.vals, h.vbuf, (uint32_t)h.n, rt};
    if (h.n > 1) rt += (uint32_t)((h.n + TILE - 1) / TILE);
  }
  if (batch) {
    cudaError_t e = cudaSuccess;
    launch(PK_H2D, st, [&] {
      e = cudaMemcpyAsync(c.arrs, tab.data(), narr * sizeof(ArrDesc), cudaMemcpyHostToDevice, st);
    });
    if (e != cudaSuccess) return DFR_ERR_CUDA;
  }
  const uint32_t root_words = (uint32_t)((size_t)narr * sizeof(RootAcc<K>) / 4);
  {
    const uint32_t words = (uint32_t)(sizeof(Ctl) / 4) + root_words;
    const uint32_t g = (words + 255) / 256 < 1024u ? (words + 255) / 256 : 1024u;
    launch(PK_INIT, st, [&] { k_init<K><<<g, 256, 0, st>>>(c, tab[0], batch ? 0 : 1, root_words); });
  }
  auto kr = k_root_count<K, SNT, TILE>;
  const int g_rc = rt_grid((const void*)kr, SNT, 0);
  launch(PK_ROOT_COUNT, st, [&] { kr<<<rt < (uint32_t)g_rc ? rt : g_rc, SNT, 0, st>>>(c, rt); });
  auto krc = k_root_classify<K, V, TILE, TCTA>;
  const int g_rcl = rt_grid((const void*)krc, 256, 0);
  launch(PK_ROOT_CLASSIFY, st, [&] { krc<<<narr < (uint32_t)g_rcl ? narr : g_rcl, 256, 0, st>>>(c, ntot); });

  auto klc = k_level_count<K, SNT, TILE>;
  auto ksc = k_scatter<K, V, SNT, SKPT>;
  auto kcl = k_classify<K, V, TILE, TCTA>;
  constexpr size_t sc_smem = scatter_smem_bytes<K, V, SNT, SKPT>();
  const int g_lc = rt_grid((const void*)klc, SNT, 0);
  const int g_sc = rt_grid((const void*)ksc, SNT, sc_smem);
  const int g_cl = rt_grid((const void*)kcl, 256, 0);
  const uint32_t lc_grid = lay.tilecap < (uint32_t)g_lc ? lay.tilecap : (uint32_t)g_lc;
  const uint32_t sc_grid = lay.tilecap < (uint32_t)g_sc ? lay.tilecap : (uint32_t)g_sc;
  const uint32_t cl_grid = lay.segcap < (uint32_t)g_cl ? lay.segcap : (uint32_t)g_cl;
  for (int L = 0; L < (int)sizeof(K); ++L) {
    launch(PK_LEVEL_COUNT, st, [&] { klc<<<lc_grid, SNT, 0, st>>>(c, L); });
    launch(PK_SCATTER, st, [&] { ksc<<<sc_grid, SNT, sc_smem, st>>>(c, L); });
    launch(PK_CLASSIFY, st, [&] { kcl<<<cl_grid, 256, 0, st>>>(c, L); });
  }
  auto kcs = k_ctasort<K, V, CNT, CKPT>;
  constexpr size_t cs_smem = ctasort_smem_bytes<K, V, CNT, CKPT>();
  const int g_cs = rt_grid((const void*)kcs, CNT, cs_smem);
  const uint32_t cs_grid = lay.ctacap < (uint32_t)g_cs ? lay.ctacap : (uint32_t)g_cs;
  launch(PK_CTASORT, st, [&] { kcs<<<cs_grid, CNT, cs_smem, st>>>(c); });
  auto kcp = k_copy<K, V, SNT, TILE>;
  const int g_cp = rt_grid((const void*)kcp, SNT, 0);
  const uint32_t cp_grid = lay.copytilecap < (uint32_t)g_cp ? lay.copytilecap : (uint32_t)g_cp;
  launch(PK_COPY, st, [&] { kcp<<<cp_grid, SNT, 0, st>>>(c); });
  return cudaGetLastError() == cudaSuccess ? DFR_OK : DFR_ERR_CUDA;
}

// Entry points instantiated per key type (dfr_u32.cu, ...).
int run_u32(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st);
int run_u32_kv(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st);
int run_u64(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st);
int run_u64_kv(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st);
size_t ws_u32(uint64_t ntot, uint32_t narr);
size_t ws_u32_kv(uint64_t ntot, uint32_t narr);
size_t ws_u64(uint64_t ntot, uint32_t narr);
size_t ws_u64_kv(uint64_t ntot, uint32_t narr);

}  // namespace dfr
