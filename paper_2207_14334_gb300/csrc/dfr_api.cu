// dfr_api.cu -- the C ABI declared in include/dfr.h: argument marshalling to
// the per-type drivers, device status and statistics readback, debug knobs
// and launch profiling.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "dfr_host.cuh"

namespace dfr {

namespace {

constexpr uint32_t kDefaultSpinLimit = 1u << 18;

std::atomic<uint32_t> g_spin_limit{kDefaultSpinLimit};
std::atomic<int> g_force_timeout{0};
std::atomic<int> g_profile{0};
std::atomic<uint64_t> g_launches{0};

struct ProfRec {
  int kind;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pending;  // start event of the launch in flight

std::mutex g_grid_mu;
std::map<std::pair<const void*, int>, int> g_grid_cache;

// The tuning table: built-in entries written by the autotuner, overridable.
constexpr int kKeyTypes = 6;
const dfr_tune_t kBuiltinTune[kKeyTypes][DFR_TUNE_CLASSES] = {
#include "dfr_tune_table.inc"
};
std::mutex g_tune_mu;
dfr_tune_t g_tune[kKeyTypes][DFR_TUNE_CLASSES];
bool g_tune_init = false;

void tune_init_locked() {
  if (g_tune_init) return;
  for (int k = 0; k < kKeyTypes; ++k)
    for (int c = 0; c < DFR_TUNE_CLASSES; ++c) g_tune[k][c] = kBuiltinTune[k][c];
  g_tune_init = true;
}

bool tune_valid(const dfr_tune_t& t) {
  if (t.target_log2 < 6 || t.target_log2 > 13) return false;
  if (t.max_bits < 4 || t.max_bits > (uint32_t)RB) return false;
  if (t.warp_max < DFR_TUNE_WARP_MIN || t.warp_max > DFR_TUNE_WARP_MAX) return false;
  if (t.scatter_ctas_per_sm > 4 || t.ctasort_ctas_per_sm > 4) return false;
  if (t.schedule > DFR_SCHED_DFR) return false;
  if (t.launch > DFR_LAUNCH_PERSISTENT) return false;
  return t.reserved == 0;
}

}  // namespace

int rt_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

dfr_tune_t rt_tune(int key_type, uint64_t mean_keys) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  tune_init_locked();
  return g_tune[key_type][dfr_tune_class(mean_keys)];
}

uint32_t rt_spin_limit() { return g_spin_limit.load(); }
int rt_force_timeout() { return g_force_timeout.load(); }
void rt_count_launch() { g_launches.fetch_add(1); }

void rt_prof_begin(int, cudaStream_t st) {
  if (!g_profile.load()) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, st);
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof_pending.push_back(e);
}

void rt_prof_end(int kind, cudaStream_t st) {
  if (!g_profile.load()) return;
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (g_prof_pending.empty()) return;
  cudaEvent_t a = g_prof_pending.back();
  g_prof_pending.pop_back();
  cudaEvent_t b;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return;
  }
  cudaEventRecord(b, st);
  g_prof_recs.push_back(ProfRec{kind, a, b});
}

int rt_grid(const void* kern, int threads, size_t smem) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(g_grid_mu);
  auto key = std::make_pair(kern, dev);
  auto it = g_grid_cache.find(key);
  if (it != g_grid_cache.end()) return it->second;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  if (sms < 1) sms = 1;
  const int grid = sms * per_sm;
  g_grid_cache[key] = grid;
  return grid;
}

int map_device_status(uint32_t err) {
  if (err & DERR_TIMEOUT) return DFR_ERR_TIMEOUT;
  if (err & DERR_BOUNDS) return DFR_ERR_BOUNDS;
  if (err & DERR_CAPACITY) return DFR_ERR_WORKSPACE;
  return DFR_OK;
}

int run_typed(int key_type, const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st,
              int fmt, bool persist_ok) {
  switch (key_type) {
    case DFR_U32: return run_u32(a, n, batch, ws, wsb, st, fmt, persist_ok);
    case DFR_U32_KV: return run_u32_kv(a, n, batch, ws, wsb, st, fmt, persist_ok);
    case DFR_U64_KV64: return run_u64_kv64(a, n, batch, ws, wsb, st, fmt, persist_ok);
    case DFR_U32_KV64: return run_u32_kv64(a, n, batch, ws, wsb, st, fmt, persist_ok);
    case DFR_U64: return run_u64(a, n, batch, ws, wsb, st, fmt, persist_ok);
    case DFR_U64_KV: return run_u64_kv(a, n, batch, ws, wsb, st, fmt, persist_ok);
    default: return DFR_ERR_INVALID_ARG;
  }
}

int graph_typed(int key_type, const HostArr* a, uint32_t n, void* ws, size_t wsb, cudaGraphExec_t* out,
                uint32_t* nodes) {
  switch (key_type) {
    case DFR_U32: return graph_u32(a, n, ws, wsb, out, nodes);
    case DFR_U32_KV: return graph_u32_kv(a, n, ws, wsb, out, nodes);
    case DFR_U64_KV64: return graph_u64_kv64(a, n, ws, wsb, out, nodes);
    case DFR_U32_KV64: return graph_u32_kv64(a, n, ws, wsb, out, nodes);
    case DFR_U64: return graph_u64(a, n, ws, wsb, out, nodes);
    case DFR_U64_KV: return graph_u64_kv(a, n, ws, wsb, out, nodes);
    default: return DFR_ERR_INVALID_ARG;
  }
}

int ws_typed(int key_type, uint64_t ntot, uint32_t narr, size_t* bytes) {
  switch (key_type) {
    case DFR_U32: *bytes = ws_u32(ntot, narr); return DFR_OK;
    case DFR_U32_KV: *bytes = ws_u32_kv(ntot, narr); return DFR_OK;
    case DFR_U64_KV64: *bytes = ws_u64_kv64(ntot, narr); return DFR_OK;
    case DFR_U32_KV64: *bytes = ws_u32_kv64(ntot, narr); return DFR_OK;
    case DFR_U64: *bytes = ws_u64(ntot, narr); return DFR_OK;
    case DFR_U64_KV: *bytes = ws_u64_kv(ntot, narr); return DFR_OK;
    default: return DFR_ERR_INVALID_ARG;
  }
}

}  // namespace dfr

using namespace dfr;

extern "C" {

uint64_t dfr_lsd_min_keys(int key_type) {
  switch (key_type) {
    case DFR_U32: return lsd_min_n<uint32_t, NoVal>();
    case DFR_U32_KV: return lsd_min_n<uint32_t, uint32_t>();
    case DFR_U64_KV64: return lsd_min_n<uint64_t, uint64_t>();
    case DFR_U32_KV64: return lsd_min_n<uint32_t, uint64_t>();
    case DFR_U64: return lsd_min_n<uint64_t, NoVal>();
    case DFR_U64_KV: return lsd_min_n<uint64_t, uint32_t>();
    default: return 0;
  }
}

int dfr_workspace_bytes(int key_type, uint64_t n, size_t* bytes) {
  if (!bytes || n > DFR_MAX_N) return DFR_ERR_INVALID_ARG;
  return ws_typed(key_type, n, 1u, bytes);
}

int dfr_sort_u32(uint32_t* keys, uint32_t* buf, uint64_t n, void* ws, size_t ws_bytes, dfr_stream_t stream) {
  const HostArr a{keys, buf, nullptr, nullptr, n};
  return run_u32(&a, 1u, false, ws, ws_bytes, (cudaStream_t)stream, DFR_FMT_UNSIGNED, true);
}

int dfr_sort_u64(uint64_t* keys, uint64_t* buf, uint64_t n, void* ws, size_t ws_bytes, dfr_stream_t stream) {
  const HostArr a{keys, buf, nullptr, nullptr, n};
  return run_u64(&a, 1u, false, ws, ws_bytes, (cudaStream_t)stream, DFR_FMT_UNSIGNED, true);
}

int dfr_sort_u64_kv(uint64_t* keys, uint32_t* vals, uint64_t* kbuf, uint32_t* vbuf, uint64_t n, void* ws,
                    size_t ws_bytes, dfr_stream_t stream) {
  const HostArr a{keys, kbuf, vals, vbuf, n};
  return run_u64_kv(&a, 1u, false, ws, ws_bytes, (cudaStream_t)stream, DFR_FMT_UNSIGNED, true);
}

int dfr_sort_u32_kv(uint32_t* keys, uint32_t* vals, uint32_t* kbuf, uint32_t* vbuf, uint64_t n, void* ws,
                    size_t ws_bytes, dfr_stream_t stream) {
  const HostArr a{keys, kbuf, vals, vbuf, n};
  return run_u32_kv(&a, 1u, false, ws, ws_bytes, (cudaStream_t)stream, DFR_FMT_UNSIGNED, true);
}

int dfr_sort_u64_kv64(uint64_t* keys, uint64_t* vals, uint64_t* kbuf, uint64_t* vbuf, uint64_t n, void* ws,
                      size_t ws_bytes, dfr_stream_t stream) {
  const HostArr a{keys, kbuf, vals, vbuf, n};
  return run_u64_kv64(&a, 1u, false, ws, ws_bytes, (cudaStream_t)stream, DFR_FMT_UNSIGNED, true);
}

int dfr_sort_u32_kv64(uint32_t* keys, uint64_t* vals, uint32_t* kbuf, uint64_t* vbuf, uint64_t n, void* ws,
                      size_t ws_bytes, dfr_stream_t stream) {
  const HostArr a{keys, kbuf, vals, vbuf, n};
  return run_u32_kv64(&a, 1u, false, ws, ws_bytes, (cudaStream_t)stream, DFR_FMT_UNSIGNED, true);
}

int dfr_last_device_status(const void* ws, dfr_stream_t stream, int* status) {
  if (!ws || !status) return DFR_ERR_INVALID_ARG;
  uint32_t err = 0;
  if (cudaMemcpyAsync(&err, ws, sizeof(err), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    return DFR_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DFR_ERR_CUDA;
  *status = map_device_status(err);
  return DFR_OK;
}

int dfr_get_stats(const void* ws, dfr_stream_t stream, dfr_stats_t* out) {
  if (!ws || !out) return DFR_ERR_INVALID_ARG;
  Ctl h;
  if (cudaMemcpyAsync(&h, ws, sizeof(Ctl), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    return DFR_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DFR_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
  out->n_total = h.n_total;
  out->key_bytes = h.key_bytes;
  out->val_bytes = h.val_bytes;
  out->device_status = (uint32_t)map_device_status(h.err);
  uint32_t levels = 0;
  for (int L = 0; L < MAXLV && L < DFR_STATS_MAX_LEVELS; ++L) {
    out->level_segments[L] = h.lv[L].nseg;
    out->level_tiles[L] = h.lv[L].ntiles;
    out->level_keys[L] = h.lv[L].keys;
    out->level_hist_keys[L] = h.lv[L].hist_keys;
    if (h.lv[L].nseg) levels = (uint32_t)L + 1;
  }
  out->levels = levels;
  out->cta_buckets = h.cta_buckets;
  out->cta_keys = h.cta_keys;
  out->tiny_buckets = h.tiny_buckets;
  out->tiny_keys = h.tiny_keys;
  out->const_buckets = h.const_buckets;
  out->const_keys = h.const_keys;
  out->copy_keys = h.copy_keys;
  // Minimal bytes of the executed plan: one read of every key (root count);
  // a read and a write of every record per partition level it is dealt in;
  // a read and a write of every record sorted by a diversion sort; a read and
  // a write of every constant record that has to move back from the buffer.
  // Re-reads by per-level counts are not charged (they could be fused).
  // The LSD passes charge a read and a write of every record they deal; when
  // the estimated deal counted the keys the root count read nothing.
  const uint64_t rec = (uint64_t)h.key_bytes + h.val_bytes;
  uint64_t b = h.root_skipped ? 0 : h.n_total * h.key_bytes;
  b += 2 * rec * h.lsd_keys;
  for (int L = 0; L < MAXLV; ++L) b += 2 * rec * h.lv[L].keys;
  b += 2 * rec * (h.cta_keys + h.wsort_keys + h.tiny_keys + h.copy_keys);
  out->model_bytes = b;
  out->wsort_buckets = h.wsort_buckets;
  // 1 scatter staging, 2 scatter write, 3 CTA-sort staging, 4 warp-sort staging, 5 look-back timeout,
  // 6 LSD-pass staging, 7 LSD-pass write, 8 a segment histogram that does not add up
  out->device_error_site = h.err_site;
  out->group_buckets = h.group_buckets;
  out->schedule = h.sched;
  out->lsd_keys = h.lsd_keys;
  out->est_overflow = h.est_overflow;
  out->est_capacity = h.est_cap;
  out->est_aborted = h.est_abort;
  out->root_read = h.n_total ? (h.root_skipped ? 0u : 1u) : 0u;
  out->persistent = h.persist;
  out->wsort_keys = h.wsort_keys;
  return DFR_OK;
}

int dfr_batch_workspace_bytes(const dfr_segment_t* segs, uint32_t count, size_t* bytes) {
  if (!bytes || (!segs && count)) return DFR_ERR_INVALID_ARG;
  if (count == 0) {
    *bytes = 0;
    return DFR_OK;
  }
  const int kt = segs[0].key_type;
  uint64_t ntot = 0;
  for (uint32_t i = 0; i < count; ++i) {
    if (segs[i].key_type != kt || segs[i].n > DFR_MAX_N) return DFR_ERR_INVALID_ARG;
    ntot += segs[i].n;
  }
  return ws_typed(kt, ntot, count, bytes);
}

int dfr_sort_batch(const dfr_segment_t* segs, uint32_t count, void* ws, size_t ws_bytes, dfr_stream_t stream) {
  if (count == 0) return DFR_OK;
  if (!segs) return DFR_ERR_INVALID_ARG;
  const int kt = segs[0].key_type;
  std::vector<HostArr> a(count);
  for (uint32_t i = 0; i < count; ++i) {
    if (segs[i].key_type != kt) return DFR_ERR_INVALID_ARG;
    a[i] = HostArr{segs[i].keys, segs[i].kbuf, segs[i].vals, segs[i].vbuf, segs[i].n};
  }
  return run_typed(kt, a.data(), count, true, ws, ws_bytes, (cudaStream_t)stream);
}

struct dfr_graph {
  cudaGraphExec_t exec;
  uint32_t nodes;
};

int dfr_graph_create(dfr_graph_t** out, const dfr_segment_t* segs, uint32_t count, void* ws, size_t ws_bytes) {
  if (!out) return DFR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!segs || count == 0) return DFR_ERR_INVALID_ARG;
  const int kt = segs[0].key_type;
  std::vector<HostArr> a(count);
  for (uint32_t i = 0; i < count; ++i) {
    if (segs[i].key_type != kt) return DFR_ERR_INVALID_ARG;
    a[i] = HostArr{segs[i].keys, segs[i].kbuf, segs[i].vals, segs[i].vbuf, segs[i].n};
  }
  cudaGraphExec_t exec = nullptr;
  uint32_t nodes = 0;
  const int rc = graph_typed(kt, a.data(), count, ws, ws_bytes, &exec, &nodes);
  if (rc != DFR_OK) return rc;
  *out = new dfr_graph{exec, nodes};
  return DFR_OK;
}

int dfr_graph_launch(dfr_graph_t* g, dfr_stream_t stream) {
  if (!g || !g->exec) return DFR_ERR_INVALID_ARG;
  if (cudaGraphLaunch(g->exec, (cudaStream_t)stream) != cudaSuccess) return DFR_ERR_CUDA;
  for (uint32_t i = 0; i < g->nodes; ++i) rt_count_launch();
  return DFR_OK;
}

int dfr_graph_destroy(dfr_graph_t* g) {
  if (!g) return DFR_ERR_INVALID_ARG;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
  return DFR_OK;
}

int dfr_tune_class(uint64_t mean_keys) {
  int lg = 0;
  while (lg < 63 && (mean_keys >> (lg + 1)) != 0) ++lg;  // floor(log2), 0 for 0 and 1
  const int c = (lg - 10) / 2;
  return lg < 12 ? 0 : (c >= DFR_TUNE_CLASSES ? DFR_TUNE_CLASSES - 1 : c);
}

int dfr_tune_get(int key_type, int size_class, dfr_tune_t* out) {
  if (!out || key_type < 0 || key_type >= kKeyTypes || size_class < 0 || size_class >= DFR_TUNE_CLASSES)
    return DFR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_tune_mu);
  tune_init_locked();
  *out = g_tune[key_type][size_class];
  return DFR_OK;
}

int dfr_tune_set(int key_type, int size_class, const dfr_tune_t* t) {
  if (!t || key_type < 0 || key_type >= kKeyTypes || size_class < 0 || size_class >= DFR_TUNE_CLASSES ||
      !tune_valid(*t))
    return DFR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_tune_mu);
  tune_init_locked();
  g_tune[key_type][size_class] = *t;
  return DFR_OK;
}

int dfr_tune_reset(void) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_init = false;
  tune_init_locked();
  return DFR_OK;
}

int dfr_sort_format(int key_type, int key_format, void* keys, void* vals, void* kbuf, void* vbuf,
                    uint64_t n, void* ws, size_t ws_bytes, dfr_stream_t stream) {
  const HostArr a{keys, kbuf, vals, vbuf, n};
  return run_typed(key_type, &a, 1u, false, ws, ws_bytes, (cudaStream_t)stream, key_format);
}

int dfr_sort_batch_format(const dfr_segment_t* segs, uint32_t count, int key_format, void* ws, size_t ws_bytes,
                          dfr_stream_t stream) {
  if (count == 0) return fmt_valid(key_format) ? DFR_OK : DFR_ERR_INVALID_ARG;
  if (!segs) return DFR_ERR_INVALID_ARG;
  const int kt = segs[0].key_type;
  std::vector<HostArr> a(count);
  for (uint32_t i = 0; i < count; ++i) {
    if (segs[i].key_type != kt) return DFR_ERR_INVALID_ARG;
    a[i] = HostArr{segs[i].keys, segs[i].kbuf, segs[i].vals, segs[i].vbuf, segs[i].n};
  }
  return run_typed(kt, a.data(), count, true, ws, ws_bytes, (cudaStream_t)stream, key_format);
}

int dfr_set_debug(uint32_t spin_limit, int force_timeout) {
  g_spin_limit.store(spin_limit ? spin_limit : kDefaultSpinLimit);
  g_force_timeout.store(force_timeout ? 1 : 0);
  return DFR_OK;
}

int dfr_profile_enable(int on) {
  g_profile.store(on ? 1 : 0);
  return DFR_OK;
}

int dfr_profile_read(double* ms_total, uint64_t* launches) {
  if (!ms_total || !launches) return DFR_ERR_INVALID_ARG;
  for (int i = 0; i < DFR_PROFILE_KINDS; ++i) {
    ms_total[i] = 0.0;
    launches[i] = 0;
  }
  std::lock_guard<std::mutex> g(g_prof_mu);
  int rc = DFR_OK;
  for (auto& r : g_prof_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      rc = DFR_ERR_CUDA;
    if (r.kind >= 0 && r.kind < DFR_PROFILE_KINDS) {
      ms_total[r.kind] += ms;
      launches[r.kind] += 1;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof_recs.clear();
  return rc;
}

const char* dfr_profile_kind_name(int kind) {
  static const char* names[DFR_PROFILE_KINDS] = {"init",     "root_count", "root_classify", "level_count",
                                                  "scatter",  "classify",   "ctasort",       "copy",
                                                  "h2d",      "warpsort",     "keyfmt",        "lsd_pass",
                                                  "lsd_plan", "persist"};
  return (kind >= 0 && kind < DFR_PROFILE_KINDS) ? names[kind] : "unknown";
}

uint64_t dfr_launch_count(void) { return g_launches.load(); }

const char* dfr_status_string(int status) {
  switch (status) {
    case DFR_OK: return "ok";
    case DFR_ERR_INVALID_ARG: return "invalid argument";
    case DFR_ERR_WORKSPACE: return "workspace too small or device queue overflow";
    case DFR_ERR_CUDA: return "CUDA runtime error";
    case DFR_ERR_TIMEOUT: return "device-side wait timed out";
    case DFR_ERR_OVER_BUDGET: return "request exceeds the memory budget";
    case DFR_ERR_BUSY: return "busy";
    case DFR_ERR_BOUNDS: return "device-side bounds check failed";
    case DFR_ERR_TOO_LARGE: return "more keys than the fixed no-allocation scratch holds";
    case DFR_ERR_HOST: return "host resource (thread or host memory) unavailable";
    default: return "unknown status";
  }
}

}  // extern "C"
