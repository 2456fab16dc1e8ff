// dfr_noalloc.cu -- dfr_sort_u32_noalloc: the plain u32 sort for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where a cudaMalloc is not allowed or not
// wanted -- a plug-in inside a host application that owns every byte of
// device memory through its own allocator, a library called under a strict
// per-process memory quota, or a latency-critical loop where the implicit
// device synchronisation of cudaMalloc/cudaFree is unacceptable.  Such a
// caller can hand over its keys but not a scratch buffer and a workspace.
//
// How: the scratch buffer (the sort's extra buffer) and the workspace live in
// one file-scope device array of fixed size, which every GPU that loads this
// library holds until the process exits.  Host code never uses the array's
// name as an address: once per device, with that device current, the first
// call asks the runtime for the array's device address
// (cudaGetSymbolAddress) and caches it together with the launch grid sizes.
// That first call should therefore come before any stream capture.
//
// Sharing: every call on a device uses the same array, which keeps whatever
// the previous call left in it.  The launch sequence clears what must start
// at zero (control block and root accumulators) and writes every other region
// before reading it.  Two calls whose work overlaps on the GPU (different
// streams, or different host threads without ordering) race on the array:
// the caller must serialise them.
//
// No device or host allocation happens in this file: no cudaMalloc, no
// cudaFree, no allocating library routine, no heap containers.
#include <mutex>

#include "dfr_host.cuh"

namespace dfr {
namespace {

// Largest array the fixed scratch holds, and the scratch size: the u32
// scratch buffer (4 bytes per key) plus the u32 workspace for that many keys,
// with slack.  setup() verifies the fit against the real workspace layout.
constexpr uint64_t kNoAllocMaxN = DFR_NOALLOC_MAX_N;
constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
  bool ready;
  int status;
  unsigned char* base;  // device address of g_noalloc_scratch on this device
  int g_rc, g_rcl, g_lc, g_sc, g_cl, g_cs, g_cp;
};

constexpr int kMaxDevices = 64;
NoAllocDevice g_dev[kMaxDevices];
std::mutex g_noalloc_mu;

using K = uint32_t;
using V = NoVal;
using C = Cfg<K, V>;
constexpr int SNT = C::SNT, SKPT = C::SKPT, TILE = SNT * SKPT;
constexpr int CNT = C::CNT, CKPT = C::CKPT, TCTA = CNT * CKPT;
constexpr size_t kScatterSmem = scatter_smem_bytes<K, V, SNT, SKPT>();
constexpr size_t kCtaSmem = ctasort_smem_bytes<K, V, CNT, CKPT>();

int grid_of(const void* kern, int threads, size_t smem, int sms) {
  int per_sm = 0;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) return -1;
  return (per_sm < 1 ? 1 : per_sm) * sms;
}

// Once per device, with the device current: resolve the scratch address and
// the persistent grid sizes.  Returns a DFR status.
int setup(int dev, NoAllocDevice* d) {
  const size_t need = align256(kNoAllocMaxN * sizeof(K)) + make_layout<K, V>(kNoAllocMaxN, 1u).total;
  if (need > kNoAllocScratchBytes) return DFR_ERR_WORKSPACE;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return DFR_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return DFR_ERR_CUDA;
  d->g_rc = grid_of((const void*)k_root_count<K, SNT, TILE>, SNT, 0, sms);
  d->g_rcl = grid_of((const void*)k_root_classify<K, V, TILE, TCTA>, 256, 0, sms);
  d->g_lc = grid_of((const void*)k_level_count<K, SNT, TILE>, SNT, 0, sms);
  d->g_sc = grid_of((const void*)k_scatter<K, V, SNT, SKPT>, SNT, kScatterSmem, sms);
  d->g_cl = grid_of((const void*)k_classify<K, V, TILE, TCTA>, 256, 0, sms);
  d->g_cs = grid_of((const void*)k_ctasort<K, V, CNT, CKPT>, CNT, kCtaSmem, sms);
  d->g_cp = grid_of((const void*)k_copy<K, V, SNT, TILE>, SNT, 0, sms);
  if (d->g_rc < 0 || d->g_rcl < 0 || d->g_lc < 0 || d->g_sc < 0 || d->g_cl < 0 || d->g_cs < 0 || d->g_cp < 0)
    return DFR_ERR_CUDA;
  d->base = static_cast<unsigned char*>(p);
  return DFR_OK;
}

inline uint32_t min_u32(uint32_t a, uint32_t b) { return a < b ? a : b; }

}  // namespace
}  // namespace dfr

using namespace dfr;

extern "C" int dfr_sort_u32_noalloc(uint32_t* keys, uint64_t n, dfr_stream_t stream) {
  if (n <= 1) return DFR_OK;
  if (!keys || ((uintptr_t)keys % sizeof(uint32_t))) return DFR_ERR_INVALID_ARG;
  if (n > kNoAllocMaxN) return DFR_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DFR_ERR_CUDA;
  NoAllocDevice* d = &g_dev[dev];
  {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!d->ready) {
      d->status = setup(dev, d);
      d->ready = true;
    }
  }
  if (d->status != DFR_OK) return d->status;
  cudaStream_t st = (cudaStream_t)stream;

  // scratch buffer first, then the workspace (both 256-byte aligned)
  unsigned char* buf = d->base;
  void* ws = d->base + align256(n * sizeof(K));
  if (ranges_overlap(keys, n * sizeof(K), d->base, kNoAllocScratchBytes)) return DFR_ERR_INVALID_ARG;
  const Layout lay = make_layout<K, V>(n, 1u);
  Ctx c = make_ctx(ws, lay, 1u);
  c.spin_limit = rt_spin_limit();
  c.force_timeout = 0u;

  const uint32_t rt = (uint32_t)((n + TILE - 1) / TILE);
  const ArrDesc a0{keys, buf, nullptr, nullptr, (uint32_t)n, 0u};
  const uint32_t root_words = (uint32_t)(sizeof(RootAcc<K>) / 4);
  const uint32_t words = (uint32_t)(sizeof(Ctl) / 4) + root_words;
  k_init<K><<<(words + 255) / 256, 256, 0, st>>>(c, a0, 1, root_words);
  rt_count_launch();
  k_root_count<K, SNT, TILE><<<min_u32(rt, (uint32_t)d->g_rc), SNT, 0, st>>>(c, rt);
  rt_count_launch();
  k_root_classify<K, V, TILE, TCTA><<<1, 256, 0, st>>>(c, (unsigned long long)n);
  rt_count_launch();
  const uint32_t lc_grid = min_u32(lay.tilecap, (uint32_t)d->g_lc);
  const uint32_t sc_grid = min_u32(lay.tilecap, (uint32_t)d->g_sc);
  const uint32_t cl_grid = min_u32(lay.segcap, (uint32_t)d->g_cl);
  for (int L = 0; L < (int)sizeof(K); ++L) {
    k_level_count<K, SNT, TILE><<<lc_grid, SNT, 0, st>>>(c, L);
    rt_count_launch();
    k_scatter<K, V, SNT, SKPT><<<sc_grid, SNT, kScatterSmem, st>>>(c, L);
    rt_count_launch();
    k_classify<K, V, TILE, TCTA><<<cl_grid, 256, 0, st>>>(c, L);
    rt_count_launch();
  }
  k_ctasort<K, V, CNT, CKPT><<<min_u32(lay.ctacap, (uint32_t)d->g_cs), CNT, kCtaSmem, st>>>(c);
  rt_count_launch();
  k_copy<K, V, SNT, TILE><<<min_u32(lay.copytilecap, (uint32_t)d->g_cp), SNT, 0, st>>>(c);
  rt_count_launch();
  return cudaGetLastError() == cudaSuccess ? DFR_OK : DFR_ERR_CUDA;
}
