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
  bool ready;           // set-up succeeded on this device (a failed set-up is retried by the next call)
  unsigned char* base;  // device address of g_noalloc_scratch on this device
  Grids grids;
  int sms;
};

constexpr int kMaxDevices = 64;
NoAllocDevice g_dev[kMaxDevices];
std::mutex g_noalloc_mu;

using K = uint32_t;
using V = NoVal;
constexpr int G = 1;  // arrays of at most 2^20 keys: the small-array geometry
using T = Kernels<K, V, G>;

// Once per device, with the device current: resolve the scratch address and
// the persistent grid sizes.  Returns a DFR status.
int setup(int dev, NoAllocDevice* d) {
  const size_t need = align256(kNoAllocMaxN * sizeof(K)) + make_layout<K, V, G>(kNoAllocMaxN, 1u).total;
  if (need > kNoAllocScratchBytes) return DFR_ERR_WORKSPACE;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return DFR_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return DFR_ERR_CUDA;
  auto grid_of = [sms](const void* kern, int threads, size_t smem) -> int {
    int per_sm = 0;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) return -1;
    return (per_sm < 1 ? 1 : per_sm) * sms;
  };
  if (!T::grids(grid_of, &d->grids)) return DFR_ERR_CUDA;
  d->sms = sms;
  d->base = static_cast<unsigned char*>(p);
  return DFR_OK;
}

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
      const int rc = setup(dev, d);
      if (rc != DFR_OK) {
        // Leave the device un-set-up so that a later call retries (the failure
        // may be transient, e.g. a first call made inside a stream capture),
        // and take back the non-sticky error the failed runtime call left, so
        // that the caller's next cudaGetLastError does not report it.
        cudaGetLastError();
        return rc;
      }
      d->ready = true;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;

  // scratch buffer first, then the workspace (both 256-byte aligned)
  unsigned char* buf = d->base;
  void* ws = d->base + align256(n * sizeof(K));
  if (ranges_overlap(keys, n * sizeof(K), d->base, kNoAllocScratchBytes)) return DFR_ERR_INVALID_ARG;
  const Layout lay = make_layout<K, V, G>(n, 1u);
  Ctx c = make_ctx(ws, lay, 1u);
  c.spin_limit = rt_spin_limit();
  c.force_timeout = 0u;
  c.nlev = (uint32_t)T::nlev;
  const dfr_tune_t tune = rt_tune(DFR_U32, n);
  ctx_plan<K, V>(&c, tune);
  Grids g = d->grids;
  apply_tune(tune, d->sms, &g);
  const uint32_t rt = (uint32_t)((n + T::TILE - 1) / T::TILE);
  const ArrDesc a0{keys, buf, nullptr, nullptr, (uint32_t)n, 0u};
  enqueue_sort<K, V, G>(c, lay, g, 1u, rt, (unsigned long long)n, a0, true, st,
                     [](int, cudaStream_t, auto&& fn) {
                       fn();
                       rt_count_launch();
                     });
  return cudaGetLastError() == cudaSuccess ? DFR_OK : DFR_ERR_CUDA;
}
