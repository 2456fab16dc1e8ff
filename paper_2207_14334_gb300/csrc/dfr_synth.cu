// dfr_synth.cu -- seeded synthetic keys generated on the device.
//
// Benchmarks of the served form generate each request's keys at its arrival,
// because the total stream (about 10^11 keys) cannot be staged in advance.
// The generator is SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): output i (0-based) of the
// stream seeded with s is
//     z  = s + (i + 1) * 0x9E3779B97F4A7C15
//     z  = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
//     z  = (z ^ (z >> 27)) * 0x94D049BB133111EB
//     out = z ^ (z >> 31)
// A u32 key is the high half of the output.  The host-side generator module
// implements the same definition in numpy, so any request can be regenerated
// on the CPU and checked against the CPU sort.  Nothing here belongs to the
// sort itself.
#include "dfr_host.cuh"

namespace dfr {
namespace {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t s, uint64_t i) {
  uint64_t z = s + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_fill_splitmix64(void* keys, void* vals, int vwide, uint64_t n, int wide, uint64_t seed) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t z = splitmix64_at(seed, i);
    if (wide)
      static_cast<uint64_t*>(keys)[i] = z;
    else
      static_cast<uint32_t*>(keys)[i] = (uint32_t)(z >> 32);
    if (vals) {
      if (vwide)
        static_cast<uint64_t*>(vals)[i] = i;
      else
        static_cast<uint32_t*>(vals)[i] = (uint32_t)i;
    }
  }
}

}  // namespace
}  // namespace dfr

using namespace dfr;

extern "C" int dfr_fill_splitmix64(int key_type, void* keys, void* vals, uint64_t n, uint64_t seed,
                                   dfr_stream_t stream) {
  if (!key_type_valid(key_type)) return DFR_ERR_INVALID_ARG;
  if (n == 0) return DFR_OK;
  const bool wide = key_bytes_of(key_type) == 8u;
  const bool kv = has_vals(key_type);
  const size_t vb = val_bytes_of(key_type);
  if (!keys || ((uintptr_t)keys % (wide ? 8u : 4u))) return DFR_ERR_INVALID_ARG;
  if (kv && (!vals || ((uintptr_t)vals % vb))) return DFR_ERR_INVALID_ARG;
  if (n > DFR_MAX_N) return DFR_ERR_INVALID_ARG;
  const int threads = 256;
  const uint64_t want = (n + threads - 1) / threads;
  const int blocks = (int)(want < 4096 ? want : 4096);
  k_fill_splitmix64<<<blocks, threads, 0, (cudaStream_t)stream>>>(keys, kv ? vals : nullptr, vb == 8u ? 1 : 0, n,
                                                                  wide ? 1 : 0, seed);
  rt_count_launch();
  return cudaGetLastError() == cudaSuccess ? DFR_OK : DFR_ERR_CUDA;
}
