// dfr_u32_kv.cu -- instantiation of the DFR sort driver for key type uint32_t, payload uint32_t.
#include "dfr_host.cuh"

namespace dfr {

int run_u32_kv(const HostArr* a, uint32_t n, bool batch, void* ws, size_t wsb, cudaStream_t st, int fmt, bool persist_ok) {
  return run_sort<uint32_t, uint32_t>(a, n, batch, ws, wsb, st, fmt, persist_ok);
}

size_t ws_u32_kv(uint64_t ntot, uint32_t narr) { return workspace_bytes<uint32_t, uint32_t>(ntot, narr); }

int graph_u32_kv(const HostArr* a, uint32_t n, void* ws, size_t wsb, cudaGraphExec_t* out, uint32_t* nodes) {
  return build_graph<uint32_t, uint32_t>(a, n, ws, wsb, out, nodes);
}

}  // namespace dfr
