// dfr_server.cu -- the served form: a request loop over the batched sort.
//
// Requests (one array each, in caller-owned device buffers) are admitted in
// arrival order under a device-memory budget, coalesced into batches of one
// key type and sorted with the batched launch sequence (the dfr_sort_batch
// path) on one of several streams, so that batches overlap on the device.
// Requests that arrive while batches run are admitted as soon as memory and a
// stream free up (continuous batching).  Each request is timestamped when it
// is submitted and when its batch completes on the device (a host function
// enqueued behind the batch), which gives its latency.
//
// Memory: the server owns one device pool of `mem_budget_bytes`, allocated at
// creation and sub-allocated first-fit in 256-byte granules.  A batch takes
// one block: its workspace followed by scratch buffers for the requests that
// did not bring their own.  The block is returned when the batch completes.
//
// Threads: one dispatcher thread forms and launches batches and retires the
// finished ones.  The host function that marks a batch complete runs on a
// CUDA-owned thread; it makes no CUDA call and takes only `done_mu`, which no
// thread holds across a CUDA call.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dfr_host.cuh"
#include "dfr_tickets.h"

namespace dfr {
namespace {

double now_us() {
  using namespace std::chrono;
  return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

// First-fit allocator over [0, size) in 256-byte granules.
class Pool {
 public:
  explicit Pool(size_t size) {
    if (size) free_[0] = size;
  }
  size_t largest() const {
    size_t m = 0;
    for (const auto& h : free_) m = h.second > m ? h.second : m;
    return m;
  }
  // The offset of a block of `bytes` (a multiple of 256), or SIZE_MAX.
  size_t alloc(size_t bytes) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;  // offset -> length of each hole
};

struct Request {
  uint64_t ticket = 0;
  dfr_segment_t seg{};
  cudaEvent_t ready = nullptr;  // the batch's stream waits on it before sorting
  double t_submit = 0.0;
  double latency_us = 0.0;
  int status = DFR_OK;
  bool done = false;
};

constexpr size_t kMaxBatch = 4096;  // default cap on requests per batched launch sequence
constexpr int kStatusSlot = 64;     // bytes of pinned memory per batch for its error word


// Scratch bytes the server provides for a request without its own buffers.
size_t scratch_bytes(const dfr_segment_t& s) {
  size_t b = 0;
  if (!s.kbuf) b += align256(s.n * key_bytes_of(s.key_type));
  if (has_vals(s.key_type) && !s.vbuf) b += align256(s.n * val_bytes_of(s.key_type));
  return b;
}

size_t ws_bytes(int kt, uint64_t ntot, uint32_t count) {
  size_t w = 0;
  ws_typed(kt, ntot, count, &w);
  return align256(w);
}

}  // namespace
}  // namespace dfr

using namespace dfr;

struct dfr_server {
  struct Batch {
    std::vector<Request*> reqs;
    size_t off = 0, bytes = 0;  // pool block
    int stream = 0;
    int slot = 0;  // error-word slot in status_host
    int launch_status = DFR_OK;
    // written by the completion host function under done_mu
    bool finished = false;
    double t_done = 0.0;
    dfr_server* server = nullptr;
  };

  int device = 0;
  size_t budget = 0;
  unsigned char* base = nullptr;
  uint32_t* status_host = nullptr;  // pinned, one error-word slot per batch slot
  std::vector<int> free_slots;
  Pool* pool = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<uint32_t> stream_load;  // batches in flight per stream

  std::mutex mu;  // everything below, except the Batch completion fields
  std::condition_variable cv;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> requests;
  std::vector<Batch*> inflight;
  uint64_t next_ticket = 1;
  uint64_t launched_batches = 0;
  size_t max_batch = kMaxBatch;
  uint32_t max_inflight = 1;  // batches in flight per stream
  bool stop = false;

  std::mutex done_mu;
  std::thread thread;

  static void CUDART_CB on_done(void* p);
  Batch* form_batch(std::vector<dfr_segment_t>* segs);  // with mu held
  void launch(Batch* b, std::vector<dfr_segment_t>& segs);
  void retire();  // with mu held
  void run();
};

void CUDART_CB dfr_server::on_done(void* p) {
  Batch* b = static_cast<Batch*>(p);
  dfr_server* s = b->server;
  {
    std::lock_guard<std::mutex> g(s->done_mu);
    b->finished = true;
    b->t_done = now_us();
  }
  s->cv.notify_all();
}

// Take the oldest pending request and the later requests of its key type, in
// arrival order, while their batch (workspace + missing scratch) still fits
// the largest free block of the pool; reserve that block and a free stream.
dfr_server::Batch* dfr_server::form_batch(std::vector<dfr_segment_t>* segs) {
  int st = -1;
  for (size_t i = 0; i < streams.size(); ++i)
    if (stream_load[i] < max_inflight && (st < 0 || stream_load[i] < stream_load[(size_t)st])) st = (int)i;
  if (st < 0 || pending.empty() || free_slots.empty()) return nullptr;
  const int kt = pending.front()->seg.key_type;
  const size_t room = pool->largest();
  std::vector<Request*> take;
  uint64_t ntot = 0;
  size_t scratch = 0, total = 0;
  for (Request* r : pending) {
    if (r->seg.key_type != kt) continue;
    if (take.size() >= max_batch) break;
    const size_t need = ws_bytes(kt, ntot + r->seg.n, (uint32_t)take.size() + 1) + scratch + scratch_bytes(r->seg);
    if (need > room) break;  // later requests wait behind this one
    take.push_back(r);
    ntot += r->seg.n;
    scratch += scratch_bytes(r->seg);
    total = need;
  }
  if (take.empty()) return nullptr;
  Batch* b = new Batch();
  b->server = this;
  b->stream = st;
  b->reqs = take;
  b->bytes = total;
  b->off = pool->alloc(total);
  ++stream_load[st];
  b->slot = free_slots.back();
  free_slots.pop_back();
  // hand out scratch after the workspace
  size_t at = b->off + ws_bytes(kt, ntot, (uint32_t)take.size());
  segs->clear();
  for (Request* r : take) {
    dfr_segment_t g = r->seg;
    if (!g.kbuf) {
      g.kbuf = base + at;
      at += align256(g.n * key_bytes_of(kt));
    }
    if (has_vals(kt) && !g.vbuf) {
      g.vbuf = base + at;
      at += align256(g.n * val_bytes_of(kt));
    }
    segs->push_back(g);
  }
  // drop the taken requests from the queue (they are in queue order)
  size_t j = 0;
  std::deque<Request*> rest;
  for (Request* r : pending) {
    if (j < take.size() && r == take[j]) {
      ++j;
      continue;
    }
    rest.push_back(r);
  }
  pending.swap(rest);
  return b;
}

// Enqueue the waits on the requests' ready events, the batch, the read-back
// of its device error word and the completion host function on the batch's
// stream.  A batch of one request takes the plain single-array launch
// sequence.  Runs without mu.
void dfr_server::launch(Batch* b, std::vector<dfr_segment_t>& segs) {
  cudaStream_t st = streams[b->stream];
  uint32_t* slot = status_host + (size_t)b->slot * (kStatusSlot / sizeof(uint32_t));
  *slot = 0;
  void* ws = base + b->off;
  int rc = DFR_OK;
  for (Request* r : b->reqs)
    if (r->ready && cudaStreamWaitEvent(st, r->ready, 0) != cudaSuccess) rc = DFR_ERR_CUDA;
  if (rc == DFR_OK) {
    std::vector<HostArr> arrs(segs.size());
    for (size_t i = 0; i < segs.size(); ++i)
      arrs[i] = HostArr{segs[i].keys, segs[i].kbuf, segs[i].vals, segs[i].vbuf, segs[i].n};
    // With several streams the batches take the level sequence: they run side
    // by side, which a cooperative launch's whole-grid residency would
    // serialise.  A one-stream server runs its batches one after another, as
    // plain calls do, so it takes their launch form.
    rc = run_typed(segs[0].key_type, arrs.data(), (uint32_t)arrs.size(), arrs.size() > 1, ws, b->bytes, st,
                   DFR_FMT_UNSIGNED, streams.size() == 1);
  }
  bool any = false;
  for (const auto& g : segs) any = any || g.n > 1;
  if (rc == DFR_OK && any && cudaMemcpyAsync(slot, ws, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = DFR_ERR_CUDA;
  b->launch_status = rc;
  if (cudaLaunchHostFunc(st, &dfr_server::on_done, b) != cudaSuccess) {
    cudaStreamSynchronize(st);
    b->launch_status = b->launch_status == DFR_OK ? DFR_ERR_CUDA : b->launch_status;
    on_done(b);
  }
}

// Give back the memory and stream of every finished batch and complete its
// requests: latency = completion time on the device - submission time.
void dfr_server::retire() {
  for (size_t i = 0; i < inflight.size();) {
    Batch* b = inflight[i];
    bool fin;
    double t;
    {
      std::lock_guard<std::mutex> g(done_mu);
      fin = b->finished;
      t = b->t_done;
    }
    if (!fin) {
      ++i;
      continue;
    }
    const uint32_t* slot = status_host + (size_t)b->slot * (kStatusSlot / sizeof(uint32_t));
    const int st = b->launch_status != DFR_OK ? b->launch_status : map_device_status(*slot);
    free_slots.push_back(b->slot);
    for (Request* r : b->reqs) {
      r->status = st;
      r->latency_us = t - r->t_submit;
      r->done = true;
    }
    pool->release(b->off, b->bytes);
    --stream_load[b->stream];
    inflight.erase(inflight.begin() + (long)i);
    delete b;
    cv.notify_all();
  }
}

void dfr_server::run() {
  cudaSetDevice(device);
  std::vector<dfr_segment_t> segs;
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    retire();
    Batch* b = form_batch(&segs);
    if (b) {
      inflight.push_back(b);
      ++launched_batches;
      lk.unlock();
      launch(b, segs);
      lk.lock();
      continue;
    }
    if (stop && pending.empty() && inflight.empty()) break;
    // completions notify without mu held: the timeout bounds a missed wake-up
    cv.wait_for(lk, std::chrono::microseconds(100));
  }
}

extern "C" {

int dfr_server_create(dfr_server_t** out, int device, size_t mem_budget_bytes, int n_streams) {
  if (!out) return DFR_ERR_INVALID_ARG;
  *out = nullptr;
  if (mem_budget_bytes < 4096 || n_streams < 1 || n_streams > DFR_SERVER_MAX_STREAMS) return DFR_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return DFR_ERR_CUDA;
  dfr_server* s = new (std::nothrow) dfr_server();
  if (!s) return DFR_ERR_HOST;
  s->device = device;
  s->budget = mem_budget_bytes & ~(size_t)255;
  int rc = DFR_OK;
  auto release = [s] {
    for (auto x : s->streams) cudaStreamDestroy(x);
    if (s->status_host) cudaFreeHost(s->status_host);
    if (s->base) cudaFree(s->base);
    delete s->pool;
    delete s;
  };
  try {
    bool ok = cudaMalloc(&s->base, s->budget) == cudaSuccess;
    const size_t nslots = (size_t)n_streams * DFR_SERVER_MAX_INFLIGHT;
    ok = ok && cudaMallocHost(&s->status_host, nslots * kStatusSlot) == cudaSuccess;
    for (size_t i = 0; ok && i < nslots; ++i) s->free_slots.push_back((int)(nslots - 1 - i));
    for (int i = 0; ok && i < n_streams; ++i) {
      cudaStream_t st;
      ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) {
        s->streams.push_back(st);
        s->stream_load.push_back(0u);
      }
    }
    if (!ok) rc = DFR_ERR_CUDA;
    if (rc == DFR_OK) s->pool = new Pool(s->budget);
  } catch (...) {  // host memory for the bookkeeping (std::bad_alloc)
    rc = DFR_ERR_HOST;
  }
  if (rc == DFR_OK && !start_thread(&s->thread, [s] { s->run(); }, SpawnStdThread{})) rc = DFR_ERR_HOST;
  if (rc != DFR_OK) {
    release();
    return rc;
  }
  *out = s;
  return DFR_OK;
}

int dfr_submit_after(dfr_server_t* s, const dfr_segment_t* req, void* ready_event, uint64_t* ticket) {
  if (!s || !req || !ticket) return DFR_ERR_INVALID_ARG;
  const dfr_segment_t& g = *req;
  if (!key_type_valid(g.key_type) || g.n > DFR_MAX_N) return DFR_ERR_INVALID_ARG;
  if (g.n > 1) {
    const size_t kb = key_bytes_of(g.key_type);
    if (!g.keys || ((uintptr_t)g.keys % kb) || (g.kbuf && ((uintptr_t)g.kbuf % kb))) return DFR_ERR_INVALID_ARG;
    const size_t vb = val_bytes_of(g.key_type);
    if (has_vals(g.key_type) && (!g.vals || ((uintptr_t)g.vals % vb) || (g.vbuf && ((uintptr_t)g.vbuf % vb))))
      return DFR_ERR_INVALID_ARG;
  }
  if (ws_bytes(g.key_type, g.n, 1u) + scratch_bytes(g) > s->budget) return DFR_ERR_OVER_BUDGET;
  Request* r = new Request();
  r->seg = g;
  r->ready = static_cast<cudaEvent_t>(ready_event);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return DFR_ERR_BUSY;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = now_us();
    s->requests[r->ticket] = r;
    s->pending.push_back(r);
    *ticket = r->ticket;
  }
  s->cv.notify_all();
  return DFR_OK;
}

int dfr_submit(dfr_server_t* s, const dfr_segment_t* req, uint64_t* ticket) {
  return dfr_submit_after(s, req, nullptr, ticket);
}

int dfr_server_set_limits(dfr_server_t* s, uint32_t max_batch, uint32_t max_inflight_per_stream) {
  if (!s || max_batch < 1 || max_batch > kMaxBatch || max_inflight_per_stream < 1 ||
      max_inflight_per_stream > DFR_SERVER_MAX_INFLIGHT)
    return DFR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->max_batch = max_batch;
  s->max_inflight = max_inflight_per_stream;
  return DFR_OK;
}

int dfr_poll(dfr_server_t* s, uint64_t ticket, int* done, double* latency_us) {
  if (!s || !done) return DFR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  Request* r = nullptr;
  const Ticket t = take_if_done(s->requests, ticket, &r);
  *done = t == Ticket::done ? 1 : 0;
  if (t == Ticket::unknown) return DFR_ERR_INVALID_ARG;
  if (t == Ticket::pending) return DFR_OK;
  if (latency_us) *latency_us = r->latency_us;
  const int st = r->status;
  delete r;
  return st;
}

int dfr_wait(dfr_server_t* s, uint64_t ticket, double* latency_us) {
  if (!s) return DFR_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  Request* r = nullptr;
  if (wait_and_take(lk, s->cv, s->requests, ticket, &r) != Ticket::done) return DFR_ERR_INVALID_ARG;
  if (latency_us) *latency_us = r->latency_us;
  const int st = r->status;
  delete r;
  return st;
}

int dfr_server_stats(dfr_server_t* s, uint64_t* batches, uint64_t* pending, uint64_t* inflight) {
  if (!s) return DFR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->launched_batches;
  if (pending) *pending = s->pending.size();
  if (inflight) *inflight = s->inflight.size();
  return DFR_OK;
}

int dfr_server_destroy(dfr_server_t* s) {
  if (!s) return DFR_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->thread.joinable()) s->thread.join();
  cudaSetDevice(s->device);
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFreeHost(s->status_host);
  cudaFree(s->base);
  for (auto& kv : s->requests) delete kv.second;
  delete s->pool;
  delete s;
  return DFR_OK;
}

}  // extern "C"
