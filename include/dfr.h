/*
 * dfr.h -- C ABI of the GB300 (sm_103a) Diverting Fast Radix sort library.
 *
 * The library sorts unsigned integer keys (optionally with 32-bit payloads)
 * ascending and STABLY, with the hot path of the paper's Diverting Fast Radix
 * method: a recursive most-significant-digit radix partition (count, convert
 * the counts into indices, deal; Preliminaries and Section "Most Significant
 * Digit (MSD) Radix Sorts"), where every bucket below a size threshold is
 * diverted to a different, stable small-bucket sort (Algorithm 2 and Section
 * "Analysis", the diversion threshold N_d) and buckets holding one repeated
 * key are left alone (Section MSD: last-digit buckets hold equal keys).
 *
 * Conventions shared by every call:
 *   - Pointers to keys, payloads, scratch buffers and workspace are DEVICE
 *     pointers owned by the caller (allocate them however you like, e.g. with
 *     PyTorch).  The library allocates no device memory in these calls.
 *   - Every sort call is asynchronous on `stream` (0 = legacy default stream):
 *     it only enqueues kernels and returns.  Device-side failures are recorded
 *     in a status word inside the workspace; read them with
 *     dfr_last_device_status().
 *   - The result lands in place in `keys` (and `vals`).  `buf`/`vbuf` are the
 *     paper's extra buffer, as large as the input (Section MSD); their
 *     contents are undefined afterwards.
 *   - n == 0 and n == 1 return DFR_OK without touching the GPU.
 *   - A single array may hold at most DFR_MAX_N keys.
 *   - Ranges [keys, keys+n) and [buf, buf+n) (and the payload pair) must not
 *     overlap; overlap returns DFR_ERR_INVALID_ARG.  The workspace must not
 *     overlap any of them either, and the arrays of one batch must be
 *     disjoint from one another; these two are not checked (the result is
 *     undefined).
 *   - The workspace must be at least dfr_workspace_bytes() bytes and 256-byte
 *     aligned.  One workspace serves one call at a time: calls sharing a
 *     workspace must be ordered on one stream (or otherwise serialised).
 *
 * Return codes: DFR_OK on success, otherwise one of the DFR_ERR_* values;
 * a call that returns an error enqueues nothing.
 */
#ifndef DFR_H
#define DFR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; declared here so this header needs no CUDA
 * include. */
typedef struct CUstream_st* dfr_stream_t;

enum dfr_status {
    DFR_OK = 0,
    DFR_ERR_INVALID_ARG = 1,  /* null pointer, overlap, n too large, misaligned workspace */
    DFR_ERR_WORKSPACE = 2,    /* workspace smaller than required, or a device queue overflowed */
    DFR_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    DFR_ERR_TIMEOUT = 4,      /* a device-side wait gave up after its iteration limit */
    DFR_ERR_OVER_BUDGET = 5,  /* a served request exceeds the server's memory budget */
    DFR_ERR_BUSY = 6,         /* the server cannot take the request now */
    DFR_ERR_BOUNDS = 7,       /* a device-side bounds check rejected a write (result invalid) */
    DFR_ERR_TOO_LARGE = 8,    /* more keys than dfr_sort_u32_noalloc's fixed scratch holds */
    DFR_ERR_HOST = 9          /* a host resource (a thread, host memory) could not be obtained */
};

enum dfr_key_type {
    DFR_U32 = 0,       /* uint32 keys */
    DFR_U64 = 1,       /* uint64 keys */
    DFR_U64_KV = 2,    /* uint64 keys with uint32 payloads */
    DFR_U32_KV = 3,    /* uint32 keys with uint32 payloads */
    DFR_U64_KV64 = 4,  /* uint64 keys with uint64 payloads */
    DFR_U32_KV64 = 5   /* uint32 keys with uint64 payloads */
};

/* Largest number of keys in one array (the decoupled look-back keeps 30-bit
 * counts per digit). */
#define DFR_MAX_N ((uint64_t)((1u << 30) - 1u))

/*
 * dfr_workspace_bytes -- bytes of device workspace one sort of n keys of
 * `key_type` needs.  Pure host arithmetic, no CUDA call.
 * Errors: DFR_ERR_INVALID_ARG for an unknown key type, n > DFR_MAX_N or a
 * null `bytes`.
 */
int dfr_workspace_bytes(int key_type, uint64_t n, size_t* bytes);

/*
 * dfr_sort_u32 -- sort n uint32 keys ascending in place (the whole DFR path:
 * count, prefix, deal per level; divert small buckets; leave constant buckets).
 *   keys  [n] device, in/out
 *   buf   [n] device scratch (the extra buffer of Algorithm 2)
 *   ws    device workspace of ws_bytes >= dfr_workspace_bytes(DFR_U32, n)
 */
int dfr_sort_u32(uint32_t* keys, uint32_t* buf, uint64_t n, void* ws, size_t ws_bytes,
                 dfr_stream_t stream);

/* dfr_sort_u64 -- as dfr_sort_u32 for uint64 keys (DFR_U64 workspace). */
int dfr_sort_u64(uint64_t* keys, uint64_t* buf, uint64_t n, void* ws, size_t ws_bytes,
                 dfr_stream_t stream);

/*
 * dfr_sort_u64_kv -- stable sort of (uint64 key, uint32 payload) records by
 * key: each payload moves with its key and equal keys keep their input order
 * (Section MSD: stable with an extra buffer and a stable diversion).
 *   keys/vals [n] device in/out;  kbuf/vbuf [n] device scratch.
 */
int dfr_sort_u64_kv(uint64_t* keys, uint32_t* vals, uint64_t* kbuf, uint32_t* vbuf, uint64_t n,
                    void* ws, size_t ws_bytes, dfr_stream_t stream);

/* dfr_sort_u32_kv -- as dfr_sort_u64_kv for uint32 keys (DFR_U32_KV workspace). */
int dfr_sort_u32_kv(uint32_t* keys, uint32_t* vals, uint32_t* kbuf, uint32_t* vbuf, uint64_t n,
                    void* ws, size_t ws_bytes, dfr_stream_t stream);

/*
 * dfr_sort_u64_kv64 / dfr_sort_u32_kv64 -- the same stable key-value sort with
 * 64-bit payloads: records of the paper's statement of the problem carry
 * data beside their key (Preliminaries), and a 64-bit payload holds a
 * pointer, an offset into a large table or a second key word.  Payloads are
 * moved, never read as numbers.  `vals`/`vbuf` must be 8-byte aligned;
 * workspace of type DFR_U64_KV64 / DFR_U32_KV64.
 */
int dfr_sort_u64_kv64(uint64_t* keys, uint64_t* vals, uint64_t* kbuf, uint64_t* vbuf, uint64_t n,
                      void* ws, size_t ws_bytes, dfr_stream_t stream);
int dfr_sort_u32_kv64(uint32_t* keys, uint64_t* vals, uint32_t* kbuf, uint64_t* vbuf, uint64_t n,
                      void* ws, size_t ws_bytes, dfr_stream_t stream);

/*
 * dfr_last_device_status -- wait for `stream`, then report the device status
 * word of the last call that used `ws`: DFR_OK, DFR_ERR_TIMEOUT,
 * DFR_ERR_BOUNDS or DFR_ERR_WORKSPACE (queue capacity), in *status.
 * Returns DFR_ERR_CUDA if the copy or the synchronisation fails.
 */
int dfr_last_device_status(const void* ws, dfr_stream_t stream, int* status);

/* Per-call counters, filled from the workspace by dfr_get_stats(). */
#define DFR_STATS_MAX_LEVELS 16
typedef struct {
    uint64_t n_total;                                  /* keys in the call (all arrays) */
    uint32_t key_bytes, val_bytes;                     /* w and v */
    uint32_t levels;                                   /* partition levels that did work */
    uint32_t device_status;                            /* as dfr_last_device_status */
    uint64_t level_segments[DFR_STATS_MAX_LEVELS];     /* large segments partitioned per level */
    uint64_t level_tiles[DFR_STATS_MAX_LEVELS];        /* tiles per level */
    uint64_t level_keys[DFR_STATS_MAX_LEVELS];         /* keys dealt per level */
    uint64_t level_hist_keys[DFR_STATS_MAX_LEVELS];    /* keys re-read by a per-level count */
    uint64_t cta_buckets, cta_keys;                    /* diverted to the CTA shared-memory sort */
    uint64_t tiny_buckets, tiny_keys;                  /* diverted to the warp sort */
    uint64_t const_buckets, const_keys;                /* constant buckets left alone */
    uint64_t copy_keys;                                /* constant keys moved back from buf */
    uint64_t model_bytes;                              /* minimal bytes of the executed plan */
    uint64_t wsort_buckets, wsort_keys;                /* diverted to the warp shared-memory sort */
    uint32_t device_error_site;                        /* first failed device check (0 = none; see dfr_api.cu) */
    uint32_t schedule;                                 /* how the top digits were sorted: DFR_SCHED_MSD, _LSD or
                                                          _DFR (an estimate that failed reports DFR_SCHED_MSD) */
    uint64_t group_buckets;                            /* diverted key-only buckets finished by one counting pass
                                                          plus in-group ranking */
    uint64_t lsd_keys;                                 /* keys dealt by the LSD passes (both passes; includes the
                                                          part of a failed estimated pass that ran) */
    uint64_t est_overflow;                             /* keys the estimated deal sent to overflow regions */
    uint32_t est_capacity;                             /* keys per estimated bucket (0 unless DFR_SCHED_DFR ran) */
    uint32_t est_aborted;                              /* 1: an overflow region filled up and the MSD schedule
                                                          sorted the array instead */
    uint32_t root_read;                                /* 1: the root count read the keys (0 when the estimated
                                                          deal counted them) */
    uint32_t persistent;                               /* 1: the call ran as one persistent launch
                                                          (DFR_LAUNCH_*) */
} dfr_stats_t;

/* dfr_get_stats -- wait for `stream` and copy the counters of the last call
 * that used `ws` into *out.  DFR_ERR_CUDA on a failed copy. */
int dfr_get_stats(const void* ws, dfr_stream_t stream, dfr_stats_t* out);

/*
 * dfr_sort_u32_noalloc -- dfr_sort_u32 for callers that cannot allocate
 * device memory.  The paper has no counterpart: it is a deployment variant.
 *
 * Some callers cannot hand over a scratch buffer and a workspace: a plug-in
 * inside a host application that owns all device memory through its own
 * allocator, code running under a strict per-process memory quota, or a
 * latency-critical loop that must not pay cudaMalloc's implicit device
 * synchronisation.  This call needs only the keys: its scratch buffer and
 * workspace live in a fixed device array inside the library, which every GPU
 * that loads the library holds until the process exits.
 *   keys  [n] device, in/out;  n <= DFR_NOALLOC_MAX_N.
 * Returns DFR_ERR_TOO_LARGE for n > DFR_NOALLOC_MAX_N (nothing enqueued),
 * DFR_ERR_INVALID_ARG for a null or misaligned `keys` or keys inside the
 * fixed array, DFR_ERR_CUDA if the launch or the one-time set-up fails (a
 * failed set-up is retried by the next call).  It calls no cudaMalloc, no
 * cudaFree and no allocating library routine.
 * The first call on a device (with that device current) resolves the fixed
 * array's device address; make that first call before any stream capture.
 * Every call on a device shares the one array, which keeps the previous
 * call's contents; the call clears what must start at zero itself.  Calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * the array: serialise them.
 * Device-side status: there is no caller-visible workspace, so the device
 * status word of this call cannot be read back.  For u32 key-only arrays of
 * at most DFR_NOALLOC_MAX_N keys the launch sequence contains no device-side
 * wait (tiles claim bucket runs with atomics; the look-back of the LSD
 * schedules only serves larger arrays), so DFR_ERR_TIMEOUT cannot arise, and
 * the bounds and queue-capacity checks fail only after an internal fault.  If
 * one did fail, the keys would be left unsorted with nothing reported:
 * callers that must see the device status use dfr_sort_u32 with their own
 * workspace and dfr_last_device_status().
 */
#define DFR_NOALLOC_MAX_N ((uint64_t)1u << 20)
int dfr_sort_u32_noalloc(uint32_t* keys, uint64_t n, dfr_stream_t stream);

/* ---------------------------------------------------------------- batch -- */

/* One array of a batch.  All arrays of one batch call share `key_type`. */
typedef struct {
    int key_type;   /* one of enum dfr_key_type */
    void* keys;     /* [n] device, in/out */
    void* vals;     /* [n] device payloads of 4 or 8 bytes (kv types only, else NULL) */
    void* kbuf;     /* [n] device scratch for keys */
    void* vbuf;     /* [n] device scratch for payloads (kv types only) */
    uint64_t n;
} dfr_segment_t;

/*
 * dfr_batch_workspace_bytes -- workspace bytes for one dfr_sort_batch call
 * over `count` arrays (host array `segs`).  No CUDA call.
 */
int dfr_batch_workspace_bytes(const dfr_segment_t* segs, uint32_t count, size_t* bytes);

/*
 * dfr_sort_batch -- sort `count` independent arrays with one launch sequence:
 * every kernel is persistent and pulls tiles and buckets of all arrays from
 * device work queues, so thousands of uneven arrays cost the same number of
 * launches as one.  Each array's result is exactly that of sorting it alone.
 * The descriptor table is copied to the device before the call returns, so
 * `segs` may be reused at once.
 * Errors: DFR_ERR_INVALID_ARG for mixed key types, null pointers, overlap
 * within one array's buffers or an array above DFR_MAX_N; DFR_ERR_WORKSPACE
 * for a short workspace.  Distinct arrays must not share memory (unchecked).
 */
int dfr_sort_batch(const dfr_segment_t* segs, uint32_t count, void* ws, size_t ws_bytes,
                   dfr_stream_t stream);

/* ----------------------------------------------------------- key formats -- */

/*
 * Signed, floating-point and descending keys.  The sort orders unsigned
 * integers; other orders are reduced to it by an order-preserving bijection
 * of the key's bits, applied in place before the sort and undone after it
 * (two extra read+write passes over the keys):
 *   DFR_FMT_SIGNED      two's complement (int32 / int64): flip the sign bit;
 *   DFR_FMT_FLOAT       IEEE 754 binary32 / binary64 in totalOrder:
 *                       -NaN < -inf < ... < -0.0 < +0.0 < ... < +inf < +NaN
 *                       (NaNs ordered by their payload bits): flip every bit
 *                       of a negative value, set the sign bit of a positive one;
 *   DFR_FMT_DESCENDING  flag: largest key first; equal keys still keep input
 *                       order (stable): complement the image.
 * The width comes from the key type (DFR_U32, DFR_U32_KV, DFR_U32_KV64:
 * 32-bit keys; DFR_U64, DFR_U64_KV, DFR_U64_KV64: 64-bit keys); payloads are
 * unchanged.  Workspace and
 * buffers as for the unsigned sorts.  DFR_ERR_INVALID_ARG for an unknown
 * format.
 */
enum dfr_key_format {
    DFR_FMT_UNSIGNED = 0,
    DFR_FMT_SIGNED = 1,
    DFR_FMT_FLOAT = 2,
    DFR_FMT_DESCENDING = 0x100
};
int dfr_sort_format(int key_type, int key_format, void* keys, void* vals, void* kbuf, void* vbuf,
                    uint64_t n, void* ws, size_t ws_bytes, dfr_stream_t stream);
int dfr_sort_batch_format(const dfr_segment_t* segs, uint32_t count, int key_format, void* ws, size_t ws_bytes,
                          dfr_stream_t stream);

/* --------------------------------------------------------------- graphs -- */

/*
 * A sort captured once into a CUDA graph and launched many times: for
 * callers that sort the same buffers repeatedly (refilling the keys between
 * launches), one graph launch replaces the call's ~24 kernel launches.  The
 * graph is bound to the segments' pointers and lengths and to `ws` (which it
 * owns while it lives: no other call may use that workspace), and to the
 * launch plan in force at creation.  dfr_graph_create uploads the descriptor
 * table synchronously and captures on a private stream; it fails like
 * dfr_sort_batch on bad arguments (DFR_ERR_INVALID_ARG, DFR_ERR_WORKSPACE) or
 * with DFR_ERR_CUDA.  dfr_graph_launch enqueues one complete sort on
 * `stream`; device errors land in `ws` as for the other calls.
 */
typedef struct dfr_graph dfr_graph_t;
int dfr_graph_create(dfr_graph_t** graph, const dfr_segment_t* segs, uint32_t count, void* ws, size_t ws_bytes);
int dfr_graph_launch(dfr_graph_t* graph, dfr_stream_t stream);
int dfr_graph_destroy(dfr_graph_t* graph);

/* --------------------------------------------------------------- served -- */

/*
 * The served form: a stream of independent sort requests under a device
 * memory budget.  The paper sorts one array at a time and has no such loop;
 * this is the standard request-batching pattern of a serving system put over
 * dfr_sort_batch.  A server owns one device pool of the budget's size and a
 * dispatcher thread.  Requests are admitted in arrival order; the oldest
 * pending request and the later ones of its key type are coalesced into one
 * batched launch sequence while their workspace and scratch fit the pool's
 * largest free block; up to `n_streams` batches run at once, each on its own
 * stream.  A request's result is exactly that of sorting its array alone.
 *
 * Ownership: the caller's `keys` / `vals` (and optional `kbuf` / `vbuf`)
 * device buffers must stay valid and untouched from dfr_submit until the
 * request is done.  Requests with NULL `kbuf` / `vbuf` get scratch from the
 * pool.  The caller orders its own writes of the inputs before dfr_submit
 * (e.g. cudaStreamSynchronize on the producing stream); the server's streams
 * do not wait on any caller stream.
 */
typedef struct dfr_server dfr_server_t;
#define DFR_SERVER_MAX_STREAMS 64

/* dfr_server_create -- a server on `device` owning `mem_budget_bytes` of
 * device memory (allocated here, >= 4096) with `n_streams` streams (1 ..
 * DFR_SERVER_MAX_STREAMS).  DFR_ERR_CUDA if a device allocation or stream
 * fails; DFR_ERR_HOST if host memory or the dispatcher thread cannot be had
 * (everything created so far is released; *server stays NULL). */
int dfr_server_create(dfr_server_t** server, int device, size_t mem_budget_bytes, int n_streams);

/* dfr_submit -- queue one request (`req` is copied) and return its ticket.
 * Errors (nothing queued): DFR_ERR_INVALID_ARG for an unknown key type,
 * n > DFR_MAX_N, a null or misaligned buffer; DFR_ERR_OVER_BUDGET when the
 * request's workspace plus its server-provided scratch alone exceed the
 * budget; DFR_ERR_BUSY once the server is being destroyed. */
int dfr_submit(dfr_server_t* server, const dfr_segment_t* req, uint64_t* ticket);

/* dfr_submit_after -- as dfr_submit, for inputs still being produced on the
 * device: the stream that sorts the request first waits on `ready_event` (a
 * cudaEvent_t recorded by the caller after the work that writes the
 * request's buffers; NULL = no wait).  The event must stay alive until the
 * request is done; recording it again before then is allowed only for later
 * work of the same stream (the wait then covers that work too). */
int dfr_submit_after(dfr_server_t* server, const dfr_segment_t* req, void* ready_event, uint64_t* ticket);

/* dfr_server_set_limits -- `max_batch`: cap on requests coalesced into one
 * launch sequence (1 .. 4096, default 4096); 1 serves every request alone
 * with the plain single-array launch sequence.  `max_inflight_per_stream`:
 * batches enqueued on one stream before the server waits for one of them to
 * complete (1 .. DFR_SERVER_MAX_INFLIGHT, default 1); with 1 stream,
 * max_batch 1 and a deep in-flight limit, requests are sorted by back-to-back
 * plain launches in arrival order. */
#define DFR_SERVER_MAX_INFLIGHT 64
int dfr_server_set_limits(dfr_server_t* server, uint32_t max_batch, uint32_t max_inflight_per_stream);

/* dfr_poll -- *done = 1 once the request's sort has completed on the device;
 * then *latency_us (may be NULL) = completion time - submission time in
 * microseconds, the ticket is released and the request's status is returned
 * (DFR_OK; a device error: DFR_ERR_TIMEOUT, DFR_ERR_BOUNDS,
 * DFR_ERR_WORKSPACE; or DFR_ERR_CUDA when its batch could not be enqueued).
 * While pending: *done = 0 and DFR_OK.  An unknown or released ticket gives
 * DFR_ERR_INVALID_ARG.
 *
 * Any thread may poll or wait on any ticket.  A ticket is released once:
 * when several threads poll or wait on the same ticket, the first one to see
 * it done gets its status and latency, and the others get
 * DFR_ERR_INVALID_ARG (released ticket). */
int dfr_poll(dfr_server_t* server, uint64_t ticket, int* done, double* latency_us);

/* dfr_wait -- block until the request is done; then as dfr_poll.  A wait
 * whose ticket another thread releases meanwhile returns
 * DFR_ERR_INVALID_ARG. */
int dfr_wait(dfr_server_t* server, uint64_t ticket, double* latency_us);

/* dfr_server_stats -- batches launched so far, requests pending and batches
 * in flight (each pointer may be NULL). */
int dfr_server_stats(dfr_server_t* server, uint64_t* batches, uint64_t* pending, uint64_t* inflight);

/* dfr_server_destroy -- finish every queued request, then free the pool, the
 * streams and the server.  Tickets not yet polled are released. */
int dfr_server_destroy(dfr_server_t* server);

/* ---------------------------------------------------------------- tuning -- */

/*
 * Per-size-class launch plan.  None of these knobs changes a result (the sort
 * is exact whatever they are); they trade levels, diversion and occupancy.
 * The built-in table comes from the project's autotuner (tune.py, measured on
 * a GB300 and checked in); dfr_tune_set overrides an entry for this process.
 * A call picks the entry of its key type and of the size class of its mean
 * array length (n_total / arrays).
 */
typedef struct {
    uint32_t target_log2;          /* radix window per level chosen so buckets come out near 2^target_log2
                                      keys (6 .. 13); narrower windows mean more levels, smaller buckets */
    uint32_t max_bits;             /* radix bits per level, 4 .. 8 (the launched levels always suffice:
                                      a level widens its window when fewer levels remain) */
    uint32_t warp_max;             /* diverted runs of at most this many keys go to the warp sort, larger
                                      ones to the CTA sort (128 .. 512) */
    uint32_t scatter_ctas_per_sm;  /* scatter grid: CTAs per SM, 0 = as many as fit */
    uint32_t ctasort_ctas_per_sm;  /* CTA-sort grid: CTAs per SM, 0 = as many as fit */
    uint32_t schedule;             /* how a single array sorts its top two digits (DFR_SCHED_*); batches
                                      always use DFR_SCHED_MSD */
    uint32_t launch;               /* how the call is launched (DFR_LAUNCH_*) */
    uint32_t reserved;             /* zero */
} dfr_tune_t;

/*
 * Launch forms of a plain call or a dfr_sort_batch call (a server with more
 * than one stream always uses the level sequence).  Both give the same
 * result.
 *   DFR_LAUNCH_AUTO        one persistent launch for calls of fewer than
 *                          DFR_PERSIST_AUTO_KEYS keys in all, the level
 *                          sequence otherwise;
 *   DFR_LAUNCH_LEVELS      the level sequence: every phase of every level is
 *                          its own kernel (about 24 launches per call);
 *   DFR_LAUNCH_PERSISTENT  one persistent, cooperative launch in which every
 *                          CTA pulls the count, deal, classification, diverted
 *                          bucket and copy-back items of all arrays from device
 *                          queues, phases separated by bounded grid-wide
 *                          barriers (a wait that runs out records
 *                          DFR_ERR_TIMEOUT), levels run until none is left.
 * The LSD schedules of the top digits always run as the level sequence.
 */
enum dfr_launch { DFR_LAUNCH_AUTO = 0, DFR_LAUNCH_LEVELS = 1, DFR_LAUNCH_PERSISTENT = 2 };
#define DFR_PERSIST_AUTO_KEYS ((uint64_t)1 << 25)

/*
 * Schedules of the top digits (paper, Section "Diverting Fast Radix").
 *   DFR_SCHED_MSD  every level counts its digit, then deals it (diverting MSD,
 *                  the paper's Algorithm 2);
 *   DFR_SCHED_LSD  one upfront read counts the top two digits; they are dealt
 *                  least significant first, then the 16-bit prefix buckets are
 *                  diverted or recursed on (diverting LSD, Algorithm 4);
 *   DFR_SCHED_DFR  as DFR_SCHED_LSD, but the first deal uses estimated bucket
 *                  sizes (N/256) with overflow regions instead of a counting
 *                  read (Fast Radix, Algorithm 3); if an overflow region fills
 *                  up, that deal is discarded and DFR_SCHED_MSD sorts the array.
 * All three give the same result.  The LSD schedules apply to single arrays of
 * at least 256 x the CTA-sort capacity keys (dfr_lsd_min_keys); smaller arrays
 * and batches use DFR_SCHED_MSD whatever the plan says.
 */
#define DFR_SCHED_MSD 0
#define DFR_SCHED_LSD 1
#define DFR_SCHED_DFR 2
uint64_t dfr_lsd_min_keys(int key_type);

/* Size classes: 0 = mean array length below 2^12 keys, c = [2^(10+2c), 2^(12+2c)),
 * DFR_TUNE_CLASSES-1 = 2^28 keys and above. */
#define DFR_TUNE_CLASSES 10
#define DFR_TUNE_WARP_MIN 128
#define DFR_TUNE_WARP_MAX 512
int dfr_tune_class(uint64_t mean_keys);

/* dfr_tune_get / dfr_tune_set -- read or override the entry of (key_type,
 * size_class).  dfr_tune_set validates every field (DFR_ERR_INVALID_ARG) and
 * affects later calls of this process.  dfr_tune_reset restores the built-in
 * table. */
int dfr_tune_get(int key_type, int size_class, dfr_tune_t* out);
int dfr_tune_set(int key_type, int size_class, const dfr_tune_t* t);
int dfr_tune_reset(void);

/* ---------------------------------------------------- synthetic inputs -- */

/*
 * dfr_fill_splitmix64 -- write n seeded pseudo-random keys on the device (for
 * benchmarks and tests; not part of the sort).  Key i is output i of the
 * SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014) seeded with
 * `seed`: z = seed + (i+1)*0x9E3779B97F4A7C15, then the generator's mixing
 * function; u32 keys take its high 32 bits.  For the kv key types
 * vals[i] = i (the original index, 4 or 8 bytes by the key type); `vals` is
 * ignored otherwise.
 * Asynchronous on `stream`.  Errors: DFR_ERR_INVALID_ARG for an unknown key
 * type, n > DFR_MAX_N, or a null or misaligned pointer.
 */
int dfr_fill_splitmix64(int key_type, void* keys, void* vals, uint64_t n, uint64_t seed,
                        dfr_stream_t stream);

/* ---------------------------------------------------- debug and profiling -- */

/*
 * dfr_set_debug -- process-wide debug knobs (not for production use).
 *   spin_limit     iterations a device-side wait may spin before it gives up
 *                  and records DFR_ERR_TIMEOUT (0 = default limit);
 *   force_timeout  1 = the decoupled look-back and the persistent launch's
 *                  grid-wide barriers wait on a status word that nothing ever
 *                  sets, so they must time out (tests the timeout path without
 *                  hanging anything); 0 = normal.
 */
int dfr_set_debug(uint32_t spin_limit, int force_timeout);

/* dfr_profile_enable -- 1: record CUDA events around every kernel launch of
 * later calls (per kernel kind), 0: stop.  dfr_profile_read() waits for the
 * device, returns per-kind totals and clears them.  Kinds are listed by
 * dfr_profile_kind_name(). */
int dfr_profile_enable(int on);
#define DFR_PROFILE_KINDS 14
int dfr_profile_read(double* ms_total /*[DFR_PROFILE_KINDS]*/, uint64_t* launches /*[DFR_PROFILE_KINDS]*/);
const char* dfr_profile_kind_name(int kind);

/* dfr_launch_count -- kernels this process has launched through the library. */
uint64_t dfr_launch_count(void);

/* dfr_status_string -- short text for a status code. */
const char* dfr_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* DFR_H */
