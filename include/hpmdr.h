/*
 * hpmdr.h - C ABI of the GB300 (sm_103a) progressive data refactoring library.
 *
 * Method: HP-MDR (arXiv 2505.00227).  A field is decomposed into multilevel
 * coefficients (Sec. 3), each level is aligned to its maximum exponent and
 * split into bitplanes (Sec. 4, Algorithm 1), every four bitplanes are merged
 * and stored with Huffman, RLE or direct copy (Sec. 5, Algorithm 2), and a
 * retrieval fetches only the bitplane groups needed for an L-infinity or QoI
 * error bound (Sec. 3, Sec. 6.2, Algorithm 3), incrementally over earlier
 * retrievals of the same handle.
 *
 * Conventions
 *   - Every call returns an hpmdr_status; nothing else crosses the boundary.
 *   - Arrays are C order, dims[0] slowest (z), dims[2] fastest (x); a 1D or 2D
 *     field passes ndims = 1 or 2 and its sizes in the last entries.
 *   - "on_device" flags tell whether a pointer is CUDA device memory (1) or
 *     host memory (0).  Host memory may be pageable or pinned.
 *   - The caller owns every input and output buffer.  The library owns
 *     contexts, handles and everything they hold; views stay valid until the
 *     owning object is freed.
 *   - All GPU work is ordered on the context's CUDA stream.  A call returns
 *     when its results are complete (output buffers written, info filled).
 *   - No call falls back to the CPU: without a usable sm_103a device every
 *     compute call returns HPMDR_ERR_CUDA.
 */
#ifndef HPMDR_H
#define HPMDR_H
#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HPMDR_API __attribute__((visibility("default")))
#else
#define HPMDR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HPMDR_OK = 0,
  HPMDR_ERR_ARG = -1,           /* bad argument, unsupported shape or value range */
  HPMDR_ERR_NOMEM = -2,         /* an allocation failed or the budget is spent */
  HPMDR_ERR_CUDA = -3,          /* a CUDA call failed (message: hpmdr_last_error) */
  HPMDR_ERR_CORRUPT = -4,       /* stored bytes failed a bounds or format check */
  HPMDR_ERR_UNATTAINABLE = -5,  /* even all bitplanes cannot meet the bound */
  HPMDR_ERR_TIMEOUT = -6,       /* a bounded wait gave up (serving: a request queued past
                                   its deadline) */
  HPMDR_ERR_BUSY = -7,          /* request not finished yet (serving) */
  HPMDR_ERR_CANCELLED = -8      /* request cancelled before it started (serving) */
} hpmdr_status;

typedef enum { HPMDR_F32 = 0, HPMDR_F64 = 1 } hpmdr_dtype;

/* storage method of a merged bitplane group (Sec. 5.1); non-leading planes of
 * a group hold a placeholder entry (Algorithm 2) */
typedef enum { HPMDR_DC = 0, HPMDR_HUFFMAN = 1, HPMDR_RLE = 2, HPMDR_PLACEHOLDER = 3 } hpmdr_method;

/* Optional allocator hook for device memory.  alloc returns device memory
 * usable on `stream`, or NULL; free releases it after work on `stream`. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, void* stream, void* user);
  void* user;
} hpmdr_allocator;

/* Parameters of Algorithm 2 (Sec. 5.2).  Zero fields take the defaults:
 * group_m = 4 planes, size_threshold T_s = 4096 bytes, compression-ratio
 * threshold T_cr = cr_num/cr_den = 2/1.  T_cr must be >= 1. */
typedef struct {
  int group_m;              /* only 4 is supported */
  uint64_t size_threshold;  /* T_s: groups of S <= T_s bytes are copied */
  uint32_t cr_num, cr_den;  /* T_cr = cr_num / cr_den */
  int32_t method;           /* 0: Algorithm 2 picks per group; 1 + HPMDR_DC / HPMDR_HUFFMAN /
                               HPMDR_RLE: every group stored with that method (the lossless-
                               strategy comparison of Sec. 7.2.2; slots sized for the worst case) */
  int32_t reserved0;
  uint64_t reserved[3];
} hpmdr_config;

typedef struct hpmdr_ctx hpmdr_ctx;        /* stream, allocator, workspace */
typedef struct hpmdr_handle hpmdr_handle;  /* one refactored field + retrieval state */

typedef struct {
  double est_linf;              /* rigorous L-infinity bound of this reconstruction */
  double requested_abs;         /* the absolute bound that was asked for */
  uint64_t est_units_hi, est_units_lo;  /* est_linf exactly, in units of 2^(E_f-51-B) */
  uint64_t bytes_fetched_total; /* stored bytes of all groups fetched so far */
  uint64_t bytes_fetched_new;   /* stored bytes fetched by this call */
  int groups_per_level[64];     /* bitplane groups used per level (level 0 = root) */
  int nlevels;
  int status;                   /* HPMDR_OK or HPMDR_ERR_UNATTAINABLE */
} hpmdr_retrieve_info;

/* ---- context ------------------------------------------------------------ */
/* cfg and alloc may be NULL (defaults; stream-ordered CUDA pool allocation).
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream). */
HPMDR_API hpmdr_status hpmdr_ctx_create(hpmdr_ctx** ctx, const hpmdr_config* cfg,
                              const hpmdr_allocator* alloc, void* cuda_stream);
HPMDR_API void hpmdr_ctx_destroy(hpmdr_ctx* ctx);
HPMDR_API hpmdr_status hpmdr_ctx_set_stream(hpmdr_ctx* ctx, void* cuda_stream);

/* ---- refactor (Sec. 3 pipeline: decompose, align + Algorithm 1, Algorithm 2)
 * field: N = prod(dims) values of dtype; dims[d] >= 1, N < 2^32.
 * Values must be finite with max|f| < 2^121 (F32) or in [2^-1001, 2^1017)
 * (F64, or an all-zero field); otherwise HPMDR_ERR_ARG.
 * On success *out is a new handle (free with hpmdr_handle_free). */
HPMDR_API hpmdr_status hpmdr_refactor(hpmdr_ctx* ctx, const void* field, int field_on_device, int ndims,
                            const uint64_t dims[3], hpmdr_dtype dtype, hpmdr_handle** out);

/* ---- retrieve (Sec. 3 "error control", Algorithm 3's copy_to_device/recompose)
 * Reconstructs the whole field into `out` (N values of the handle's dtype)
 * from the shortest prefix of the handle's greedy group sequence whose error
 * estimate meets the bound.  Only groups not fetched by an earlier call on
 * this handle are decoded (incremental).  rel_linf_bound is relative to the
 * value range max(f) - min(f); hpmdr_retrieve_abs takes an absolute bound.
 * Returns HPMDR_ERR_UNATTAINABLE, with the best reconstruction written and
 * info filled, when all groups together cannot meet the bound.  info may be NULL. */
HPMDR_API hpmdr_status hpmdr_retrieve(hpmdr_ctx* ctx, hpmdr_handle* h, double rel_linf_bound, void* out,
                            int out_on_device, hpmdr_retrieve_info* info);
HPMDR_API hpmdr_status hpmdr_retrieve_abs(hpmdr_ctx* ctx, hpmdr_handle* h, double abs_linf_bound, void* out,
                                int out_on_device, hpmdr_retrieve_info* info);

/* Asynchronous retrieval: the same work as hpmdr_retrieve with the output on
 * the device, enqueued on the context stream; the call returns without waiting
 * for the GPU, so back-to-back retrievals (of one handle, incremental as
 * usual, or of several) run without host round trips between them.  *info
 * (may be NULL; host memory owned by the caller) is filled by hpmdr_ctx_wait,
 * which waits for everything enqueued on the context stream and returns
 * HPMDR_OK, or the first status of a pending retrieval that was not OK (each
 * info carries its own).  Up to 64 retrievals may be pending; one more waits
 * first.  The handle, out and info must stay valid until hpmdr_ctx_wait. */
HPMDR_API hpmdr_status hpmdr_retrieve_async(hpmdr_ctx* ctx, hpmdr_handle* h, double rel_linf_bound,
                                            void* out, hpmdr_retrieve_info* info);
/* as hpmdr_retrieve_async with the output in host memory (page-locked for
 * overlap): the reconstruction goes to one of two device buffers of the
 * context and is copied out on a stream of its own, so the copy of one
 * retrieval overlaps the kernels of the next; out is complete at
 * hpmdr_ctx_wait. */
HPMDR_API hpmdr_status hpmdr_retrieve_async_host(hpmdr_ctx* ctx, hpmdr_handle* h,
                                                 double rel_linf_bound, void* out,
                                                 hpmdr_retrieve_info* info);
HPMDR_API hpmdr_status hpmdr_ctx_wait(hpmdr_ctx* ctx);

/* ---- out-of-core pipeline (Sec. 5.3, the refactoring and retrieval pipelines)
 * nvars variables of one shape (dims, ndims entries as for hpmdr_refactor) in
 * host memory, cut into chunks as for hpmdr_refactor_chunked, are refactored
 * unit by unit, unit u = v * nchunks + c, into serialized streams in host
 * memory (the hpmdr_handle_export format, one per unit), and retrieved back
 * from them.  Three queues, one CUDA stream each: host -> device copies,
 * kernels, device -> host copies; unit u + 1's input goes in while unit u's
 * kernels run and unit u - 1's result comes out; two device input (output)
 * buffers alternate and at most three units' handles are on the device.
 * queues = 3 runs that pipeline; queues = 1 puts every step of every unit on
 * one stream, in order (nothing overlaps: the baseline of Sec. 5.3's
 * comparison).  Overlap needs page-locked host memory for fields, streams and
 * outputs.
 * hpmdr_refactor_pipeline: out == NULL sets *total to a bound on the bytes of
 * all streams; else out (16-byte aligned, *total bytes) receives the streams
 * back to back, each 16-byte aligned, offsets[u] / sizes[u] (nvars * nchunks
 * entries) their placement, and *total the bytes used.
 * hpmdr_retrieve_pipeline: every unit of variable v at rel_bounds[v], relative
 * to v's whole range (from the streams' headers), into the host array outs[v]
 * (dims); infos (may be NULL) gets one record per unit.  Returns HPMDR_OK, or
 * HPMDR_ERR_UNATTAINABLE when some unit could not meet its bound. */
HPMDR_API hpmdr_status hpmdr_refactor_pipeline(hpmdr_ctx* ctx, int nvars, const void* const* fields,
                                               int ndims, const uint64_t dims[3],
                                               const uint64_t chunk[3], hpmdr_dtype dtype,
                                               int queues, void* out, uint64_t* total,
                                               uint64_t* offsets, uint64_t* sizes);
HPMDR_API hpmdr_status hpmdr_retrieve_pipeline(hpmdr_ctx* ctx, int nvars, const void* streams,
                                               const uint64_t* offsets, const uint64_t* sizes,
                                               int ndims, const uint64_t dims[3],
                                               const uint64_t chunk[3], const double* rel_bounds,
                                               int queues, void* const* outs,
                                               hpmdr_retrieve_info* infos);

/* ---- QoI retrieval (Sec. 6.2, Algorithm 3) for the velocity magnitude
 * |v| = sqrt(vx^2 + vy^2 + vz^2) of three FP32 handles of equal shape.
 * rel_qoi_bound is relative to max|v| - min|v| of the refactored data.
 * Writes the three components (out[c], may be NULL) and |v| (out_vmag).
 * info[0..2] describe the components, info[3] the QoI (est_linf = QoI bound). */
HPMDR_API hpmdr_status hpmdr_qoi_prepare_vmag(hpmdr_ctx* ctx, hpmdr_handle* v[3], const void* vx,
                                    const void* vy, const void* vz, int on_device);
HPMDR_API hpmdr_status hpmdr_retrieve_qoi_vmag(hpmdr_ctx* ctx, hpmdr_handle* v[3], double rel_qoi_bound,
                                     void* out[3], void* out_vmag, int on_device,
                                     hpmdr_retrieve_info info[4]);

/* ---- iterated QoI retrieval (Sec. 6.2, Algorithm 3) for the total velocity
 * V = vx^2 + vy^2 + vz^2 of three FP32 handles of equal shape (V evaluated in
 * FP64, written as FP32).  hpmdr_qoi_prepare_vtotal records the range of V of
 * the original data (it must fit FP32).  hpmdr_retrieve_qoi_vtotal starts from
 * eps_i = (tau / max V) * (max v_i - min v_i), tau = rel_qoi_bound * (max V -
 * min V), and repeats: retrieve every variable to eps_i, bound the QoI error
 * pointwise (2 |x_hat| E + E^2 per variable plus the output rounding; the
 * maximum tau' is computed on the device), stop if tau' <= tau, else choose
 * the next bounds with the estimator:
 *   HPMDR_EST_CP    halve all bounds until the point of the largest tau'
 *                   meets tau (reconstruction held fixed);
 *   HPMDR_EST_MA    one more merged bitplane group per variable;
 *   HPMDR_EST_MAPE  p = tau'/tau: bounds E_i / p while p > c (0: c = 10),
 *                   MA once p <= c.
 * Components go to out[i] (may be NULL) and V_hat to out_qoi; rep (may be
 * NULL) receives the iterations, the final bound and data estimates.
 * HPMDR_ERR_UNATTAINABLE when every variable is fully retrieved and tau' > tau. */
typedef enum { HPMDR_EST_CP = 0, HPMDR_EST_MA = 1, HPMDR_EST_MAPE = 2 } hpmdr_qoi_estimator;
typedef struct {
  int status, iterations;
  double tau_abs;                /* requested QoI bound */
  double est;                    /* final QoI error bound tau' */
  double eps[3];                 /* final data error estimates */
  int prefix[3];                 /* greedy-sequence steps retrieved per variable */
  int pad;
  uint64_t bytes_fetched_total;  /* stored bytes used, over the three variables */
} hpmdr_qoi_report;
HPMDR_API hpmdr_status hpmdr_qoi_prepare_vtotal(hpmdr_ctx* ctx, hpmdr_handle* v[3], const void* vx,
                                                const void* vy, const void* vz, int on_device);
HPMDR_API hpmdr_status hpmdr_retrieve_qoi_vtotal(hpmdr_ctx* ctx, hpmdr_handle* v[3],
                                                 double rel_qoi_bound, int estimator, double c,
                                                 void* out[3], void* out_qoi, int on_device,
                                                 hpmdr_qoi_report* rep);
/* One bounding step of hpmdr_retrieve_qoi_vtotal (Sec. 6.2, Algorithm 3's QoI
 * error estimate) on given components: out[i] = V_hat = RN32(RN64(RN64(vx^2 +
 * vy^2) + vz^2)) (squares exact in FP64), and the largest pointwise bound on
 * |V_hat - V| for |x_hat_i - x_i| <= e[i] (2 |x_hat_i| e_i + e_i^2 summed, plus
 * the FP32 rounding of V_hat: 2^-24 V_hat, 2^-150 below the normal range,
 * +inf past FLT_MAX, and 2^-50 V_hat for the FP64 additions; FP64, every
 * operation rounded to nearest) with its first point.  vx, vy, vz, out: device
 * arrays of n FP32 values (caller owned); e: host, 3 values >= 0; *bound and
 * *point: host.  Synchronous on the context stream.  HPMDR_ERR_ARG for n = 0,
 * a NULL pointer or a negative e. */
HPMDR_API hpmdr_status hpmdr_qoi_vtotal_bound(hpmdr_ctx* ctx, const float* vx, const float* vy,
                                              const float* vz, uint64_t n, const double e[3],
                                              float* out, double* bound, uint64_t* point);

/* ---- handle inspection -------------------------------------------------- */
HPMDR_API hpmdr_status hpmdr_handle_field_info(const hpmdr_handle* h, int* dtype, uint64_t dims[3],
                                     int* nlevels, int* E_f, int* input_exact,
                                     double stats[4] /* max|f|, min, max, range */);
HPMDR_API hpmdr_status hpmdr_handle_level_info(const hpmdr_handle* h, int level, uint64_t* n, int* bl,
                                     int* ngroups, int* exact);
/* stored bytes of one group copied to host `buf` (NULL: only *len); method
 * and the Huffman / RLE size estimates of Sec. 5.2 (est may be NULL) */
HPMDR_API hpmdr_status hpmdr_handle_group(const hpmdr_handle* h, int level, int group, void* buf,
                                uint64_t* len, int* method, uint64_t est[2]);
/* the level's (B+1) bitplanes as produced by Algorithm 1 (host copy) */
HPMDR_API hpmdr_status hpmdr_handle_planes(const hpmdr_handle* h, int level, void* buf, uint64_t* len);
/* the tau-independent greedy group sequence (level index per step) */
HPMDR_API hpmdr_status hpmdr_handle_sequence(const hpmdr_handle* h, int* seq, int cap, int* len);
/* serialized handle (stored groups + metadata); buf NULL: *len = size needed */
HPMDR_API hpmdr_status hpmdr_handle_export(const hpmdr_handle* h, void* buf, uint64_t* len);
HPMDR_API hpmdr_status hpmdr_handle_import(hpmdr_ctx* ctx, const void* buf, uint64_t len,
                                 hpmdr_handle** out);
/* forget the fetched groups; poison != 0 also overwrites the device copies of
 * Huffman/RLE groups so that the next retrieval must decode them again */
HPMDR_API hpmdr_status hpmdr_handle_reset(hpmdr_ctx* ctx, hpmdr_handle* h, int poison);
HPMDR_API void hpmdr_handle_free(hpmdr_handle* h);

/* ---- device plane cache -------------------------------------------------
 * A refactored handle keeps its full plane buffer (the encoder's output; DC
 * groups are read from it).  hpmdr_handle_compact packs every group's stored
 * bytes, DC groups included, into one device buffer and releases the planes:
 * the handle then holds only its compressed streams, and the plane buffer
 * becomes a cache that the next retrieval allocates and fills with the groups
 * it selects (Huffman/RLE decoded, DC copied), growing incrementally as later
 * retrievals tighten the bound.  hpmdr_handle_drop_cache releases that cache
 * (compacting first if needed).  Results do not depend on the cache state. */
HPMDR_API hpmdr_status hpmdr_handle_compact(hpmdr_ctx* ctx, hpmdr_handle* h);
HPMDR_API hpmdr_status hpmdr_handle_drop_cache(hpmdr_ctx* ctx, hpmdr_handle* h);
/* device bytes: resident = held until hpmdr_handle_free (streams, metadata,
 * and the planes of a handle that is not compact); cache = plane cache and
 * recompose grids held now; cache_max = the most a retrieval holds (those
 * plus its transient staging).  Any pointer may be NULL. */
HPMDR_API hpmdr_status hpmdr_handle_memory(const hpmdr_handle* h, uint64_t* resident, uint64_t* cache,
                                           uint64_t* cache_max);

/* ---- chunk streaming (Sec. 5.3 pipeline) ------------------------------------
 * A field of dims (ndims entries, as for hpmdr_refactor) is cut into
 * independent sub-blocks of `chunk` (the last ones along an axis may be
 * smaller), numbered in C order over the chunk grid; each is refactored as a
 * field of its own.  Chunk c runs on stream c mod nstreams (1..16 streams
 * ordered after the context stream): its host<->device copy overlaps the
 * kernels of the chunks on the other streams.  Overlap needs page-locked host
 * memory; pageable memory works but serializes the copies.
 * hpmdr_refactor_chunked: out == NULL only sets *nchunks; else out[0..cap)
 * receives *nchunks new handles (cap >= *nchunks).
 * hpmdr_retrieve_chunked: hs are those handles in the same order; every chunk
 * is retrieved with the absolute bound rel_linf_bound * (max_c max f - min_c
 * min f), i.e. relative to the whole field's range, and written into its box
 * of out (prod(dims) values).  infos (may be NULL) receives one entry per
 * chunk.  Returns HPMDR_ERR_UNATTAINABLE if any chunk is. */
HPMDR_API hpmdr_status hpmdr_refactor_chunked(hpmdr_ctx* ctx, const void* field, int field_on_device,
                                              int ndims, const uint64_t dims[3],
                                              const uint64_t chunk[3], hpmdr_dtype dtype,
                                              int nstreams, hpmdr_handle** out, uint64_t cap,
                                              uint64_t* nchunks);
HPMDR_API hpmdr_status hpmdr_retrieve_chunked(hpmdr_ctx* ctx, hpmdr_handle* const* hs, uint64_t n,
                                              int ndims, const uint64_t dims[3],
                                              const uint64_t chunk[3], double rel_linf_bound,
                                              void* out, int out_on_device, int nstreams,
                                              hpmdr_retrieve_info* infos);

/* ---- serving ---------------------------------------------------------------
 * A request loop over refactored fields.  hpmdr_server_add_field compacts a
 * handle (see hpmdr_handle_compact) and admits its stored bytes against the
 * HBM budget (HPMDR_ERR_NOMEM if they do not fit).  hpmdr_server_submit queues
 * a request and returns at once; max_slots worker threads, each with its own
 * CUDA stream, run requests concurrently.  A request starts as soon as a slot
 * is free, none of its handles is used by a running request, and the budget
 * has room for the plane caches it fills (idle caches are evicted least
 * recently used first); requests that cannot start do not block later ones.
 * keep_cache = 0 gives the plain per-request path: every request decodes all
 * groups it uses and drops them afterwards.  A request's result does not
 * depend on the requests before or beside it.  Outputs are device buffers of
 * the caller, valid until the request is polled done.  Handles must stay
 * alive and must not be used outside the server while it runs. */
typedef struct hpmdr_server hpmdr_server;
typedef enum { HPMDR_REQ_FIELD = 0, HPMDR_REQ_VMAG = 1 } hpmdr_request_kind;
typedef struct {
  int kind;             /* hpmdr_request_kind */
  hpmdr_handle* h[3];   /* FIELD: h[0]; VMAG: the (vx, vy, vz) triplet, prepared with
                           hpmdr_qoi_prepare_vmag */
  double rel_bound;     /* relative L-infinity bound (FIELD) or relative QoI bound (VMAG) */
  void* out[3];         /* FIELD: out[0] receives the field; VMAG: components (entries may
                           be NULL) */
  void* out_vmag;       /* VMAG: receives |v| */
} hpmdr_request;
typedef struct {
  int max_slots;        /* requests running at once, 1..64 */
  int keep_cache;       /* 1: keep plane caches between requests; 0: plain path */
  uint64_t hbm_budget;  /* device bytes for stored fields + plane caches + QoI scratch */
  double queue_timeout_s;  /* > 0: a request still queued this long after its submit
                              fails with HPMDR_ERR_TIMEOUT instead of starting; 0: none */
} hpmdr_server_config;
HPMDR_API hpmdr_status hpmdr_server_create(hpmdr_ctx* ctx, const hpmdr_server_config* cfg,
                                           hpmdr_server** out);
/* drops queued requests, waits for running ones */
HPMDR_API void hpmdr_server_destroy(hpmdr_server* s);
HPMDR_API hpmdr_status hpmdr_server_add_field(hpmdr_server* s, hpmdr_ctx* ctx, hpmdr_handle* h);
/* HPMDR_ERR_ARG for a handle not added, HPMDR_ERR_NOMEM if the request cannot
 * fit in the budget even with every other cache evicted */
HPMDR_API hpmdr_status hpmdr_server_submit(hpmdr_server* s, const hpmdr_request* r, uint64_t* ticket);
/* The request's status once done (the ticket is then consumed), else
 * HPMDR_ERR_BUSY (wait = 0) or block until done (wait != 0).  info: 1 entry
 * for FIELD, 4 for VMAG (may be NULL).  times: submit, start and completion
 * instants in seconds of the monotonic clock (may be NULL). */
HPMDR_API hpmdr_status hpmdr_server_poll(hpmdr_server* s, uint64_t ticket, int wait,
                                         hpmdr_retrieve_info info[4], double times[3]);
/* Host-side cancellation: a request still queued is dropped (HPMDR_OK; its
 * poll then returns HPMDR_ERR_CANCELLED); a request that has started or
 * finished is not (HPMDR_ERR_BUSY; it completes and its poll gives its
 * status); HPMDR_ERR_ARG for an unknown or already polled ticket.  The paper
 * has no counterpart (its retrieval has no request stream). */
HPMDR_API hpmdr_status hpmdr_server_cancel(hpmdr_server* s, uint64_t ticket);
/* budget bytes in use, peak, cache evictions, completed, queued, running */
HPMDR_API hpmdr_status hpmdr_server_stats(hpmdr_server* s, uint64_t stats[6]);

/* ---- batched persistent path ---------------------------------------------
 * Many fields of uneven sizes (one dtype) refactored, then retrieved, each
 * pass as one CUDA-graph launch whose every stage is one persistent kernel
 * over the work units (tiles, chunks, groups) of all fields.  Results are
 * bit-identical to hpmdr_refactor / hpmdr_retrieve field by field.
 * hpmdr_batch_create plans n fields of dims[3 j .. 3 j + 2] (C order, as for
 * hpmdr_refactor with ndims = 3) and allocates their handles once; the batch
 * owns them (hpmdr_batch_handle gives views usable with every handle entry
 * point; do not free them) and must be destroyed before its context.
 * hpmdr_batch_refactor: fields[j] are device pointers, 16-byte aligned.
 * hpmdr_batch_retrieve: relative L-infinity bound and device output per field,
 * incremental per handle like hpmdr_retrieve; infos (may be NULL) gets n
 * entries.  Returns the first error, else HPMDR_ERR_UNATTAINABLE if any field
 * is, else HPMDR_OK.
 * hpmdr_batch_autotune times both graphs under each candidate tuning
 * {persistent CTAs per SM of the tile and chunk kernels, values per unit of
 * the statistics pass, persistent CTAs per SM of the decoder} and keeps the
 * fastest (written to best, may be NULL); it leaves the batch refactored from
 * `fields` with empty retrieval state.  hpmdr_batch_last_ms: device time of
 * the last refactor and retrieval call (graph launch to results on host). */
typedef struct hpmdr_batch hpmdr_batch;
HPMDR_API hpmdr_status hpmdr_batch_create(hpmdr_ctx* ctx, uint64_t n, const uint64_t* dims,
                                          hpmdr_dtype dtype, hpmdr_batch** out);
HPMDR_API void hpmdr_batch_destroy(hpmdr_batch* b);
HPMDR_API hpmdr_status hpmdr_batch_handle(hpmdr_batch* b, uint64_t i, hpmdr_handle** h);
HPMDR_API hpmdr_status hpmdr_batch_refactor(hpmdr_batch* b, const void* const* fields);
HPMDR_API hpmdr_status hpmdr_batch_retrieve(hpmdr_batch* b, const double* rel_bounds,
                                            void* const* outs, hpmdr_retrieve_info* infos);
HPMDR_API hpmdr_status hpmdr_batch_autotune(hpmdr_batch* b, const void* const* fields,
                                            const double* rel_bounds, void* const* outs,
                                            uint32_t best[3]);
HPMDR_API hpmdr_status hpmdr_batch_set_tuning(hpmdr_batch* b, const uint32_t tuning[3]);
HPMDR_API hpmdr_status hpmdr_batch_get_tuning(const hpmdr_batch* b, uint32_t tuning[3]);
HPMDR_API hpmdr_status hpmdr_batch_last_ms(const hpmdr_batch* b, double ms[2]);

/* ---- stage entry points (device pointers, ordered on `stream`) ---------- */
/* Algorithm 1 on one level: q holds n aligned integers (uint32 for B = 32,
 * uint64 for B = 64), sign n bytes (0/1).  planes receives (B+1) planes of
 * 4*ceil(n/128) uint32 words: plane 0 = sign, plane 1+p = bit B-1-p; element
 * j at word j>>5, bit j&31; padding bits zero. */
HPMDR_API hpmdr_status hpmdr_bitplane_encode(const void* q, const uint8_t* sign, uint64_t n, int B,
                                   uint32_t* planes, void* stream);
/* inverse: keeps the top k magnitude planes (k = 0..B); sign_out gets the
 * sign plane when k > 0, else zeros */
HPMDR_API hpmdr_status hpmdr_bitplane_decode(const uint32_t* planes, uint64_t n, int B, int k, void* q_out,
                                   uint8_t* sign_out, void* stream);
/* The bitplane encoder designs of Sec. 4 for B = 32, all writing the layout of
 * hpmdr_bitplane_encode byte for byte (and decoding as hpmdr_bitplane_decode):
 * the register block of Sec. 4.3 (the production encoder), the locality block
 * of Sec. 4.1 (a thread moves the bits of 32 contiguous elements one at a
 * time), and register shuffling (Sec. 4.2; a thread per element, a warp per
 * word) with each of the four warp instructions.  The shuffle designs share one
 * decoder (a broadcast per plane).  q (uint32) and planes must be 16-byte
 * aligned; n < 2^32 - 256; k = 0..32.  HPMDR_ERR_ARG otherwise. */
typedef enum {
  HPMDR_BP_REGISTER_BLOCK = 0,
  HPMDR_BP_LOCALITY_BLOCK = 1,
  HPMDR_BP_SHUFFLE_BALLOT = 2,
  HPMDR_BP_SHUFFLE_SHIFT = 3,
  HPMDR_BP_SHUFFLE_MATCH_ANY = 4,
  HPMDR_BP_SHUFFLE_REDUCE = 5
} hpmdr_bp_design;
HPMDR_API hpmdr_status hpmdr_bitplane_encode_design(const uint32_t* q, const uint8_t* sign,
                                                    uint64_t n, int design, uint32_t* planes,
                                                    void* stream);
HPMDR_API hpmdr_status hpmdr_bitplane_decode_design(const uint32_t* planes, uint64_t n, int design,
                                                    int k, uint32_t* q_out, uint8_t* sign_out,
                                                    void* stream);
/* Algorithm 2 on one byte group G (device memory, S bytes): force = -1 picks the
 * method as Algorithm 2 does, else HPMDR_DC / HPMDR_HUFFMAN / HPMDR_RLE.
 * out (device) needs cap bytes; *len receives the stored length. */
HPMDR_API hpmdr_status hpmdr_encode_group(hpmdr_ctx* ctx, const uint8_t* G, uint64_t S, int force,
                                uint8_t* out, uint64_t cap, uint64_t* len, int* method);
HPMDR_API hpmdr_status hpmdr_decode_group(hpmdr_ctx* ctx, const uint8_t* in, uint64_t len, int method,
                                uint8_t* G, uint64_t S);
/* The last step of recomposition (Sec. 3, Algorithm 3's recompose; the output
 * rounding of the fixed-point reading): out[i] = RN(X[i]) * 2^(E_f-48)
 * in the output type, RN the round-to-nearest-even conversion of the integer,
 * for FP32 followed by an exact power-of-two scale when -78 <= E_f <= 121 and
 * else rounded through FP64 first; exactly what every retrieval writes.  X and
 * out are device arrays of n values (out 4 or 8 bytes each); synchronous on the
 * context stream.  HPMDR_ERR_ARG for a NULL pointer with n > 0, another dtype,
 * or an E_f no field of the type has (FP32: -148..128, FP64: -1073..1024). */
HPMDR_API hpmdr_status hpmdr_fixed_to_float(hpmdr_ctx* ctx, const int64_t* X, uint64_t n, int E_f,
                                            hpmdr_dtype dtype, void* out);
/* hpmdr_encode_group for callers that cannot allocate device memory: a
 * solver that owns all of HBM, or one that forbids cudaMalloc/cudaFree between
 * steps because they may synchronize the device.  The paper has no
 * counterpart: this is the encoder of hpmdr_encode_group, bit for bit (same
 * method choice, same stored bytes), with its scratch in a static device
 * array of about 70 KB that every GPU loading the library holds until exit.
 * G (device, 16-byte aligned) holds S <= 16 MiB bytes; larger groups give
 * HPMDR_ERR_ARG.  size_threshold / cr_num / cr_den are hpmdr_encode_group's
 * size and ratio thresholds (the hpmdr_config fields of the same names;
 * 0 = defaults).  out (device) has cap bytes; the coded bytes not fitting
 * gives HPMDR_ERR_ARG.  The call is synchronous: it waits on `stream` before
 * returning.  The first call on a device looks up the array's address; make
 * it before any stream capture.  Calls share the array, which keeps the last
 * call's contents: calls that overlap on the GPU race and must be serialized. */
HPMDR_API hpmdr_status hpmdr_encode_group_noalloc(const uint8_t* G, uint64_t S, int force,
                                                  uint64_t size_threshold, uint32_t cr_num,
                                                  uint32_t cr_den, uint8_t* out, uint64_t cap,
                                                  uint64_t* len, int* method, void* stream);

/* ---- measurement -------------------------------------------------------- */
/* Kernels launched by this library in this process so far. */
HPMDR_API uint64_t hpmdr_kernel_launches(void);
/* enable != 0: record CUDA events on the context stream around every kernel
 * stage (and clear the totals); 0: stop recording. */
HPMDR_API hpmdr_status hpmdr_ctx_profile(hpmdr_ctx* ctx, int enable);
/* as hpmdr_ctx_profile(ctx, 1), but only the stages whose bit (1 << index, the
 * index of hpmdr_ctx_profile_entry) is set record events: two events per
 * launch of a chosen stage, none elsewhere (0: stop recording) */
HPMDR_API hpmdr_status hpmdr_ctx_profile_stages(hpmdr_ctx* ctx, uint64_t stage_mask);
/* totals of stage `index` (0 .. count-1; HPMDR_ERR_ARG past the end): name,
 * summed event time in ms, launches, and algorithmic bytes (the bytes the
 * method must read and write in that stage; 0 where not defined) */
HPMDR_API hpmdr_status hpmdr_ctx_profile_entry(hpmdr_ctx* ctx, int index, const char** name,
                                               double* total_ms, uint64_t* launches, double* bytes);

HPMDR_API const char* hpmdr_strerror(hpmdr_status s);
HPMDR_API const char* hpmdr_last_error(void);  /* text of the last CUDA failure on this thread */

#ifdef __cplusplus
}
#endif
#endif
