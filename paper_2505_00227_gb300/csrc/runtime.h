// Host-side objects of the runtime (contexts, plans, handles) shared by the
// translation units that implement the C ABI: runtime.cu (single-field and
// chunk-streamed paths) and batch.cu (batched persistent launches).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/hpmdr.h"
#include "internal.h"

extern thread_local std::string g_last_error;

// ------------------------------------------------------------------ profiling
// Optional per-stage CUDA events on the context stream: elapsed time per
// kernel stage plus the stage's algorithmic bytes (what the method must move).
enum Stage {
  ST_STATS, ST_FINALIZE, ST_LEVELMAX, ST_BITLEN, ST_ENCODE, ST_CHUNK_STATS, ST_DECIDE,
  ST_HUFF_BITS, ST_OFFSETS, ST_HUFF_ENC, ST_RLE_ENC, ST_HEADERS, ST_SEQUENCE, ST_SELECT,
  ST_DECODE, ST_ROOT, ST_COPY, ST_LEVEL, ST_COPY_OUT, ST_LEVEL_OUT, ST_VMAG, ST_CELLS_MAX,
  ST_CELLS_ENC, ST_CELLS_REC, ST_CELLS_REC_OUT, ST_SMALL, ST_GCELLS_MAX, ST_GCELLS_ENC, ST_PACK,
  ST_UNPACK, ST_GCELLS_REC, ST_GCELLS_REC_OUT, NSTAGE
};
extern const char* kStageName[NSTAGE];

struct ProfEntry {
  int stage;
  cudaEvent_t a, b;
  double bytes;
};

struct Profiler {
  bool on = false;
  uint64_t mask = ~0ull;  // stages that record events (bit = Stage)
  std::vector<cudaEvent_t> pool;
  std::vector<ProfEntry> pending;
  double ms[NSTAGE] = {}, bytes[NSTAGE] = {};
  uint64_t calls[NSTAGE] = {};
  cudaEvent_t get() {
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }
  size_t begin(int stage, double b, cudaStream_t s) {
    if (!on || !((mask >> stage) & 1u)) return SIZE_MAX;
    ProfEntry p{stage, get(), get(), b};
    cudaEventRecord(p.a, s);
    pending.push_back(p);
    return pending.size() - 1;
  }
  void end(size_t i, cudaStream_t s) {
    if (i != SIZE_MAX) cudaEventRecord(pending[i].b, s);
  }
  void patch(size_t i, double b) {
    if (i != SIZE_MAX && i < pending.size()) pending[i].bytes = b;
  }
  void resolve() {
    for (auto& p : pending) {
      float t = 0;
      cudaEventSynchronize(p.b);
      cudaEventElapsedTime(&t, p.a, p.b);
      ms[p.stage] += t;
      bytes[p.stage] += p.bytes;
      calls[p.stage]++;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void reset() {
    resolve();
    for (int i = 0; i < NSTAGE; i++) ms[i] = bytes[i] = 0, calls[i] = 0;
  }
  ~Profiler() {
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct ProfScope {
  Profiler* P;
  size_t i;
  cudaStream_t s;
  ProfScope(Profiler* p, int stage, double bytes, cudaStream_t st)
      : P(p), i(p ? p->begin(stage, bytes, st) : SIZE_MAX), s(st) {}
  ~ProfScope() {
    if (P) P->end(i, s);
  }
};

#define HP_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      g_last_error = std::string(#call) + ": " + cudaGetErrorString(e_);           \
      return HPMDR_ERR_CUDA;                                                       \
    }                                                                              \
  } while (0)

#define HP_TRY(expr)                \
  do {                              \
    hpmdr_status s_ = (expr);       \
    if (s_ != HPMDR_OK) return s_;  \
  } while (0)

struct Allocator {
  hpmdr_allocator hook{};
  bool has_hook = false;
  cudaMemPool_t pool = nullptr;

  hpmdr_status alloc(void** p, size_t bytes, cudaStream_t s) const {
    *p = nullptr;
    if (bytes == 0) return HPMDR_OK;
    bytes = (bytes + 255) & ~(size_t)255;
    if (has_hook) {
      *p = hook.alloc(bytes, (void*)s, hook.user);
      return *p ? HPMDR_OK : HPMDR_ERR_NOMEM;
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
      g_last_error = std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? HPMDR_ERR_NOMEM : HPMDR_ERR_CUDA;
    }
    return HPMDR_OK;
  }
  void release(void* p, cudaStream_t s) const {
    if (!p) return;
    if (has_hook) hook.free(p, (void*)s, hook.user);
    else cudaFreeAsync(p, s);
  }
};

// an asynchronous retrieval waiting for hpmdr_ctx_wait: where its results land
// and the profiler entries to patch once its selection is known
struct PendingRetrieval {
  hpmdr_handle* H = nullptr;
  hpmdr_retrieve_info* info = nullptr;
  int slot = 0;
  std::vector<std::pair<size_t, int>> prof_lv;
  size_t prof_decode = SIZE_MAX, prof_small = SIZE_MAX;
  int small_end = 0;
};

struct hpmdr_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  uint64_t Ts = 4096;
  uint32_t cr_num = 2, cr_den = 1;
  int force = -1;  // -1: Algorithm 2; else the method every group is stored with
  Allocator A;
  Profiler prof;
  std::vector<cudaStream_t> aux;  // extra streams of the chunk pipelines (created on demand)
  // asynchronous retrievals: a ring of page-locked result slots (selection
  // record + device status) filled by copies on the stream, read at wait
  static constexpr int kRing = 64;
  void* pinned = nullptr;      // mapped: written by a kernel (launch_to_host)
  void* pinned_dev = nullptr;  // its device address
  // the refactor's metadata mirror, written the same way
  void* pinned_meta = nullptr;
  void* pinned_meta_dev = nullptr;
  int ring_next = 0;
  std::vector<PendingRetrieval> pending;
  // asynchronous retrievals into host memory: two device output buffers, the
  // copy of one to the host (on copy_stream) overlapping the next retrieval
  void* out_stage[2] = {nullptr, nullptr};
  size_t out_stage_bytes = 0;
  int out_next = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
  bool copied_pending[2] = {false, false};
  // a retrieval's root and small levels recomposed beside its decode
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  Profiler* P() { return prof.on ? &prof : nullptr; }
  ~hpmdr_ctx() {
    if (side) cudaStreamSynchronize(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
    if (copy_stream) cudaStreamSynchronize(copy_stream);
    for (int i = 0; i < 2; i++) {
      A.release(out_stage[i], stream);
      if (ev_ready[i]) cudaEventDestroy(ev_ready[i]);
      if (ev_copied[i]) cudaEventDestroy(ev_copied[i]);
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
    for (cudaStream_t s : aux) cudaStreamDestroy(s);
    if (pinned) cudaFreeHost(pinned);
    if (pinned_meta) cudaFreeHost(pinned_meta);
  }
};

// The geometry of one field shape under one coder configuration: the level
// descriptors, the tile order, the chunk -> group map and the initial
// FieldMeta (group sizes, chunk ranges, slot layout).  It depends only on
// (dims, B, T_s, T_cr), so it is built and uploaded once and shared by every
// handle of that shape: refactoring the same shape again, or the chunks of a
// streamed field, repeats no host planning and no metadata upload.
struct Plan {
  uint64_t dims[3] = {1, 1, 1}, N = 1;
  int B = 32, ngroups = 8, nlev = 0;
  std::vector<LevelDesc> levels;
  std::vector<uint32_t> perm;         // per level: processing order of its tiles
  std::vector<uint32_t> chunk_group;  // global chunk -> flat group index
  uint32_t total_tiles = 0, generic_tiles = 0, total_chunks = 0;
  uint64_t plane_bytes = 0, slot_bytes = 0;
  // general cell levels: nodes of the largest one, and of all of them
  uint64_t gstage_max = 0, gstage_sum = 0;
  std::unique_ptr<FieldMeta> meta0{new FieldMeta()};
  // one device buffer holding levels, perm, chunk map and meta0
  unsigned char* d_buf = nullptr;
  LevelDesc* d_levels = nullptr;
  uint32_t* d_perm = nullptr;
  uint32_t* d_chunk_group = nullptr;
  FieldMeta* d_meta0 = nullptr;
  ~Plan() {
    if (d_buf) cudaFree(d_buf);
  }
};

struct hpmdr_handle {
  Allocator A;
  cudaStream_t stream = nullptr;  // stream used to free device memory
  int dtype = 0, B = 32, nlev = 0, ngroups = 8;
  uint64_t dims[3] = {1, 1, 1}, N = 1;
  std::shared_ptr<const Plan> plan;
  std::vector<LevelDesc> levels;  // host copy of plan->levels
  uint32_t total_tiles = 0, generic_tiles = 0, total_chunks = 0, max_items = 0;
  uint64_t plane_bytes = 0, slot_bytes = 0;
  const LevelDesc* d_levels = nullptr;      // owned by the plan
  const uint32_t* d_perm = nullptr;         // owned by the plan
  const uint32_t* d_chunk_group = nullptr;  // owned by the plan
  uint8_t* d_planes = nullptr;  // plane buffer (refactor output, retrieval plane cache)
  uint8_t* d_slots = nullptr;
  FieldMeta* d_meta = nullptr;
  RetrieveDev* d_rd = nullptr;
  int64_t* d_xa = nullptr;  // |G_2| int64 (recompose scratch)
  int64_t* d_xb = nullptr;  // |G_4| int64
  int64_t* d_xroot = nullptr;
  uint64_t xa_elems = 0, xb_elems = 0;
  // compact: every group's stored bytes (DC groups included) live in the slot
  // buffer, packed; the plane buffer is then only a cache of decoded planes,
  // allocated on the first retrieval and released by hpmdr_handle_drop_cache
  bool compact = false;
  std::unique_ptr<FieldMeta> meta{new FieldMeta()};  // host mirror after refactor/import
  bool qoi_ready = false;
  float qmin = 0, qmax = 0;
  bool vt_ready = false;  // total velocity range of the triplet this handle belongs to
  double vt_min = 0, vt_max = 0;
  // profiler entries of the last retrieval, patched with bytes known after it
  std::vector<std::pair<size_t, int>> prof_lv;  // (entry, level*4 + kind)
  size_t prof_decode = SIZE_MAX, prof_small = SIZE_MAX;
  int small_end = 0;

  void release_cache(cudaStream_t s) {
    A.release(d_planes, s);
    A.release(d_xa, s);
    A.release(d_xb, s);
    d_planes = nullptr;
    d_xa = d_xb = nullptr;
  }
  ~hpmdr_handle() {
    A.release(d_planes, stream);
    A.release(d_slots, stream);
    A.release(d_meta, stream);
    A.release(d_rd, stream);
    A.release(d_xa, stream);
    A.release(d_xb, stream);
    A.release(d_xroot, stream);
  }
};

uint64_t round16(uint64_t v);
size_t align256(size_t v);
hpmdr_status check_dims(int ndims, const uint64_t dims_in[3], uint64_t dims[3], uint64_t* N);
hpmdr_status get_plan(int device, const uint64_t dims[3], int dtype, uint64_t Ts, uint32_t num,
                      uint32_t den, int force, std::shared_ptr<const Plan>* out);
// a handle with the plan of (ndims, dims, dtype) under ctx's coder settings
hpmdr_status new_handle(hpmdr_ctx* ctx, int ndims, const uint64_t dims_in[3], int dtype,
                        const std::shared_ptr<const Plan>* plan_in,
                        std::unique_ptr<hpmdr_handle>& H);
void count_items(hpmdr_handle* H);
hpmdr_status ensure_retrieve_buffers(hpmdr_handle* H, cudaStream_t s);
hpmdr_status collect_info(hpmdr_ctx* ctx, hpmdr_handle* H, hpmdr_retrieve_info* info,
                          cudaStream_t s);
