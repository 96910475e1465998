// Batched refactor and retrieval of many fields of uneven sizes: every stage
// is one persistent launch over the work units (tiles, chunks, groups) of all
// fields, and each pass (refactor; retrieve) is one CUDA-graph launch.
//
// The batch owns one handle per field, allocated once; a refactor or
// retrieval only uploads the job table (field and output pointers, bounds)
// and launches the pass's graph.  The stage kernels are the single-field
// kernels' per-unit bodies, so a batched result is bit-identical to the
// per-field path.  Recomposition is level-sequential inside a field, so the
// retrieval graph runs it in rounds: round r recomposes level small_end+1+r of
// every field that has it.
//
// Tuning (picked by hpmdr_batch_autotune, by timing the graphs):
//   grid_mul  persistent CTAs per SM of the tile and chunk kernels
//   seg       values per work unit of the statistics pass
//   dec_mul   persistent CTAs per SM of the decoder
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "../../include/hpmdr.h"
#include "dev_common.cuh"
#include "runtime.h"

using namespace hp;

namespace {

struct Tuning {
  uint32_t grid_mul = 4, seg = 65536, dec_mul = 6;
};

struct Round {
  uint32_t ncells = 0, ngen = 0, ngc = 0;
  uint32_t cells_total = 0, copy_total = 0, level_total = 0, unpack_total = 0, gc_total = 0;
  size_t o_cells_refs = 0, o_cells_u0 = 0, o_gen_refs = 0, o_copy_u0 = 0, o_level_u0 = 0;
  size_t o_gc_refs = 0, o_unpack_u0 = 0, o_gc_u0 = 0;
};

uint32_t gcell_units(const LevelDesc& D) {  // 256 cells per unit
  return (uint32_t)(((uint64_t)D.gc[0] * D.gc[1] * D.gc[2] + 255) / 256);
}

// a device table section: bytes appended to a host image, 256-byte aligned
struct Image {
  std::vector<unsigned char> bytes;
  template <typename T>
  size_t add(const std::vector<T>& v) {
    const size_t o = bytes.size();
    bytes.resize(o + align256(std::max<size_t>(v.size() * sizeof(T), 1)), 0);
    if (!v.empty()) memcpy(bytes.data() + o, v.data(), v.size() * sizeof(T));
    return o;
  }
};

std::vector<uint32_t> prefix(const std::vector<uint32_t>& units) {
  std::vector<uint32_t> p(units.size() + 1, 0);
  for (size_t j = 0; j < units.size(); j++) p[j + 1] = p[j] + units[j];
  return p;
}

}  // namespace

struct hpmdr_batch {
  // copies of the creating context's settings: the batch outlives nothing of
  // it but the CUDA stream it orders its calls after
  Allocator A;
  cudaStream_t user = nullptr;  // the context's stream at creation
  cudaStream_t s = nullptr;     // the batch's own stream (graphs capture on it)
  cudaEvent_t ev = nullptr;
  uint64_t Ts = 4096;
  uint32_t cr_num = 2, cr_den = 1;
  int force = -1;
  int dtype = 0;
  uint32_t n = 0;
  int sms = 152;
  std::vector<std::unique_ptr<hpmdr_handle>> hs;
  std::vector<BatchJob> jobs;
  Tuning tune;
  // device: static tables (unit prefixes, level entries), the job table,
  // per-job coder scratch, gathered metadata and retrieval records
  unsigned char* d_tab = nullptr;
  BatchJob* d_jobs = nullptr;
  unsigned char* d_scratch = nullptr;
  FieldMeta* d_metas = nullptr;
  RetrieveDev* d_rds = nullptr;
  int32_t* d_status = nullptr;
  uint32_t* d_u_dec = nullptr;
  // pinned host mirrors
  BatchJob* h_jobs = nullptr;
  FieldMeta* h_metas = nullptr;
  RetrieveDev* h_rds = nullptr;
  int32_t* h_status = nullptr;
  // unit tables (offsets into d_tab) and totals
  size_t o_stats = 0, o_gen = 0, o_chunks = 0, o_groups = 0, o_cells_refs = 0, o_cells_u0 = 0;
  uint32_t t_stats = 0, t_gen = 0, t_chunks = 0, t_groups = 0, t_cells = 0, n_cells_refs = 0;
  size_t o_gc_refs = 0, o_gc_u0 = 0, o_pack_u0 = 0;
  uint32_t n_gc_refs = 0, t_gc = 0, t_pack = 0;
  std::vector<std::vector<uint64_t>> soff;  // per job and level: staging offset
  std::vector<Round> rounds;
  cudaGraphExec_t g_ref = nullptr, g_ret = nullptr;
  uint64_t k_ref = 0, k_ret = 0;  // kernel launches per graph
  bool refactored = false;
  float last_ms[2] = {0, 0};

  template <typename T>
  T* tab(size_t o) const { return reinterpret_cast<T*>(d_tab + o); }

  void drop_graphs() {
    if (g_ref) cudaGraphExecDestroy(g_ref);
    if (g_ret) cudaGraphExecDestroy(g_ret);
    g_ref = g_ret = nullptr;
  }

  ~hpmdr_batch() {
    drop_graphs();
    if (s) {
      cudaStreamSynchronize(s);
      A.release(d_tab, s);
      A.release(d_jobs, s);
      A.release(d_scratch, s);
      A.release(d_metas, s);
      A.release(d_rds, s);
      A.release(d_status, s);
      A.release(d_u_dec, s);
      hs.clear();  // the handles free their memory on s
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    if (ev) cudaEventDestroy(ev);
    if (h_jobs) cudaFreeHost(h_jobs);
    if (h_metas) cudaFreeHost(h_metas);
    if (h_rds) cudaFreeHost(h_rds);
    if (h_status) cudaFreeHost(h_status);
  }

  // order this call after the work already on the creating context's stream
  void enter() {
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(s, ev, 0);
  }

  // unit tables for the current tuning (field sizes fixed at creation)
  hpmdr_status build_tables() {
    Image im;
    std::vector<uint32_t> u_stats(n), u_gen(n), u_chunks(n), u_groups(n);
    std::vector<LevelRef> cells, gcs;
    std::vector<uint32_t> u_cells, u_gc, u_pack;
    soff.assign(n, {});
    for (uint32_t j = 0; j < n; j++) {
      const hpmdr_handle* H = hs[j].get();
      u_stats[j] = (uint32_t)((H->N + tune.seg - 1) / tune.seg);
      u_gen[j] = H->generic_tiles;
      u_chunks[j] = H->total_chunks;
      u_groups[j] = (uint32_t)(H->nlev * H->ngroups);
      soff[j].assign(H->nlev, 0);
      uint64_t so = 0;
      for (const LevelDesc& D : H->levels) {
        LevelRef R;
        memset(&R, 0, sizeof(R));
        R.job = j;
        R.level = (uint32_t)D.level;
        if (D.fast == 1) {
          cells.push_back(R);
          u_cells.push_back(cell_tiles(D));
        } else if (D.fast == 2) {
          R.soff = so;
          soff[j][D.level] = so;
          so += D.n;
          gcs.push_back(R);
          u_gc.push_back(gcell_units(D));
          u_pack.push_back(D.ntiles);
        }
      }
    }
    const auto p_stats = prefix(u_stats), p_gen = prefix(u_gen), p_chunks = prefix(u_chunks),
               p_groups = prefix(u_groups), p_cells = prefix(u_cells);
    t_stats = p_stats.back();
    t_gen = p_gen.back();
    t_chunks = p_chunks.back();
    t_groups = p_groups.back();
    t_cells = p_cells.back();
    n_cells_refs = (uint32_t)cells.size();
    o_stats = im.add(p_stats);
    o_gen = im.add(p_gen);
    o_chunks = im.add(p_chunks);
    o_groups = im.add(p_groups);
    o_cells_refs = im.add(cells);
    o_cells_u0 = im.add(p_cells);
    {
      const auto p_gc = prefix(u_gc), p_pack = prefix(u_pack);
      n_gc_refs = (uint32_t)gcs.size();
      t_gc = p_gc.back();
      t_pack = p_pack.back();
      o_gc_refs = im.add(gcs);
      o_gc_u0 = im.add(p_gc);
      o_pack_u0 = im.add(p_pack);
    }
    // recomposition rounds
    rounds.clear();
    for (uint32_t r = 0;; r++) {
      std::vector<LevelRef> rc, rg, rgc;
      std::vector<uint32_t> uc, ucopy, ulev, uunpack, ugc;
      for (uint32_t j = 0; j < n; j++) {
        const hpmdr_handle* H = hs[j].get();
        const int L = H->nlev - 1, se = jobs[j].small_end, l = se + 1 + (int)r;
        if (l > L) continue;
        LevelRef R;
        memset(&R, 0, sizeof(R));
        R.job = j;
        R.level = (uint32_t)l;
        R.final = l == L;
        // the grid of level l - 1 (same alternation as the single-field path)
        if (l - 1 == 0) R.coarse = H->d_xroot;
        else R.coarse = ((L - (l - 1)) % 2 == 1) ? H->d_xa : H->d_xb;
        R.dst = R.final ? nullptr : (((L - l) % 2 == 1) ? H->d_xa : H->d_xb);
        const LevelDesc& D = H->levels[l];
        if (D.fast == 1) {
          rc.push_back(R);
          uc.push_back(cell_tiles(D));
        } else if (D.fast == 2) {
          R.soff = soff[j][l];
          rgc.push_back(R);
          uunpack.push_back(D.ntiles);
          ugc.push_back(gcell_units(D));
        } else {
          rg.push_back(R);
          ucopy.push_back((uint32_t)(((uint64_t)D.gc[0] * D.gc[1] * D.gc[2] + 255) / 256));
          ulev.push_back(D.ntiles);
        }
      }
      if (rc.empty() && rg.empty() && rgc.empty()) break;
      Round R;
      R.ncells = (uint32_t)rc.size();
      R.ngen = (uint32_t)rg.size();
      R.ngc = (uint32_t)rgc.size();
      {
        const auto pu = prefix(uunpack), pg = prefix(ugc);
        R.unpack_total = pu.back();
        R.gc_total = pg.back();
        R.o_gc_refs = im.add(rgc);
        R.o_unpack_u0 = im.add(pu);
        R.o_gc_u0 = im.add(pg);
      }
      const auto pc = prefix(uc), pcopy = prefix(ucopy), plev = prefix(ulev);
      R.cells_total = pc.back();
      R.copy_total = pcopy.back();
      R.level_total = plev.back();
      R.o_cells_refs = im.add(rc);
      R.o_cells_u0 = im.add(pc);
      R.o_gen_refs = im.add(rg);
      R.o_copy_u0 = im.add(pcopy);
      R.o_level_u0 = im.add(plev);
      rounds.push_back(R);
    }
    A.release(d_tab, s);
    d_tab = nullptr;
    HP_TRY(A.alloc((void**)&d_tab, im.bytes.size(), s));
    HP_CUDA(cudaMemcpyAsync(d_tab, im.bytes.data(), im.bytes.size(), cudaMemcpyHostToDevice, s));
    HP_CUDA(cudaStreamSynchronize(s));
    return HPMDR_OK;
  }

  uint32_t grid(uint32_t mul) const { return (uint32_t)sms * mul; }

  void enqueue_refactor(cudaStream_t s) {
    const uint32_t g = grid(tune.grid_mul);
    launch_b_init(d_jobs, n, s);
    launch_b_stats(d_jobs, tab<uint32_t>(o_stats), n, t_stats, tune.seg, dtype, g, s);
    launch_b_finalize(d_jobs, n, s);
    launch_b_cells_levelmax(d_jobs, tab<LevelRef>(o_cells_refs), tab<uint32_t>(o_cells_u0),
                            n_cells_refs, t_cells, g, dtype, s);
    launch_b_gcells_levelmax(d_jobs, tab<LevelRef>(o_gc_refs), tab<uint32_t>(o_gc_u0), n_gc_refs,
                             t_gc, dtype, g, s);
    launch_b_levelmax(d_jobs, tab<uint32_t>(o_gen), n, t_gen, dtype, g, s);
    launch_b_bitlen(d_jobs, n, s);
    launch_b_cells_encode(d_jobs, tab<LevelRef>(o_cells_refs), tab<uint32_t>(o_cells_u0),
                          n_cells_refs, t_cells, g, dtype, s);
    launch_b_gcells_encode(d_jobs, tab<LevelRef>(o_gc_refs), tab<uint32_t>(o_gc_u0), n_gc_refs,
                           t_gc, dtype, g, s);
    launch_b_pack(d_jobs, tab<LevelRef>(o_gc_refs), tab<uint32_t>(o_pack_u0), n_gc_refs, t_pack,
                  dtype == 0 ? 32 : 64, g, s);
    launch_b_encode(d_jobs, tab<uint32_t>(o_gen), n, t_gen, dtype, g, s);
    launch_b_chunk_stats(d_jobs, tab<uint32_t>(o_chunks), n, t_chunks, g, s);
    launch_b_decide(d_jobs, tab<uint32_t>(o_groups), n, t_groups, Ts, cr_num, cr_den, force, g, s);
    launch_b_huff_bits(d_jobs, tab<uint32_t>(o_chunks), n, t_chunks, g, s);
    launch_b_group_offsets(d_jobs, tab<uint32_t>(o_groups), n, t_groups, g, s);
    launch_b_huff_encode(d_jobs, tab<uint32_t>(o_chunks), n, t_chunks, g, s);
    launch_b_rle_encode(d_jobs, tab<uint32_t>(o_chunks), n, t_chunks, g, s);
    launch_b_headers(d_jobs, tab<uint32_t>(o_groups), n, t_groups, g, s);
    launch_b_sequence(d_jobs, n, s);
    launch_b_gather(d_jobs, n, d_metas, nullptr, nullptr, s);
  }

  void enqueue_retrieve(cudaStream_t s) {
    const uint32_t g = grid(tune.grid_mul);
    launch_b_select(d_jobs, n, s);
    launch_b_items_prefix(d_jobs, n, d_u_dec, s);
    launch_b_decode(d_jobs, d_u_dec, n, grid(tune.dec_mul), s);
    launch_b_recompose_small(d_jobs, n, dtype, s);
    for (const Round& R : rounds) {
      launch_b_cells_recompose(d_jobs, tab<LevelRef>(R.o_cells_refs), tab<uint32_t>(R.o_cells_u0),
                               R.ncells, R.cells_total, g, dtype, s);
      launch_b_unpack(d_jobs, tab<LevelRef>(R.o_gc_refs), tab<uint32_t>(R.o_unpack_u0), R.ngc,
                      R.unpack_total, dtype == 0 ? 32 : 64, g, s);
      launch_b_gcells_recompose(d_jobs, tab<LevelRef>(R.o_gc_refs), tab<uint32_t>(R.o_gc_u0), R.ngc,
                                R.gc_total, dtype, g, s);
      launch_b_recompose_copy(d_jobs, tab<LevelRef>(R.o_gen_refs), tab<uint32_t>(R.o_copy_u0),
                              R.ngen, R.copy_total, dtype, g, s);
      launch_b_recompose_level(d_jobs, tab<LevelRef>(R.o_gen_refs), tab<uint32_t>(R.o_level_u0),
                               R.ngen, R.level_total, dtype, g, s);
    }
    launch_b_gather(d_jobs, n, nullptr, d_rds, d_status, s);
  }

  hpmdr_status capture(bool refactor_pass) {
    cudaGraph_t graph = nullptr;
    const uint64_t k0 = hpmdr_kernel_launches();
    HP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    if (refactor_pass) enqueue_refactor(s);
    else enqueue_retrieve(s);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    const uint64_t k = hpmdr_kernel_launches() - k0;
    if (e != cudaSuccess) {
      g_last_error = std::string("batch graph capture: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return HPMDR_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g_last_error = std::string("batch graph instantiate: ") + cudaGetErrorString(e);
      return HPMDR_ERR_CUDA;
    }
    if (refactor_pass) g_ref = exec, k_ref = k;
    else g_ret = exec, k_ret = k;
    return HPMDR_OK;
  }

  // captured launches are counted once per replay, not at capture
  hpmdr_status launch(bool refactor_pass) {
    cudaGraphExec_t& g = refactor_pass ? g_ref : g_ret;
    if (!g) {
      const uint64_t before = hpmdr_kernel_launches();
      HP_TRY(capture(refactor_pass));
      unnote_launches(hpmdr_kernel_launches() - before);
    }
    HP_CUDA(cudaMemcpyAsync(d_jobs, h_jobs, sizeof(BatchJob) * n, cudaMemcpyHostToDevice, s));
    HP_CUDA(cudaGraphLaunch(g, s));
    const uint64_t k = refactor_pass ? k_ref : k_ret;
    for (uint64_t i = 0; i < k; i++) note_launch();
    return HPMDR_OK;
  }
};

extern "C" hpmdr_status hpmdr_batch_create(hpmdr_ctx* ctx, uint64_t n, const uint64_t* dims,
                                           hpmdr_dtype dtype, hpmdr_batch** out) {
  if (!ctx || !out || !dims || n == 0 || n > (1u << 20) ||
      (dtype != HPMDR_F32 && dtype != HPMDR_F64))
    return HPMDR_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<hpmdr_batch> b(new hpmdr_batch());
  b->A = ctx->A;
  b->user = ctx->stream;
  b->Ts = ctx->Ts;
  b->cr_num = ctx->cr_num;
  b->cr_den = ctx->cr_den;
  b->force = ctx->force;
  b->dtype = dtype;
  b->n = (uint32_t)n;
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  HP_CUDA(cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking));
  HP_CUDA(cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming));
  b->enter();
  const cudaStream_t s = b->s;
  b->hs.resize(n);
  b->jobs.assign(n, BatchJob{});
  // per-job coder scratch in one block
  std::vector<size_t> o_sc(n);
  size_t sc_bytes = 0;
  for (uint64_t j = 0; j < n; j++) {
    HP_TRY(new_handle(ctx, 3, dims + 3 * j, dtype, nullptr, b->hs[j]));
    hpmdr_handle* H = b->hs[j].get();
    H->stream = s;
    HP_TRY(H->A.alloc((void**)&H->d_slots, H->slot_bytes, s));
    HP_TRY(H->A.alloc((void**)&H->d_meta, sizeof(FieldMeta), s));
    HP_TRY(ensure_retrieve_buffers(H, s));  // planes, retrieval record, recompose grids
    const uint32_t ngt = (uint32_t)(H->nlev * H->ngroups), tc = std::max(H->total_chunks, 1u);
    const uint64_t gs = H->plan->gstage_sum;  // every general cell level staged at once
    o_sc[j] = sc_bytes;
    sc_bytes += align256(1024ull * ngt) + align256(8ull * ngt) + 3 * align256(4ull * tc) +
                align256(256ull * ngt) + align256(gs * (H->B / 8)) + align256(gs);
  }
  HP_TRY(b->A.alloc((void**)&b->d_scratch, sc_bytes, s));
  HP_TRY(b->A.alloc((void**)&b->d_jobs, sizeof(BatchJob) * n, s));
  HP_TRY(b->A.alloc((void**)&b->d_metas, sizeof(FieldMeta) * n, s));
  HP_TRY(b->A.alloc((void**)&b->d_rds, sizeof(RetrieveDev) * n, s));
  HP_TRY(b->A.alloc((void**)&b->d_status, 4 * n, s));
  HP_TRY(b->A.alloc((void**)&b->d_u_dec, 4 * (n + 1), s));
  HP_CUDA(cudaMallocHost((void**)&b->h_jobs, sizeof(BatchJob) * n));
  HP_CUDA(cudaMallocHost((void**)&b->h_metas, sizeof(FieldMeta) * n));
  HP_CUDA(cudaMallocHost((void**)&b->h_rds, sizeof(RetrieveDev) * n));
  HP_CUDA(cudaMallocHost((void**)&b->h_status, 4 * n));
  for (uint64_t j = 0; j < n; j++) {
    hpmdr_handle* H = b->hs[j].get();
    BatchJob& J = b->jobs[j];
    memset(&J, 0, sizeof(J));
    J.N = H->N;
    for (int d = 0; d < 3; d++) J.dims[d] = (uint32_t)H->dims[d];
    J.nlev = (uint32_t)H->nlev;
    J.ngt = (uint32_t)(H->nlev * H->ngroups);
    J.generic_tiles = H->generic_tiles;
    J.total_chunks = H->total_chunks;
    J.meta = H->d_meta;
    J.meta0 = H->plan->d_meta0;
    J.planes = H->d_planes;
    J.slots = H->d_slots;
    J.levels = H->d_levels;
    J.perm = H->d_perm;
    J.chunk_group = H->d_chunk_group;
    const uint32_t tc = std::max(H->total_chunks, 1u);
    unsigned char* p = b->d_scratch + o_sc[j];
    J.hist = (uint32_t*)p;
    p += align256(1024ull * J.ngt);
    J.gcost = (unsigned long long*)p;
    p += align256(8ull * J.ngt);
    J.ccost = (uint32_t*)p;
    p += align256(4ull * tc);
    J.cwords = (uint32_t*)p;
    p += align256(4ull * tc);
    J.cout = (uint32_t*)p;
    p += align256(4ull * tc);
    J.lens = p;
    p += align256(256ull * J.ngt);
    J.gq = p;
    p += align256(H->plan->gstage_sum * (H->B / 8));
    J.gsg = p;
    J.rd = H->d_rd;
    J.xroot = H->d_xroot;
    J.xa = H->d_xa;
    J.xb = H->d_xb;
    const int L = H->nlev - 1;
    int l_end = 0;  // same split as the single-field retrieval
    while (l_end < L && !H->levels[l_end + 1].fast && H->levels[l_end + 1].n <= kSmallLevelNodes)
      l_end++;
    J.small_end = l_end;
    H->small_end = l_end;
  }
  memcpy(b->h_jobs, b->jobs.data(), sizeof(BatchJob) * n);
  HP_TRY(b->build_tables());
  *out = b.release();
  return HPMDR_OK;
}

extern "C" void hpmdr_batch_destroy(hpmdr_batch* b) { delete b; }

extern "C" hpmdr_status hpmdr_batch_handle(hpmdr_batch* b, uint64_t i, hpmdr_handle** h) {
  if (!b || !h || i >= b->n) return HPMDR_ERR_ARG;
  *h = b->hs[i].get();
  return HPMDR_OK;
}

static hpmdr_status batch_refactor(hpmdr_batch* b, const void* const* fields, bool timed) {
  const cudaStream_t s = b->s;
  for (uint32_t j = 0; j < b->n; j++) {
    if (!fields[j] || ((uintptr_t)fields[j] & 15)) return HPMDR_ERR_ARG;
    b->h_jobs[j].f = fields[j];
  }
  b->enter();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timed) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  hpmdr_status st = b->launch(true);
  if (st == HPMDR_OK &&
      cudaMemcpyAsync(b->h_metas, b->d_metas, sizeof(FieldMeta) * b->n, cudaMemcpyDeviceToHost,
                      s) != cudaSuccess)
    st = HPMDR_ERR_CUDA;
  if (timed) cudaEventRecord(e1, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) st = HPMDR_ERR_CUDA;
  if (timed) {
    cudaEventElapsedTime(&b->last_ms[0], e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (st != HPMDR_OK) return st;
  hpmdr_status worst = HPMDR_OK;
  for (uint32_t j = 0; j < b->n; j++) {
    hpmdr_handle* H = b->hs[j].get();
    memcpy(H->meta.get(), &b->h_metas[j], sizeof(FieldMeta));
    count_items(H);
    if (H->meta->status && worst == HPMDR_OK) worst = (hpmdr_status)H->meta->status;
  }
  b->refactored = worst == HPMDR_OK;
  return worst;
}

static hpmdr_status batch_retrieve(hpmdr_batch* b, const double* rel, void* const* outs,
                                   hpmdr_retrieve_info* infos, bool timed) {
  if (!b->refactored) return HPMDR_ERR_ARG;
  const cudaStream_t s = b->s;
  for (uint32_t j = 0; j < b->n; j++) {
    if (!outs[j] || !(rel[j] >= 0.0)) return HPMDR_ERR_ARG;
    b->h_jobs[j].out = outs[j];
    b->h_jobs[j].tau = rel[j];
  }
  b->enter();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timed) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  hpmdr_status st = b->launch(false);
  if (st == HPMDR_OK &&
      (cudaMemcpyAsync(b->h_rds, b->d_rds, sizeof(RetrieveDev) * b->n, cudaMemcpyDeviceToHost, s) !=
           cudaSuccess ||
       cudaMemcpyAsync(b->h_status, b->d_status, 4 * b->n, cudaMemcpyDeviceToHost, s) !=
           cudaSuccess))
    st = HPMDR_ERR_CUDA;
  if (timed) cudaEventRecord(e1, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) st = HPMDR_ERR_CUDA;
  if (timed) {
    cudaEventElapsedTime(&b->last_ms[1], e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (st != HPMDR_OK) return st;
  hpmdr_status worst = HPMDR_OK;
  for (uint32_t j = 0; j < b->n; j++) {
    const RetrieveDev& rd = b->h_rds[j];
    const hpmdr_handle* H = b->hs[j].get();
    hpmdr_status r = b->h_status[j] ? (hpmdr_status)b->h_status[j] : (hpmdr_status)rd.status;
    if (infos) {
      hpmdr_retrieve_info& info = infos[j];
      memset(&info, 0, sizeof(info));
      info.est_linf = rd.E_abs;
      info.requested_abs = rd.tau_abs;
      info.est_units_hi = rd.E_hi;
      info.est_units_lo = rd.E_lo;
      info.bytes_fetched_total = rd.bytes_total;
      info.bytes_fetched_new = rd.bytes_new;
      info.nlevels = H->nlev;
      for (int l = 0; l < H->nlev && l < 64; l++) info.groups_per_level[l] = rd.g[l];
      info.status = r;
    }
    if (r != HPMDR_OK && (worst == HPMDR_OK || worst == HPMDR_ERR_UNATTAINABLE)) worst = r;
  }
  return worst;
}

extern "C" hpmdr_status hpmdr_batch_refactor(hpmdr_batch* b, const void* const* fields) {
  if (!b || !fields) return HPMDR_ERR_ARG;
  return batch_refactor(b, fields, true);
}

extern "C" hpmdr_status hpmdr_batch_retrieve(hpmdr_batch* b, const double* rel_bounds,
                                             void* const* outs, hpmdr_retrieve_info* infos) {
  if (!b || !rel_bounds || !outs) return HPMDR_ERR_ARG;
  return batch_retrieve(b, rel_bounds, outs, infos, true);
}

extern "C" hpmdr_status hpmdr_batch_last_ms(const hpmdr_batch* b, double ms[2]) {
  if (!b || !ms) return HPMDR_ERR_ARG;
  ms[0] = b->last_ms[0];
  ms[1] = b->last_ms[1];
  return HPMDR_OK;
}

static hpmdr_status apply_tuning(hpmdr_batch* b, const Tuning& t) {
  b->tune = t;
  b->drop_graphs();
  return b->build_tables();
}

extern "C" hpmdr_status hpmdr_batch_set_tuning(hpmdr_batch* b, const uint32_t tuning[3]) {
  if (!b || !tuning) return HPMDR_ERR_ARG;
  Tuning t;
  t.grid_mul = tuning[0];
  t.seg = tuning[1];
  t.dec_mul = tuning[2];
  if (t.grid_mul < 1 || t.grid_mul > 32 || t.dec_mul < 1 || t.dec_mul > 32 || t.seg < 1024 ||
      t.seg > (1u << 24) || t.seg % 1024)
    return HPMDR_ERR_ARG;
  return apply_tuning(b, t);
}

extern "C" hpmdr_status hpmdr_batch_get_tuning(const hpmdr_batch* b, uint32_t tuning[3]) {
  if (!b || !tuning) return HPMDR_ERR_ARG;
  tuning[0] = b->tune.grid_mul;
  tuning[1] = b->tune.seg;
  tuning[2] = b->tune.dec_mul;
  return HPMDR_OK;
}

// Times the refactor and retrieval graphs under each candidate tuning (the
// retrieval from empty plane caches each time) and keeps the fastest.  The
// handles end refactored from `fields`, with empty retrieval state.
extern "C" hpmdr_status hpmdr_batch_autotune(hpmdr_batch* b, const void* const* fields,
                                             const double* rel_bounds, void* const* outs,
                                             uint32_t best_out[3]) {
  if (!b || !fields || !rel_bounds || !outs) return HPMDR_ERR_ARG;
  const uint32_t grid_muls[] = {2, 4, 8}, segs[] = {16384, 65536}, dec_muls[] = {4, 8};
  Tuning best = b->tune;
  float best_ms = -1;
  for (uint32_t gm : grid_muls)
    for (uint32_t sg : segs)
      for (uint32_t dm : dec_muls) {
        Tuning t;
        t.grid_mul = gm;
        t.seg = sg;
        t.dec_mul = dm;
        HP_TRY(apply_tuning(b, t));
        float total = 0;
        for (int rep = 0; rep < 2; rep++) {  // the first run builds the graphs
          HP_TRY(batch_refactor(b, fields, true));
          hpmdr_status st = batch_retrieve(b, rel_bounds, outs, nullptr, true);
          if (st != HPMDR_OK && st != HPMDR_ERR_UNATTAINABLE) return st;
          total = b->last_ms[0] + b->last_ms[1];
        }
        if (best_ms < 0 || total < best_ms) best_ms = total, best = t;
      }
  HP_TRY(apply_tuning(b, best));
  HP_TRY(batch_refactor(b, fields, true));
  if (best_out) {
    best_out[0] = best.grid_mul;
    best_out[1] = best.seg;
    best_out[2] = best.dec_mul;
  }
  return HPMDR_OK;
}
