// Host runtime behind the C ABI of include/hpmdr.h: contexts, handles,
// device memory, the launch order of the refactor and retrieve paths, and
// the serialized handle format.  All arithmetic of the method runs in the
// kernels of the other .cu files; this file only plans, allocates, launches
// and copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <array>
#include <string>
#include <vector>

#include "../../include/hpmdr.h"
#include "dev_common.cuh"
#include "runtime.h"

using namespace hp;

thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

const char* kStageName[NSTAGE] = {
    "stats", "stats_finalize", "levelmax", "bitlen", "encode", "chunk_stats", "decide",
    "huff_bits", "group_offsets", "huff_encode", "rle_encode", "headers", "sequence", "select",
    "decode", "recompose_root", "recompose_copy", "recompose_level", "recompose_copy_out",
    "recompose_level_out", "vmag", "cells_levelmax", "cells_encode", "cells_recompose",
    "cells_recompose_out", "recompose_small", "gcells_levelmax", "gcells_quantize",
    "bitplane_encode", "bitplane_decode", "gcells_recompose", "gcells_recompose_out"};

void hp::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void hp::unnote_launches(uint64_t k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }

void hp::set_smem_once(const void* func, int bytes) {
  static std::mutex* mu = new std::mutex();
  static std::set<std::pair<const void*, int>>* done = new std::set<std::pair<const void*, int>>();
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(*mu);
  if (done->count({func, dev})) return;
  cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  done->insert({func, dev});
}

// ------------------------------------------------------------------ geometry
static int detail_levels(const uint64_t d[3]) {
  uint64_t n = std::max(d[0], std::max(d[1], d[2]));
  int L = 0;
  for (uint64_t h = 1; h < n; h *= 2) L++;
  return L;
}

static uint32_t axis_count(uint64_t g, int o) { return (uint32_t)(o ? g / 2 : (g + 1) / 2); }

uint64_t round16(uint64_t v) { return (v + 15) & ~15ull; }

hpmdr_status check_dims(int ndims, const uint64_t dims_in[3], uint64_t dims[3], uint64_t* N) {
  if (ndims < 1 || ndims > 3 || !dims_in) return HPMDR_ERR_ARG;
  uint64_t in[3] = {dims_in[0], dims_in[1], dims_in[2]};  // dims may alias dims_in
  dims[0] = dims[1] = dims[2] = 1;
  for (int i = 0; i < ndims; i++) dims[3 - ndims + i] = in[3 - ndims + i];
  uint64_t n = 1;
  for (int d = 0; d < 3; d++) {
    if (dims[d] == 0 || dims[d] > 0xffffffffull) return HPMDR_ERR_ARG;
    n *= dims[d];
    if (n >= 0xffffffffull) return HPMDR_ERR_ARG;
  }
  *N = n;
  return HPMDR_OK;
}

// levels below this many nodes keep the tile kernels (one launch for all of them)
static const uint32_t kGeneralCellMinNodes = 1u << 14;

static void plan_levels(Plan& P) {
  const int L = detail_levels(P.dims);
  P.nlev = L + 1;
  P.levels.assign(P.nlev, LevelDesc{});
  uint64_t poff = 0;
  uint32_t tile = 0, gtile = 0;
  for (int l = 0; l < P.nlev; l++) {
    LevelDesc& D = P.levels[l];
    memset(&D, 0, sizeof(D));
    D.level = l;
    D.hlog = l == 0 ? -1 : (L - l);
    uint64_t h = l == 0 ? (1ull << L) * 2 : (1ull << (L - l));
    for (int d = 0; d < 3; d++) {
      D.g[d] = (uint32_t)((P.dims[d] + h - 1) / h);
      D.gc[d] = (D.g[d] + 1) / 2;
    }
    uint64_t n = 0;
    if (l == 0) {
      n = 1;
      for (int t = 0; t <= 8; t++) D.off[t] = 0;
      D.off[8] = 1;
    } else {
      D.off[0] = D.off[1] = 0;
      for (int t = 1; t < 8; t++) {
        int oz = (t >> 2) & 1, oy = (t >> 1) & 1, ox = t & 1;
        D.cnt[t][0] = axis_count(D.g[0], oz);
        D.cnt[t][1] = axis_count(D.g[1], oy);
        D.cnt[t][2] = axis_count(D.g[2], ox);
        D.dx[t] = make_fastdiv(std::max(D.cnt[t][2], 1u));
        D.dy[t] = make_fastdiv(std::max(D.cnt[t][1], 1u));
        uint64_t c = (uint64_t)D.cnt[t][0] * D.cnt[t][1] * D.cnt[t][2];
        D.off[t] = (uint32_t)n;
        n += c;
      }
      D.off[8] = (uint32_t)n;
    }
    D.n = (uint32_t)n;
    D.W = (uint32_t)(4 * ((n + 127) / 128));
    // every level starts on a 256-byte boundary of the plane buffer (padding
    // between levels, never inside a group): with W a multiple of 8 words, a
    // warp's 32 consecutive words of a plane then cover 4 whole 32-byte
    // sectors instead of straddling 5
    poff = (poff + 255) & ~(uint64_t)255;
    D.plane_off = poff;
    poff += (uint64_t)(P.B + 1) * D.W * 4;
    D.tile0 = tile;
    D.ntiles = (uint32_t)((n + HP_TILE - 1) / HP_TILE);
    tile += D.ntiles;
    // cells of the level (its coarse grid), for the general cell kernels
    D.dx[0] = make_fastdiv(std::max(D.gc[2], 1u));
    D.dy[0] = make_fastdiv(std::max(D.gc[1], 1u));
    if (cell_path_ok(D, P.B)) D.fast = 1;
    else if (D.hlog >= 0 && D.n >= kGeneralCellMinNodes) D.fast = 2;
    else D.fast = 0;
    if (D.fast == 2) {
      P.gstage_max = std::max<uint64_t>(P.gstage_max, D.n);
      P.gstage_sum += D.n;
    }
    D.gtile0 = gtile;
    if (!D.fast) gtile += D.ntiles;
  }
  P.plane_bytes = poff;
  P.total_tiles = tile;
  P.generic_tiles = gtile;
  // Tile order: a tile starting at node j0 of parity type t sits at relative
  // position (j0 - off_t) / count_t of its type's raster; sorting by that
  // position makes the tiles of all seven types that cover the same region of
  // the grid run together, so their shared coarse neighbours and field rows
  // are read from L2 instead of being streamed from HBM once per type.
  P.perm.assign(tile, 0);
  for (int l = 0; l < P.nlev; l++) {
    const LevelDesc& D = P.levels[l];
    std::vector<std::pair<double, uint32_t>> key(D.ntiles);
    for (uint32_t q = 0; q < D.ntiles; q++) {
      const uint32_t j0 = q * HP_TILE;
      int t = 1;
      for (int k = 2; k <= 7; k++)
        if (j0 >= D.off[k]) t = k;
      const uint32_t cnt = D.off[t + 1] - D.off[t];
      const double rel = (l == 0 || cnt == 0) ? 0.0 : (double)(j0 - D.off[t]) / (double)cnt;
      key[q] = {rel + 1e-9 * t, q};
    }
    std::sort(key.begin(), key.end());
    for (uint32_t q = 0; q < D.ntiles; q++) P.perm[D.tile0 + q] = key[q].second;
  }
}

// group geometry (Sec. 5.2: B/4 groups of 4 planes, the sign plane in group 0)
// and slot capacities; fills meta0
static void plan_groups(Plan& P, uint64_t Ts, uint32_t num, uint32_t den, int force) {
  FieldMeta& M = *P.meta0;
  uint32_t chunk = 0;
  uint64_t slot = 0;
  P.chunk_group.clear();
  for (int l = 0; l < P.nlev; l++) {
    const LevelDesc& D = P.levels[l];
    for (int g = 0; g < P.ngroups; g++) {
      GroupMeta& G = M.grp[l][g];
      memset(&G, 0, sizeof(G));
      G.S = (uint64_t)(g == 0 ? 5 : 4) * D.W * 4;
      G.plane_off = D.plane_off + (g == 0 ? 0 : (uint64_t)(4 * g + 1) * D.W * 4);
      G.nchunks = (uint32_t)((G.S + HP_CHUNK - 1) / HP_CHUNK);
      G.chunk0 = chunk;
      for (uint32_t c = 0; c < G.nchunks; c++)
        P.chunk_group.push_back((uint32_t)(l * P.ngroups + g));
      chunk += G.nchunks;
      G.stored_len = G.S;
      if (force == HPMDR_HUFFMAN || force == HPMDR_RLE) {
        // forced coding: the worst case (16 bits per Huffman symbol, or one
        // (byte, length) record per byte) plus header and word padding
        G.cap = round16(2 * G.S + 4ull * G.nchunks + 512);
        G.slot_off = slot;
        slot += G.cap;
      } else if (force < 0 && G.S > Ts) {
        // a coded group is chosen only if S / est > num / den, so est < S den / num
        G.cap = round16((G.S * den + num - 1) / num) + 16;
        G.slot_off = slot;
        slot += G.cap;
      }
    }
  }
  P.total_chunks = chunk;
  P.slot_bytes = slot;
}

static void init_meta(FieldMeta& M, int dtype, int B, int nlev, int ngroups) {
  memset(&M, 0, sizeof(M));
  M.status = 0;
  M.dtype = dtype;
  M.B = B;
  M.nlev = nlev;
  M.ngroups = ngroups;
  M.E_f = 0;
  M.input_exact = 1;
  M.key_absmax = 0;
  M.key_min = ~0ull;
  M.key_max = 0;
  M.floored = 0;
  M.lsb_min = INT32_MAX;
  for (int l = 0; l < HP_MAX_LEVELS; l++) M.exact[l] = 1;
  M.seq_len = 0;
  M.compact = 0;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Plans are cached process-wide per (device, shape, B, T_s, T_cr).  Handles
// hold a reference, so a plan evicted from the cache lives on while used.
hpmdr_status get_plan(int device, const uint64_t dims[3], int dtype, uint64_t Ts,
                             uint32_t num, uint32_t den, int force, std::shared_ptr<const Plan>* out) {
  typedef std::array<uint64_t, 9> Key;
  static std::mutex* mu = new std::mutex();  // never destroyed: usable during exit
  static std::map<Key, std::shared_ptr<const Plan>>* cache =
      new std::map<Key, std::shared_ptr<const Plan>>();
  const Key key = {(uint64_t)device, dims[0], dims[1], dims[2], (uint64_t)dtype, Ts,
                   (uint64_t)num, (uint64_t)den, (uint64_t)(force + 1)};
  {
    std::lock_guard<std::mutex> lock(*mu);
    auto it = cache->find(key);
    if (it != cache->end()) {
      *out = it->second;
      return HPMDR_OK;
    }
  }
  std::shared_ptr<Plan> P(new Plan());
  for (int d = 0; d < 3; d++) P->dims[d] = dims[d];
  P->N = dims[0] * dims[1] * dims[2];
  P->B = dtype == HPMDR_F32 ? 32 : 64;
  P->ngroups = P->B / 4;
  plan_levels(*P);
  if (P->nlev > HP_MAX_LEVELS) return HPMDR_ERR_ARG;
  init_meta(*P->meta0, dtype, P->B, P->nlev, P->ngroups);
  plan_groups(*P, Ts, num, den, force);
  const size_t o_lv = 0, o_perm = align256(sizeof(LevelDesc) * P->nlev);
  const size_t o_cg = o_perm + align256(4ull * std::max(P->total_tiles, 1u));
  const size_t o_meta = o_cg + align256(4ull * std::max(P->total_chunks, 1u));
  const size_t bytes = o_meta + align256(sizeof(FieldMeta));
  std::vector<unsigned char> host(bytes, 0);
  memcpy(host.data() + o_lv, P->levels.data(), sizeof(LevelDesc) * P->nlev);
  memcpy(host.data() + o_perm, P->perm.data(), 4ull * P->total_tiles);
  memcpy(host.data() + o_cg, P->chunk_group.data(), 4ull * P->total_chunks);
  memcpy(host.data() + o_meta, P->meta0.get(), sizeof(FieldMeta));
  HP_CUDA(cudaMalloc((void**)&P->d_buf, bytes));
  HP_CUDA(cudaMemcpy(P->d_buf, host.data(), bytes, cudaMemcpyHostToDevice));
  P->d_levels = (LevelDesc*)(P->d_buf + o_lv);
  P->d_perm = (uint32_t*)(P->d_buf + o_perm);
  P->d_chunk_group = (uint32_t*)(P->d_buf + o_cg);
  P->d_meta0 = (FieldMeta*)(P->d_buf + o_meta);
  std::lock_guard<std::mutex> lock(*mu);
  if (cache->size() >= 1024) cache->clear();
  auto ins = cache->insert({key, P});
  *out = ins.first->second;
  return HPMDR_OK;
}

// a handle with the plan of (ndims, dims, dtype) under ctx's coder settings
hpmdr_status new_handle(hpmdr_ctx* ctx, int ndims, const uint64_t dims_in[3], int dtype,
                               const std::shared_ptr<const Plan>* plan_in,
                               std::unique_ptr<hpmdr_handle>& H) {
  if (dtype != HPMDR_F32 && dtype != HPMDR_F64) return HPMDR_ERR_ARG;
  H.reset(new hpmdr_handle());
  HP_TRY(check_dims(ndims, dims_in, H->dims, &H->N));
  if (plan_in) H->plan = *plan_in;
  else
    HP_TRY(get_plan(ctx->device, H->dims, dtype, ctx->Ts, ctx->cr_num, ctx->cr_den, ctx->force,
                    &H->plan));
  const Plan& P = *H->plan;
  H->A = ctx->A;
  H->stream = ctx->stream;
  H->dtype = dtype;
  H->B = P.B;
  H->ngroups = P.ngroups;
  H->nlev = P.nlev;
  H->levels = P.levels;
  H->total_tiles = P.total_tiles;
  H->generic_tiles = P.generic_tiles;
  H->total_chunks = P.total_chunks;
  H->plane_bytes = P.plane_bytes;
  H->slot_bytes = P.slot_bytes;
  H->d_levels = P.d_levels;
  H->d_perm = P.d_perm;
  H->d_chunk_group = P.d_chunk_group;
  memcpy(H->meta.get(), P.meta0.get(), sizeof(FieldMeta));
  return HPMDR_OK;
}

void count_items(hpmdr_handle* H) {
  H->max_items = 0;
  for (int l = 0; l < H->nlev; l++)
    for (int g = 0; g < H->ngroups; g++)
      if (H->compact || H->meta->grp[l][g].method != HPMDR_DC)
        H->max_items += H->meta->grp[l][g].nchunks;
}

// ------------------------------------------------------------------- context
extern "C" hpmdr_status hpmdr_ctx_create(hpmdr_ctx** out, const hpmdr_config* cfg,
                                         const hpmdr_allocator* alloc, void* stream) {
  if (!out) return HPMDR_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<hpmdr_ctx> c(new hpmdr_ctx());
  if (cfg) {
    if (cfg->group_m != 0 && cfg->group_m != 4) return HPMDR_ERR_ARG;
    if (cfg->size_threshold) c->Ts = cfg->size_threshold;
    if (cfg->cr_num || cfg->cr_den) {
      if (!cfg->cr_num || !cfg->cr_den || cfg->cr_num < cfg->cr_den) return HPMDR_ERR_ARG;
      c->cr_num = cfg->cr_num;
      c->cr_den = cfg->cr_den;
    }
    if (cfg->method < 0 || cfg->method > 3) return HPMDR_ERR_ARG;
    c->force = cfg->method - 1;
  }
  int ndev = 0;
  HP_CUDA(cudaGetDeviceCount(&ndev));
  if (ndev <= 0) return HPMDR_ERR_CUDA;
  HP_CUDA(cudaGetDevice(&c->device));
  c->stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    c->A.hook = *alloc;
    c->A.has_hook = true;
  } else {
    HP_CUDA(cudaDeviceGetDefaultMemPool(&c->A.pool, c->device));
    uint64_t thr = ~0ull;  // keep freed blocks cached in the pool
    HP_CUDA(cudaMemPoolSetAttribute(c->A.pool, cudaMemPoolAttrReleaseThreshold, &thr));
  }
  *out = c.release();
  return HPMDR_OK;
}

extern "C" void hpmdr_ctx_destroy(hpmdr_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  ctx->pending.clear();
  for (cudaStream_t s : ctx->aux) cudaStreamSynchronize(s);
  delete ctx;
}

extern "C" hpmdr_status hpmdr_ctx_set_stream(hpmdr_ctx* ctx, void* stream) {
  if (!ctx) return HPMDR_ERR_ARG;
  ctx->stream = (cudaStream_t)stream;
  return HPMDR_OK;
}

// ------------------------------------------------------------------ refactor
struct RefactorProf {
  size_t hbits = SIZE_MAX, henc = SIZE_MAX, renc = SIZE_MAX;
};

// Every device step of a refactor, enqueued on s without waiting: reads the
// field f (device, 16-byte aligned, H's dims), allocates and writes H's
// planes, slots and device metadata.
static hpmdr_status refactor_enqueue(hpmdr_ctx* ctx, hpmdr_handle* H, const void* f,
                                     cudaStream_t s, RefactorProf* rp) {
  const size_t esz = H->dtype == HPMDR_F32 ? 4 : 8;
  const int ngt = H->nlev * H->ngroups;
  const uint32_t tc = std::max(H->total_chunks, 1u);
  HP_TRY(H->A.alloc((void**)&H->d_planes, H->plane_bytes, s));
  HP_TRY(H->A.alloc((void**)&H->d_slots, H->slot_bytes, s));
  HP_TRY(H->A.alloc((void**)&H->d_meta, sizeof(FieldMeta), s));
  // per-call scratch in one block: group histograms and RLE sizes (zeroed,
  // accumulated by atomics), chunk costs, chunk words, chunk offsets, lengths
  const size_t o_hist = 0, o_gcost = align256(1024ull * ngt);
  const size_t o_counts = o_gcost + align256(8ull * ngt), o_cost = o_counts + 256;
  const size_t o_words = o_cost + align256(4ull * tc), o_out = o_words + align256(4ull * tc);
  const size_t o_lens = o_out + align256(4ull * tc), o_gq = o_lens + align256(256ull * ngt);
  // staging of the general cell levels (one level at a time)
  const uint64_t gmax = H->plan->gstage_max;
  const size_t o_gsg = o_gq + align256(gmax * (H->B / 8)), o_lists = o_gsg + align256(gmax);
  const size_t scratch_bytes = o_lists + align256(8ull * tc);
  unsigned char* sc = nullptr;
  HP_TRY(H->A.alloc((void**)&sc, scratch_bytes, s));
  uint32_t* d_hist = (uint32_t*)(sc + o_hist);
  unsigned long long* d_gcost = (unsigned long long*)(sc + o_gcost);
  uint32_t* d_cost = (uint32_t*)(sc + o_cost);
  uint32_t* d_words = (uint32_t*)(sc + o_words);
  uint32_t* d_out = (uint32_t*)(sc + o_out);
  uint8_t* d_lens = (uint8_t*)(sc + o_lens);
  void* d_gq = sc + o_gq;
  uint8_t* d_gsg = sc + o_gsg;
  uint32_t* d_counts = (uint32_t*)(sc + o_counts);  // zeroed with the histograms
  uint32_t* d_lists = (uint32_t*)(sc + o_lists);
  if (cudaMemsetAsync(sc, 0, o_cost, s) != cudaSuccess ||
      cudaMemcpyAsync(H->d_meta, H->plan->d_meta0, sizeof(FieldMeta), cudaMemcpyDeviceToDevice,
                      s) != cudaSuccess) {
    H->A.release(sc, s);
    g_last_error = "refactor setup copy failed";
    return HPMDR_ERR_CUDA;
  }
  ChunkMap cm{H->d_chunk_group, H->total_chunks};
  Profiler* P = ctx->P();
  const double fb = (double)H->N * esz, pb = (double)H->plane_bytes, cb = 4.0 * tc + 1032.0 * ngt;
  // FP32 with a cell-path finest level: the statistics and that level's
  // estimate share one read of the field
  const LevelDesc& Dfin = H->levels[H->nlev - 1];
  const bool fused = stats_cells_ok(H->dtype, Dfin);
  { ProfScope p(P, ST_STATS, fb, s);
    if (fused) launch_stats_cells((const float*)f, H->dims, H->d_levels + Dfin.level, Dfin,
                                  H->d_meta, s);
    else launch_stats(f, H->N, H->dtype, H->d_meta, s); }
  { ProfScope p(P, ST_FINALIZE, 0, s); launch_stats_finalize(H->d_meta, s); }
  // algorithmic bytes: the field once (split over the level kernels by node
  // count) and each level's planes once
  auto lvl_bytes = [&](const LevelDesc& D, bool planes_too) {
    return (double)D.n * esz + (planes_too ? (double)(H->B + 1) * D.W * 4.0 : 0.0);
  };
  double gen_f = 0, gen_p = 0;
  for (const LevelDesc& D : H->levels)
    if (!D.fast) gen_f += (double)D.n * esz, gen_p += (double)(H->B + 1) * D.W * 4.0;
  for (const LevelDesc& D : H->levels)
    if (D.fast == 1) {
      ProfScope p(P, ST_CELLS_MAX, lvl_bytes(D, false), s);
      launch_cells_levelmax(f, H->dtype, H->dims, H->d_levels + D.level, D, H->d_meta, s,
                            fused && D.level == Dfin.level);
    } else if (D.fast == 2) {
      ProfScope p(P, ST_GCELLS_MAX, lvl_bytes(D, false), s);
      launch_gcells_levelmax(f, H->dtype, H->dims, H->d_levels + D.level, D, H->d_meta, s);
    }
  if (H->generic_tiles) {
    ProfScope p(P, ST_LEVELMAX, gen_f, s);
    launch_levelmax(f, H->dtype, H->dims, H->d_levels, H->nlev, H->generic_tiles, H->d_perm,
                    H->d_meta, s);
  }
  { ProfScope p(P, ST_BITLEN, 0, s); launch_bitlen(H->d_meta, s); }
  const double qb = H->B / 8 + 1;  // staged bytes per node
  for (const LevelDesc& D : H->levels)
    if (D.fast == 1) {
      ProfScope p(P, ST_CELLS_ENC, lvl_bytes(D, true), s);
      launch_cells_encode(f, H->dtype, H->dims, H->d_levels + D.level, D, H->d_meta,
                          (uint32_t*)H->d_planes, s);
    } else if (D.fast == 2) {
      { ProfScope p(P, ST_GCELLS_ENC, lvl_bytes(D, false) + qb * D.n, s);
        launch_gcells_encode(f, H->dtype, H->dims, H->d_levels + D.level, D, H->d_meta, d_gq,
                             d_gsg, s); }
      { ProfScope p(P, ST_PACK, qb * D.n + (double)(H->B + 1) * D.W * 4.0, s);
        launch_bitplane_encode(d_gq, d_gsg, D.n, H->B, (uint32_t*)(H->d_planes + D.plane_off),
                               s); }
    }
  if (H->generic_tiles) {
    ProfScope p(P, ST_ENCODE, gen_f + gen_p, s);
    launch_encode(f, H->dtype, H->dims, H->d_levels, H->nlev, H->generic_tiles, H->d_perm,
                  H->d_meta, (uint32_t*)H->d_planes, s);
  }
  { ProfScope p(P, ST_CHUNK_STATS, pb + cb, s);
    launch_chunk_stats(H->d_planes, H->d_meta, cm, d_hist, d_gcost, d_cost, s); }
  { ProfScope p(P, ST_DECIDE, cb, s);
    launch_decide(H->d_meta, ngt, d_hist, d_gcost, d_lens, ctx->Ts, ctx->cr_num, ctx->cr_den,
                  ctx->force, s); }
  launch_coder_lists(H->d_meta, cm, d_lists, d_counts, s);
  { ProfScope p(P, ST_HUFF_BITS, 0, s); rp->hbits = p.i;
    launch_huff_bits_list(H->d_planes, H->d_meta, cm, d_lens, d_words, d_lists, d_counts, s); }
  { ProfScope p(P, ST_OFFSETS, 0, s);
    launch_group_offsets(H->d_meta, ngt, d_words, d_cost, d_out, s); }
  { ProfScope p(P, ST_HUFF_ENC, 0, s); rp->henc = p.i;
    launch_huff_encode_list(H->d_planes, H->d_meta, cm, d_lens, d_out, H->d_slots, d_lists,
                            d_counts, s); }
  { ProfScope p(P, ST_RLE_ENC, 0, s); rp->renc = p.i;
    launch_rle_encode_list(H->d_planes, H->d_meta, cm, d_out, H->d_slots, d_lists, d_counts, s); }
  { ProfScope p(P, ST_HEADERS, 0, s); launch_headers(H->d_meta, ngt, d_lens, d_out, H->d_slots, s); }
  { ProfScope p(P, ST_SEQUENCE, 0, s); launch_sequence(H->d_meta, s); }
  H->A.release(sc, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_last_error = std::string("refactor launch: ") + cudaGetErrorString(e);
    return HPMDR_ERR_CUDA;
  }
  return HPMDR_OK;
}

// page-locked host memory the device writes through its mapped address
static hpmdr_status alloc_mapped(size_t bytes, void** host, void** dev) {
  if (cudaHostAlloc(host, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    *host = nullptr;
    cudaGetLastError();
    return HPMDR_ERR_NOMEM;
  }
  if (cudaHostGetDevicePointer(dev, *host, 0) != cudaSuccess) {
    cudaFreeHost(*host);
    *host = nullptr;
    g_last_error = "cudaHostGetDevicePointer failed";
    cudaGetLastError();
    return HPMDR_ERR_CUDA;
  }
  return HPMDR_OK;
}

static_assert(sizeof(FieldMeta) % 4 == 0 && sizeof(RetrieveDev) % 4 == 0,
              "word copies to the host");

// waits for H's refactor on s and mirrors its metadata to the host (a kernel
// writes it to page-locked memory: a copy-engine transfer would wait behind
// large copies still running on other streams)
static hpmdr_status refactor_finish(hpmdr_ctx* ctx, hpmdr_handle* H, cudaStream_t s,
                                    const RefactorProf& rp) {
  if (!ctx->pinned_meta) HP_TRY(alloc_mapped(sizeof(FieldMeta), &ctx->pinned_meta, &ctx->pinned_meta_dev));
  launch_to_host(H->d_meta, ctx->pinned_meta_dev, sizeof(FieldMeta), nullptr, nullptr, 0, s);
  HP_CUDA(cudaGetLastError());
  HP_CUDA(cudaStreamSynchronize(s));
  std::memcpy(H->meta.get(), ctx->pinned_meta, sizeof(FieldMeta));
  count_items(H);
  if (H->meta->status) return (hpmdr_status)H->meta->status;
  if (ctx->prof.on) {  // bytes of the coder stages, known once the methods are chosen
    double hS = 0, hC = 0, rS = 0, rC = 0;
    for (int l = 0; l < H->nlev; l++)
      for (int g = 0; g < H->ngroups; g++) {
        const GroupMeta& G = H->meta->grp[l][g];
        if (G.method == HPMDR_HUFFMAN) hS += G.S, hC += G.stored_len;
        if (G.method == HPMDR_RLE) rS += G.S, rC += G.stored_len;
      }
    ctx->prof.patch(rp.hbits, hS);
    ctx->prof.patch(rp.henc, hS + hC);
    ctx->prof.patch(rp.renc, rS + rC);
  }
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_refactor(hpmdr_ctx* ctx, const void* field, int field_on_device,
                                       int ndims, const uint64_t dims_in[3], hpmdr_dtype dtype,
                                       hpmdr_handle** out) {
  if (!ctx || !field || !out) return HPMDR_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<hpmdr_handle> H;
  HP_TRY(new_handle(ctx, ndims, dims_in, dtype, nullptr, H));
  const cudaStream_t s = ctx->stream;
  const size_t esz = dtype == HPMDR_F32 ? 4 : 8;
  const void* f = field;
  void* d_field = nullptr;
  // host input, or a device pointer without 16-byte alignment (the kernels read
  // rows with 16-byte loads): stage it in an aligned device buffer
  if (!field_on_device || ((uintptr_t)field & 15)) {
    HP_TRY(H->A.alloc(&d_field, H->N * esz, s));
    if (cudaMemcpyAsync(d_field, field, H->N * esz,
                        field_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        s) != cudaSuccess) {
      H->A.release(d_field, s);
      g_last_error = "field upload failed";
      return HPMDR_ERR_CUDA;
    }
    f = d_field;
  }
  RefactorProf rp;
  hpmdr_status st = refactor_enqueue(ctx, H.get(), f, s, &rp);
  H->A.release(d_field, s);
  if (st != HPMDR_OK) return st;
  HP_TRY(refactor_finish(ctx, H.get(), s, rp));
  *out = H.release();
  return HPMDR_OK;
}

// ------------------------------------------------------------ chunk streaming
// A field too large to stage at once is cut into independent sub-blocks
// ("chunks") that are refactored and retrieved as separate fields (Sec. 5.3's
// pipeline).  Chunk c of the grid (ceil(Z/cz), ceil(Y/cy), ceil(X/cx)), in C
// order, runs on stream c mod nstreams: its host<->device copy overlaps the
// kernels of the chunks on the other streams.
struct ChunkGrid {
  uint64_t dims[3], chunk[3], count[3], n;
  void box(uint64_t c, uint64_t org[3], uint64_t ext[3]) const {
    const uint64_t cc[3] = {c / (count[1] * count[2]), (c / count[2]) % count[1], c % count[2]};
    for (int d = 0; d < 3; d++) {
      org[d] = cc[d] * chunk[d];
      ext[d] = std::min(chunk[d], dims[d] - org[d]);
    }
  }
};

static hpmdr_status chunk_grid(int ndims, const uint64_t dims_in[3], const uint64_t chunk_in[3],
                               ChunkGrid* G) {
  uint64_t N = 0;
  HP_TRY(check_dims(ndims, dims_in, G->dims, &N));
  if (!chunk_in) return HPMDR_ERR_ARG;
  uint64_t c[3] = {1, 1, 1};
  for (int i = 0; i < ndims; i++) c[3 - ndims + i] = chunk_in[3 - ndims + i];
  G->n = 1;
  for (int d = 0; d < 3; d++) {
    if (c[d] == 0) return HPMDR_ERR_ARG;
    G->chunk[d] = std::min(c[d], G->dims[d]);
    G->count[d] = (G->dims[d] + G->chunk[d] - 1) / G->chunk[d];
    G->n *= G->count[d];
  }
  return HPMDR_OK;
}

// copy the box (org, ext) between a dense (Z, Y, X) array and a dense ext-sized one
static hpmdr_status copy_box(void* dst, const void* src, const ChunkGrid& G, const uint64_t org[3],
                             const uint64_t ext[3], size_t esz, bool to_chunk, cudaMemcpyKind kind,
                             cudaStream_t s) {
  cudaMemcpy3DParms p;
  memset(&p, 0, sizeof(p));
  const cudaPitchedPtr full =
      make_cudaPitchedPtr(to_chunk ? (void*)src : dst, G.dims[2] * esz, G.dims[2] * esz, G.dims[1]);
  const cudaPitchedPtr part =
      make_cudaPitchedPtr(to_chunk ? dst : (void*)src, ext[2] * esz, ext[2] * esz, ext[1]);
  const cudaPos at = make_cudaPos(org[2] * esz, org[1], org[0]);
  if (to_chunk) {
    p.srcPtr = full;
    p.srcPos = at;
    p.dstPtr = part;
  } else {
    p.srcPtr = part;
    p.dstPtr = full;
    p.dstPos = at;
  }
  p.extent = make_cudaExtent(ext[2] * esz, ext[1], ext[0]);
  p.kind = kind;
  HP_CUDA(cudaMemcpy3DAsync(&p, s));
  return HPMDR_OK;
}

// nstreams streams ordered after ctx->stream
static hpmdr_status pipeline_streams(hpmdr_ctx* ctx, int nstreams, std::vector<cudaStream_t>& ss) {
  if (nstreams < 1 || nstreams > 16) return HPMDR_ERR_ARG;
  while ((int)ctx->aux.size() < nstreams) {
    cudaStream_t s = nullptr;
    HP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ctx->aux.push_back(s);
  }
  ss.assign(ctx->aux.begin(), ctx->aux.begin() + nstreams);
  cudaEvent_t e = nullptr;
  HP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEventRecord(e, ctx->stream);
  for (cudaStream_t s : ss) cudaStreamWaitEvent(s, e, 0);
  cudaEventDestroy(e);
  return HPMDR_OK;
}

static hpmdr_status join_streams(const std::vector<cudaStream_t>& ss) {
  hpmdr_status st = HPMDR_OK;
  for (cudaStream_t s : ss)
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      g_last_error = "chunk pipeline stream failed";
      st = HPMDR_ERR_CUDA;
    }
  return st;
}

extern "C" hpmdr_status hpmdr_refactor_chunked(hpmdr_ctx* ctx, const void* field,
                                               int field_on_device, int ndims,
                                               const uint64_t dims[3], const uint64_t chunk[3],
                                               hpmdr_dtype dtype, int nstreams,
                                               hpmdr_handle** out, uint64_t cap,
                                               uint64_t* nchunks) {
  if (!ctx || !nchunks || (dtype != HPMDR_F32 && dtype != HPMDR_F64)) return HPMDR_ERR_ARG;
  ChunkGrid G;
  HP_TRY(chunk_grid(ndims, dims, chunk, &G));
  *nchunks = G.n;
  if (!out) return HPMDR_OK;  // size query
  if (!field || cap < G.n) return HPMDR_ERR_ARG;
  for (uint64_t c = 0; c < G.n; c++) out[c] = nullptr;
  std::vector<cudaStream_t> ss;
  HP_TRY(pipeline_streams(ctx, nstreams, ss));
  const size_t esz = dtype == HPMDR_F32 ? 4 : 8;
  const size_t stage_bytes = G.chunk[0] * G.chunk[1] * G.chunk[2] * esz;
  std::vector<void*> stage(ss.size(), nullptr);
  std::vector<std::unique_ptr<hpmdr_handle>> hs(G.n);
  std::vector<RefactorProf> rps(G.n);
  std::shared_ptr<const Plan> full_plan;  // every interior chunk shares one plan
  hpmdr_status st = HPMDR_OK;
  for (size_t i = 0; i < ss.size() && st == HPMDR_OK; i++)
    st = ctx->A.alloc(&stage[i], stage_bytes, ss[i]);
  for (uint64_t c = 0; c < G.n && st == HPMDR_OK; c++) {
    const cudaStream_t s = ss[c % ss.size()];
    uint64_t org[3], ext[3];
    G.box(c, org, ext);
    const bool full = ext[0] == G.chunk[0] && ext[1] == G.chunk[1] && ext[2] == G.chunk[2];
    if ((st = new_handle(ctx, 3, ext, dtype, full && full_plan ? &full_plan : nullptr, hs[c])))
      break;
    if (full && !full_plan) full_plan = hs[c]->plan;
    void* buf = stage[c % ss.size()];
    if ((st = copy_box(buf, field, G, org, ext, esz, true,
                       field_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s)))
      break;
    st = refactor_enqueue(ctx, hs[c].get(), buf, s, &rps[c]);
  }
  for (size_t i = 0; i < ss.size(); i++) ctx->A.release(stage[i], ss[i]);
  hpmdr_status js = join_streams(ss);
  if (st == HPMDR_OK) st = js;
  for (uint64_t c = 0; c < G.n && st == HPMDR_OK; c++)
    st = refactor_finish(ctx, hs[c].get(), ss[c % ss.size()], rps[c]);
  if (st != HPMDR_OK) return st;
  for (uint64_t c = 0; c < G.n; c++) out[c] = hs[c].release();
  return HPMDR_OK;
}

// ------------------------------------------------------------------ retrieve
hpmdr_status ensure_retrieve_buffers(hpmdr_handle* H, cudaStream_t s) {
  if (!H->d_planes) HP_TRY(H->A.alloc((void**)&H->d_planes, H->plane_bytes, s));
  if (!H->d_rd) HP_TRY(H->A.alloc((void**)&H->d_rd, sizeof(RetrieveDev), s));
  if (!H->d_xroot) HP_TRY(H->A.alloc((void**)&H->d_xroot, 8, s));
  const int L = H->nlev - 1;
  if (L >= 2 && !H->d_xa) {
    const LevelDesc& D = H->levels[L];  // h = 1: coarse grid is G_2
    H->xa_elems = (uint64_t)D.gc[0] * D.gc[1] * D.gc[2];
    HP_TRY(H->A.alloc((void**)&H->d_xa, 8 * H->xa_elems, s));
  }
  if (L >= 3 && !H->d_xb) {
    const LevelDesc& D = H->levels[L - 1];  // h = 2: coarse grid is G_4
    H->xb_elems = (uint64_t)D.gc[0] * D.gc[1] * D.gc[2];
    HP_TRY(H->A.alloc((void**)&H->d_xb, 8 * H->xb_elems, s));
  }
  return HPMDR_OK;
}

// enqueue select -> decode -> recompose for one handle (device-resident out)
static hpmdr_status enqueue_retrieve(hpmdr_ctx* ctx, hpmdr_handle* H, double tau, int is_abs,
                                     void* d_out, cudaStream_t s) {
  HP_TRY(ensure_retrieve_buffers(H, s));
  Profiler* P = ctx->P();
  H->prof_lv.clear();
  H->prof_decode = SIZE_MAX;
  H->prof_small = SIZE_MAX;
  const uint32_t* Pl = (const uint32_t*)H->d_planes;
  const int L = H->nlev - 1;
  // the root and the leading run of small generic levels run in one CTA
  int l_end = 0;
  while (l_end < L && !H->levels[l_end + 1].fast && H->levels[l_end + 1].n <= kSmallLevelNodes)
    l_end++;
  // When every group of those levels is a direct copy already in the plane
  // buffer (not a compact handle, whose copies the decode makes), their
  // recomposition needs nothing from the decode and runs beside it on the
  // side stream, joined before the next level.
  // Their groups per level are computed on the host too (host_select_small, the
  // same choice k_select makes, which k_select checks), so the kernel starts with
  // k_select rather than after it.
  bool fork = !H->meta->compact;
  for (int l = 0; fork && l <= l_end; l++)
    for (int g = 0; g < H->ngroups; g++)
      if (H->meta->grp[l][g].method != HPMDR_DC) fork = false;
  SmallSel hs;
  hs.l_end = -1;
  if (fork) host_select_small(*H->meta, tau, is_abs, l_end, &hs);
  auto small = [&](cudaStream_t st, const SmallSel* sel) {
    ProfScope p(P, ST_SMALL, 0, st);
    H->prof_small = p.i;
    H->small_end = l_end;
    launch_recompose_small(Pl, H->d_meta, H->d_levels, H->levels.data(), l_end, H->nlev,
                           H->d_xroot, H->d_xa, H->d_xb, d_out, H->dtype, st, sel);
  };
  if (fork) {
    if (!ctx->side) {
      HP_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
      HP_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
      HP_CUDA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    }
    HP_CUDA(cudaEventRecord(ctx->ev_fork, s));  // after the previous retrieval's kernels
    HP_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    small(ctx->side, &hs);
  }
  { ProfScope p(P, ST_SELECT, 0, s);
    launch_select(H->d_meta, tau, is_abs, H->d_rd, s, fork ? &hs : nullptr); }
  { ProfScope p(P, ST_DECODE, 0, s); H->prof_decode = p.i;
    launch_decode(H->d_slots, H->d_meta, H->d_rd, H->max_items, H->d_planes, s); }
  if (fork) {
    HP_CUDA(cudaEventRecord(ctx->ev_join, ctx->side));
    HP_CUDA(cudaStreamWaitEvent(s, ctx->ev_join, 0));
  } else {
    small(s, nullptr);  // after the decode, which may write the planes it reads
  }
  // staging of the general cell levels: scratch of this retrieval only
  // (stream-ordered), so that it is not part of the handle's cache
  const uint64_t gmax = H->plan->gstage_max;
  void* d_gq = nullptr;
  if (gmax) HP_TRY(H->A.alloc(&d_gq, gmax * (H->B / 8 + 1), s));
  uint8_t* d_gsg = (uint8_t*)d_gq + gmax * (H->B / 8);
  const int64_t* coarse =
      l_end == 0 ? H->d_xroot : (((L - l_end) % 2 == 1) ? H->d_xa : H->d_xb);
  for (int l = l_end + 1; l <= L; l++) {
    const bool final = l == L;
    void* dst = final ? d_out : (void*)(((L - l) % 2 == 1) ? H->d_xa : H->d_xb);
    const int fd = final ? H->dtype : -1;
    if (H->levels[l].fast == 1) {
      ProfScope p(P, final ? ST_CELLS_REC_OUT : ST_CELLS_REC, 0, s);
      H->prof_lv.push_back({p.i, l * 8 + (final ? 3 : 1)});
      H->prof_lv.push_back({SIZE_MAX - 1, l * 8 + (final ? 2 : 0)});  // copy folded in
      launch_cells_recompose(Pl, H->d_meta, H->d_levels + l, H->levels[l], coarse, dst,
                             final ? 1 : 0, H->B, s);
    } else if (H->levels[l].fast == 2) {
      { ProfScope p(P, ST_UNPACK, 0, s);
        H->prof_lv.push_back({p.i, l * 8 + 4});
        launch_level_unpack(Pl, H->d_meta, H->d_levels + l, H->levels[l], H->B, d_gq, d_gsg,
                            s); }
      { ProfScope p(P, final ? ST_GCELLS_REC_OUT : ST_GCELLS_REC, 0, s);
        H->prof_lv.push_back({p.i, l * 8 + (final ? 6 : 5)});
        launch_gcells_recompose(H->d_meta, H->d_levels + l, H->levels[l], H->dtype, d_gq, d_gsg,
                                coarse, dst, final ? 1 : 0, s); }
    } else {
      { ProfScope p(P, final ? ST_COPY_OUT : ST_COPY, 0, s);
        H->prof_lv.push_back({p.i, l * 8 + (final ? 2 : 0)});
        launch_recompose_copy(H->d_levels + l, H->levels[l], coarse, dst, fd, H->d_meta, s); }
      { ProfScope p(P, final ? ST_LEVEL_OUT : ST_LEVEL, 0, s);
        H->prof_lv.push_back({p.i, l * 8 + (final ? 3 : 1)});
        launch_recompose_level(Pl, H->d_meta, H->d_levels + l, H->levels[l], H->d_perm, coarse,
                               dst, H->B, fd, s); }
    }
    coarse = (const int64_t*)dst;
  }
  H->A.release(d_gq, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_last_error = std::string("retrieve launch: ") + cudaGetErrorString(e);
    return HPMDR_ERR_CUDA;
  }
  return HPMDR_OK;
}

// algorithmic bytes of a retrieval's stages, once its selection is known: the
// stored bytes a decode reads and the plane bytes it writes; for the
// recomposition, the plane words of the selected groups a launch reads and
// the values it writes.  The int64 coarse grids a level reads and the staging
// of the general cell levels are intermediates of this implementation, not
// bytes of the method: they appear in the measured DRAM traffic only.
static void patch_retrieve_bytes(hpmdr_ctx* ctx, hpmdr_handle* H, const RetrieveDev& rd,
                                 const std::vector<std::pair<size_t, int>>& prof_lv,
                                 size_t prof_decode, size_t prof_small, int small_end) {
  if (!ctx->prof.on) return;
  const int ng = H->ngroups;
  const double esz = H->dtype == HPMDR_F32 ? 4.0 : 8.0;
  double dec = 0;
  for (uint32_t i = 0; i < rd.n_new && i < HP_SEQ_MAX; i++) {
    const GroupMeta& G = H->meta->grp[rd.new_gi[i] / ng][rd.new_gi[i] % ng];
    dec += (double)G.stored_len + (double)G.S;
  }
  ctx->prof.patch(prof_decode, dec);
  {  // small levels: their planes and the values they write
    double b = 0;
    for (int l = 1; l <= small_end; l++) {
      const LevelDesc& D = H->levels[l];
      const double coarse = (double)D.gc[0] * D.gc[1] * D.gc[2];
      const double osz = l == H->nlev - 1 ? esz : 8.0;
      const int g = rd.g[l];
      b += (g > 0 ? (double)(4 * g + 1) * D.W * 4.0 : 0.0) + ((double)D.n + coarse) * osz;
    }
    ctx->prof.patch(prof_small, b);
  }
  size_t last = SIZE_MAX;
  double last_b = 0;
  for (auto& pe : prof_lv) {
    const int l = pe.second / 8, kind = pe.second % 8;
    const LevelDesc& D = H->levels[l];
    const double coarse = (double)D.gc[0] * D.gc[1] * D.gc[2];
    const double osz = (kind == 2 || kind == 3 || kind == 6) ? esz : 8.0;
    const int g = rd.g[l];
    const double planes = g > 0 ? (double)(4 * g + 1) * D.W * 4.0 : 0.0;
    double b;
    if (kind == 0 || kind == 2) {  // the coarse nodes copied into the level grid
      b = coarse * osz;
    } else if (kind == 4) {  // planes -> staging
      b = planes;
    } else if (kind >= 5) {  // staging + coarse grid -> level grid (coarse nodes included)
      b = ((double)D.n + coarse) * osz;
    } else {  // planes + coarse grid -> the level's nodes
      b = planes + (double)D.n * osz;
    }
    if (pe.first == SIZE_MAX - 1) {  // a cell kernel also wrote the coarse nodes
      last_b += coarse * osz;
      ctx->prof.patch(last, last_b);
      continue;
    }
    ctx->prof.patch(pe.first, b);
    last = pe.first;
    last_b = b;
  }
}

void fill_info(const hpmdr_handle* H, const RetrieveDev& rd, hpmdr_retrieve_info* info);

hpmdr_status collect_info(hpmdr_ctx* ctx, hpmdr_handle* H, hpmdr_retrieve_info* info,
                                 cudaStream_t s) {
  RetrieveDev rd;
  int32_t mstatus = 0;
  HP_CUDA(cudaMemcpyAsync(&rd, H->d_rd, sizeof(rd), cudaMemcpyDeviceToHost, s));
  HP_CUDA(cudaMemcpyAsync(&mstatus, &H->d_meta->status, 4, cudaMemcpyDeviceToHost, s));
  HP_CUDA(cudaStreamSynchronize(s));
  if (mstatus) return (hpmdr_status)mstatus;
  patch_retrieve_bytes(ctx, H, rd, H->prof_lv, H->prof_decode, H->prof_small, H->small_end);
  fill_info(H, rd, info);
  return (hpmdr_status)rd.status;
}

void fill_info(const hpmdr_handle* H, const RetrieveDev& rd, hpmdr_retrieve_info* info) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->est_linf = rd.E_abs;
    info->requested_abs = rd.tau_abs;
    info->est_units_hi = rd.E_hi;
    info->est_units_lo = rd.E_lo;
    info->bytes_fetched_total = rd.bytes_total;
    info->bytes_fetched_new = rd.bytes_new;
    info->nlevels = H->nlev;
    for (int l = 0; l < H->nlev && l < 64; l++) info->groups_per_level[l] = rd.g[l];
    info->status = rd.status;
  }
}

static hpmdr_status retrieve_common(hpmdr_ctx* ctx, hpmdr_handle* H, double tau, int is_abs,
                                    void* out, int out_on_device, hpmdr_retrieve_info* info) {
  if (!ctx || !H || !out || !(tau >= 0.0)) return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  const size_t bytes = H->N * (H->dtype == HPMDR_F32 ? 4 : 8);
  void* d_out = out;
  if (!out_on_device) HP_TRY(H->A.alloc(&d_out, bytes, s));
  hpmdr_status st = enqueue_retrieve(ctx, H, tau, is_abs, d_out, s);
  if (st == HPMDR_OK && !out_on_device &&
      cudaMemcpyAsync(out, d_out, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    st = HPMDR_ERR_CUDA;
  hpmdr_status st2 = st == HPMDR_OK ? collect_info(ctx, H, info, s) : st;
  if (!out_on_device) H->A.release(d_out, s);
  return st2;
}

extern "C" hpmdr_status hpmdr_retrieve(hpmdr_ctx* ctx, hpmdr_handle* h, double rel, void* out,
                                       int out_on_device, hpmdr_retrieve_info* info) {
  return retrieve_common(ctx, h, rel, 0, out, out_on_device, info);
}

extern "C" hpmdr_status hpmdr_retrieve_abs(hpmdr_ctx* ctx, hpmdr_handle* h, double tau, void* out,
                                           int out_on_device, hpmdr_retrieve_info* info) {
  return retrieve_common(ctx, h, tau, 1, out, out_on_device, info);
}

// Retrieval of a chunk-streamed field: every chunk is retrieved with the same
// absolute bound tau = rel * (max_c vmax_c - min_c vmin_c), so the whole field
// meets the relative bound against its global range.  Each chunk's
// reconstruction goes to out (a dense (Z, Y, X) array) through a per-stream
// staging buffer; the copy of one chunk overlaps the kernels of the next.
// ------------------------------------------------ asynchronous retrieval
static constexpr size_t kSlotBytes = (sizeof(RetrieveDev) + 16 + 255) / 256 * 256;

static hpmdr_status ctx_wait(hpmdr_ctx* ctx) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (ctx->copy_stream) {
    const cudaError_t e2 = cudaStreamSynchronize(ctx->copy_stream);
    if (e == cudaSuccess) e = e2;
  }
  hpmdr_status first = HPMDR_OK;
  if (e != cudaSuccess) {
    g_last_error = std::string("wait: ") + cudaGetErrorString(e);
    first = HPMDR_ERR_CUDA;
  }
  for (PendingRetrieval& p : ctx->pending) {
    const unsigned char* slot = (const unsigned char*)ctx->pinned + (size_t)p.slot * kSlotBytes;
    const RetrieveDev& rd = *reinterpret_cast<const RetrieveDev*>(slot);
    const int32_t mstatus = *reinterpret_cast<const int32_t*>(slot + sizeof(RetrieveDev));
    hpmdr_status st = HPMDR_OK;
    if (e != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
    } else if (mstatus) {
      st = (hpmdr_status)mstatus;
    } else {
      patch_retrieve_bytes(ctx, p.H, rd, p.prof_lv, p.prof_decode, p.prof_small, p.small_end);
      fill_info(p.H, rd, p.info);
      st = (hpmdr_status)rd.status;
    }
    if (p.info && st != (hpmdr_status)rd.status) p.info->status = st;
    if (first == HPMDR_OK && st != HPMDR_OK) first = st;
  }
  ctx->pending.clear();
  return first;
}

static hpmdr_status retrieve_async_impl(hpmdr_ctx* ctx, hpmdr_handle* H, double rel, void* out,
                                       int out_on_device, hpmdr_retrieve_info* info);

extern "C" hpmdr_status hpmdr_retrieve_async(hpmdr_ctx* ctx, hpmdr_handle* H, double rel,
                                             void* out, hpmdr_retrieve_info* info) {
  return retrieve_async_impl(ctx, H, rel, out, 1, info);
}

extern "C" hpmdr_status hpmdr_retrieve_async_host(hpmdr_ctx* ctx, hpmdr_handle* H, double rel,
                                                  void* out, hpmdr_retrieve_info* info) {
  return retrieve_async_impl(ctx, H, rel, out, 0, info);
}

static hpmdr_status retrieve_async_impl(hpmdr_ctx* ctx, hpmdr_handle* H, double rel, void* out,
                                       int out_on_device, hpmdr_retrieve_info* info) {
  if (!ctx || !H || !out || !(rel >= 0.0)) return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  if (!ctx->pinned) HP_TRY(alloc_mapped(kSlotBytes * hpmdr_ctx::kRing, &ctx->pinned, &ctx->pinned_dev));
  if ((int)ctx->pending.size() == hpmdr_ctx::kRing) {  // every slot in flight: drain
    const hpmdr_status st = ctx_wait(ctx);
    if (st != HPMDR_OK && st != HPMDR_ERR_UNATTAINABLE) return st;
  }
  int b = -1;
  void* d_out = out;
  if (!out_on_device) {  // into one of the two device buffers, then copied out
    const size_t bytes = H->N * (H->dtype == HPMDR_F32 ? 4 : 8);
    if (!ctx->copy_stream) {
      HP_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
      for (int i = 0; i < 2; i++) {
        HP_CUDA(cudaEventCreateWithFlags(&ctx->ev_ready[i], cudaEventDisableTiming));
        HP_CUDA(cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming));
      }
    }
    if (ctx->out_stage_bytes < bytes) {  // grow: wait for the copies still reading them
      HP_CUDA(cudaStreamSynchronize(ctx->copy_stream));
      for (int i = 0; i < 2; i++) {
        ctx->A.release(ctx->out_stage[i], s);
        ctx->out_stage[i] = nullptr;
        ctx->copied_pending[i] = false;
      }
      ctx->out_stage_bytes = 0;
      for (int i = 0; i < 2; i++) HP_TRY(ctx->A.alloc(&ctx->out_stage[i], bytes, s));
      ctx->out_stage_bytes = bytes;
    }
    b = ctx->out_next;
    ctx->out_next ^= 1;
    if (ctx->copied_pending[b]) HP_CUDA(cudaStreamWaitEvent(s, ctx->ev_copied[b], 0));
    d_out = ctx->out_stage[b];
  }
  HP_TRY(enqueue_retrieve(ctx, H, rel, 0, d_out, s));
  if (b >= 0) {
    const size_t bytes = H->N * (H->dtype == HPMDR_F32 ? 4 : 8);
    HP_CUDA(cudaEventRecord(ctx->ev_ready[b], s));
    HP_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_ready[b], 0));
    HP_CUDA(cudaMemcpyAsync(out, d_out, bytes, cudaMemcpyDeviceToHost, ctx->copy_stream));
    HP_CUDA(cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream));
    ctx->copied_pending[b] = true;
  }
  PendingRetrieval p;
  p.H = H;
  p.info = info;
  p.slot = ctx->ring_next;
  ctx->ring_next = (ctx->ring_next + 1) % hpmdr_ctx::kRing;
  // the selection record and the status, by a kernel (not behind the copy
  // engine's queue of output transfers)
  unsigned char* slot = (unsigned char*)ctx->pinned_dev + (size_t)p.slot * kSlotBytes;
  launch_to_host(H->d_rd, slot, sizeof(RetrieveDev), &H->d_meta->status, slot + sizeof(RetrieveDev),
                 4, s);
  HP_CUDA(cudaGetLastError());
  p.prof_lv = H->prof_lv;
  p.prof_decode = H->prof_decode;
  p.prof_small = H->prof_small;
  p.small_end = H->small_end;
  ctx->pending.push_back(std::move(p));
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_ctx_wait(hpmdr_ctx* ctx) {
  if (!ctx) return HPMDR_ERR_ARG;
  return ctx_wait(ctx);
}

extern "C" hpmdr_status hpmdr_retrieve_chunked(hpmdr_ctx* ctx, hpmdr_handle* const* hs,
                                               uint64_t n, int ndims, const uint64_t dims[3],
                                               const uint64_t chunk[3], double rel, void* out,
                                               int out_on_device, int nstreams,
                                               hpmdr_retrieve_info* infos) {
  if (!ctx || !hs || !out || !(rel >= 0.0)) return HPMDR_ERR_ARG;
  ChunkGrid G;
  HP_TRY(chunk_grid(ndims, dims, chunk, &G));
  if (n != G.n || n == 0) return HPMDR_ERR_ARG;
  double lo = 0, hi = 0;
  for (uint64_t c = 0; c < n; c++) {
    const hpmdr_handle* H = hs[c];
    if (!H || H->dtype != hs[0]->dtype) return HPMDR_ERR_ARG;
    uint64_t org[3], ext[3];
    G.box(c, org, ext);
    for (int d = 0; d < 3; d++)
      if (H->dims[d] != ext[d]) return HPMDR_ERR_ARG;
    if (c == 0 || H->meta->vmin < lo) lo = H->meta->vmin;
    if (c == 0 || H->meta->vmax > hi) hi = H->meta->vmax;
  }
  const double tau = rel * (hi - lo);
  const size_t esz = hs[0]->dtype == HPMDR_F32 ? 4 : 8;
  std::vector<cudaStream_t> ss;
  HP_TRY(pipeline_streams(ctx, nstreams, ss));
  const size_t stage_bytes = G.chunk[0] * G.chunk[1] * G.chunk[2] * esz;
  std::vector<void*> stage(ss.size(), nullptr);
  hpmdr_status st = HPMDR_OK;
  for (size_t i = 0; i < ss.size() && st == HPMDR_OK; i++)
    st = ctx->A.alloc(&stage[i], stage_bytes, ss[i]);
  for (uint64_t c = 0; c < n && st == HPMDR_OK; c++) {
    const cudaStream_t s = ss[c % ss.size()];
    uint64_t org[3], ext[3];
    G.box(c, org, ext);
    void* buf = stage[c % ss.size()];
    if ((st = enqueue_retrieve(ctx, hs[c], tau, 1, buf, s))) break;
    st = copy_box(out, buf, G, org, ext, esz, false,
                  out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  }
  for (size_t i = 0; i < ss.size(); i++) ctx->A.release(stage[i], ss[i]);
  hpmdr_status js = join_streams(ss);
  if (st != HPMDR_OK) return st;
  if (js != HPMDR_OK) return js;
  hpmdr_status worst = HPMDR_OK;
  for (uint64_t c = 0; c < n; c++) {
    hpmdr_status r = collect_info(ctx, hs[c], infos ? &infos[c] : nullptr, ss[c % ss.size()]);
    if (r != HPMDR_OK && r != HPMDR_ERR_UNATTAINABLE) return r;
    if (r != HPMDR_OK) worst = r;
  }
  return worst;
}

// ----------------------------------------------------------------------- QoI
extern "C" hpmdr_status hpmdr_qoi_prepare_vmag(hpmdr_ctx* ctx, hpmdr_handle* v[3], const void* vx,
                                               const void* vy, const void* vz, int on_device) {
  if (!ctx || !v || !v[0] || !v[1] || !v[2] || !vx || !vy || !vz) return HPMDR_ERR_ARG;
  for (int c = 0; c < 3; c++)
    if (v[c]->dtype != HPMDR_F32 || v[c]->N != v[0]->N) return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  const uint64_t N = v[0]->N;
  const void* src[3] = {vx, vy, vz};
  void* tmp[3] = {nullptr, nullptr, nullptr};
  float* d_q = nullptr;
  hpmdr_status st = HPMDR_OK;
  float q[2];
  do {
    for (int c = 0; c < 3 && !on_device; c++) {
      if ((st = ctx->A.alloc(&tmp[c], N * 4, s))) break;
      if (cudaMemcpyAsync(tmp[c], src[c], N * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = HPMDR_ERR_CUDA;
        break;
      }
      src[c] = tmp[c];
    }
    if (st) break;
    if ((st = ctx->A.alloc((void**)&d_q, 8, s))) break;
    launch_vmag_range((const float*)src[0], (const float*)src[1], (const float*)src[2], N, d_q, s);
    if (cudaMemcpyAsync(q, d_q, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    if (!(q[1] >= ldexpf(1.0f, -60))) st = HPMDR_ERR_ARG;  // |v| too small for FP32 squares
    for (int c = 0; c < 3; c++) {
      v[c]->qmin = q[0];
      v[c]->qmax = q[1];
      v[c]->qoi_ready = st == HPMDR_OK;
    }
  } while (0);
  for (int c = 0; c < 3; c++) ctx->A.release(tmp[c], s);
  ctx->A.release(d_q, s);
  return st;
}

// bounds of the velocity-magnitude QoI: |(|v_hat| - |v|)| <= sqrt(sum eps_c^2),
// plus the FP32 evaluation error of |v| on both sides (< 3 ulps relative each)
static double qoi_component_bound(double tau_q, double qmax) {
  const double u = ldexp(1.0, -24);
  double slack = 7.0 * u * (qmax + tau_q);
  double eps = (tau_q - slack) / sqrt(3.0);
  eps = eps * (1.0 - ldexp(1.0, -50));
  return eps > 0.0 ? eps : 0.0;
}

static double qoi_estimate(const double E[3], double qmax) {
  const double u = ldexp(1.0, -24);
  double r = sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
  return (r + 7.0 * u * (qmax + r)) * (1.0 + ldexp(1.0, -50));
}

extern "C" hpmdr_status hpmdr_retrieve_qoi_vmag(hpmdr_ctx* ctx, hpmdr_handle* v[3], double rel,
                                                void* out[3], void* out_vmag, int on_device,
                                                hpmdr_retrieve_info info[4]) {
  if (!ctx || !v || !out_vmag || !(rel >= 0.0)) return HPMDR_ERR_ARG;
  for (int c = 0; c < 3; c++)
    if (!v[c] || !v[c]->qoi_ready || v[c]->N != v[0]->N) return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  const uint64_t N = v[0]->N;
  const double tau_q = rel * ((double)v[0]->qmax - (double)v[0]->qmin);
  const double eps = qoi_component_bound(tau_q, (double)v[0]->qmax);
  void* comp[3] = {nullptr, nullptr, nullptr};
  bool own[3] = {false, false, false};
  void* d_vm = on_device ? out_vmag : nullptr;
  hpmdr_status st = HPMDR_OK, worst = HPMDR_OK;
  hpmdr_retrieve_info tmp[4];
  hpmdr_retrieve_info* inf = info ? info : tmp;
  double E[3];
  do {
    for (int c = 0; c < 3; c++) {
      if (on_device && out && out[c]) comp[c] = out[c];
      else {
        if ((st = ctx->A.alloc(&comp[c], N * 4, s))) break;
        own[c] = true;
      }
    }
    if (st) break;
    if (!d_vm && (st = ctx->A.alloc(&d_vm, N * 4, s))) break;
    // the three component retrievals and |v| are enqueued back to back; each
    // selection record and status is written by a kernel into a page-locked
    // slot of the context's ring, read after the one wait below
    if (!ctx->pending.empty()) {  // earlier asynchronous retrievals own ring slots
      const hpmdr_status r = ctx_wait(ctx);
      if (r != HPMDR_OK && r != HPMDR_ERR_UNATTAINABLE) {
        st = r;
        break;
      }
    }
    if (!ctx->pinned &&
        (st = alloc_mapped(kSlotBytes * hpmdr_ctx::kRing, &ctx->pinned, &ctx->pinned_dev)))
      break;
    PendingRetrieval pr[3];
    for (int c = 0; c < 3; c++) {
      if ((st = enqueue_retrieve(ctx, v[c], eps, 1, comp[c], s))) break;
      unsigned char* slot = (unsigned char*)ctx->pinned_dev + (size_t)c * kSlotBytes;
      launch_to_host(v[c]->d_rd, slot, sizeof(RetrieveDev), &v[c]->d_meta->status,
                     slot + sizeof(RetrieveDev), 4, s);
      pr[c].H = v[c];
      pr[c].prof_lv = v[c]->prof_lv;
      pr[c].prof_decode = v[c]->prof_decode;
      pr[c].prof_small = v[c]->prof_small;
      pr[c].small_end = v[c]->small_end;
    }
    if (st) break;
    { ProfScope p(ctx->P(), ST_VMAG, 16.0 * N, s);
      launch_vmag((const float*)comp[0], (const float*)comp[1], (const float*)comp[2], N,
                  (float*)d_vm, s); }
    if (!on_device) {
      for (int c = 0; c < 3; c++)
        if (out && out[c] && cudaMemcpyAsync(out[c], comp[c], N * 4, cudaMemcpyDeviceToHost, s) !=
                                 cudaSuccess)
          st = HPMDR_ERR_CUDA;
      if (cudaMemcpyAsync(out_vmag, d_vm, N * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = HPMDR_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    for (int c = 0; c < 3 && st == HPMDR_OK; c++) {
      const unsigned char* slot = (const unsigned char*)ctx->pinned + (size_t)c * kSlotBytes;
      const RetrieveDev& rd = *reinterpret_cast<const RetrieveDev*>(slot);
      const int32_t mstatus = *reinterpret_cast<const int32_t*>(slot + sizeof(RetrieveDev));
      if (mstatus) {
        st = (hpmdr_status)mstatus;
        break;
      }
      patch_retrieve_bytes(ctx, v[c], rd, pr[c].prof_lv, pr[c].prof_decode, pr[c].prof_small,
                           pr[c].small_end);
      fill_info(v[c], rd, &inf[c]);
      const hpmdr_status r = (hpmdr_status)rd.status;
      if (r != HPMDR_OK && r != HPMDR_ERR_UNATTAINABLE) st = r;
      else if (r != HPMDR_OK) worst = r;
      E[c] = inf[c].est_linf;
    }
    if (st) break;
    memset(&inf[3], 0, sizeof(inf[3]));
    inf[3].est_linf = qoi_estimate(E, (double)v[0]->qmax);
    inf[3].requested_abs = tau_q;
    inf[3].status = worst;
    for (int c = 0; c < 3; c++) {
      inf[3].bytes_fetched_new += inf[c].bytes_fetched_new;
      inf[3].bytes_fetched_total += inf[c].bytes_fetched_total;
    }
    if (worst == HPMDR_OK && inf[3].est_linf > tau_q) worst = HPMDR_ERR_UNATTAINABLE;
    inf[3].status = worst;
  } while (0);
  for (int c = 0; c < 3; c++)
    if (own[c]) ctx->A.release(comp[c], s);
  if (!on_device) ctx->A.release(d_vm, s);
  return st != HPMDR_OK ? st : worst;
}

// ------------------------------------------- iterated QoI: total velocity
extern "C" hpmdr_status hpmdr_qoi_prepare_vtotal(hpmdr_ctx* ctx, hpmdr_handle* v[3],
                                                 const void* vx, const void* vy, const void* vz,
                                                 int on_device) {
  if (!ctx || !v || !v[0] || !v[1] || !v[2] || !vx || !vy || !vz) return HPMDR_ERR_ARG;
  for (int c = 0; c < 3; c++)
    if (v[c]->dtype != HPMDR_F32 || v[c]->N != v[0]->N) return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  const uint64_t N = v[0]->N;
  const void* src[3] = {vx, vy, vz};
  void* tmp[3] = {nullptr, nullptr, nullptr};
  double* d_r = nullptr;
  double r[2] = {0, 0};
  hpmdr_status st = HPMDR_OK;
  do {
    for (int c = 0; c < 3 && !on_device; c++) {
      if ((st = ctx->A.alloc(&tmp[c], N * 4, s))) break;
      if (cudaMemcpyAsync(tmp[c], src[c], N * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = HPMDR_ERR_CUDA;
        break;
      }
      src[c] = tmp[c];
    }
    if (st) break;
    if ((st = ctx->A.alloc((void**)&d_r, 16, s))) break;
    launch_vtotal_range((const float*)src[0], (const float*)src[1], (const float*)src[2], N, d_r, s);
    if (cudaMemcpyAsync(r, d_r, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    if (!(r[1] <= 0x1.fffffep127)) st = HPMDR_ERR_ARG;  // V must fit FP32
    for (int c = 0; c < 3; c++) {
      v[c]->vt_min = r[0];
      v[c]->vt_max = r[1];
      v[c]->vt_ready = st == HPMDR_OK;
    }
  } while (0);
  for (int c = 0; c < 3; c++) ctx->A.release(tmp[c], s);
  ctx->A.release(d_r, s);
  return st;
}

// absolute estimate after the first k steps of the handle's greedy sequence
static double prefix_estimate(const hpmdr_handle* H, int k) {
  const FieldMeta& M = *H->meta;
  if (k > M.seq_len) k = M.seq_len;
  const double v = ldexp((double)M.E_hi[k], 64) + (double)M.E_lo[k];
  return ldexp(v, M.E_f - 51 - H->B);
}

// the pointwise bound at one point (same operations as the device's)
static double vtotal_point_bound_host(const float xs[3], const double e[3]) {
  double b = 0.0;
  for (int i = 0; i < 3; i++) {
    double t = 2.0 * fabs((double)xs[i]);
    t = t * e[i];
    const double u = e[i] * e[i];
    t = t + u;
    b = b + t;
  }
  const double a = (double)xs[0] * (double)xs[0], bb = (double)xs[1] * (double)xs[1];
  const double c = (double)xs[2] * (double)xs[2];
  const double v = (a + bb) + c;
  if (v > 0x1.fffffep127) return INFINITY;
  b = b + v * 0x1p-24;
  if (v != 0.0) b = b + 0x1p-150;
  b = b + v * 0x1p-50;
  return b;
}

// Algorithm 3 for V = vx^2 + vy^2 + vz^2: retrieve every variable to its data
// bound, bound the QoI error on the device, and choose the next bounds by the
// requested estimator until the bound meets tau.
extern "C" hpmdr_status hpmdr_retrieve_qoi_vtotal(hpmdr_ctx* ctx, hpmdr_handle* v[3], double rel,
                                                  int estimator, double c, void* out[3],
                                                  void* out_qoi, int on_device,
                                                  hpmdr_qoi_report* rep) {
  if (!ctx || !v || !out_qoi || !(rel >= 0.0) || estimator < 0 || estimator > 2) return HPMDR_ERR_ARG;
  for (int i = 0; i < 3; i++)
    if (!v[i] || !v[i]->vt_ready || v[i]->N != v[0]->N) return HPMDR_ERR_ARG;
  if (c == 0.0) c = 10.0;  // the paper's threshold
  const cudaStream_t s = ctx->stream;
  const uint64_t N = v[0]->N;
  const double vt_min = v[0]->vt_min, vt_max = v[0]->vt_max;
  const double tau = rel * (vt_max - vt_min);
  hpmdr_qoi_report R;
  memset(&R, 0, sizeof(R));
  R.tau_abs = tau;
  double eps[3], E[3];
  int nseq[3];
  for (int i = 0; i < 3; i++) {
    eps[i] = vt_max > 0.0 ? (tau / vt_max) * v[i]->meta->range : 0.0;
    nseq[i] = v[i]->meta->seq_len;
  }
  void* comp[3] = {nullptr, nullptr, nullptr};
  bool own[3] = {false, false, false};
  void* d_q = on_device ? out_qoi : nullptr;
  unsigned long long* d_best = nullptr;
  hpmdr_status st = HPMDR_OK, status = HPMDR_ERR_UNATTAINABLE;
  do {
    for (int i = 0; i < 3; i++) {
      if (on_device && out && out[i]) comp[i] = out[i];
      else {
        if ((st = ctx->A.alloc(&comp[i], N * 4, s))) break;
        own[i] = true;
      }
    }
    if (st) break;
    if (!d_q && (st = ctx->A.alloc(&d_q, N * 4, s))) break;
    if ((st = ctx->A.alloc((void**)&d_best, vtotal_bound_scratch(N), s))) break;
    for (int it = 1; it <= 4096 && st == HPMDR_OK; it++) {
      bool full = true;
      uint64_t fetched = 0;
      // With three distinct handles the retrievals and the bound are enqueued back
      // to back: the bound kernels read each variable's error estimate from its
      // selection record, and one wait brings back the records, the statuses and
      // the bound.  A handle given twice has one record, which its second
      // retrieval overwrites: then each record is read right after its retrieval
      // and the estimates are copied into the bound's own slots.
      const bool distinct = v[0] != v[1] && v[0] != v[2] && v[1] != v[2];
      RetrieveDev rdh[3];
      int32_t msth[3] = {0, 0, 0};
      bool ok = true;
      for (int i = 0; i < 3 && st == HPMDR_OK && ok; i++) {
        st = enqueue_retrieve(ctx, v[i], eps[i], 1, comp[i], s);
        if (st == HPMDR_OK && !distinct)
          ok = cudaMemcpyAsync(&rdh[i], v[i]->d_rd, sizeof(RetrieveDev), cudaMemcpyDeviceToHost,
                               s) == cudaSuccess &&
               cudaMemcpyAsync(&msth[i], &v[i]->d_meta->status, 4, cudaMemcpyDeviceToHost, s) ==
                   cudaSuccess &&
               cudaStreamSynchronize(s) == cudaSuccess;
      }
      if (st) break;
      double* d_e = vtotal_bound_e(d_best, N);
      if (!distinct && ok) {
        const double eh[3] = {rdh[0].E_abs, rdh[1].E_abs, rdh[2].E_abs};
        ok = cudaMemcpyAsync(d_e, eh, 24, cudaMemcpyHostToDevice, s) == cudaSuccess;
      }
      const double* const ep[3] = {
          distinct ? &v[0]->d_rd->E_abs : d_e, distinct ? &v[1]->d_rd->E_abs : d_e + 1,
          distinct ? &v[2]->d_rd->E_abs : d_e + 2};
      if (ok)
        launch_vtotal_bound((const float*)comp[0], (const float*)comp[1], (const float*)comp[2],
                            N, ep, (float*)d_q, d_best, s);
      unsigned long long best[2];
      ok = ok && cudaGetLastError() == cudaSuccess &&
           cudaMemcpyAsync(best, d_best, 16, cudaMemcpyDeviceToHost, s) == cudaSuccess;
      for (int i = 0; i < 3 && ok && distinct; i++)
        ok = cudaMemcpyAsync(&rdh[i], v[i]->d_rd, sizeof(RetrieveDev), cudaMemcpyDeviceToHost,
                             s) == cudaSuccess &&
             cudaMemcpyAsync(&msth[i], &v[i]->d_meta->status, 4, cudaMemcpyDeviceToHost, s) ==
                 cudaSuccess;
      if (!ok || cudaStreamSynchronize(s) != cudaSuccess) {
        st = HPMDR_ERR_CUDA;
        break;
      }
      for (int i = 0; i < 3 && st == HPMDR_OK; i++) {
        if (msth[i]) {
          st = (hpmdr_status)msth[i];
          break;
        }
        patch_retrieve_bytes(ctx, v[i], rdh[i], v[i]->prof_lv, v[i]->prof_decode,
                             v[i]->prof_small, v[i]->small_end);
        hpmdr_retrieve_info inf;
        fill_info(v[i], rdh[i], &inf);
        const hpmdr_status r = (hpmdr_status)rdh[i].status;
        if (r != HPMDR_OK && r != HPMDR_ERR_UNATTAINABLE) {
          st = r;
          break;
        }
        E[i] = inf.est_linf;
        int k = 0;
        for (int l = 0; l < inf.nlevels; l++) k += inf.groups_per_level[l];
        R.prefix[i] = k;
        if (k < nseq[i]) full = false;
        fetched += inf.bytes_fetched_total;
      }
      if (st) break;
      double bmax;
      memcpy(&bmax, &best[0], 8);
      const double bound = bmax * (1.0 + 0x1p-40);
      R.iterations = it;
      R.est = bound;
      R.bytes_fetched_total = fetched;
      for (int i = 0; i < 3; i++) R.eps[i] = E[i];
      if (bound <= tau) {
        status = HPMDR_OK;
        break;
      }
      if (full) break;
      bool ma = estimator == HPMDR_EST_MA;
      if (estimator == HPMDR_EST_MAPE) {
        const double p = bound / tau;
        if (p > c) {
          for (int i = 0; i < 3; i++) eps[i] = E[i] / p;
        } else {
          ma = true;
        }
      } else if (estimator == HPMDR_EST_CP) {
        float xs[3];
        for (int i = 0; i < 3; i++)
          if (cudaMemcpyAsync(&xs[i], (const float*)comp[i] + best[1], 4, cudaMemcpyDeviceToHost,
                              s) != cudaSuccess)
            st = HPMDR_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) st = HPMDR_ERR_CUDA;
        double e[3] = {E[0], E[1], E[2]};
        for (int k = 0; k < 1100; k++) {
          for (int i = 0; i < 3; i++) e[i] = e[i] * 0.5;
          if (vtotal_point_bound_host(xs, e) * (1.0 + 0x1p-40) <= tau) break;
        }
        for (int i = 0; i < 3; i++) eps[i] = e[i];
      }
      if (ma)
        for (int i = 0; i < 3; i++)
          if (R.prefix[i] < nseq[i]) eps[i] = prefix_estimate(v[i], R.prefix[i] + 1);
    }
    if (st) break;
    if (!on_device) {
      for (int i = 0; i < 3; i++)
        if (out && out[i] && cudaMemcpyAsync(out[i], comp[i], N * 4, cudaMemcpyDeviceToHost, s) !=
                                 cudaSuccess)
          st = HPMDR_ERR_CUDA;
      if (cudaMemcpyAsync(out_qoi, d_q, N * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = HPMDR_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) st = HPMDR_ERR_CUDA;
  } while (0);
  for (int i = 0; i < 3; i++)
    if (own[i]) ctx->A.release(comp[i], s);
  if (!on_device) ctx->A.release(d_q, s);
  ctx->A.release(d_best, s);
  R.status = st != HPMDR_OK ? st : status;
  if (rep) *rep = R;
  return (hpmdr_status)R.status;
}

// ------------------------------------------------------------- inspection
extern "C" hpmdr_status hpmdr_handle_field_info(const hpmdr_handle* h, int* dtype, uint64_t dims[3],
                                                int* nlevels, int* E_f, int* input_exact,
                                                double stats[4]) {
  if (!h) return HPMDR_ERR_ARG;
  if (dtype) *dtype = h->dtype;
  if (dims) memcpy(dims, h->dims, sizeof(h->dims));
  if (nlevels) *nlevels = h->nlev;
  if (E_f) *E_f = h->meta->E_f;
  if (input_exact) *input_exact = h->meta->input_exact;
  if (stats) {
    stats[0] = h->meta->maxabs;
    stats[1] = h->meta->vmin;
    stats[2] = h->meta->vmax;
    stats[3] = h->meta->range;
  }
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_handle_level_info(const hpmdr_handle* h, int level, uint64_t* n,
                                                int* bl, int* ngroups, int* exact) {
  if (!h || level < 0 || level >= h->nlev) return HPMDR_ERR_ARG;
  if (n) *n = h->levels[level].n;
  if (bl) *bl = h->meta->bl[level];
  if (ngroups) *ngroups = h->ngroups;
  if (exact) *exact = h->meta->exact[level];
  return HPMDR_OK;
}

static const uint8_t* group_src(const hpmdr_handle* h, int l, int g) {
  const GroupMeta& G = h->meta->grp[l][g];
  return (G.method == HPMDR_DC && !h->compact) ? h->d_planes + G.plane_off
                                               : h->d_slots + G.slot_off;
}

extern "C" hpmdr_status hpmdr_handle_group(const hpmdr_handle* h, int level, int group, void* buf,
                                           uint64_t* len, int* method, uint64_t est[2]) {
  if (!h || !len || level < 0 || level >= h->nlev || group < 0 || group >= h->ngroups)
    return HPMDR_ERR_ARG;
  const GroupMeta& G = h->meta->grp[level][group];
  if (method) *method = G.method;
  if (est) {
    est[0] = G.est_H;
    est[1] = G.est_R;
  }
  if (!buf) {
    *len = G.stored_len;
    return HPMDR_OK;
  }
  if (*len < G.stored_len) return HPMDR_ERR_ARG;
  *len = G.stored_len;
  HP_CUDA(cudaMemcpy(buf, group_src(h, level, group), G.stored_len, cudaMemcpyDeviceToHost));
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_handle_planes(const hpmdr_handle* h, int level, void* buf,
                                            uint64_t* len) {
  if (!h || !len || level < 0 || level >= h->nlev) return HPMDR_ERR_ARG;
  const LevelDesc& D = h->levels[level];
  const uint64_t need = (uint64_t)(h->B + 1) * D.W * 4;
  if (!buf) {
    *len = need;
    return HPMDR_OK;
  }
  if (*len < need || !h->d_planes) return HPMDR_ERR_ARG;  // compact handle without a cache
  *len = need;
  HP_CUDA(cudaMemcpy(buf, h->d_planes + D.plane_off, need, cudaMemcpyDeviceToHost));
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_handle_sequence(const hpmdr_handle* h, int* seq, int cap, int* len) {
  if (!h || !len) return HPMDR_ERR_ARG;
  *len = h->meta->seq_len;
  for (int i = 0; seq && i < h->meta->seq_len && i < cap; i++) seq[i] = h->meta->seq[i];
  return HPMDR_OK;
}

// ------------------------------------------------------------ serialization
// Layout (little-endian): "HPMDR1\0\0", u32 version=1, u32 reserved,
// i32 dtype, B, nlev, ngroups, E_f, input_exact, u64 dims[3],
// f64 maxabs, vmin, vmax, range, f32 qmin, qmax, i32 qoi_ready, i32 seq_len,
// per level: i32 bl, i32 exact;  per (level, group): u64 stored_len, i32 method,
// i32 reserved, u64 est_H, u64 est_R;  u8 seq[seq_len] padded to 8;
// u64 E_hi[seq_len+1], E_lo[seq_len+1];  then each group's stored bytes in
// (level, group) order, each padded to 16 bytes.
namespace {
struct Writer {
  uint8_t* p;
  uint64_t n = 0;
  void put(const void* v, size_t k) {
    if (p) memcpy(p + n, v, k);
    n += k;
  }
  template <typename T>
  void val(T v) { put(&v, sizeof(T)); }
  void pad(size_t a) {
    while (n % a) val<uint8_t>(0);
  }
};
struct Reader {
  const uint8_t* p;
  uint64_t len, n = 0;
  bool ok = true;
  void get(void* v, size_t k) {
    if (n + k > len) {
      ok = false;
      memset(v, 0, k);
      return;
    }
    memcpy(v, p + n, k);
    n += k;
  }
  template <typename T>
  T val() {
    T v;
    get(&v, sizeof(T));
    return v;
  }
  void pad(size_t a) { n = (n + a - 1) / a * a; }
};
}  // namespace

// one copy per run of byte ranges that are contiguous on both sides
struct CopyRuns {
  std::vector<std::array<uint64_t, 3>> v;  // dst, src, len
  void add(void* dst, const void* src, uint64_t len) {
    const uint64_t d = (uint64_t)(uintptr_t)dst, s = (uint64_t)(uintptr_t)src;
    if (!v.empty() && v.back()[0] + v.back()[2] == d && v.back()[1] + v.back()[2] == s)
      v.back()[2] += len;
    else
      v.push_back({d, s, len});
  }
  hpmdr_status issue(cudaMemcpyKind kind, cudaStream_t st) const {
    for (const auto& c : v)
      HP_CUDA(cudaMemcpyAsync((void*)(uintptr_t)c[0], (const void*)(uintptr_t)c[1], c[2], kind, st));
    return HPMDR_OK;
  }
};

// The export stream of h: its header written to buf (nullptr: sizes only),
// and where each stored group goes (byte offset in the stream, length), in
// (level, group) order.  Returns the stream length.
static uint64_t export_layout(const hpmdr_handle* h, uint8_t* buf,
                              std::vector<std::pair<uint64_t, uint64_t>>* pos) {
  const FieldMeta& M = *h->meta;
  Writer w{buf};
  w.put("HPMDR1\0\0", 8);
  w.val<uint32_t>(1);
  w.val<uint32_t>(0);
  w.val<int32_t>(h->dtype);
  w.val<int32_t>(h->B);
  w.val<int32_t>(h->nlev);
  w.val<int32_t>(h->ngroups);
  w.val<int32_t>(M.E_f);
  w.val<int32_t>(M.input_exact);
  for (int d = 0; d < 3; d++) w.val<uint64_t>(h->dims[d]);
  w.val<double>(M.maxabs);
  w.val<double>(M.vmin);
  w.val<double>(M.vmax);
  w.val<double>(M.range);
  w.val<float>(h->qmin);
  w.val<float>(h->qmax);
  w.val<int32_t>(h->qoi_ready ? 1 : 0);
  w.val<int32_t>(M.seq_len);
  for (int l = 0; l < h->nlev; l++) {
    w.val<int32_t>(M.bl[l]);
    w.val<int32_t>(M.exact[l]);
  }
  for (int l = 0; l < h->nlev; l++)
    for (int g = 0; g < h->ngroups; g++) {
      const GroupMeta& G = M.grp[l][g];
      w.val<uint64_t>(G.stored_len);
      w.val<int32_t>(G.method);
      w.val<int32_t>(0);
      w.val<uint64_t>(G.est_H);
      w.val<uint64_t>(G.est_R);
    }
  w.put(M.seq, M.seq_len);
  w.pad(8);
  for (int i = 0; i <= M.seq_len; i++) w.val<uint64_t>(M.E_hi[i]);
  for (int i = 0; i <= M.seq_len; i++) w.val<uint64_t>(M.E_lo[i]);
  w.pad(16);
  if (pos) pos->clear();
  for (int l = 0; l < h->nlev; l++)
    for (int g = 0; g < h->ngroups; g++) {
      const GroupMeta& G = M.grp[l][g];
      if (pos) pos->push_back({w.n, G.stored_len});
      w.n += G.stored_len;  // the group's bytes are copied by the caller
      w.pad(16);
    }
  return w.n;
}

// largest export stream of a handle of this plan: header + every group stored
// directly (a coded group is kept only when smaller) + alignment
static uint64_t export_bound(const Plan& P) {
  const uint64_t groups = (uint64_t)P.nlev * P.ngroups;
  return 4096 + 8ull * P.nlev + 32 * groups + 17ull * (HP_SEQ_MAX + 1) + P.plane_bytes +
         16 * groups;
}

extern "C" hpmdr_status hpmdr_handle_export(const hpmdr_handle* h, void* buf, uint64_t* len) {
  if (!h || !len) return HPMDR_ERR_ARG;
  std::vector<std::pair<uint64_t, uint64_t>> pos;
  const uint64_t n = export_layout(h, nullptr, &pos);
  if (!buf) {
    *len = n;
    return HPMDR_OK;
  }
  if (*len < n) return HPMDR_ERR_ARG;
  export_layout(h, (uint8_t*)buf, nullptr);
  size_t k = 0;
  for (int l = 0; l < h->nlev; l++)
    for (int g = 0; g < h->ngroups; g++, k++) {
      uint8_t* dst = (uint8_t*)buf + pos[k].first;
      HP_CUDA(cudaMemcpy(dst, group_src(h, l, g), pos[k].second, cudaMemcpyDeviceToHost));
    }
  *len = n;
  return HPMDR_OK;
}

// A handle from an export stream: header parsed on the host, device buffers
// allocated and the stored groups and metadata copied on stream s (not waited
// for: buf must stay valid until s passes the copies).
static hpmdr_status import_enqueue(hpmdr_ctx* ctx, const void* buf, uint64_t len,
                                   const std::shared_ptr<const Plan>* plan, cudaStream_t s,
                                   std::unique_ptr<hpmdr_handle>& out) {
  Reader r{(const uint8_t*)buf, len};
  char magic[8];
  r.get(magic, 8);
  if (!r.ok || memcmp(magic, "HPMDR1\0\0", 8) != 0) return HPMDR_ERR_CORRUPT;
  if (r.val<uint32_t>() != 1) return HPMDR_ERR_CORRUPT;
  r.val<uint32_t>();
  const int32_t dtype = r.val<int32_t>(), B = r.val<int32_t>();
  const int nlev = r.val<int32_t>();
  const int32_t ngroups = r.val<int32_t>();
  if (!r.ok || (dtype != 0 && dtype != 1) || B != (dtype ? 64 : 32) || ngroups != B / 4)
    return HPMDR_ERR_CORRUPT;
  const int32_t E_f = r.val<int32_t>(), input_exact = r.val<int32_t>();
  uint64_t dims[3], N = 0;
  for (int d = 0; d < 3; d++) dims[d] = r.val<uint64_t>();
  if (!r.ok || check_dims(3, dims, dims, &N) != HPMDR_OK) return HPMDR_ERR_CORRUPT;
  std::unique_ptr<hpmdr_handle> H;
  if (plan && *plan) {
    const uint64_t* pd = (*plan)->dims;
    if (pd[0] != dims[0] || pd[1] != dims[1] || pd[2] != dims[2] || (*plan)->B != B) plan = nullptr;
  }
  HP_TRY(new_handle(ctx, 3, dims, dtype, plan, H));
  if (H->nlev != nlev || nlev > HP_MAX_LEVELS) return HPMDR_ERR_CORRUPT;
  FieldMeta& M = *H->meta;
  M.E_f = E_f;
  M.input_exact = input_exact;
  M.maxabs = r.val<double>();
  M.vmin = r.val<double>();
  M.vmax = r.val<double>();
  M.range = r.val<double>();
  H->qmin = r.val<float>();
  H->qmax = r.val<float>();
  H->qoi_ready = r.val<int32_t>() != 0;
  M.seq_len = r.val<int32_t>();
  if (M.seq_len < 0 || M.seq_len > HP_SEQ_MAX) return HPMDR_ERR_CORRUPT;
  for (int l = 0; l < nlev; l++) {
    M.bl[l] = r.val<int32_t>();
    M.exact[l] = r.val<int32_t>();
  }
  // the plan's group geometry stays; coded groups get slots of their exact size
  uint64_t slot = 0;
  for (int l = 0; l < nlev; l++)
    for (int g = 0; g < H->ngroups; g++) {
      GroupMeta& G = M.grp[l][g];
      G.stored_len = r.val<uint64_t>();
      G.method = r.val<int32_t>();
      r.val<int32_t>();
      G.est_H = r.val<uint64_t>();
      G.est_R = r.val<uint64_t>();
      if (G.method < 0 || G.method > 2 || (G.method == HPMDR_DC && G.stored_len != G.S))
        return HPMDR_ERR_CORRUPT;
      if (G.method != HPMDR_DC) {
        G.cap = round16(G.stored_len);
        G.slot_off = slot;
        slot += G.cap;
      } else {
        G.cap = 0;
        G.slot_off = 0;
      }
    }
  H->slot_bytes = slot;
  r.get(M.seq, M.seq_len);
  r.pad(8);
  for (int i = 0; i <= M.seq_len; i++) M.E_hi[i] = r.val<uint64_t>();
  for (int i = 0; i <= M.seq_len; i++) M.E_lo[i] = r.val<uint64_t>();
  for (int i = 0; i < M.seq_len; i++)
    if (M.seq[i] >= nlev) return HPMDR_ERR_CORRUPT;
  r.pad(16);
  if (!r.ok) return HPMDR_ERR_CORRUPT;
  HP_TRY(H->A.alloc((void**)&H->d_planes, H->plane_bytes, s));
  HP_TRY(H->A.alloc((void**)&H->d_slots, H->slot_bytes, s));
  HP_TRY(H->A.alloc((void**)&H->d_meta, sizeof(FieldMeta), s));
  CopyRuns runs;
  for (int l = 0; l < nlev; l++)
    for (int g = 0; g < H->ngroups; g++) {
      const GroupMeta& G = M.grp[l][g];
      if (r.n + G.stored_len > len) return HPMDR_ERR_CORRUPT;
      uint8_t* dst = G.method == HPMDR_DC ? H->d_planes + G.plane_off : H->d_slots + G.slot_off;
      if (G.stored_len) runs.add(dst, r.p + r.n, G.stored_len);
      r.n += G.stored_len;
      r.pad(16);
    }
  HP_TRY(runs.issue(cudaMemcpyHostToDevice, s));
  HP_CUDA(cudaMemcpyAsync(H->d_meta, H->meta.get(), sizeof(FieldMeta), cudaMemcpyHostToDevice, s));
  count_items(H.get());
  out = std::move(H);
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_handle_import(hpmdr_ctx* ctx, const void* buf, uint64_t len,
                                            hpmdr_handle** out) {
  if (!ctx || !buf || !out) return HPMDR_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<hpmdr_handle> H;
  HP_TRY(import_enqueue(ctx, buf, len, nullptr, ctx->stream, H));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  *out = H.release();
  return HPMDR_OK;
}

// ------------------------------------------- out-of-core pipeline (Sec. 5.3)
// Units u = v * nchunks + c ((variable, chunk) pairs) pass through three
// queues, one CUDA stream each: host -> device copies (q1), kernels (q2) and
// device -> host copies (q3).  Two device input/output buffers alternate, so
// unit u + 1's copy in and unit u - 1's copy out overlap unit u's kernels; the
// host reads a unit's metadata (to lay out its stream) while the GPU works on
// the next one.
struct UnitEvents {
  std::vector<cudaEvent_t> ev;
  ~UnitEvents() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  hpmdr_status make(size_t n) {
    ev.assign(n, nullptr);
    for (auto& e : ev) HP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return HPMDR_OK;
  }
};

static hpmdr_status pipeline_units(ChunkGrid& G, int nvars, int ndims, const uint64_t dims[3],
                                   const uint64_t chunk[3], uint64_t* U) {
  if (nvars < 1 || nvars > 4096) return HPMDR_ERR_ARG;
  HP_TRY(chunk_grid(ndims, dims, chunk, &G));
  *U = (uint64_t)nvars * G.n;
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_refactor_pipeline(hpmdr_ctx* ctx, int nvars,
                                                const void* const* fields, int ndims,
                                                const uint64_t dims[3], const uint64_t chunk[3],
                                                hpmdr_dtype dtype, int queues, void* out,
                                                uint64_t* total, uint64_t* offsets,
                                                uint64_t* sizes) {
  if (!ctx || !total || (dtype != HPMDR_F32 && dtype != HPMDR_F64) || (queues != 1 && queues != 3))
    return HPMDR_ERR_ARG;
  ChunkGrid G;
  uint64_t U = 0;
  HP_TRY(pipeline_units(G, nvars, ndims, dims, chunk, &U));
  const size_t esz = dtype == HPMDR_F32 ? 4 : 8;
  // stream bound: per unit, the largest stream of its chunk shape
  std::vector<uint64_t> bound(G.n);
  {
    std::shared_ptr<const Plan> full;
    for (uint64_t c = 0; c < G.n; c++) {
      uint64_t org[3], ext[3];
      G.box(c, org, ext);
      std::unique_ptr<hpmdr_handle> H;
      HP_TRY(new_handle(ctx, 3, ext, dtype, nullptr, H));
      bound[c] = round16(export_bound(*H->plan));
    }
  }
  uint64_t need = 0;
  for (uint64_t u = 0; u < U; u++) need += bound[u % G.n];
  if (!out) {
    *total = need;
    return HPMDR_OK;
  }
  if (!fields || !offsets || !sizes || *total < need || ((uintptr_t)out & 15)) return HPMDR_ERR_ARG;
  for (int v = 0; v < nvars; v++)
    if (!fields[v]) return HPMDR_ERR_ARG;
  std::vector<cudaStream_t> q;
  HP_TRY(pipeline_streams(ctx, queues, q));
  if (queues == 1) q.assign(3, q[0]);  // one queue: nothing overlaps (the baseline)
  const size_t in_bytes = G.chunk[0] * G.chunk[1] * G.chunk[2] * esz;
  void* in[2] = {nullptr, nullptr};
  FieldMeta* pm = nullptr;  // page-locked metadata copies, one per unit in flight
  UnitEvents eH, eC, eD;
  hpmdr_status st = eH.make(U);
  if (st == HPMDR_OK) st = eC.make(U);
  if (st == HPMDR_OK) st = eD.make(U);
  for (int i = 0; i < 2 && st == HPMDR_OK; i++) st = ctx->A.alloc(&in[i], in_bytes, q[1]);
  if (st == HPMDR_OK && cudaHostAlloc((void**)&pm, 3 * sizeof(FieldMeta), cudaHostAllocDefault) !=
                            cudaSuccess) {
    pm = nullptr;
    st = HPMDR_ERR_NOMEM;
  }
  std::vector<std::unique_ptr<hpmdr_handle>> hs(U);
  std::vector<RefactorProf> rps(U);
  std::shared_ptr<const Plan> full_plan;
  uint64_t at = 0;  // next free byte of out
  // unit w's metadata is on the host: lay out its stream, copy its groups out
  auto finish = [&](uint64_t w) -> hpmdr_status {
    HP_CUDA(cudaEventSynchronize(eC.ev[w]));
    hpmdr_handle* H = hs[w].get();
    memcpy(H->meta.get(), &pm[w % 3], sizeof(FieldMeta));
    count_items(H);
    if (H->meta->status) return (hpmdr_status)H->meta->status;
    std::vector<std::pair<uint64_t, uint64_t>> pos;
    uint8_t* dst = (uint8_t*)out + at;
    const uint64_t n = export_layout(H, dst, &pos);
    HP_CUDA(cudaStreamWaitEvent(q[2], eC.ev[w], 0));
    CopyRuns runs;
    size_t k = 0;
    for (int l = 0; l < H->nlev; l++)
      for (int g = 0; g < H->ngroups; g++, k++)
        if (pos[k].second) runs.add(dst + pos[k].first, group_src(H, l, g), pos[k].second);
    HP_TRY(runs.issue(cudaMemcpyDeviceToHost, q[2]));
    HP_CUDA(cudaEventRecord(eD.ev[w], q[2]));
    offsets[w] = at;
    sizes[w] = n;
    at += round16(n);
    H->stream = q[2];  // its buffers are released after its copies out
    hs[w].reset();
    return HPMDR_OK;
  };
  for (uint64_t u = 0; u < U && st == HPMDR_OK; u++) {
    const int v = (int)(u / G.n);
    const uint64_t c = u % G.n;
    uint64_t org[3], ext[3];
    G.box(c, org, ext);
    void* buf = in[u % 2];
    // q1: the input buffer is free once unit u - 2's kernels are done
    if (u >= 2 && (st = cudaStreamWaitEvent(q[0], eC.ev[u - 2], 0) ? HPMDR_ERR_CUDA : HPMDR_OK))
      break;
    if ((st = copy_box(buf, fields[v], G, org, ext, esz, true, cudaMemcpyHostToDevice, q[0])))
      break;
    if (cudaEventRecord(eH.ev[u], q[0]) != cudaSuccess) { st = HPMDR_ERR_CUDA; break; }
    // q2: the kernels, then the metadata to the host
    const bool fullc = ext[0] == G.chunk[0] && ext[1] == G.chunk[1] && ext[2] == G.chunk[2];
    if ((st = new_handle(ctx, 3, ext, dtype, fullc && full_plan ? &full_plan : nullptr, hs[u])))
      break;
    if (fullc && !full_plan) full_plan = hs[u]->plan;
    if (cudaStreamWaitEvent(q[1], eH.ev[u], 0) != cudaSuccess) { st = HPMDR_ERR_CUDA; break; }
    if ((st = refactor_enqueue(ctx, hs[u].get(), buf, q[1], &rps[u]))) break;
    if (cudaMemcpyAsync(&pm[u % 3], hs[u]->d_meta, sizeof(FieldMeta), cudaMemcpyDeviceToHost,
                        q[1]) != cudaSuccess ||
        cudaEventRecord(eC.ev[u], q[1]) != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    // host: unit u - 1 (its kernels overlap unit u's copy in)
    if (u >= 1) st = finish(u - 1);
  }
  if (st == HPMDR_OK && U >= 1) st = finish(U - 1);
  hpmdr_status js = join_streams(q);
  hs.clear();
  for (int i = 0; i < 2; i++) ctx->A.release(in[i], q[1]);
  join_streams(q);
  if (pm) cudaFreeHost(pm);
  if (st != HPMDR_OK) return st;
  *total = at;
  return js;
}

extern "C" hpmdr_status hpmdr_retrieve_pipeline(hpmdr_ctx* ctx, int nvars, const void* streams,
                                                const uint64_t* offsets, const uint64_t* sizes,
                                                int ndims, const uint64_t dims[3],
                                                const uint64_t chunk[3], const double* rel_bounds,
                                                int queues, void* const* outs,
                                                hpmdr_retrieve_info* infos) {
  if (!ctx || !streams || !offsets || !sizes || !rel_bounds || !outs || (queues != 1 && queues != 3))
    return HPMDR_ERR_ARG;
  ChunkGrid G;
  uint64_t U = 0;
  HP_TRY(pipeline_units(G, nvars, ndims, dims, chunk, &U));
  for (int v = 0; v < nvars; v++)
    if (!outs[v] || !(rel_bounds[v] >= 0.0)) return HPMDR_ERR_ARG;
  const uint8_t* base = (const uint8_t*)streams;
  // the global range of each variable, from the streams' headers (Sec. 5.3's
  // sub-domains meet the bound relative to the whole variable)
  std::vector<double> lo(nvars, 0.0), hi(nvars, 0.0);
  int dtype = -1;
  for (uint64_t u = 0; u < U; u++) {
    Reader r{base + offsets[u], sizes[u]};
    char magic[8];
    r.get(magic, 8);
    r.val<uint32_t>();
    r.val<uint32_t>();
    const int32_t dt = r.val<int32_t>();
    for (int k = 0; k < 5; k++) r.val<int32_t>();
    for (int d = 0; d < 3; d++) r.val<uint64_t>();
    r.val<double>();
    const double vmin = r.val<double>(), vmax = r.val<double>();
    if (!r.ok || memcmp(magic, "HPMDR1\0\0", 8) != 0 || (dtype >= 0 && dt != dtype))
      return HPMDR_ERR_CORRUPT;
    dtype = dt;
    const int v = (int)(u / G.n);
    if (u % G.n == 0 || vmin < lo[v]) lo[v] = vmin;
    if (u % G.n == 0 || vmax > hi[v]) hi[v] = vmax;
  }
  const size_t esz = dtype == 0 ? 4 : 8;
  std::vector<cudaStream_t> q;
  HP_TRY(pipeline_streams(ctx, queues, q));
  if (queues == 1) q.assign(3, q[0]);  // one queue: nothing overlaps (the baseline)
  const size_t box_bytes = G.chunk[0] * G.chunk[1] * G.chunk[2] * esz;
  void* ob[2] = {nullptr, nullptr};
  RetrieveDev* prd = nullptr;  // page-locked selection records, one per unit
  UnitEvents eH, eC, eD;
  hpmdr_status st = eH.make(U);
  if (st == HPMDR_OK) st = eC.make(U);
  if (st == HPMDR_OK) st = eD.make(U);
  for (int i = 0; i < 2 && st == HPMDR_OK; i++) st = ctx->A.alloc(&ob[i], box_bytes, q[1]);
  if (st == HPMDR_OK &&
      cudaHostAlloc((void**)&prd, U * sizeof(RetrieveDev), cudaHostAllocDefault) != cudaSuccess) {
    prd = nullptr;
    st = HPMDR_ERR_NOMEM;
  }
  std::vector<std::unique_ptr<hpmdr_handle>> hs(U);
  std::shared_ptr<const Plan> full_plan;
  for (uint64_t u = 0; u < U && st == HPMDR_OK; u++) {
    const int v = (int)(u / G.n);
    const uint64_t c = u % G.n;
    uint64_t org[3], ext[3];
    G.box(c, org, ext);
    // q1: unit u's stream in (at most two units' handles on the device)
    if (u >= 2 && cudaStreamWaitEvent(q[0], eC.ev[u - 2], 0) != cudaSuccess) { st = HPMDR_ERR_CUDA; break; }
    if ((st = import_enqueue(ctx, base + offsets[u], sizes[u], full_plan ? &full_plan : nullptr,
                             q[0], hs[u])))
      break;
    const bool fullc = ext[0] == G.chunk[0] && ext[1] == G.chunk[1] && ext[2] == G.chunk[2];
    for (int d = 0; d < 3; d++)
      if (hs[u]->dims[d] != ext[d]) st = HPMDR_ERR_CORRUPT;
    if (st != HPMDR_OK) break;
    if (fullc && !full_plan) full_plan = hs[u]->plan;
    if (cudaEventRecord(eH.ev[u], q[0]) != cudaSuccess) { st = HPMDR_ERR_CUDA; break; }
    // q2: select, decode, recompose into the free output buffer
    if (cudaStreamWaitEvent(q[1], eH.ev[u], 0) != cudaSuccess ||
        (u >= 2 && cudaStreamWaitEvent(q[1], eD.ev[u - 2], 0) != cudaSuccess)) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    hpmdr_handle* H = hs[u].get();
    if ((st = enqueue_retrieve(ctx, H, rel_bounds[v] * (hi[v] - lo[v]), 1, ob[u % 2], q[1])))
      break;
    if (cudaMemcpyAsync(&prd[u], H->d_rd, sizeof(RetrieveDev), cudaMemcpyDeviceToHost, q[1]) !=
            cudaSuccess ||
        cudaEventRecord(eC.ev[u], q[1]) != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    // q3: the box out
    if (cudaStreamWaitEvent(q[2], eC.ev[u], 0) != cudaSuccess) { st = HPMDR_ERR_CUDA; break; }
    if ((st = copy_box(outs[v], ob[u % 2], G, org, ext, esz, false, cudaMemcpyDeviceToHost, q[2])))
      break;
    if (cudaEventRecord(eD.ev[u], q[2]) != cudaSuccess) { st = HPMDR_ERR_CUDA; break; }
    H->stream = q[1];
    // unit u's device buffers go back to the pool once its kernels are done
    // (the host object stays for the infos)
    for (void** pp : {(void**)&H->d_planes, (void**)&H->d_slots, (void**)&H->d_meta,
                      (void**)&H->d_rd, (void**)&H->d_xa, (void**)&H->d_xb, (void**)&H->d_xroot}) {
      H->A.release(*pp, q[1]);
      *pp = nullptr;
    }
  }
  hpmdr_status js = join_streams(q);
  hpmdr_status worst = HPMDR_OK;
  if (st == HPMDR_OK && js == HPMDR_OK) {
    for (uint64_t u = 0; u < U; u++) {
      hpmdr_status r = (hpmdr_status)prd[u].status;
      fill_info(hs[u].get(), prd[u], infos ? &infos[u] : nullptr);
      if (r != HPMDR_OK && worst == HPMDR_OK) worst = r;
    }
  }
  hs.clear();
  for (int i = 0; i < 2; i++) ctx->A.release(ob[i], q[1]);
  join_streams(q);
  if (prd) cudaFreeHost(prd);
  if (st != HPMDR_OK) return st;
  if (js != HPMDR_OK) return js;
  return worst;
}

__global__ void k_reset(FieldMeta* m) {
  hp::pdl_enter();
  for (int l = 0; l < HP_MAX_LEVELS; l++) {
    m->fetched[l] = 0;
    m->cur[l] = 0;
  }
}

extern "C" hpmdr_status hpmdr_handle_reset(hpmdr_ctx* ctx, hpmdr_handle* h, int poison) {
  if (!ctx || !h) return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  hp::note_launch(), hp::launch_pdl(k_reset, 1, 1, 0, s, h->d_meta);
  if (poison && h->d_planes)
    for (int l = 0; l < h->nlev; l++)
      for (int g = 0; g < h->ngroups; g++) {
        const GroupMeta& G = h->meta->grp[l][g];
        if (G.method != HPMDR_DC || h->compact)
          HP_CUDA(cudaMemsetAsync(h->d_planes + G.plane_off, 0xA5, G.S, s));
      }
  HP_CUDA(cudaStreamSynchronize(s));
  return HPMDR_OK;
}

// Packs every group's stored bytes (DC groups included) into one slot buffer
// and releases the plane buffer: the handle then holds only its compressed
// streams, and the planes become a cache that the next retrieval allocates
// and fills by decoding (DC groups by copying).
extern "C" hpmdr_status hpmdr_handle_compact(hpmdr_ctx* ctx, hpmdr_handle* h) {
  if (!ctx || !h) return HPMDR_ERR_ARG;
  if (h->compact) return HPMDR_OK;
  if (!h->d_planes) return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  FieldMeta& M = *h->meta;
  std::vector<uint64_t> off((size_t)h->nlev * h->ngroups);
  uint64_t total = 0;
  for (int l = 0; l < h->nlev; l++)
    for (int g = 0; g < h->ngroups; g++) {
      off[(size_t)l * h->ngroups + g] = total;
      total += round16(M.grp[l][g].stored_len);
    }
  uint8_t* slots = nullptr;
  HP_TRY(h->A.alloc((void**)&slots, total, s));
  for (int l = 0; l < h->nlev; l++)
    for (int g = 0; g < h->ngroups; g++)
      if (cudaMemcpyAsync(slots + off[(size_t)l * h->ngroups + g], group_src(h, l, g),
                          M.grp[l][g].stored_len, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        h->A.release(slots, s);
        cudaStreamSynchronize(s);
        g_last_error = "compaction copy failed";
        return HPMDR_ERR_CUDA;
      }
  for (int l = 0; l < h->nlev; l++)
    for (int g = 0; g < h->ngroups; g++) {
      GroupMeta& G = M.grp[l][g];
      G.slot_off = off[(size_t)l * h->ngroups + g];
      G.cap = round16(G.stored_len);
    }
  M.compact = 1;
  for (int l = 0; l < HP_MAX_LEVELS; l++) M.fetched[l] = M.cur[l] = 0;
  HP_CUDA(cudaMemcpyAsync(h->d_meta, h->meta.get(), sizeof(FieldMeta), cudaMemcpyHostToDevice, s));
  h->A.release(h->d_slots, s);
  h->d_slots = slots;
  h->slot_bytes = total;
  h->release_cache(s);
  h->compact = true;
  count_items(h);
  HP_CUDA(cudaStreamSynchronize(s));
  return HPMDR_OK;
}

// Releases the plane cache of a handle (compacting it first if needed); the
// next retrieval decodes every group it uses again.
extern "C" hpmdr_status hpmdr_handle_drop_cache(hpmdr_ctx* ctx, hpmdr_handle* h) {
  if (!ctx || !h) return HPMDR_ERR_ARG;
  if (!h->compact) return hpmdr_handle_compact(ctx, h);
  if (!h->d_planes) return HPMDR_OK;
  const cudaStream_t s = ctx->stream;
  hp::note_launch(), hp::launch_pdl(k_reset, 1, 1, 0, s, h->d_meta);
  h->release_cache(s);
  HP_CUDA(cudaGetLastError());
  return HPMDR_OK;
}

static uint64_t cache_scratch_bytes(const hpmdr_handle* h) {
  const int L = h->nlev - 1;
  uint64_t b = h->plan->gstage_max * (h->B / 8 + 1);
  if (L >= 2) {
    const LevelDesc& D = h->levels[L];
    b += 8ull * D.gc[0] * D.gc[1] * D.gc[2];
  }
  if (L >= 3) {
    const LevelDesc& D = h->levels[L - 1];
    b += 8ull * D.gc[0] * D.gc[1] * D.gc[2];
  }
  return b;
}

extern "C" hpmdr_status hpmdr_handle_memory(const hpmdr_handle* h, uint64_t* resident,
                                            uint64_t* cache, uint64_t* cache_max) {
  if (!h) return HPMDR_ERR_ARG;
  const uint64_t fixed = h->slot_bytes + sizeof(FieldMeta) + sizeof(RetrieveDev) + 8;
  const uint64_t scratch = cache_scratch_bytes(h);
  if (resident) *resident = fixed + (h->compact ? 0 : h->plane_bytes);
  if (cache)
    *cache = (h->compact && h->d_planes ? h->plane_bytes : 0) + (h->d_xa ? 8 * h->xa_elems : 0) +
             (h->d_xb ? 8 * h->xb_elems : 0);
  if (cache_max) *cache_max = (h->compact ? h->plane_bytes : 0) + scratch;
  return HPMDR_OK;
}

extern "C" void hpmdr_handle_free(hpmdr_handle* h) { delete h; }

// --------------------------------------------------------- stage entry points
extern "C" hpmdr_status hpmdr_bitplane_encode(const void* q, const uint8_t* sign, uint64_t n, int B,
                                              uint32_t* planes, void* stream) {
  if (!q || !sign || !planes || n == 0 || n >= 0xffffffffull || (B != 32 && B != 64))
    return HPMDR_ERR_ARG;
  launch_bitplane_encode(q, sign, n, B, planes, (cudaStream_t)stream);
  HP_CUDA(cudaGetLastError());
  HP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_bitplane_decode(const uint32_t* planes, uint64_t n, int B, int k,
                                              void* q_out, uint8_t* sign_out, void* stream) {
  if (!planes || !q_out || !sign_out || n == 0 || n >= 0xffffffffull || (B != 32 && B != 64) ||
      k < 0 || k > B)
    return HPMDR_ERR_ARG;
  launch_bitplane_decode(planes, n, B, k, q_out, sign_out, (cudaStream_t)stream);
  HP_CUDA(cudaGetLastError());
  HP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_bitplane_encode_design(const uint32_t* q, const uint8_t* sign,
                                                     uint64_t n, int design, uint32_t* planes,
                                                     void* stream) {
  if (!q || !sign || !planes || n == 0 || n >= 0xffffff00ull || design < 0 || design > 5 ||
      ((uintptr_t)q & 15) || ((uintptr_t)planes & 15))
    return HPMDR_ERR_ARG;
  launch_bpd_encode(q, sign, n, design, planes, (cudaStream_t)stream);
  HP_CUDA(cudaGetLastError());
  HP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_bitplane_decode_design(const uint32_t* planes, uint64_t n, int design,
                                                     int k, uint32_t* q_out, uint8_t* sign_out,
                                                     void* stream) {
  if (!planes || !q_out || !sign_out || n == 0 || n >= 0xffffff00ull || design < 0 || design > 5 ||
      k < 0 || k > 32 || ((uintptr_t)q_out & 15) || ((uintptr_t)planes & 15))
    return HPMDR_ERR_ARG;
  launch_bpd_decode(planes, n, design, k, q_out, sign_out, (cudaStream_t)stream);
  HP_CUDA(cudaGetLastError());
  HP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return HPMDR_OK;
}

// one group as a one-level, one-group "field" through the same kernels
extern "C" hpmdr_status hpmdr_encode_group(hpmdr_ctx* ctx, const uint8_t* G, uint64_t S, int force,
                                           uint8_t* out, uint64_t cap, uint64_t* len, int* method) {
  if (!ctx || !G || !out || !len || S == 0 || S >= 0xffffffffull || force < -1 || force > 2)
    return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  std::unique_ptr<FieldMeta> M(new FieldMeta());
  memset(M.get(), 0, sizeof(FieldMeta));
  M->nlev = 1;
  M->ngroups = 1;
  GroupMeta& gm = M->grp[0][0];
  gm.S = S;
  gm.nchunks = (uint32_t)((S + HP_CHUNK - 1) / HP_CHUNK);
  gm.chunk0 = 0;
  gm.cap = cap;
  gm.slot_off = 0;
  gm.plane_off = 0;
  const uint32_t nc = gm.nchunks;
  std::vector<uint32_t> cg(nc, 0u);
  FieldMeta* d_meta = nullptr;
  uint8_t *d_G = nullptr, *d_lens = nullptr;
  uint32_t *d_cg = nullptr, *d_hist = nullptr, *d_cost = nullptr, *d_words = nullptr,
           *d_off = nullptr;
  unsigned long long* d_gcost = nullptr;
  hpmdr_status st = HPMDR_OK;
  do {
    if ((st = ctx->A.alloc((void**)&d_meta, sizeof(FieldMeta), s))) break;
    if ((st = ctx->A.alloc((void**)&d_G, round16(S), s))) break;
    if ((st = ctx->A.alloc((void**)&d_lens, 256, s))) break;
    if ((st = ctx->A.alloc((void**)&d_cg, 4ull * nc, s))) break;
    if ((st = ctx->A.alloc((void**)&d_hist, 1024ull, s))) break;
    if ((st = ctx->A.alloc((void**)&d_gcost, 8ull, s))) break;
    if (cudaMemsetAsync(d_hist, 0, 1024ull, s) != cudaSuccess ||
        cudaMemsetAsync(d_gcost, 0, 8ull, s) != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    if ((st = ctx->A.alloc((void**)&d_cost, 4ull * nc, s))) break;
    if ((st = ctx->A.alloc((void**)&d_words, 4ull * nc, s))) break;
    if ((st = ctx->A.alloc((void**)&d_off, 4ull * nc, s))) break;
    if (cudaMemcpyAsync(d_G, G, S, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_meta, M.get(), sizeof(FieldMeta), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_cg, cg.data(), 4ull * nc, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    ChunkMap cm{d_cg, nc};
    launch_chunk_stats(d_G, d_meta, cm, d_hist, d_gcost, d_cost, s);
    launch_decide(d_meta, 1, d_hist, d_gcost, d_lens, ctx->Ts, ctx->cr_num, ctx->cr_den, force, s);
    launch_huff_bits(d_G, d_meta, cm, d_lens, d_words, s);
    launch_group_offsets(d_meta, 1, d_words, d_cost, d_off, s);
    launch_huff_encode(d_G, d_meta, cm, d_lens, d_off, out, s);
    launch_rle_encode(d_G, d_meta, cm, d_off, out, s);
    launch_headers(d_meta, 1, d_lens, d_off, out, s);
    if (cudaMemcpyAsync(M.get(), d_meta, sizeof(FieldMeta), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    *len = M->grp[0][0].stored_len;
    if (method) *method = M->grp[0][0].method;
    if (M->status) {
      st = HPMDR_ERR_ARG;  // the coded bytes did not fit in cap
      break;
    }
    if (M->grp[0][0].method == HPMDR_DC) {
      if (cap < S) {
        st = HPMDR_ERR_ARG;
        break;
      }
      if (cudaMemcpyAsync(out, G, S, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        st = HPMDR_ERR_CUDA;
    }
  } while (0);
  ctx->A.release(d_meta, s);
  ctx->A.release(d_G, s);
  ctx->A.release(d_lens, s);
  ctx->A.release(d_cg, s);
  ctx->A.release(d_hist, s);
  ctx->A.release(d_gcost, s);
  ctx->A.release(d_cost, s);
  ctx->A.release(d_words, s);
  ctx->A.release(d_off, s);
  cudaStreamSynchronize(s);
  return st;
}

extern "C" hpmdr_status hpmdr_fixed_to_float(hpmdr_ctx* ctx, const int64_t* X, uint64_t n,
                                             int E_f, hpmdr_dtype dtype, void* out) {
  if (!ctx || (n && (!X || !out)) || (dtype != HPMDR_F32 && dtype != HPMDR_F64)) return HPMDR_ERR_ARG;
  if (dtype == HPMDR_F32 ? (E_f < -148 || E_f > 128) : (E_f < -1073 || E_f > 1024))
    return HPMDR_ERR_ARG;
  launch_convert_fixed(X, n, E_f, (int)dtype, out, ctx->stream);
  HP_CUDA(cudaGetLastError());
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_qoi_vtotal_bound(hpmdr_ctx* ctx, const float* vx, const float* vy,
                                               const float* vz, uint64_t n, const double e[3],
                                               float* out, double* bound, uint64_t* point) {
  if (!ctx || !n || !vx || !vy || !vz || !e || !out || !bound || !point) return HPMDR_ERR_ARG;
  for (int i = 0; i < 3; i++)
    if (!(e[i] >= 0.0)) return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  unsigned long long* d_best = nullptr;
  HP_TRY(ctx->A.alloc((void**)&d_best, vtotal_bound_scratch(n), s));
  double* d_e = vtotal_bound_e(d_best, n);
  const double* const ep[3] = {d_e, d_e + 1, d_e + 2};
  unsigned long long best[2] = {0, 0};
  hpmdr_status st = HPMDR_OK;
  if (cudaMemcpyAsync(d_e, e, 24, cudaMemcpyHostToDevice, s) != cudaSuccess) st = HPMDR_ERR_CUDA;
  if (st == HPMDR_OK) launch_vtotal_bound(vx, vy, vz, n, ep, out, d_best, s);
  if (st != HPMDR_OK || cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(best, d_best, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    st = HPMDR_ERR_CUDA;
  ctx->A.release(d_best, s);
  if (st) return st;
  memcpy(bound, &best[0], 8);
  *point = best[1];
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_decode_group(hpmdr_ctx* ctx, const uint8_t* in, uint64_t len,
                                           int method, uint8_t* G, uint64_t S) {
  if (!ctx || !in || !G || S == 0 || S >= 0xffffffffull || method < 0 || method > 2)
    return HPMDR_ERR_ARG;
  const cudaStream_t s = ctx->stream;
  if (method == HPMDR_DC) {
    if (len != S) return HPMDR_ERR_CORRUPT;
    HP_CUDA(cudaMemcpyAsync(G, in, S, cudaMemcpyDeviceToDevice, s));
    HP_CUDA(cudaStreamSynchronize(s));
    return HPMDR_OK;
  }
  std::unique_ptr<FieldMeta> M(new FieldMeta());
  memset(M.get(), 0, sizeof(FieldMeta));
  M->nlev = 1;
  M->ngroups = 1;
  GroupMeta& gm = M->grp[0][0];
  gm.S = S;
  gm.nchunks = (uint32_t)((S + HP_CHUNK - 1) / HP_CHUNK);
  gm.stored_len = len;
  gm.method = method;
  std::unique_ptr<RetrieveDev> rd(new RetrieveDev());
  memset(rd.get(), 0, sizeof(RetrieveDev));
  rd->n_new = 1;
  rd->new_gi[0] = 0;
  rd->new_pref[0] = 0;
  rd->new_pref[1] = gm.nchunks;
  rd->items = gm.nchunks;
  FieldMeta* d_meta = nullptr;
  RetrieveDev* d_rd = nullptr;
  uint8_t *d_in = nullptr, *d_G = nullptr;
  hpmdr_status st = HPMDR_OK;
  do {
    if ((st = ctx->A.alloc((void**)&d_meta, sizeof(FieldMeta), s))) break;
    if ((st = ctx->A.alloc((void**)&d_rd, sizeof(RetrieveDev), s))) break;
    if ((st = ctx->A.alloc((void**)&d_in, round16(len), s))) break;
    if ((st = ctx->A.alloc((void**)&d_G, round16(S), s))) break;
    if (cudaMemcpyAsync(d_in, in, len, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_meta, M.get(), sizeof(FieldMeta), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_rd, rd.get(), sizeof(RetrieveDev), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    launch_decode(d_in, d_meta, d_rd, gm.nchunks, d_G, s);
    int32_t ms = 0;
    if (cudaMemcpyAsync(&ms, &d_meta->status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(G, d_G, S, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = HPMDR_ERR_CUDA;
      break;
    }
    if (ms) st = (hpmdr_status)ms;
  } while (0);
  ctx->A.release(d_meta, s);
  ctx->A.release(d_rd, s);
  ctx->A.release(d_in, s);
  ctx->A.release(d_G, s);
  cudaStreamSynchronize(s);
  return st;
}

// ----------------------------------------------------------------- profiling
extern "C" uint64_t hpmdr_kernel_launches(void) { return g_launches.load(); }

extern "C" hpmdr_status hpmdr_ctx_profile(hpmdr_ctx* ctx, int enable) {
  if (!ctx) return HPMDR_ERR_ARG;
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->prof.reset();
  ctx->prof.on = enable != 0;
  ctx->prof.mask = ~0ull;
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_ctx_profile_stages(hpmdr_ctx* ctx, uint64_t stage_mask) {
  if (!ctx) return HPMDR_ERR_ARG;
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->prof.reset();
  ctx->prof.on = stage_mask != 0;
  ctx->prof.mask = stage_mask;
  return HPMDR_OK;
}

extern "C" hpmdr_status hpmdr_ctx_profile_entry(hpmdr_ctx* ctx, int index, const char** name,
                                                double* total_ms, uint64_t* launches,
                                                double* bytes) {
  if (!ctx || index < 0) return HPMDR_ERR_ARG;
  if (index >= NSTAGE) return HPMDR_ERR_ARG;
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->prof.resolve();
  if (name) *name = kStageName[index];
  if (total_ms) *total_ms = ctx->prof.ms[index];
  if (launches) *launches = ctx->prof.calls[index];
  if (bytes) *bytes = ctx->prof.bytes[index];
  return HPMDR_OK;
}

// ------------------------------------------------------------------- errors
extern "C" const char* hpmdr_strerror(hpmdr_status s) {
  switch (s) {
    case HPMDR_OK: return "ok";
    case HPMDR_ERR_ARG: return "invalid argument";
    case HPMDR_ERR_NOMEM: return "out of memory";
    case HPMDR_ERR_CUDA: return "CUDA error";
    case HPMDR_ERR_CORRUPT: return "corrupt stored data";
    case HPMDR_ERR_UNATTAINABLE: return "error bound unattainable";
    case HPMDR_ERR_TIMEOUT: return "timeout";
    case HPMDR_ERR_BUSY: return "busy";
    case HPMDR_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

extern "C" const char* hpmdr_last_error(void) { return g_last_error.c_str(); }
