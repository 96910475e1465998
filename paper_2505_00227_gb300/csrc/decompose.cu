// Multilevel decomposition, per-level exponent alignment and the bitplane
// transpose (Sec. 3 decomposer; Sec. 4 Algorithm 1 and its register-block
// design, Sec. 4.3).
//
// Coefficients are exact integers: F = floor(f / U) with U = 2^(E_f-48), and
// for a node of parity type t (odd axes O) at half-stride h the coefficient is
// C8 = (8/k) (k F_i - sum of its k = 2^|O| corner values), the corners being
// the neighbours at +-h along the odd axes (a right neighbour outside the
// grid is replaced by the left one).  Level l's nodes are ordered by type
// t = 1..7, then in raster order.
//
// Work decomposition: one warp owns a tile of 1024 consecutive level-linear
// nodes = 32 words of every bitplane.  Phase A computes the 1024 aligned
// integers with lane = node (consecutive lanes read consecutive x), staging
// them in shared memory; phase B gives lane L the 32 integers of word L, which
// it transposes in registers (register block, no inter-thread exchange) and
// stores as one word per plane, so that every plane store of the warp is a
// coalesced 128-byte line.
#include "dev_common.cuh"

namespace hp {

template <typename T>
struct FieldView {
  const T* __restrict__ f;
  uint32_t ny, nx;
  int E_f;
};

template <typename T>
__device__ __forceinline__ int64_t load_F(const FieldView<T>& v, uint32_t z, uint32_t y, uint32_t x,
                                          uint32_t& fl) {
  return fixed_point(__ldg(v.f + ((size_t)z * v.ny + y) * v.nx + x), v.E_f, fl);
}

// C8 of node j of level L; `fl` collects whether the node's own value lost bits
template <typename T>
__device__ __forceinline__ int64_t level_c8(const FieldView<T>& v, const LevelDesc& L, uint32_t j,
                                            uint32_t& fl) {
  if (L.hlog < 0) return 8 * load_F(v, 0, 0, 0, fl);
  NodePos p = node_pos(L, j);
  const int hl = L.hlog;
  uint32_t ign = 0;
  int64_t Fi = load_F(v, p.gz << hl, p.gy << hl, p.gx << hl, fl);
  uint32_t zs[2] = {p.gz, p.gz}, ys[2] = {p.gy, p.gy}, xs[2] = {p.gx, p.gx};
  int nz = 1, ny = 1, nx = 1;
  if (p.t & 4) { axis_nb(p.gz, L.g[0], zs[0], zs[1]); nz = 2; }
  if (p.t & 2) { axis_nb(p.gy, L.g[1], ys[0], ys[1]); ny = 2; }
  if (p.t & 1) { axis_nb(p.gx, L.g[2], xs[0], xs[1]); nx = 2; }
  int64_t sum = 0;
  for (int a = 0; a < nz; a++)
    for (int b = 0; b < ny; b++)
      for (int c = 0; c < nx; c++) sum += load_F(v, zs[a] << hl, ys[b] << hl, xs[c] << hl, ign);
  const int nodd = __popc(p.t);
  const int64_t D = ((int64_t)1 << nodd) * Fi - sum;
  return D * (int64_t)(8 >> nodd);
}

__device__ __forceinline__ int find_level(const uint32_t* tile0, int l, uint32_t tile) {
  while (tile >= tile0[l + 1]) l++;
  return l;
}

// ------------------------------------------------------------ pass: level max
// one warp: max |C8| over the 1024-node tile at `base` of level L
template <typename T>
__device__ __forceinline__ void levelmax_tile(const FieldView<T>& v, const LevelDesc& L,
                                              uint32_t base, FieldMeta* meta) {
  const int lane = threadIdx.x & 31;
  uint64_t mx = 0;
  uint32_t fl = 0;
#pragma unroll 4
  for (int r = 0; r < 32; r++) {  // unrolled: several rows' loads in flight
    uint32_t j = base + r * 32 + lane;
    if (j < L.n) {
      uint64_t m = umag(level_c8(v, L, j, fl));
      mx = m > mx ? m : mx;
    }
  }
  mx = warp_max_u64(mx);
  unsigned anyfl = __any_sync(HP_FULL, fl != 0);
  if (lane == 0) {
    if (mx) atomicMax((unsigned long long*)&meta->m8[L.level], (unsigned long long)mx);
    if (anyfl) atomicOr(&meta->floored, 1u);
  }
}

// single field: one CTA per tile, each warp 4 of its 32 rows (the generic
// levels left to these kernels are small, so latency, not bandwidth, sets
// their time: a tile's rows are computed side by side)
template <typename T>
__global__ void __launch_bounds__(256) k_levelmax(FieldView<T> v, const LevelDesc* __restrict__ levels,
                                                  int nlev, uint32_t total_tiles,
                                                  const uint32_t* __restrict__ perm, FieldMeta* meta) {
  hp::pdl_enter();
  __shared__ uint32_t s_tile0[HP_MAX_LEVELS + 1];
  for (int l = threadIdx.x; l <= nlev; l += blockDim.x)
    s_tile0[l] = l < nlev ? levels[l].gtile0 : total_tiles;
  __syncthreads();
  if (meta->status) return;
  v.E_f = meta->E_f;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, rpw = 32 / (blockDim.x >> 5);
  int l = 0;
  for (uint32_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
    l = find_level(s_tile0, l, tile);
    const LevelDesc& L = levels[l];
    const uint32_t base = perm[L.tile0 + (tile - L.gtile0)] * HP_TILE;
    uint64_t mx = 0;
    uint32_t fl = 0;
#pragma unroll 4
    for (int rr = 0; rr < rpw; rr++) {
      const uint32_t j = base + (w * rpw + rr) * 32 + lane;
      if (j < L.n) {
        const uint64_t m = umag(level_c8(v, L, j, fl));
        mx = m > mx ? m : mx;
      }
    }
    mx = warp_max_u64(mx);
    const unsigned anyfl = __any_sync(HP_FULL, fl != 0);
    if (lane == 0) {
      if (mx) atomicMax((unsigned long long*)&meta->m8[L.level], (unsigned long long)mx);
      if (anyfl) atomicOr(&meta->floored, 1u);
    }
  }
}

static int sm_count() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

void launch_levelmax(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* levels,
                     int nlev, uint32_t total_tiles, const uint32_t* perm, FieldMeta* meta,
                     cstream s) {
  uint32_t blocks = total_tiles;
  uint32_t cap = (uint32_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  if (dtype == 0) {
    FieldView<float> v{(const float*)f, (uint32_t)dims[1], (uint32_t)dims[2], 0};
    hp::note_launch(), hp::launch_pdl(k_levelmax<float>, blocks, 256, 0, s, v, levels, nlev,
                                      total_tiles, perm, meta);
  } else {
    FieldView<double> v{(const double*)f, (uint32_t)dims[1], (uint32_t)dims[2], 0};
    hp::note_launch(), hp::launch_pdl(k_levelmax<double>, blocks, 256, 0, s, v, levels, nlev,
                                      total_tiles, perm, meta);
  }
}

// bl_l = bit length of max|C8|; input exactness from the floor flags and the
// least set-bit exponent of the fused statistics pass
__device__ __forceinline__ void bitlen_level(FieldMeta* meta, int l) {
  if (l < meta->nlev) meta->bl[l] = meta->m8[l] ? bitlen64(meta->m8[l]) : 0;
  if (l == 0)
    meta->input_exact = (meta->floored || meta->lsb_min < meta->E_f - 48) ? 0 : 1;
}

__global__ void k_bitlen(FieldMeta* meta) {
  hp::pdl_enter();
  bitlen_level(meta, threadIdx.x);
}

void launch_bitlen(FieldMeta* meta, cstream s) {
  hp::note_launch(), hp::launch_pdl(k_bitlen, 1, HP_MAX_LEVELS, 0, s, meta);
}

// ------------------------------------------------- register-block transpose out
// Lane L holds in shared memory (row L, padded to 33 words) the 32 aligned
// integers of word `wi`; it transposes them and writes one word per plane.
// For B = 64 the high and low halves are transposed in turn.
template <int B>
__device__ __forceinline__ void emit_word(const uint32_t* row_hi, const uint32_t* row_lo,
                                          uint32_t sign_word, uint32_t* __restrict__ planes,
                                          uint32_t W, uint32_t wi) {
  uint32_t a[32];
#pragma unroll
  for (int b = 0; b < 32; b++) a[b] = row_hi[b];
  transpose32(a);  // a[c] bit b = bit c of element b
  planes[wi] = sign_word;
#pragma unroll
  for (int p = 0; p < 32; p++) planes[(size_t)(1 + p) * W + wi] = a[31 - p];
  if (B == 64) {
#pragma unroll
    for (int b = 0; b < 32; b++) a[b] = row_lo[b];
    transpose32(a);
#pragma unroll
    for (int p = 0; p < 32; p++) planes[(size_t)(33 + p) * W + wi] = a[31 - p];
  }
}

// ------------------------------------------------ pass: quantize + Algorithm 1
// one warp: the 1024-node tile at `base` of level L, hi/lo its shared rows
template <typename T, int B>
__device__ __forceinline__ void encode_tile(const FieldView<T>& v, const LevelDesc& L,
                                            uint32_t base, FieldMeta* meta,
                                            uint32_t* __restrict__ planes, uint32_t* hi,
                                            uint32_t* lo) {
  const int lane = threadIdx.x & 31;
  const int bl = meta->bl[L.level];
  uint64_t low = 0;
  uint32_t my_sign = 0, fl = 0;
  // phase A: lane = node (unrolled: several rows' loads in flight)
#pragma unroll 4
  for (int r = 0; r < 32; r++) {
    uint32_t j = base + r * 32 + lane;
    uint64_t q = 0;
    bool neg = false;
    if (j < L.n) {
      int64_t c8 = level_c8(v, L, j, fl);
      uint64_t m = umag(c8);
      neg = c8 < 0;
      if (bl == 0) q = 0;
      else if (B >= bl) q = m << (B - bl);
      else {
        q = m >> (bl - B);
        low |= m & ((1ull << (bl - B)) - 1ull);
      }
    }
    uint32_t sw = __ballot_sync(HP_FULL, neg);
    if (lane == r) my_sign = sw;
    if (B == 64) {
      hi[r * 33 + lane] = (uint32_t)(q >> 32);
      lo[r * 33 + lane] = (uint32_t)q;
    } else {
      hi[r * 33 + lane] = (uint32_t)q;
    }
  }
  low = warp_or_u64(low);
  if (lane == 0 && low)
    atomicOr((unsigned long long*)&meta->lowbits[L.level], (unsigned long long)low);
  __syncwarp();
  // phase B: lane = word
  const uint32_t wi = base / 32 + lane;
  if (wi < L.W) emit_word<B>(hi + lane * 33, lo + lane * 33, my_sign, planes + L.plane_off / 4, L.W, wi);
  __syncwarp();
}

// single field: one CTA per tile (as k_levelmax); the warps stage the tile's
// rows, then one warp transposes them into the plane words
template <typename T, int B>
__global__ void __launch_bounds__(B == 32 ? 256 : 128)
    k_encode(FieldView<T> v, const LevelDesc* __restrict__ levels, int nlev, uint32_t total_tiles,
             const uint32_t* __restrict__ perm, FieldMeta* meta, uint32_t* __restrict__ planes) {
  hp::pdl_enter();
  constexpr int RPW = B == 32 ? 4 : 8;  // rows per warp
  __shared__ uint32_t s_tile0[HP_MAX_LEVELS + 1];
  __shared__ uint32_t s_hi[32 * 33];
  __shared__ uint32_t s_lo[B == 64 ? 32 * 33 : 1];
  __shared__ uint32_t s_sign[32];
  for (int l = threadIdx.x; l <= nlev; l += blockDim.x)
    s_tile0[l] = l < nlev ? levels[l].gtile0 : total_tiles;
  __syncthreads();
  if (meta->status) return;
  v.E_f = meta->E_f;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int l = 0;
  for (uint32_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
    l = find_level(s_tile0, l, tile);
    const LevelDesc& L = levels[l];
    const uint32_t base = perm[L.tile0 + (tile - L.gtile0)] * HP_TILE;
    const int bl = meta->bl[L.level];
    uint64_t low = 0;
    uint32_t fl = 0;
#pragma unroll
    for (int rr = 0; rr < RPW; rr++) {
      const int r = w * RPW + rr;
      const uint32_t j = base + r * 32 + lane;
      uint64_t q = 0;
      bool neg = false;
      if (j < L.n) {
        const int64_t c8 = level_c8(v, L, j, fl);
        const uint64_t m = umag(c8);
        neg = c8 < 0;
        if (bl == 0) q = 0;
        else if (B >= bl) q = m << (B - bl);
        else {
          q = m >> (bl - B);
          low |= m & ((1ull << (bl - B)) - 1ull);
        }
      }
      const uint32_t sw = __ballot_sync(HP_FULL, neg);
      if (lane == 0) s_sign[r] = sw;
      if (B == 64) {
        s_hi[r * 33 + lane] = (uint32_t)(q >> 32);
        s_lo[r * 33 + lane] = (uint32_t)q;
      } else {
        s_hi[r * 33 + lane] = (uint32_t)q;
      }
    }
    low = warp_or_u64(low);
    if (lane == 0 && low)
      atomicOr((unsigned long long*)&meta->lowbits[L.level], (unsigned long long)low);
    __syncthreads();
    if (w == 0) {
      const uint32_t wi = base / 32 + lane;
      if (wi < L.W)
        emit_word<B>(s_hi + lane * 33, s_lo + (B == 64 ? lane * 33 : 0), s_sign[lane],
                     planes + L.plane_off / 4, L.W, wi);
    }
    __syncthreads();
  }
}

void launch_encode(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* levels,
                   int nlev, uint32_t total_tiles, const uint32_t* perm, FieldMeta* meta,
                   uint32_t* planes, cstream s) {
  uint32_t blocks = total_tiles;
  uint32_t cap = (uint32_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  if (dtype == 0) {
    FieldView<float> v{(const float*)f, (uint32_t)dims[1], (uint32_t)dims[2], 0};
    hp::note_launch(), hp::launch_pdl(k_encode<float, 32>, blocks, 256, 0, s, v, levels, nlev,
                                      total_tiles, perm, meta, planes);
  } else {
    FieldView<double> v{(const double*)f, (uint32_t)dims[1], (uint32_t)dims[2], 0};
    hp::note_launch(), hp::launch_pdl(k_encode<double, 64>, blocks, 128, 0, s, v, levels, nlev,
                                      total_tiles, perm, meta, planes);
  }
}

// ------------------------------------------------------------------ batched
// warp unit = one generic tile of one job (the job's generic tiles in its
// level-then-perm order)
__device__ __forceinline__ int generic_level(const LevelDesc* __restrict__ levels, int nlev,
                                             uint32_t tile) {
  int l = 0;
  while (l + 1 < nlev && levels[l + 1].gtile0 <= tile) l++;
  return l;
}

template <typename T>
__global__ void __launch_bounds__(256) kb_levelmax(const BatchJob* __restrict__ jobs,
                                                   const uint32_t* __restrict__ unit0,
                                                   uint32_t njobs, uint32_t total) {
  hp::pdl_enter();
  const uint32_t wpb = blockDim.x >> 5;
  for (uint32_t u = blockIdx.x * wpb + (threadIdx.x >> 5); u < total; u += gridDim.x * wpb) {
    const uint32_t j = unit_owner(unit0, njobs, u);
    const BatchJob& J = jobs[j];
    FieldMeta* meta = J.meta;
    if (meta->status) continue;
    const uint32_t tile = u - unit0[j];
    const LevelDesc& L = J.levels[generic_level(J.levels, J.nlev, tile)];
    FieldView<T> v{reinterpret_cast<const T*>(J.f), J.dims[1], J.dims[2], meta->E_f};
    levelmax_tile(v, L, J.perm[L.tile0 + (tile - L.gtile0)] * HP_TILE, meta);
  }
}

void launch_b_levelmax(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                       int dtype, uint32_t grid, cstream s) {
  if (!total) return;
  const uint32_t need = (total + 7) / 8;
  if (grid > need) grid = need;
  if (dtype == 0) hp::note_launch(), hp::launch_pdl(kb_levelmax<float>, grid, 256, 0, s, jobs,
                                                    unit0, njobs, total);
  else hp::note_launch(), hp::launch_pdl(kb_levelmax<double>, grid, 256, 0, s, jobs, unit0, njobs,
                                         total);
}

__global__ void kb_bitlen(const BatchJob* __restrict__ jobs) {
  hp::pdl_enter();
  bitlen_level(jobs[blockIdx.x].meta, threadIdx.x);
}

void launch_b_bitlen(const BatchJob* jobs, uint32_t njobs, cstream s) {
  if (njobs) hp::note_launch(), hp::launch_pdl(kb_bitlen, njobs, HP_MAX_LEVELS, 0, s, jobs);
}

template <typename T, int B>
__global__ void __launch_bounds__(B == 32 ? 256 : 128)
    kb_encode(const BatchJob* __restrict__ jobs, const uint32_t* __restrict__ unit0, uint32_t njobs,
              uint32_t total) {
  hp::pdl_enter();
  constexpr int WPB = B == 32 ? 8 : 4;
  __shared__ uint32_t s_hi[WPB][32 * 33];
  __shared__ uint32_t s_lo[B == 64 ? WPB : 1][B == 64 ? 32 * 33 : 1];
  const int w = threadIdx.x >> 5;
  for (uint32_t u = blockIdx.x * WPB + w; u < total; u += gridDim.x * WPB) {
    const uint32_t j = unit_owner(unit0, njobs, u);
    const BatchJob& J = jobs[j];
    FieldMeta* meta = J.meta;
    if (meta->status) continue;
    const uint32_t tile = u - unit0[j];
    const LevelDesc& L = J.levels[generic_level(J.levels, J.nlev, tile)];
    FieldView<T> v{reinterpret_cast<const T*>(J.f), J.dims[1], J.dims[2], meta->E_f};
    encode_tile<T, B>(v, L, J.perm[L.tile0 + (tile - L.gtile0)] * HP_TILE, meta,
                      reinterpret_cast<uint32_t*>(J.planes), s_hi[w], s_lo[B == 64 ? w : 0]);
  }
}

void launch_b_encode(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                     int dtype, uint32_t grid, cstream s) {
  if (!total) return;
  const uint32_t wpb = dtype == 0 ? 8 : 4, need = (total + wpb - 1) / wpb;
  if (grid > need) grid = need;
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(kb_encode<float, 32>, grid, 256, 0, s, jobs, unit0, njobs,
                                      total);
  else
    hp::note_launch(), hp::launch_pdl(kb_encode<double, 64>, grid, 128, 0, s, jobs, unit0, njobs,
                                      total);
}

// ------------------------------------------- stand-alone Algorithm 1 and inverse
// one warp: Algorithm 1 on the 1024 elements of the tile at `base`
template <int B>
__device__ __forceinline__ void pack_tile(const void* __restrict__ qv,
                                          const uint8_t* __restrict__ sign, uint32_t n, uint32_t W,
                                          uint32_t* __restrict__ planes, uint32_t base, uint32_t* hi,
                                          uint32_t* lo) {
  const int lane = threadIdx.x & 31;
  uint32_t my_sign = 0;
#pragma unroll 4
  for (int r = 0; r < 32; r++) {
    uint32_t j = base + r * 32 + lane;
    uint64_t q = 0;
    bool neg = false;
    if (j < n) {
      q = B == 64 ? ((const uint64_t*)qv)[j] : ((const uint32_t*)qv)[j];
      neg = sign[j] != 0;
    }
    uint32_t sw = __ballot_sync(HP_FULL, neg);
    if (lane == r) my_sign = sw;
    hi[r * 33 + lane] = B == 64 ? (uint32_t)(q >> 32) : (uint32_t)q;
    if (B == 64) lo[r * 33 + lane] = (uint32_t)q;
  }
  __syncwarp();
  const uint32_t wi = base / 32 + lane;
  if (wi < W) emit_word<B>(hi + lane * 33, lo + lane * 33, my_sign, planes, W, wi);
  __syncwarp();
}

template <int B>
__global__ void __launch_bounds__(B == 32 ? 256 : 128)
    k_bitplane_encode(const void* __restrict__ qv, const uint8_t* __restrict__ sign, uint32_t n,
                      uint32_t W, uint32_t* __restrict__ planes) {
  hp::pdl_enter();
  constexpr int WPB = B == 32 ? 8 : 4;
  __shared__ uint32_t s_hi[WPB][32 * 33];
  __shared__ uint32_t s_lo[B == 64 ? WPB : 1][B == 64 ? 32 * 33 : 1];
  const int w = threadIdx.x >> 5;
  const uint32_t ntiles = (n + HP_TILE - 1) / HP_TILE;
  for (uint32_t tile = blockIdx.x * WPB + w; tile < ntiles; tile += gridDim.x * WPB)
    pack_tile<B>(qv, sign, n, W, planes, tile * HP_TILE, s_hi[w], s_lo[B == 64 ? w : 0]);
}

// one warp: the 1024 elements of the tile at `base`, keeping the top k planes
template <int B>
__device__ __forceinline__ void unpack_tile(const uint32_t* __restrict__ planes, uint32_t n,
                                            uint32_t W, int k, void* __restrict__ qv,
                                            uint8_t* __restrict__ sign, uint32_t base, uint32_t* hi,
                                            uint32_t* lo, uint32_t* sgn) {
  const int lane = threadIdx.x & 31;
  const uint32_t wi = base / 32 + lane;
  uint32_t a[32];
  if (wi < W) {
#pragma unroll
    for (int p = 0; p < 32; p++) a[31 - p] = (p < k) ? planes[(size_t)(1 + p) * W + wi] : 0u;
    if (k) transpose32(a);
#pragma unroll
    for (int b = 0; b < 32; b++) hi[lane * 33 + b] = a[b];
    if (B == 64) {
#pragma unroll
      for (int p = 0; p < 32; p++)
        a[31 - p] = (32 + p < k) ? planes[(size_t)(33 + p) * W + wi] : 0u;
      if (k > 32) transpose32(a);
#pragma unroll
      for (int b = 0; b < 32; b++) lo[lane * 33 + b] = a[b];
    }
    sgn[lane] = k > 0 ? planes[wi] : 0u;
  }
  __syncwarp();
  for (int r = 0; r < 32; r++) {
    uint32_t j = base + r * 32 + lane;
    if (j < n) {
      if (B == 64)
        ((uint64_t*)qv)[j] = ((uint64_t)hi[r * 33 + lane] << 32) | lo[r * 33 + lane];
      else
        ((uint32_t*)qv)[j] = hi[r * 33 + lane];
      sign[j] = (uint8_t)((sgn[r] >> lane) & 1u);
    }
  }
  __syncwarp();
}

template <int B>
__global__ void __launch_bounds__(B == 32 ? 256 : 128)
    k_bitplane_decode(const uint32_t* __restrict__ planes, uint32_t n, uint32_t W, int k,
                      void* __restrict__ qv, uint8_t* __restrict__ sign) {
  hp::pdl_enter();
  constexpr int WPB = B == 32 ? 8 : 4;
  __shared__ uint32_t s_hi[WPB][32 * 33];
  __shared__ uint32_t s_lo[B == 64 ? WPB : 1][B == 64 ? 32 * 33 : 1];
  __shared__ uint32_t s_sign[WPB][32];
  const int w = threadIdx.x >> 5;
  const uint32_t ntiles = (n + HP_TILE - 1) / HP_TILE;
  for (uint32_t tile = blockIdx.x * WPB + w; tile < ntiles; tile += gridDim.x * WPB)
    unpack_tile<B>(planes, n, W, k, qv, sign, tile * HP_TILE, s_hi[w], s_lo[B == 64 ? w : 0],
                   s_sign[w]);
}

// a level's planes to its level-linear staging buffer, keeping the planes of
// the groups the current reconstruction uses (k = 4 cur[l], set by selection)
template <int B>
__global__ void __launch_bounds__(B == 32 ? 256 : 128)
    k_level_unpack(const uint32_t* __restrict__ planes, const FieldMeta* __restrict__ meta,
                   const LevelDesc* __restrict__ Lp, void* __restrict__ qv,
                   uint8_t* __restrict__ sign) {
  hp::pdl_enter();
  constexpr int WPB = B == 32 ? 8 : 4;
  __shared__ uint32_t s_hi[WPB][32 * 33];
  __shared__ uint32_t s_lo[B == 64 ? WPB : 1][B == 64 ? 32 * 33 : 1];
  __shared__ uint32_t s_sign[WPB][32];
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const int w = threadIdx.x >> 5, k = 4 * meta->cur[L.level];
  const uint32_t* P = planes + L.plane_off / 4;
  for (uint32_t tile = blockIdx.x * WPB + w; tile < L.ntiles; tile += gridDim.x * WPB)
    unpack_tile<B>(P, L.n, L.W, k, qv, sign, tile * HP_TILE, s_hi[w], s_lo[B == 64 ? w : 0],
                   s_sign[w]);
}

void launch_level_unpack(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* Ld,
                         const LevelDesc& Lh, int B, void* q, uint8_t* sign, cstream s) {
  const uint32_t wpb = B == 32 ? 8 : 4;
  uint32_t blocks = (Lh.ntiles + wpb - 1) / wpb, cap = (uint32_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  if (B == 32)
    hp::note_launch(), hp::launch_pdl(k_level_unpack<32>, blocks, 256, 0, s, planes, meta, Ld, q,
                                      sign);
  else
    hp::note_launch(), hp::launch_pdl(k_level_unpack<64>, blocks, 128, 0, s, planes, meta, Ld, q,
                                      sign);
}

void launch_bitplane_encode(const void* q, const uint8_t* sign, uint64_t n, int B, uint32_t* planes,
                            cstream s) {
  uint32_t W = (uint32_t)(4 * ((n + 127) / 128));
  uint32_t ntiles = (uint32_t)((n + HP_TILE - 1) / HP_TILE);
  uint32_t wpb = B == 32 ? 8 : 4;
  uint32_t blocks = (ntiles + wpb - 1) / wpb;
  uint32_t cap = (uint32_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  if (B == 32)
    hp::note_launch(), hp::launch_pdl(k_bitplane_encode<32>, blocks, 256, 0, s, q, sign,
                                      (uint32_t)n, W, planes);
  else
    hp::note_launch(), hp::launch_pdl(k_bitplane_encode<64>, blocks, 128, 0, s, q, sign,
                                      (uint32_t)n, W, planes);
}

void launch_bitplane_decode(const uint32_t* planes, uint64_t n, int B, int k, void* q,
                            uint8_t* sign, cstream s) {
  uint32_t W = (uint32_t)(4 * ((n + 127) / 128));
  uint32_t ntiles = (uint32_t)((n + HP_TILE - 1) / HP_TILE);
  uint32_t wpb = B == 32 ? 8 : 4;
  uint32_t blocks = (ntiles + wpb - 1) / wpb;
  uint32_t cap = (uint32_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  if (B == 32)
    hp::note_launch(), hp::launch_pdl(k_bitplane_decode<32>, blocks, 256, 0, s, planes, (uint32_t)n,
                                      W, k, q, sign);
  else
    hp::note_launch(), hp::launch_pdl(k_bitplane_decode<64>, blocks, 128, 0, s, planes, (uint32_t)n,
                                      W, k, q, sign);
}

// batched Algorithm 1 / inverse over general cell levels: warp unit = one tile
// of one (job, level) entry; the staging of entry e starts at element R.soff
template <int B>
__global__ void __launch_bounds__(B == 32 ? 256 : 128)
    kb_pack(const BatchJob* __restrict__ jobs, const LevelRef* __restrict__ refs,
            const uint32_t* __restrict__ unit0, uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
  constexpr int WPB = B == 32 ? 8 : 4;
  __shared__ uint32_t s_hi[WPB][32 * 33];
  __shared__ uint32_t s_lo[B == 64 ? WPB : 1][B == 64 ? 32 * 33 : 1];
  const int w = threadIdx.x >> 5;
  for (uint32_t u = blockIdx.x * WPB + w; u < total; u += gridDim.x * WPB) {
    const uint32_t e = unit_owner(unit0, nrefs, u);
    const LevelRef R = refs[e];
    const BatchJob& J = jobs[R.job];
    if (J.meta->status) continue;
    const LevelDesc& L = J.levels[R.level];
    const void* q = reinterpret_cast<const uint8_t*>(J.gq) + R.soff * (B / 8);
    pack_tile<B>(q, J.gsg + R.soff, L.n, L.W,
                 reinterpret_cast<uint32_t*>(J.planes + L.plane_off), (u - unit0[e]) * HP_TILE,
                 s_hi[w], s_lo[B == 64 ? w : 0]);
  }
}

template <int B>
__global__ void __launch_bounds__(B == 32 ? 256 : 128)
    kb_unpack(const BatchJob* __restrict__ jobs, const LevelRef* __restrict__ refs,
              const uint32_t* __restrict__ unit0, uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
  constexpr int WPB = B == 32 ? 8 : 4;
  __shared__ uint32_t s_hi[WPB][32 * 33];
  __shared__ uint32_t s_lo[B == 64 ? WPB : 1][B == 64 ? 32 * 33 : 1];
  __shared__ uint32_t s_sign[WPB][32];
  const int w = threadIdx.x >> 5;
  for (uint32_t u = blockIdx.x * WPB + w; u < total; u += gridDim.x * WPB) {
    const uint32_t e = unit_owner(unit0, nrefs, u);
    const LevelRef R = refs[e];
    const BatchJob& J = jobs[R.job];
    const FieldMeta* meta = J.meta;
    if (meta->status) continue;
    const LevelDesc& L = J.levels[R.level];
    void* q = reinterpret_cast<uint8_t*>(J.gq) + R.soff * (B / 8);
    unpack_tile<B>(reinterpret_cast<const uint32_t*>(J.planes + L.plane_off), L.n, L.W,
                   4 * meta->cur[L.level], q, J.gsg + R.soff, (u - unit0[e]) * HP_TILE, s_hi[w],
                   s_lo[B == 64 ? w : 0], s_sign[w]);
  }
}

void launch_b_pack(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                   uint32_t nrefs, uint32_t total, int B, uint32_t grid, cstream s) {
  if (!total) return;
  const uint32_t wpb = B == 32 ? 8 : 4, need = (total + wpb - 1) / wpb;
  if (grid > need) grid = need;
  if (B == 32) hp::note_launch(), hp::launch_pdl(kb_pack<32>, grid, 256, 0, s, jobs, refs, unit0,
                                                 nrefs, total);
  else hp::note_launch(), hp::launch_pdl(kb_pack<64>, grid, 128, 0, s, jobs, refs, unit0, nrefs,
                                         total);
}

void launch_b_unpack(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                     uint32_t nrefs, uint32_t total, int B, uint32_t grid, cstream s) {
  if (!total) return;
  const uint32_t wpb = B == 32 ? 8 : 4, need = (total + wpb - 1) / wpb;
  if (grid > need) grid = need;
  if (B == 32) hp::note_launch(), hp::launch_pdl(kb_unpack<32>, grid, 256, 0, s, jobs, refs, unit0,
                                                 nrefs, total);
  else hp::note_launch(), hp::launch_pdl(kb_unpack<64>, grid, 128, 0, s, jobs, refs, unit0, nrefs,
                                         total);
}

}  // namespace hp
