// Cell-based kernels for the large, regular levels (FP32, level grid x-extent
// a multiple of 64): level max, quantize + Algorithm 1 bitplane encoding, and
// recomposition.  They compute exactly what the generic tile kernels compute
// (same coefficients, same bits), organised around 2x2x2 cells instead of the
// level-linear order.
//
// A cell (cz, cy, cx) of the level grid G_h is the node (2cz, 2cy, 2cx) of the
// coarse grid plus its seven neighbours of parity type t = o_x + 2 o_y + 4 o_z;
// all eight corners any of those seven nodes needs are the coarse nodes
// (2cz + 2dz, 2cy + 2dy, 2cx + 2dx), d in {0,1}^3, a right corner outside the
// grid being replaced by the left one.  When g_x is a multiple of 64 every type
// has g_x/2 nodes per row, a multiple of 32, so 32 consecutive cells along x
// own exactly one word of every bitplane of every type.
//
// CTA tile: 1024 cells = XW cells along x (XW = 32 NW, NW <= 8 words) times
// RY = 32/NW rows along y, in one z slice.  Phase "cells": thread = 4
// consecutive cells (coalesced row loads, corner sums shared by the types).
// Phase "words": thread = (type, row, word), a 32x32 in-register bit transpose
// between the per-cell integers (in padded shared memory) and the plane words.
#include "dev_common.cuh"

namespace hp {

struct CellGeom {
  uint32_t g[3];   // level grid
  uint32_t c[3];   // cells per axis: ceil(g / 2)
  uint32_t NW, XW, RY, tiles_x, tiles_y;
  uint32_t ntiles;
};

__host__ __device__ inline CellGeom cell_geom(const LevelDesc& L) {
  CellGeom G;
  for (int d = 0; d < 3; d++) {
    G.g[d] = L.g[d];
    G.c[d] = (L.g[d] + 1) / 2;
  }
  const uint32_t m = G.c[2] / 32;  // words per row; NW must divide it
  G.NW = m % 8 == 0 ? 8 : (m % 4 == 0 ? 4 : (m % 2 == 0 ? 2 : 1));
  G.XW = 32 * G.NW;
  G.RY = 32 / G.NW;
  G.tiles_x = G.c[2] / G.XW;
  G.tiles_y = (G.c[1] + G.RY - 1) / G.RY;
  G.ntiles = G.tiles_x * G.tiles_y * G.c[0];
  return G;
}

bool cell_path_ok(const LevelDesc& L, int B) {
  return B == 32 && L.hlog >= 0 && L.g[2] % 64 == 0 && L.g[2] >= 64;
}

// ------------------------------------------------------------ refactor side
// fixed-point values of one thread's 4 cells: the 20 coarse corners
// (rows z in {Z0, Z2} x y in {Y0, Y2}, x = 2cx, 2cx+2, ..., 2cx+8 clamped) and
// the 28 type nodes
struct CellF {
  int64_t co[2][2][5];  // [dz][dy][i]: coarse value at x = 2cx + 2i
  int64_t nd[7][4];     // [t-1][k]: type-t node of cell cx + k
};

template <bool SELF_FLOOR>
__device__ __forceinline__ void load_cell_F(const float* __restrict__ f, const CellGeom& G,
                                            uint32_t ny, uint32_t nx, int hl, int E_f, uint32_t cz,
                                            uint32_t cy, uint32_t cx, CellF& F, uint32_t& fl) {
  // level-grid coordinates -> field coordinates by << hl
  const uint32_t Z0 = 2 * cz, Y0 = 2 * cy, X0 = 2 * cx;
  const bool hz = Z0 + 1 < G.g[0], hy = Y0 + 1 < G.g[1];
  const uint32_t Z1 = hz ? Z0 + 1 : Z0, Y1 = hy ? Y0 + 1 : Y0;
  const uint32_t Z2 = Z0 + 2 < G.g[0] ? Z0 + 2 : Z0, Y2 = Y0 + 2 < G.g[1] ? Y0 + 2 : Y0;
  const uint32_t Xe = X0 + 8 < G.g[2] ? X0 + 8 : X0 + 6;
  uint32_t ign = 0;
#pragma unroll
  for (int t = 0; t < 7; t++)
#pragma unroll
    for (int k = 0; k < 4; k++) F.nd[t][k] = 0;
  if (hl == 0) {  // finest level: 2 x 16-byte loads give the 8 values of a row segment
    uint32_t& sf0 = SELF_FLOOR ? fl : ign;
    auto row8 = [&](uint32_t z, uint32_t y, float v[8]) {
      const float4* r4 = reinterpret_cast<const float4*>(f + ((size_t)z * ny + y) * nx + X0);
      const float4 a = __ldg(r4), b = __ldg(r4 + 1);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    };
    float v[8];
    const uint32_t zz0[2] = {Z0, Z2}, yy0[2] = {Y0, Y2};
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int b = 0; b < 2; b++) {
        row8(zz0[a], yy0[b], v);
#pragma unroll
        for (int i = 0; i < 4; i++) F.co[a][b][i] = fixed_point(v[2 * i], E_f, ign);
        F.co[a][b][4] = fixed_point(__ldg(f + ((size_t)zz0[a] * ny + yy0[b]) * nx + Xe), E_f, ign);
        if (a == 0 && b == 0)
#pragma unroll
          for (int k = 0; k < 4; k++) F.nd[0][k] = fixed_point(v[2 * k + 1], E_f, sf0);
      }
    if (hy) {
      row8(Z0, Y1, v);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        F.nd[1][k] = fixed_point(v[2 * k], E_f, sf0);
        F.nd[2][k] = fixed_point(v[2 * k + 1], E_f, sf0);
      }
    }
    if (hz) {
      row8(Z1, Y0, v);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        F.nd[3][k] = fixed_point(v[2 * k], E_f, sf0);
        F.nd[4][k] = fixed_point(v[2 * k + 1], E_f, sf0);
      }
    }
    if (hz && hy) {
      row8(Z1, Y1, v);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        F.nd[5][k] = fixed_point(v[2 * k], E_f, sf0);
        F.nd[6][k] = fixed_point(v[2 * k + 1], E_f, sf0);
      }
    }
    return;
  }
  auto row = [&](uint32_t z, uint32_t y) {
    return f + ((size_t)(z << hl) * ny + (y << hl)) * nx;
  };
  auto ld = [&](const float* r, uint32_t x) { return __ldg(r + ((size_t)x << hl)); };
  const uint32_t zz[2] = {Z0, Z2}, yy[2] = {Y0, Y2};
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const float* r = row(zz[a], yy[b]);
#pragma unroll
      for (int i = 0; i < 4; i++) F.co[a][b][i] = fixed_point(ld(r, X0 + 2 * i), E_f, ign);
      F.co[a][b][4] = fixed_point(ld(r, Xe), E_f, ign);
    }
  uint32_t& sf = SELF_FLOOR ? fl : ign;
  {
    const float* r = row(Z0, Y0);
#pragma unroll
    for (int k = 0; k < 4; k++) F.nd[0][k] = fixed_point(ld(r, X0 + 2 * k + 1), E_f, sf);
  }
  if (hy) {
    const float* r = row(Z0, Y1);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      F.nd[1][k] = fixed_point(ld(r, X0 + 2 * k), E_f, sf);
      F.nd[2][k] = fixed_point(ld(r, X0 + 2 * k + 1), E_f, sf);
    }
  }
  if (hz) {
    const float* r = row(Z1, Y0);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      F.nd[3][k] = fixed_point(ld(r, X0 + 2 * k), E_f, sf);
      F.nd[4][k] = fixed_point(ld(r, X0 + 2 * k + 1), E_f, sf);
    }
  }
  if (hz && hy) {
    const float* r = row(Z1, Y1);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      F.nd[5][k] = fixed_point(ld(r, X0 + 2 * k), E_f, sf);
      F.nd[6][k] = fixed_point(ld(r, X0 + 2 * k + 1), E_f, sf);
    }
  }
}

// C8 of the 7 type nodes of cell k (types that do not exist are skipped by the caller)
__device__ __forceinline__ void cell_c8(const CellF& F, int k, int64_t c8[7]) {
  const int64_t c000 = F.co[0][0][k], c001 = F.co[0][0][k + 1];
  const int64_t c010 = F.co[0][1][k], c011 = F.co[0][1][k + 1];
  const int64_t c100 = F.co[1][0][k], c101 = F.co[1][0][k + 1];
  const int64_t c110 = F.co[1][1][k], c111 = F.co[1][1][k + 1];
  const int64_t sx0 = c000 + c001, sx1 = c010 + c011, sx2 = c100 + c101, sx3 = c110 + c111;
  // D = k F - sum of corners, C8 = D * 8 / k
  c8[0] = (2 * F.nd[0][k] - sx0) * 4;                          // t=1 (x)
  c8[1] = (2 * F.nd[1][k] - (c000 + c010)) * 4;                // t=2 (y)
  c8[2] = (4 * F.nd[2][k] - (sx0 + sx1)) * 2;                  // t=3 (x, y)
  c8[3] = (2 * F.nd[3][k] - (c000 + c100)) * 4;                // t=4 (z)
  c8[4] = (4 * F.nd[4][k] - (sx0 + sx2)) * 2;                  // t=5 (x, z)
  c8[5] = (4 * F.nd[5][k] - (c000 + c010 + c100 + c110)) * 2;  // t=6 (y, z)
  c8[6] = 8 * F.nd[6][k] - (sx0 + sx1 + sx2 + sx3);            // t=7 (x, y, z)
}

__device__ __forceinline__ bool type_exists(int t, bool hz, bool hy) {
  return (!((t >> 2) & 1) || hz) && (!((t >> 1) & 1) || hy);
}

__device__ __forceinline__ void tile_origin(const CellGeom& G, uint32_t tile, uint32_t& cz,
                                            uint32_t& cy0, uint32_t& x0) {
  const uint32_t tx = tile % G.tiles_x, r = tile / G.tiles_x;
  const uint32_t ty = r % G.tiles_y;
  cz = r / G.tiles_y;
  cy0 = ty * G.RY;
  x0 = tx * G.XW;
}

// level max of |C8| (and the floor flag of the level's own nodes): one tile
__device__ __forceinline__ void cells_levelmax_tile(const float* __restrict__ f, const CellGeom& G,
                                                    uint32_t ny, uint32_t nx, int hl, int E_f,
                                                    uint32_t tile, uint64_t& mx, uint32_t& fl) {
  const uint32_t i = threadIdx.x, per_row = G.XW / 4;
  uint32_t cz, cy0, x0;
  tile_origin(G, tile, cz, cy0, x0);
  const uint32_t cy = cy0 + i / per_row, cx = x0 + 4 * (i % per_row);
  if (cy >= G.c[1]) return;
  CellF F;
  load_cell_F<true>(f, G, ny, nx, hl, E_f, cz, cy, cx, F, fl);
  const bool hz = 2 * cz + 1 < G.g[0], hy = 2 * cy + 1 < G.g[1];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    int64_t c8[7];
    cell_c8(F, k, c8);
#pragma unroll
    for (int t = 1; t <= 7; t++)
      if (type_exists(t, hz, hy)) {
        const uint64_t m = umag(c8[t - 1]);
        mx = m > mx ? m : mx;
      }
  }
}

__device__ __forceinline__ void cells_levelmax_flush(FieldMeta* meta, int level, uint64_t mx,
                                                     uint32_t fl) {
  mx = warp_max_u64(mx);
  const unsigned anyfl = __any_sync(HP_FULL, fl != 0);
  if ((threadIdx.x & 31) == 0) {
    if (mx) atomicMax((unsigned long long*)&meta->m8[level], (unsigned long long)mx);
    if (anyfl) atomicOr(&meta->floored, 1u);
  }
}

__global__ void __launch_bounds__(256, 2) k_cells_levelmax(const float* __restrict__ f, uint32_t ny,
                                                        uint32_t nx, const LevelDesc* __restrict__ Lp,
                                                        FieldMeta* meta) {
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const CellGeom G = cell_geom(L);
  const int E_f = meta->E_f, hl = L.hlog;
  uint64_t mx = 0;
  uint32_t fl = 0;
  for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
    cells_levelmax_tile(f, G, ny, nx, hl, E_f, tile, mx, fl);
  cells_levelmax_flush(meta, L.level, mx, fl);
}

// quantize + Algorithm 1: one tile of 1024 cells (all 7 types)
typedef uint32_t CellQ[7][32][33];   // [type][row * NW + word][cell within word]
typedef uint8_t CellS[7][32][32];    // sign per cell

__device__ __forceinline__ void cells_zero_padding(const LevelDesc& L, uint32_t* P) {
  // the padding words past the last node of every plane are zero
  const uint32_t W = L.W, used = (L.n + 31) / 32, pad = W - used;
  for (uint32_t k = threadIdx.x; k < pad * (32 + 1); k += blockDim.x)
    P[(size_t)(k / pad) * W + used + k % pad] = 0u;
}

__device__ __forceinline__ void cells_encode_tile(const float* __restrict__ f, const CellGeom& G,
                                                  const LevelDesc& L, uint32_t ny, uint32_t nx,
                                                  int E_f, int bl, uint32_t* __restrict__ P,
                                                  uint32_t tile, uint64_t& low, CellQ& s_q,
                                                  CellS& s_s) {
  const int hl = L.hlog;
  const uint32_t i = threadIdx.x, per_row = G.XW / 4, W = L.W;
  uint32_t cz, cy0, x0;
  tile_origin(G, tile, cz, cy0, x0);
  {  // phase cells
    const uint32_t r = i / per_row, xl = 4 * (i % per_row), cy = cy0 + r, cx = x0 + xl;
    if (cy < G.c[1]) {
      CellF F;
      uint32_t ign = 0;
      load_cell_F<false>(f, G, ny, nx, hl, E_f, cz, cy, cx, F, ign);
      const bool hz = 2 * cz + 1 < G.g[0], hy = 2 * cy + 1 < G.g[1];
      const uint32_t rw = r * G.NW + xl / 32, b0 = xl % 32;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        int64_t c8[7];
        cell_c8(F, k, c8);
#pragma unroll
        for (int t = 1; t <= 7; t++) {
          uint32_t q = 0;
          uint8_t sg = 0;
          if (type_exists(t, hz, hy)) {
            const uint64_t m = umag(c8[t - 1]);
            sg = c8[t - 1] < 0;
            if (bl == 0) q = 0;
            else if (bl <= 32) q = (uint32_t)(m << (32 - bl));
            else {
              q = (uint32_t)(m >> (bl - 32));
              low |= m & ((1ull << (bl - 32)) - 1ull);
            }
          }
          s_q[t - 1][rw][b0 + k] = q;
          s_s[t - 1][rw][b0 + k] = sg;
        }
      }
    }
  }
  __syncthreads();
  if (i < 224) {  // phase words: thread = (type, row, word)
    const int t = i / 32 + 1;
    const uint32_t rw = i % 32, r = rw / G.NW, w = rw % G.NW, cy = cy0 + r;
    if (cy < L.cnt[t][1] && cz < L.cnt[t][0]) {
      uint32_t a[32];
#pragma unroll
      for (int b = 0; b < 32; b++) a[b] = s_q[t - 1][rw][b];
      transpose32(a);
      uint32_t sw = 0;
#pragma unroll
      for (int b = 0; b < 32; b++) sw |= (uint32_t)s_s[t - 1][rw][b] << b;
      const uint32_t word = (L.off[t] + (cz * L.cnt[t][1] + cy) * L.cnt[t][2] + x0) / 32 + w;
      P[word] = sw;
#pragma unroll
      for (int p = 0; p < 32; p++) P[(size_t)(1 + p) * W + word] = a[31 - p];
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void cells_lowbits_flush(FieldMeta* meta, int level, uint64_t low) {
  low = warp_or_u64(low);
  if ((threadIdx.x & 31) == 0 && low)
    atomicOr((unsigned long long*)&meta->lowbits[level], (unsigned long long)low);
}

__global__ void __launch_bounds__(256, 2) k_cells_encode(const float* __restrict__ f, uint32_t ny,
                                                      uint32_t nx, const LevelDesc* __restrict__ Lp,
                                                      FieldMeta* meta, uint32_t* __restrict__ planes) {
  __shared__ CellQ s_q;
  __shared__ CellS s_s;
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const CellGeom G = cell_geom(L);
  const int E_f = meta->E_f, bl = meta->bl[L.level];
  uint32_t* P = planes + L.plane_off / 4;
  uint64_t low = 0;
  if (blockIdx.x == 0) cells_zero_padding(L, P);
  for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
    cells_encode_tile(f, G, L, ny, nx, E_f, bl, P, tile, low, s_q, s_s);
  cells_lowbits_flush(meta, L.level, low);
}

static int nsm() {
  int dev = 0, n = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

void launch_cells_levelmax(const float* f, const uint64_t dims[3], const LevelDesc* Ld,
                           const LevelDesc& Lh, FieldMeta* meta, cstream s) {
  const CellGeom G = cell_geom(Lh);
  uint32_t blocks = G.ntiles, cap = (uint32_t)nsm() * 8;
  if (blocks > cap) blocks = cap;
  if (!blocks) return;
  hp::note_launch(), k_cells_levelmax<<<blocks, 256, 0, s>>>(f, (uint32_t)dims[1], (uint32_t)dims[2],
                                                          Ld, meta);
}

void launch_cells_encode(const float* f, const uint64_t dims[3], const LevelDesc* Ld,
                         const LevelDesc& Lh, FieldMeta* meta, uint32_t* planes, cstream s) {
  const CellGeom G = cell_geom(Lh);
  uint32_t blocks = G.ntiles, cap = (uint32_t)nsm() * 6;
  if (blocks > cap) blocks = cap;
  if (!blocks) return;
  hp::note_launch(), k_cells_encode<<<blocks, 256, 0, s>>>(f, (uint32_t)dims[1], (uint32_t)dims[2],
                                                        Ld, meta, planes);
}

// --------------------------------------------------------- retrieval side
__device__ __forceinline__ float out_f32(int64_t X, int E_f) {
  const int e = E_f - 48;
  if (e >= -126 && E_f <= 121) return __fmul_rn(__ll2float_rn(X), __int_as_float((e + 127) << 23));
  const double d = __dmul_rn(__ll2double_rn(X), __longlong_as_double((long long)(e + 1023) << 52));
  return __double2float_rn(d);
}

typedef uint32_t CellSW[7][32];

// recomposition of one tile of 1024 cells from the coarse grid and the planes
template <bool FINAL>
__device__ __forceinline__ void cells_recompose_tile(const uint32_t* __restrict__ P,
                                                     const LevelDesc& L, const CellGeom& G,
                                                     int E_f, int bl, int k,
                                                     const int64_t* __restrict__ coarse,
                                                     void* __restrict__ dst, uint32_t tile,
                                                     CellQ& s_q, CellSW& s_sw) {
  const uint32_t i = threadIdx.x, per_row = G.XW / 4;
  const uint32_t W = L.W;
  const uint32_t gc1 = L.gc[1], gc2 = L.gc[2];
  uint32_t cz, cy0, x0;
  tile_origin(G, tile, cz, cy0, x0);
  if (i < 224) {  // phase words: planes -> q_hat per cell
    const int t = i / 32 + 1;
    const uint32_t rw = i % 32, r = rw / G.NW, w = rw % G.NW, cy = cy0 + r;
    if (cy < L.cnt[t][1] && cz < L.cnt[t][0]) {
      const uint32_t word = (L.off[t] + (cz * L.cnt[t][1] + cy) * L.cnt[t][2] + x0) / 32 + w;
      uint32_t a[32];
#pragma unroll
      for (int p = 0; p < 32; p++) a[31 - p] = p < k ? __ldcs(P + (size_t)(1 + p) * W + word) : 0u;
      if (k) transpose32(a);
#pragma unroll
      for (int b = 0; b < 32; b++) s_q[t - 1][rw][b] = a[b];
      s_sw[t - 1][rw] = k ? __ldcs(P + word) : 0u;
    }
  }
  __syncthreads();
  {  // phase cells
    const uint32_t r = i / per_row, xl = 4 * (i % per_row), cy = cy0 + r, cx = x0 + xl;
    if (cy < G.c[1]) {
      const bool hz = 2 * cz + 1 < G.g[0], hy = 2 * cy + 1 < G.g[1];
      // coarse corners: rows (cz | cz+1 clamped) x (cy | cy+1 clamped), x = cx .. cx+4 clamped
      const uint32_t cz1 = 2 * cz + 2 < G.g[0] ? cz + 1 : cz, cy1 = 2 * cy + 2 < G.g[1] ? cy + 1 : cy;
      const uint32_t xe = 2 * cx + 8 < G.g[2] ? cx + 4 : cx + 3;
      int64_t C[2][2][5];
      const uint32_t zz[2] = {cz, cz1}, yy[2] = {cy, cy1};
#pragma unroll
      for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
          const int64_t* row = coarse + ((size_t)zz[a] * gc1 + yy[b]) * gc2;
          // cx is a multiple of 4 and gc2 of 32: two aligned 16-byte loads
          const longlong2 p0 = __ldg(reinterpret_cast<const longlong2*>(row + cx));
          const longlong2 p1 = __ldg(reinterpret_cast<const longlong2*>(row + cx) + 1);
          C[a][b][0] = p0.x;
          C[a][b][1] = p0.y;
          C[a][b][2] = p1.x;
          C[a][b][3] = p1.y;
          C[a][b][4] = __ldg(row + xe);
        }
      const uint32_t rw = r * G.NW + xl / 32, b0 = xl % 32;
      // one output row (2cz+oz, 2cy+oy) at a time: its even-x nodes are type
      // te = 2 oy + 4 oz (te = 0: the coarse node itself), its odd-x nodes te + 1
#pragma unroll
      for (int oz = 0; oz < 2; oz++)
#pragma unroll
        for (int oy = 0; oy < 2; oy++) {
          if ((oz && !hz) || (oy && !hy)) continue;
          const int te = 2 * oy + 4 * oz;
          int64_t V[8];
#pragma unroll
          for (int kk = 0; kk < 4; kk++) {
#pragma unroll
            for (int par = 0; par < 2; par++) {
              const int t = te + par;
              int64_t X;
              if (t == 0) {
                X = C[0][0][kk];
              } else {
                // corner sum of type t: the corners along its odd axes
                int64_t S = 0;
#pragma unroll
                for (int dz = 0; dz < 2; dz++)
#pragma unroll
                  for (int dy = 0; dy < 2; dy++)
#pragma unroll
                    for (int dx = 0; dx < 2; dx++) {
                      if ((dz && !(t & 4)) || (dy && !(t & 2)) || (dx && !(t & 1))) continue;
                      S += C[dz][dy][kk + dx];
                    }
                const uint32_t qh = s_q[t - 1][rw][b0 + kk];
                const bool neg = (s_sw[t - 1][rw] >> (b0 + kk)) & 1u;
                uint64_t mag;
                if (bl == 0) mag = 0;
                else if (bl <= 32) mag = qh >> (32 - bl);
                else mag = (uint64_t)qh << (bl - 32);
                const int64_t c8 = neg ? -(int64_t)mag : (int64_t)mag;
                const int nodd = __popc(t);
                X = (c8 * ((int64_t)1 << nodd) + 8 * S) >> (3 + nodd);
              }
              V[2 * kk + par] = X;
            }
          }
          const size_t base = ((size_t)(2 * cz + oz) * G.g[1] + (2 * cy + oy)) * G.g[2] + 2 * cx;
          if (FINAL) {
            float4* d4 = reinterpret_cast<float4*>(reinterpret_cast<float*>(dst) + base);
            d4[0] = make_float4(out_f32(V[0], E_f), out_f32(V[1], E_f), out_f32(V[2], E_f),
                                out_f32(V[3], E_f));
            d4[1] = make_float4(out_f32(V[4], E_f), out_f32(V[5], E_f), out_f32(V[6], E_f),
                                out_f32(V[7], E_f));
          } else {
            longlong2* d2 = reinterpret_cast<longlong2*>(reinterpret_cast<int64_t*>(dst) + base);
#pragma unroll
            for (int kk = 0; kk < 4; kk++) d2[kk] = make_longlong2(V[2 * kk], V[2 * kk + 1]);
          }
        }
    }
  }
  __syncthreads();
}

template <bool FINAL>
__global__ void __launch_bounds__(256, 3) k_cells_recompose(const uint32_t* __restrict__ planes,
                                                         const FieldMeta* __restrict__ meta,
                                                         const LevelDesc* __restrict__ Lp,
                                                         const int64_t* __restrict__ coarse,
                                                         void* __restrict__ dst) {
  __shared__ CellQ s_q;
  __shared__ CellSW s_sw;
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const CellGeom G = cell_geom(L);
  const int E_f = meta->E_f, bl = meta->bl[L.level], k = 4 * meta->cur[L.level];
  const uint32_t* P = planes + L.plane_off / 4;
  for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
    cells_recompose_tile<FINAL>(P, L, G, E_f, bl, k, coarse, dst, tile, s_q, s_sw);
}

void launch_cells_recompose(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* Ld,
                            const LevelDesc& Lh, const int64_t* coarse, void* dst, int final,
                            cstream s) {
  const CellGeom G = cell_geom(Lh);
  uint32_t blocks = G.ntiles, cap = (uint32_t)nsm() * 6;
  if (blocks > cap) blocks = cap;
  if (!blocks) return;
  if (final)
    hp::note_launch(), k_cells_recompose<true><<<blocks, 256, 0, s>>>(planes, meta, Ld, coarse, dst);
  else
    hp::note_launch(), k_cells_recompose<false><<<blocks, 256, 0, s>>>(planes, meta, Ld, coarse, dst);
}

// ------------------------------------------------------------------ batched
uint32_t cell_tiles(const LevelDesc& L) { return cell_geom(L).ntiles; }

// unit = one tile of 1024 cells of one (job, level) entry
__global__ void __launch_bounds__(256, 2) kb_cells_levelmax(const BatchJob* __restrict__ jobs,
                                                         const LevelRef* __restrict__ refs,
                                                         const uint32_t* __restrict__ unit0,
                                                         uint32_t nrefs, uint32_t total) {
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t e = unit_owner(unit0, nrefs, u);
    const LevelRef R = refs[e];
    const BatchJob& J = jobs[R.job];
    FieldMeta* meta = J.meta;
    if (meta->status) continue;
    const LevelDesc& L = J.levels[R.level];
    const CellGeom G = cell_geom(L);
    uint64_t mx = 0;
    uint32_t fl = 0;
    cells_levelmax_tile(reinterpret_cast<const float*>(J.f), G, J.dims[1], J.dims[2], L.hlog,
                        meta->E_f, u - unit0[e], mx, fl);
    cells_levelmax_flush(meta, L.level, mx, fl);
  }
}

__global__ void __launch_bounds__(256, 2) kb_cells_encode(const BatchJob* __restrict__ jobs,
                                                       const LevelRef* __restrict__ refs,
                                                       const uint32_t* __restrict__ unit0,
                                                       uint32_t nrefs, uint32_t total) {
  __shared__ CellQ s_q;
  __shared__ CellS s_s;
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t e = unit_owner(unit0, nrefs, u);
    const LevelRef R = refs[e];
    const BatchJob& J = jobs[R.job];
    FieldMeta* meta = J.meta;
    if (meta->status) continue;
    const LevelDesc& L = J.levels[R.level];
    const CellGeom G = cell_geom(L);
    uint32_t* P = reinterpret_cast<uint32_t*>(J.planes) + L.plane_off / 4;
    const uint32_t tile = u - unit0[e];
    if (tile == 0) cells_zero_padding(L, P);
    uint64_t low = 0;
    cells_encode_tile(reinterpret_cast<const float*>(J.f), G, L, J.dims[1], J.dims[2], meta->E_f,
                      meta->bl[L.level], P, tile, low, s_q, s_s);
    cells_lowbits_flush(meta, L.level, low);
  }
}

__global__ void __launch_bounds__(256, 3) kb_cells_recompose(const BatchJob* __restrict__ jobs,
                                                          const LevelRef* __restrict__ refs,
                                                          const uint32_t* __restrict__ unit0,
                                                          uint32_t nrefs, uint32_t total) {
  __shared__ CellQ s_q;
  __shared__ CellSW s_sw;
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t e = unit_owner(unit0, nrefs, u);
    const LevelRef R = refs[e];
    const BatchJob& J = jobs[R.job];
    const FieldMeta* meta = J.meta;
    if (meta->status) continue;
    const LevelDesc& L = J.levels[R.level];
    const CellGeom G = cell_geom(L);
    const uint32_t* P = reinterpret_cast<const uint32_t*>(J.planes) + L.plane_off / 4;
    const int E_f = meta->E_f, bl = meta->bl[L.level], k = 4 * meta->cur[L.level];
    if (R.final)
      cells_recompose_tile<true>(P, L, G, E_f, bl, k, R.coarse, J.out, u - unit0[e], s_q, s_sw);
    else
      cells_recompose_tile<false>(P, L, G, E_f, bl, k, R.coarse, R.dst, u - unit0[e], s_q, s_sw);
  }
}

void launch_b_cells_levelmax(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                             uint32_t nrefs, uint32_t total, uint32_t grid, cstream s) {
  if (!total) return;
  if (grid > total) grid = total;
  hp::note_launch(), kb_cells_levelmax<<<grid, 256, 0, s>>>(jobs, refs, unit0, nrefs, total);
}

void launch_b_cells_encode(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                           uint32_t nrefs, uint32_t total, uint32_t grid, cstream s) {
  if (!total) return;
  if (grid > total) grid = total;
  hp::note_launch(), kb_cells_encode<<<grid, 256, 0, s>>>(jobs, refs, unit0, nrefs, total);
}

void launch_b_cells_recompose(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                              uint32_t nrefs, uint32_t total, uint32_t grid, cstream s) {
  if (!total) return;
  if (grid > total) grid = total;
  hp::note_launch(), kb_cells_recompose<<<grid, 256, 0, s>>>(jobs, refs, unit0, nrefs, total);
}

}  // namespace hp
