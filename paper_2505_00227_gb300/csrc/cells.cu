// Cell-based kernels for the large, regular levels (FP32 or FP64, level grid
// x-extent a multiple of 64): level max, quantize + Algorithm 1 bitplane
// encoding, and recomposition.  They compute exactly what the generic tile kernels compute
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
  return (B == 32 || B == 64) && L.hlog >= 0 && L.g[2] % 64 == 0 && L.g[2] >= 64;
}

// ------------------------------------------------------------ refactor side
// The seven type coefficients of 4 consecutive cells (cx .. cx+3), computed
// row by row: only the coarse row (Z0, Y0) and running sums of coarse rows
// stay live, never all 48 fixed-point values at once.  visit(t, c8) gets the
// coefficients c8[k] of the type-t nodes of cells cx + k, k = 0..3; types
// that do not exist at this (cz, cy) are not visited.  Corner sums: with c_yz the coarse value
// row at (Z0 + 2 dz, Y0 + 2 dy) (clamped), a = c_00 + c_01, d = c_00 + c_10,
// b = a + c_10 + c_11; a type's corners along x are entries k and k + 1.
// FPCONV (FP32 only; no floor flag needed and -78 <= E_f): the fixed point of
// every value by fixed_point_fp on the floating-point pipes instead of the
// IEEE-field integer path; both give the same F.  T: float or double.
template <bool SELF_FLOOR, bool FPCONV = false, typename T, typename V>
__device__ __forceinline__ void cells_visit(const T* __restrict__ f, const CellGeom& G,
                                            uint32_t ny, uint32_t nx, int hl, int E_f,
                                            uint32_t cz, uint32_t cy, uint32_t cx, uint32_t& fl,
                                            V&& visit) {
  static_assert(!FPCONV || sizeof(T) == 4, "the floating-point conversion is for FP32 values");
  const uint32_t Z0 = 2 * cz, Y0 = 2 * cy, X0 = 2 * cx;
  const bool hz = Z0 + 1 < G.g[0], hy = Y0 + 1 < G.g[1];
  const uint32_t Z2 = Z0 + 2 < G.g[0] ? Z0 + 2 : Z0, Y2 = Y0 + 2 < G.g[1] ? Y0 + 2 : Y0;
  const uint32_t Xe = X0 + 8 < G.g[2] ? X0 + 8 : X0 + 6;
  const bool f32 = ((uintptr_t)f & 31u) == 0;  // rows start at multiples of 64 values
  uint32_t ign = 0;
  uint32_t& sf = SELF_FLOOR ? fl : ign;
  const float sc = FPCONV ? __int_as_float((48 - E_f + 127) << 23) : 0.0f;
  auto fixp = [&](T x, uint32_t& fla) -> int64_t {
    if constexpr (FPCONV) return fixed_point_fp(x, sc);
    else return fixed_point(x, E_f, fla);
  };
  // values at x = X0 .. X0 + 7 of level-grid row (z, y); odd x only if asked
  auto seg = [&](uint32_t z, uint32_t y, T v[8], bool odd) {
    const T* r = f + ((size_t)(z << hl) * ny + (y << hl)) * nx;
    if constexpr (sizeof(T) == 4) {
      if (hl == 0 && f32) {  // finest level, 32-byte aligned field: one 32-byte load
        ld_nc_v8f(r + X0, v);
        return;
      } else if (hl == 0) {  // two 16-byte loads
        const float4 p = __ldg(reinterpret_cast<const float4*>(r + X0));
        const float4 q = __ldg(reinterpret_cast<const float4*>(r + X0) + 1);
        v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
        v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
        return;
      }
    } else {
      if (hl == 0 && f32) {  // FP64: two 32-byte loads
        ld_nc_v4d(r + X0, v);
        ld_nc_v4d(r + X0 + 4, v + 4);
        return;
      } else if (hl == 0) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const double2 p = __ldg(reinterpret_cast<const double2*>(r + X0) + i);
          v[2 * i] = p.x;
          v[2 * i + 1] = p.y;
        }
        return;
      }
    }
#pragma unroll
    for (int i = 0; i < 8; i++)
      if (!(i & 1) || odd) v[i] = __ldg(r + ((size_t)(X0 + i) << hl));
  };
  // the coarse values of a row: x = X0, X0 + 2, X0 + 4, X0 + 6 and the clamped
  // X0 + 8; v receives the row segment (odd x too if asked)
  auto coarse = [&](uint32_t z, uint32_t y, int64_t c[5], T v[8], bool odd) {
    seg(z, y, v, odd);
#pragma unroll
    for (int i = 0; i < 4; i++) c[i] = fixp(v[2 * i], ign);
    c[4] = fixp(__ldg(f + ((size_t)(z << hl) * ny + (y << hl)) * nx + ((size_t)Xe << hl)), ign);
  };
  T v[8];
  int64_t c0[5], a[5], c[4];
  coarse(Z0, Y0, c0, v, true);  // and the t = 1 nodes at odd x
#pragma unroll
  for (int k = 0; k < 4; k++) c[k] = (2 * fixp(v[2 * k + 1], sf) - (c0[k] + c0[k + 1])) * 4;
  visit(1, c);
  if (hy) {
    coarse(Z0, Y2, a, v, false);
#pragma unroll
    for (int i = 0; i < 5; i++) a[i] += c0[i];
    seg(Z0, Y0 + 1, v, true);
#pragma unroll
    for (int k = 0; k < 4; k++) c[k] = (2 * fixp(v[2 * k], sf) - a[k]) * 4;
    visit(2, c);
#pragma unroll
    for (int k = 0; k < 4; k++) c[k] = (4 * fixp(v[2 * k + 1], sf) - (a[k] + a[k + 1])) * 2;
    visit(3, c);
  }
  if (hz) {
    int64_t c1[5];
    coarse(Z2, Y0, c1, v, false);
#pragma unroll
    for (int i = 0; i < 5; i++) c0[i] += c1[i];  // c0 becomes d
    seg(Z0 + 1, Y0, v, true);
#pragma unroll
    for (int k = 0; k < 4; k++) c[k] = (2 * fixp(v[2 * k], sf) - c0[k]) * 4;
    visit(4, c);
#pragma unroll
    for (int k = 0; k < 4; k++) c[k] = (4 * fixp(v[2 * k + 1], sf) - (c0[k] + c0[k + 1])) * 2;
    visit(5, c);
    if (hy) {
      int64_t c3[5];
      coarse(Z2, Y2, c3, v, false);
#pragma unroll
      for (int i = 0; i < 5; i++) a[i] += c1[i] + c3[i];  // a becomes b
      seg(Z0 + 1, Y0 + 1, v, true);
#pragma unroll
      for (int k = 0; k < 4; k++) c[k] = (4 * fixp(v[2 * k], sf) - a[k]) * 2;
      visit(6, c);
#pragma unroll
      for (int k = 0; k < 4; k++) c[k] = 8 * fixp(v[2 * k + 1], sf) - (a[k] + a[k + 1]);
      visit(7, c);
    }
  }
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
template <typename T>
__device__ __forceinline__ void cells_levelmax_tile(const T* __restrict__ f, const CellGeom& G,
                                                    uint32_t ny, uint32_t nx, int hl, int E_f,
                                                    uint32_t tile, uint64_t& mx, uint32_t& fl) {
  const uint32_t i = threadIdx.x, per_row = G.XW / 4;
  uint32_t cz, cy0, x0;
  tile_origin(G, tile, cz, cy0, x0);
  const uint32_t cy = cy0 + i / per_row, cx = x0 + 4 * (i % per_row);
  if (cy >= G.c[1]) return;
  cells_visit<true>(f, G, ny, nx, hl, E_f, cz, cy, cx, fl, [&](int, const int64_t* c8) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint64_t m = umag(c8[k]);
      mx = m > mx ? m : mx;
    }
  });
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

// ----------------------------------------------- level max by estimate
// The exact pass above spends most of its instructions on 64-bit fixed-point
// arithmetic, but only bl = bitlen(max |C8|) is needed.  A pass in FP32 gives
// every node's detail d = f - mean(corners) to within (k + 1) 2^(E_f - 24)
// < 2^(E_f - 20) (k <= 8 corners summed in k - 1 roundings of partial sums
// below k 2^E_f, one rounding of the difference), i.e. C8 = 8 d / U to within
// 2^31 plus 16 for the floors of the fixed point.  So max |C8| lies within
// 2^32 of 8 max|d~| / U; when that interval (widened to 2^33 for the FP64
// evaluation below) has one bit length, that is bl.  Otherwise (a maximum
// within about 2^-10 of a power of two at the usual magnitudes, a near-zero
// level, a tiny field) the exact pass runs for the level.  The floor flag of
// the level's own nodes is exact in both passes.
//
// STATS (the finest level, hl = 0): the same pass also gives the field
// statistics of Sec. 4 (max|f|, min f, max f as order keys) and the least
// set-bit exponent of the values, so the field is read once for both; the
// estimate needs no E_f (its bound is applied after E_f is known), and the
// floor flag is decided from the least exponent once E_f is (FieldMeta::lsb_min).
// Every value lies in the four rows (Z0 | Z0+1, Y0 | Y0+1) of exactly one
// thread's cells, which are the rows STATS visits.
struct FieldStats32 {
  uint32_t am, kn, kx;  // abs key max, order key min and max (as k_stats)
  int32_t lsb;          // least exponent of a set bit (INT32_MAX: none)
};

__device__ __forceinline__ void fstats_add(FieldStats32& st, float v) {
  const uint32_t u = __float_as_uint(v), a = u & 0x7fffffffu;
  const uint32_t o = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  st.am = a > st.am ? a : st.am;
  st.kn = o < st.kn ? o : st.kn;
  st.kx = o > st.kx ? o : st.kx;
  if (a) {  // v = m 2^(e - 150) (normal) or m 2^-149 (subnormal)
    const uint32_t e = a >> 23, m = e ? ((a & 0x7fffffu) | 0x800000u) : a;
    const int32_t lsb = (int32_t)(e ? e : 1u) - 151 + __ffs((int)m);
    st.lsb = lsb < st.lsb ? lsb : st.lsb;
  }
}

template <bool STATS = false>
__device__ __forceinline__ void cells_levelmax_est_tile(const float* __restrict__ f,
                                                        const CellGeom& G, uint32_t ny,
                                                        uint32_t nx, int hl, int E_f, uint32_t tile,
                                                        float& mx, uint32_t& fl,
                                                        FieldStats32* st = nullptr) {
  const uint32_t i = threadIdx.x, per_row = G.XW / 4;
  uint32_t cz, cy0, x0;
  tile_origin(G, tile, cz, cy0, x0);
  const uint32_t cy = cy0 + i / per_row, cx = x0 + 4 * (i % per_row);
  if (cy >= G.c[1]) return;
  const uint32_t Z0 = 2 * cz, Y0 = 2 * cy, X0 = 2 * cx;
  const bool hz = Z0 + 1 < G.g[0], hy = Y0 + 1 < G.g[1];
  const uint32_t Z2 = Z0 + 2 < G.g[0] ? Z0 + 2 : Z0, Y2 = Y0 + 2 < G.g[1] ? Y0 + 2 : Y0;
  const uint32_t Xe = X0 + 8 < G.g[2] ? X0 + 8 : X0 + 6;
  const bool f32 = ((uintptr_t)f & 31u) == 0;
  auto seg = [&](uint32_t z, uint32_t y, float v[8], bool odd) {
    const float* r = f + ((size_t)(z << hl) * ny + (y << hl)) * nx;
    if (hl == 0 && f32) {
      ld_nc_v8f(r + X0, v);
    } else if (hl == 0) {
      const float4 p = __ldg(reinterpret_cast<const float4*>(r + X0));
      const float4 q = __ldg(reinterpret_cast<const float4*>(r + X0) + 1);
      v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
      v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
    } else {
#pragma unroll
      for (int k = 0; k < 8; k++)
        if (!(k & 1) || odd) v[k] = __ldg(r + ((size_t)(X0 + k) << hl));
    }
  };
  auto coarse = [&](uint32_t z, uint32_t y, float c[5], float v[8], bool odd) {
    seg(z, y, v, odd);
#pragma unroll
    for (int k = 0; k < 4; k++) c[k] = v[2 * k];
    c[4] = __ldg(f + ((size_t)(z << hl) * ny + (y << hl)) * nx + ((size_t)Xe << hl));
  };
  // the floor flag on the floating-point pipes when 2^(48 - E_f) is a normal float
  const bool fp_fl = E_f >= -78;
  const float sc = __int_as_float(((fp_fl ? 48 - E_f : 0) + 127) << 23);
  auto take = [&](float node, float mean) {
    mx = fmaxf(mx, fabsf(__fsub_rn(node, mean)));
    if (!STATS) fl |= fp_fl ? float_floors_fp(node, sc) : float_floors(node, E_f);
  };
  auto own = [&](const float v[8]) {  // a row of this thread's cells (STATS)
    if (STATS) {
#pragma unroll
      for (int k = 0; k < 8; k++) fstats_add(*st, v[k]);
    }
  };
  float v[8], c0[5], a[5];
  coarse(Z0, Y0, c0, v, true);
  own(v);
#pragma unroll
  for (int k = 0; k < 4; k++) take(v[2 * k + 1], __fmul_rn(__fadd_rn(c0[k], c0[k + 1]), 0.5f));
  if (hy) {
    coarse(Z0, Y2, a, v, false);
#pragma unroll
    for (int k = 0; k < 5; k++) a[k] = __fadd_rn(a[k], c0[k]);
    seg(Z0, Y0 + 1, v, true);
    own(v);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      take(v[2 * k], __fmul_rn(a[k], 0.5f));
      take(v[2 * k + 1], __fmul_rn(__fadd_rn(a[k], a[k + 1]), 0.25f));
    }
  }
  if (hz) {
    float c1[5];
    coarse(Z2, Y0, c1, v, false);
#pragma unroll
    for (int k = 0; k < 5; k++) c0[k] = __fadd_rn(c0[k], c1[k]);
    seg(Z0 + 1, Y0, v, true);
    own(v);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      take(v[2 * k], __fmul_rn(c0[k], 0.5f));
      take(v[2 * k + 1], __fmul_rn(__fadd_rn(c0[k], c0[k + 1]), 0.25f));
    }
    if (hy) {
      float c3[5];
      coarse(Z2, Y2, c3, v, false);
#pragma unroll
      for (int k = 0; k < 5; k++) a[k] = __fadd_rn(a[k], __fadd_rn(c1[k], c3[k]));
      seg(Z0 + 1, Y0 + 1, v, true);
      own(v);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        take(v[2 * k], __fmul_rn(a[k], 0.25f));
        take(v[2 * k + 1], __fmul_rn(__fadd_rn(a[k], a[k + 1]), 0.125f));
      }
    }
  }
}

__global__ void __launch_bounds__(256, 4) k_cells_levelmax_est(const float* __restrict__ f,
                                                            uint32_t ny, uint32_t nx,
                                                            const LevelDesc* __restrict__ Lp,
                                                            FieldMeta* meta) {
  hp::pdl_enter();
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const CellGeom G = cell_geom(L);
  const int E_f = meta->E_f, hl = L.hlog;
  float mx = 0.0f;
  uint32_t fl = 0;
  for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
    cells_levelmax_est_tile(f, G, ny, nx, hl, E_f, tile, mx, fl);
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(HP_FULL, mx, o));
  const unsigned anyfl = __any_sync(HP_FULL, fl != 0);
  if ((threadIdx.x & 31) == 0) {
    if (mx > 0.0f) atomicMax(&meta->m8est[L.level], __float_as_uint(mx));  // order of >= 0 floats
    if (anyfl) atomicOr(&meta->floored, 1u);
  }
}

// field statistics and the finest level's estimate in one read (FP32, the
// finest level on the cell path); k_stats_finalize follows
__global__ void __launch_bounds__(256, 4) k_stats_cells(const float* __restrict__ f, uint32_t ny,
                                                     uint32_t nx, const LevelDesc* __restrict__ Lp,
                                                     FieldMeta* meta) {
  hp::pdl_enter();
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const CellGeom G = cell_geom(L);
  float mx = 0.0f;
  uint32_t fl = 0;
  FieldStats32 st{0u, 0xffffffffu, 0u, 0x7fffffff};
  for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
    cells_levelmax_est_tile<true>(f, G, ny, nx, 0, 0, tile, mx, fl, &st);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(HP_FULL, mx, o));
    st.am = max(st.am, __shfl_xor_sync(HP_FULL, st.am, o));
    st.kn = min(st.kn, __shfl_xor_sync(HP_FULL, st.kn, o));
    st.kx = max(st.kx, __shfl_xor_sync(HP_FULL, st.kx, o));
    st.lsb = min(st.lsb, __shfl_xor_sync(HP_FULL, st.lsb, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (mx > 0.0f) atomicMax(&meta->m8est[L.level], __float_as_uint(mx));  // order of >= 0 floats
    atomicMax((unsigned long long*)&meta->key_absmax, (unsigned long long)st.am);
    atomicMin((unsigned long long*)&meta->key_min,
              st.kn == 0xffffffffu ? ~0ull : (unsigned long long)st.kn);
    atomicMax((unsigned long long*)&meta->key_max, (unsigned long long)st.kx);
    if (st.lsb != 0x7fffffff) atomicMin(&meta->lsb_min, st.lsb);
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 4) k_cells_levelmax(const T* __restrict__ f, uint32_t ny,
                                                        uint32_t nx, const LevelDesc* __restrict__ Lp,
                                                        FieldMeta* meta) {
  hp::pdl_enter();
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  // the estimate pass settled bl: one thread records it, nothing else to do
  if (cells_bl_from_estimate(meta, L.level, false)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cells_bl_from_estimate(meta, L.level, true);
    return;
  }
  const CellGeom G = cell_geom(L);
  const int E_f = meta->E_f, hl = L.hlog;
  uint64_t mx = 0;
  uint32_t fl = 0;
  for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
    cells_levelmax_tile(f, G, ny, nx, hl, E_f, tile, mx, fl);
  cells_levelmax_flush(meta, L.level, mx, fl);
}

// quantize + Algorithm 1: one tile of 1024 cells (all 7 types)
// Shared staging of one tile: aligned integers [type][row * NW + word][cell
// within word], rows of 36 words so that the 16-byte accesses of both phases
// (a thread's 4 cells; a word's 32 cells as 8 vectors) are conflict-free; and
// the sign bits, one 4-bit nibble per 4 cells.
typedef uint32_t CellQ[7][32][36];
typedef uint8_t CellS[7][32][8];

__device__ __forceinline__ void cells_zero_padding(const LevelDesc& L, int B, uint32_t* P) {
  // the padding words past the last node of every plane are zero
  const uint32_t W = L.W, used = (L.n + 31) / 32, pad = W - used;
  for (uint32_t k = threadIdx.x; k < pad * (uint32_t)(B + 1); k += blockDim.x)
    P[(size_t)(k / pad) * W + used + k % pad] = 0u;
}

// B = 32 (FP32): 32-bit aligned integers in s_q.  B = 64 (FP64): 64-bit aligned
// integers, the high halves in s_q and the low halves in s_ql; the words phase
// then transposes each half, the high halves giving planes 1..32 and the low
// halves planes 33..64.
template <int B, bool FPCONV, typename T>
__device__ __forceinline__ void cells_encode_tile(const T* __restrict__ f, const CellGeom& G,
                                                  const LevelDesc& L, uint32_t ny, uint32_t nx,
                                                  int E_f, int bl, uint32_t* __restrict__ P,
                                                  uint32_t tile, uint64_t& low, CellQ& s_q,
                                                  CellS& s_s, CellQ* s_ql = nullptr) {
  const int hl = L.hlog;
  const uint32_t i = threadIdx.x, per_row = G.XW / 4, W = L.W;
  uint32_t cz, cy0, x0;
  tile_origin(G, tile, cz, cy0, x0);
  {  // phase cells
    const uint32_t r = i / per_row, xl = 4 * (i % per_row), cy = cy0 + r, cx = x0 + xl;
    if (cy < G.c[1]) {
      const uint32_t rw = r * G.NW + xl / 32, b0 = xl % 32;
      uint32_t ign = 0;
      cells_visit<false, FPCONV>(f, G, ny, nx, hl, E_f, cz, cy, cx, ign, [&](int t, const int64_t* c8) {
        uint32_t nib = 0;
        if constexpr (B == 32) {
          uint32_t q[4];
#pragma unroll
          for (int k = 0; k < 4; k++) {
            const uint64_t m = umag(c8[k]);
            if (bl == 0) q[k] = 0;
            else if (bl <= 32) q[k] = (uint32_t)(m << (32 - bl));
            else {
              q[k] = (uint32_t)(m >> (bl - 32));
              low |= m & ((1ull << (bl - 32)) - 1ull);
            }
            nib |= (c8[k] < 0 ? 1u : 0u) << k;
          }
          *reinterpret_cast<uint4*>(&s_q[t - 1][rw][b0]) = make_uint4(q[0], q[1], q[2], q[3]);
        } else {  // bl <= 63 < B: q = |C8| 2^(64 - bl), nothing dropped
          uint64_t q[4];
#pragma unroll
          for (int k = 0; k < 4; k++) {
            q[k] = bl == 0 ? 0ull : umag(c8[k]) << (64 - bl);
            nib |= (c8[k] < 0 ? 1u : 0u) << k;
          }
          *reinterpret_cast<uint4*>(&s_q[t - 1][rw][b0]) =
              make_uint4((uint32_t)(q[0] >> 32), (uint32_t)(q[1] >> 32), (uint32_t)(q[2] >> 32),
                         (uint32_t)(q[3] >> 32));
          *reinterpret_cast<uint4*>(&(*s_ql)[t - 1][rw][b0]) =
              make_uint4((uint32_t)q[0], (uint32_t)q[1], (uint32_t)q[2], (uint32_t)q[3]);
        }
        s_s[t - 1][rw][b0 / 4] = (uint8_t)nib;
      });
    }
  }
  __syncthreads();
  if (i < 224) {  // phase words: thread = (type, row, word)
    const int t = i / 32 + 1;
    const uint32_t rw = i % 32, r = rw / G.NW, w = rw % G.NW, cy = cy0 + r;
    if (cy < L.cnt[t][1] && cz < L.cnt[t][0]) {
      const uint32_t word = (L.off[t] + (cz * L.cnt[t][1] + cy) * L.cnt[t][2] + x0) / 32 + w;
#pragma unroll
      for (int half = 0; half < B / 32; half++) {  // planes 1 + 32 half .. 32 + 32 half
        const CellQ& src = half == 0 ? s_q : *s_ql;
        uint32_t a[32];
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const uint4 x = *reinterpret_cast<const uint4*>(&src[t - 1][rw][4 * j]);
          a[4 * j] = x.x;
          a[4 * j + 1] = x.y;
          a[4 * j + 2] = x.z;
          a[4 * j + 3] = x.w;
        }
        transpose32(a);
#pragma unroll
        for (int p = 0; p < 32; p++) P[(size_t)(1 + 32 * half + p) * W + word] = a[31 - p];
      }
      const uint2 nb = *reinterpret_cast<const uint2*>(&s_s[t - 1][rw][0]);
      uint32_t sw = 0;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        sw |= ((nb.x >> (8 * j)) & 0xfu) << (4 * j);
        sw |= ((nb.y >> (8 * j)) & 0xfu) << (16 + 4 * j);
      }
      P[word] = sw;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void cells_lowbits_flush(FieldMeta* meta, int level, uint64_t low) {
  low = warp_or_u64(low);
  if ((threadIdx.x & 31) == 0 && low)
    atomicOr((unsigned long long*)&meta->lowbits[level], (unsigned long long)low);
}

__global__ void __launch_bounds__(256, 3) k_cells_encode(const float* __restrict__ f, uint32_t ny,
                                                      uint32_t nx, const LevelDesc* __restrict__ Lp,
                                                      FieldMeta* meta, uint32_t* __restrict__ planes) {
  hp::pdl_enter();
  __shared__ CellQ s_q;
  __shared__ CellS s_s;
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const CellGeom G = cell_geom(L);
  const int E_f = meta->E_f, bl = meta->bl[L.level];
  uint32_t* P = planes + L.plane_off / 4;
  uint64_t low = 0;
  if (blockIdx.x == 0) cells_zero_padding(L, 32, P);
  if (E_f >= -78) {  // 2^(48 - E_f) is a normal float
    for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
      cells_encode_tile<32, true>(f, G, L, ny, nx, E_f, bl, P, tile, low, s_q, s_s);
  } else {
    for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
      cells_encode_tile<32, false>(f, G, L, ny, nx, E_f, bl, P, tile, low, s_q, s_s);
  }
  cells_lowbits_flush(meta, L.level, low);
}

// FP64 fields (B = 64): the staging of both halves (65 KB) is dynamic shared memory
struct CellStage64 {
  CellQ q, ql;
  CellS s;
};

__global__ void __launch_bounds__(256, 3) k_cells_encode64(const double* __restrict__ f, uint32_t ny,
                                                        uint32_t nx, const LevelDesc* __restrict__ Lp,
                                                        FieldMeta* meta,
                                                        uint32_t* __restrict__ planes) {
  hp::pdl_enter();
  extern __shared__ __align__(16) unsigned char enc64_smem[];
  CellStage64& S = *reinterpret_cast<CellStage64*>(enc64_smem);
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const CellGeom G = cell_geom(L);
  const int E_f = meta->E_f, bl = meta->bl[L.level];
  uint32_t* P = planes + L.plane_off / 4;
  uint64_t low = 0;
  if (blockIdx.x == 0) cells_zero_padding(L, 64, P);
  for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
    cells_encode_tile<64, false>(f, G, L, ny, nx, E_f, bl, P, tile, low, S.q, S.s, &S.ql);
}

static int nsm() {
  int dev = 0, n = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

// FP32: the estimate pass, then the exact pass where the estimate left bl open;
// FP64: the exact pass
void launch_cells_levelmax(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* Ld,
                           const LevelDesc& Lh, FieldMeta* meta, cstream s, bool est_done) {
  const CellGeom G = cell_geom(Lh);
  // one wave of resident CTAs (4 per SM), each looping over tiles
  uint32_t blocks = G.ntiles, cap = (uint32_t)nsm() * 4;
  if (blocks > cap) blocks = cap;
  if (!blocks) return;
  const uint32_t ny = (uint32_t)dims[1], nx = (uint32_t)dims[2];
  if (dtype == 0) {
    if (!est_done)
      hp::note_launch(), hp::launch_pdl(k_cells_levelmax_est, blocks, 256, 0, s, (const float*)f,
                                        ny, nx, Ld, meta);
    hp::note_launch(), hp::launch_pdl(k_cells_levelmax<float>, blocks, 256, 0, s, (const float*)f,
                                      ny, nx, Ld, meta);
  } else {
    hp::note_launch(), hp::launch_pdl(k_cells_levelmax<double>, blocks, 256, 0, s,
                                      (const double*)f, ny, nx, Ld, meta);
  }
}

bool stats_cells_ok(int dtype, const LevelDesc& Lh) {
  return dtype == 0 && Lh.fast == 1 && Lh.hlog == 0;
}

void launch_stats_cells(const float* f, const uint64_t dims[3], const LevelDesc* Ld,
                        const LevelDesc& Lh, FieldMeta* meta, cstream s) {
  const CellGeom G = cell_geom(Lh);
  uint32_t blocks = G.ntiles, cap = (uint32_t)nsm() * 4;
  if (blocks > cap) blocks = cap;
  if (!blocks) return;
  hp::note_launch(), hp::launch_pdl(k_stats_cells, blocks, 256, 0, s, f, (uint32_t)dims[1],
                                    (uint32_t)dims[2], Ld, meta);
}

void launch_cells_encode(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* Ld,
                         const LevelDesc& Lh, FieldMeta* meta, uint32_t* planes, cstream s) {
  const CellGeom G = cell_geom(Lh);
  uint32_t blocks = G.ntiles, cap = (uint32_t)nsm() * 3;  // one wave, 3 CTAs per SM
  if (blocks > cap) blocks = cap;
  if (!blocks) return;
  const uint32_t ny = (uint32_t)dims[1], nx = (uint32_t)dims[2];
  if (dtype == 0) {
    hp::note_launch(), hp::launch_pdl(k_cells_encode, blocks, 256, 0, s, (const float*)f, ny, nx,
                                      Ld, meta, planes);
  } else {
    set_smem_once((const void*)k_cells_encode64, (int)sizeof(CellStage64));
    hp::note_launch(), hp::launch_pdl(k_cells_encode64, blocks, 256, sizeof(CellStage64), s,
                                      (const double*)f, ny, nx, Ld, meta, planes);
  }
}

// --------------------------------------------------------- retrieval side
typedef uint32_t CellSW[7][32];

// How a level's coefficients come back, uniform over a launch: no planes
// (k = 0 or an all-zero level: c8 = 0, the planes are not touched), bl <= 32
// (c8 magnitude = q_hat >> (32 - bl)), bl > 32 (q_hat << (bl - 32)), and
// among those bl >= 35, where c8 / 8 is an integer (CR_WIDE3, below).
// CR_ANY: decided per tile at run time (one instantiation for every case).
enum { CR_NONE = 0, CR_NARROW = 1, CR_WIDE = 2, CR_ANY = 3, CR_WIDE3 = 4 };

__device__ __forceinline__ int cells_mode(int bl, int k) {
  return (k == 0 || bl == 0) ? CR_NONE
                             : (bl <= 32 ? CR_NARROW : (bl >= 35 ? CR_WIDE3 : CR_WIDE));
}

// Planes 1 .. k (k <= 32, uniform over a launch) of one word position -> the
// q_hat (top k bits) of its 32 nodes, written to a staging row of 32 words.
// With at most 8 (16) planes the transpose works on bytes (half-words) only.
__device__ __forceinline__ void cells_words_top(const uint32_t* __restrict__ P, uint32_t W,
                                                uint32_t word, int k, uint32_t* __restrict__ qrow) {
  if (k <= 8) {  // the top 8 rows only
    uint32_t r[8];
#pragma unroll
    for (int p = 0; p < 8; p++) r[7 - p] = p < k ? __ldcs(P + (size_t)(1 + p) * W + word) : 0u;
    transpose8x4(r);
#pragma unroll
    for (int j = 0; j < 8; j++) {  // out[c]: byte c >> 3 of r[c & 7] to the top byte
      const uint32_t sel = ((uint32_t)(j >> 1) << 12) | 0x444u;
      const int c0 = (4 * j) & 7;
      *reinterpret_cast<uint4*>(qrow + 4 * j) =
          make_uint4(__byte_perm(r[c0], 0u, sel), __byte_perm(r[c0 + 1], 0u, sel),
                     __byte_perm(r[c0 + 2], 0u, sel), __byte_perm(r[c0 + 3], 0u, sel));
    }
  } else if (k <= 16) {  // the top 16 rows only
    uint32_t r[16];
#pragma unroll
    for (int p = 0; p < 16; p++) r[15 - p] = p < k ? __ldcs(P + (size_t)(1 + p) * W + word) : 0u;
    transpose16x2(r);
#pragma unroll
    for (int j = 0; j < 4; j++) {
      *reinterpret_cast<uint4*>(qrow + 4 * j) =
          make_uint4(r[4 * j] << 16, r[4 * j + 1] << 16, r[4 * j + 2] << 16, r[4 * j + 3] << 16);
      *reinterpret_cast<uint4*>(qrow + 16 + 4 * j) =
          make_uint4(r[4 * j] & 0xffff0000u, r[4 * j + 1] & 0xffff0000u,
                     r[4 * j + 2] & 0xffff0000u, r[4 * j + 3] & 0xffff0000u);
    }
  } else {
    uint32_t a[32];
#pragma unroll
    for (int p = 0; p < 32; p++) a[31 - p] = p < k ? __ldcs(P + (size_t)(1 + p) * W + word) : 0u;
    transpose32(a);
#pragma unroll
    for (int j = 0; j < 8; j++)
      *reinterpret_cast<uint4*>(qrow + 4 * j) =
          make_uint4(a[4 * j], a[4 * j + 1], a[4 * j + 2], a[4 * j + 3]);
  }
}

// recomposition of one tile of 1024 cells from the coarse grid and the planes.
// SMALL (FINAL only): the retrieval's error bound proves |X| < 2^48 for every
// value and the output exponent is in the normal range, so every value takes
// the short conversion without a range test; the output is 32-byte aligned and
// each thread writes a row's 8 values with one 32-byte store.
template <bool FINAL, int MODE, bool SMALL = false>
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
  const int md = MODE == CR_ANY ? cells_mode(bl, k) : MODE;
  if (md != CR_NONE) {
    if (i < 224) {  // phase words: planes -> q_hat per cell
      const int t = i / 32 + 1;
      const uint32_t rw = i % 32, r = rw / G.NW, w = rw % G.NW, cy = cy0 + r;
      if (cy < L.cnt[t][1] && cz < L.cnt[t][0]) {
        const uint32_t word = (L.off[t] + (cz * L.cnt[t][1] + cy) * L.cnt[t][2] + x0) / 32 + w;
        cells_words_top(P, W, word, k, &s_q[t - 1][rw][0]);
        s_sw[t - 1][rw] = __ldcs(P + word);
      }
    }
    __syncthreads();
  }
  {  // phase cells: one output row (2cz + oz, 2cy + oy) at a time
    const uint32_t r = i / per_row, xl = 4 * (i % per_row), cy = cy0 + r, cx = x0 + xl;
    if (cy < G.c[1]) {
      const bool hz = 2 * cz + 1 < G.g[0], hy = 2 * cy + 1 < G.g[1];
      // coarse rows (cz | cz+1 clamped) x (cy | cy+1 clamped), x = cx .. cx+4 clamped
      const uint32_t cz1 = 2 * cz + 2 < G.g[0] ? cz + 1 : cz, cy1 = 2 * cy + 2 < G.g[1] ? cy + 1 : cy;
      const uint32_t xe = 2 * cx + 8 < G.g[2] ? cx + 4 : cx + 3;
      const uint32_t rw = r * G.NW + xl / 32, b0 = xl % 32;
      const int e = E_f - 48;
      const bool fast_e = e >= -126 && E_f <= 121;
      const float s24 = __int_as_float(((fast_e ? e : 0) + 24 + 127) << 23);
      const float s0 = __int_as_float(((fast_e ? e : 0) + 127) << 23);
      // a thread's rows of the output and of the coarse grid are 32-byte aligned
      // when the buffers are: one 32-byte access per row then
      const bool a32 = (((uintptr_t)dst | (uintptr_t)coarse) & 31u) == 0;
      auto load = [&](uint32_t z, uint32_t y, int64_t c[5]) {
        const int64_t* row = coarse + ((size_t)z * gc1 + y) * gc2;
        // cx is a multiple of 4 and gc2 of 32: aligned 32- or 16-byte loads
        if (a32) {
          ld_nc_v4s64(row + cx, c);
        } else {
          const longlong2 p0 = __ldg(reinterpret_cast<const longlong2*>(row + cx));
          const longlong2 p1 = __ldg(reinterpret_cast<const longlong2*>(row + cx) + 1);
          c[0] = p0.x;
          c[1] = p0.y;
          c[2] = p1.x;
          c[3] = p1.y;
        }
        c[4] = __ldg(row + xe);
      };
      // the staged q_hat of the type-t nodes of the thread's 4 cells and their
      // sign bits; c8 of one of them
      auto qof = [&](int t, uint32_t qh[4], uint32_t& sg) {
        if (md == CR_NONE) return;
        const uint4 x = *reinterpret_cast<const uint4*>(&s_q[t - 1][rw][b0]);
        qh[0] = x.x;
        qh[1] = x.y;
        qh[2] = x.z;
        qh[3] = x.w;
        sg = s_sw[t - 1][rw] >> b0;
      };
      auto c8at = [&](const uint32_t qh[4], uint32_t sg, int kk) -> int64_t {
        if (md == CR_NONE) return 0;
        const uint64_t mag = md == CR_NARROW ? (uint64_t)(qh[kk] >> (32 - bl))
                                             : (uint64_t)qh[kk] << (bl - 32);
        const uint64_t neg = 0ull - (uint64_t)((sg >> kk) & 1u);  // all ones if negative
        return (int64_t)((mag ^ neg) - neg);
      };
      // CR_WIDE3: c8 = +-(q_hat << s) with s = bl - 32 >= 3, so c8 / 8 is the
      // integer +-(q_hat << (s - 3)) and X = floor((c8 + E) / 8) = ex +- q_hat 2^(s-3)
      // with ex = floor(E / 8) = S >> n.  One wide multiply-add gives
      // q_hat 2^(s-3) + ex, and a negative sign is applied by complementing ex
      // before it and the sum after it (~(y + ~ex) = ex - y).
      const uint32_t p2 = MODE == CR_WIDE3 ? 1u << (bl - 35) : 0u;
      auto wide3 = [&](uint32_t qh, uint32_t sg, int kk, int64_t ex) -> int64_t {
        const uint64_t neg = (uint64_t)(int64_t)((int32_t)(sg << (31 - kk)) >> 31);
        return (int64_t)(((uint64_t)qh * p2 + ((uint64_t)ex ^ neg)) ^ neg);
      };
      // Row (oz, oy): even-x nodes are type te = 2 oy + 4 oz (te = 0: the coarse
      // node itself), odd-x nodes te + 1.  e[kk] is the sum of the row's coarse
      // corners along y and z; a type with n odd axes has
      // X = floor((c8 2^n + 8 S) / 2^(3+n)) = (c8 + S 2^(3-n)) >> 3.
      auto emit = [&](int oz, int oy, const int64_t e[5]) {
        const int te = 2 * oy + 4 * oz, ne = __popc(te), no = ne + 1;
        uint32_t qe[4] = {0, 0, 0, 0}, qo[4] = {0, 0, 0, 0}, se = 0, so = 0;
        if (te != 0) qof(te, qe, se);
        qof(te + 1, qo, so);
        const size_t base = ((size_t)(2 * cz + oz) * G.g[1] + (2 * cy + oy)) * G.g[2] + 2 * cx;
        float o8[8];  // FINAL && SMALL: the row's 8 values, one 32-byte store
#pragma unroll
        for (int hf = 0; hf < 2; hf++) {  // two cells (four nodes) at a time
          int64_t V[4];
#pragma unroll
          for (int u = 0; u < 2; u++) {
            const int kk = 2 * hf + u;
            if (MODE == CR_WIDE3) {
              V[2 * u] = te == 0 ? e[kk] : wide3(qe[kk], se, kk, e[kk] >> ne);
              V[2 * u + 1] = wide3(qo[kk], so, kk, (e[kk] + e[kk + 1]) >> no);
            } else {
              V[2 * u] = te == 0 ? e[kk] : (c8at(qe, se, kk) + e[kk] * (8 >> ne)) >> 3;
              V[2 * u + 1] = (c8at(qo, so, kk) + (e[kk] + e[kk + 1]) * (8 >> no)) >> 3;
            }
          }
          if (FINAL && SMALL) {  // (the output is 32-byte aligned on this path)
#pragma unroll
            for (int u = 0; u < 4; u++) o8[4 * hf + u] = fixed_to_f32_small(V[u], s24, s0);
          } else if (FINAL) {
            // values below 2^48 in magnitude (the rule; a partial reconstruction
            // of a rough field can pass it) take the short conversion
            uint32_t big = 0;
#pragma unroll
            for (int u = 0; u < 4; u++) big |= ((uint32_t)((uint64_t)V[u] >> 32) + 65536u) >> 17;
            float o[4];
            if (fast_e && big == 0) {
#pragma unroll
              for (int u = 0; u < 4; u++) o[u] = fixed_to_f32_small(V[u], s24, s0);
            } else {
#pragma unroll
              for (int u = 0; u < 4; u++) o[u] = fixed_to_f32(V[u], E_f);
            }
            reinterpret_cast<float4*>(reinterpret_cast<float*>(dst) + base)[hf] =
                make_float4(o[0], o[1], o[2], o[3]);
          } else if (a32) {
            st_v4s64(reinterpret_cast<int64_t*>(dst) + base + 4 * hf, V[0], V[1], V[2], V[3]);
          } else {
            longlong2* d2 = reinterpret_cast<longlong2*>(reinterpret_cast<int64_t*>(dst) + base);
            d2[2 * hf] = make_longlong2(V[0], V[1]);
            d2[2 * hf + 1] = make_longlong2(V[2], V[3]);
          }
        }
        if (FINAL && SMALL) st_v8f(reinterpret_cast<float*>(dst) + base, o8);
      };
      int64_t c0[5], a[5];
      load(cz, cy, c0);
      load(cz, cy1, a);  // both rows' loads in flight before the first row's work
      emit(0, 0, c0);
      if (hy) {
#pragma unroll
        for (int q = 0; q < 5; q++) a[q] += c0[q];
        emit(0, 1, a);
      }
      if (hz) {
        int64_t c1[5];
        load(cz1, cy, c1);
        if (hy) {
          int64_t c3[5];
          load(cz1, cy1, c3);
#pragma unroll
          for (int q = 0; q < 5; q++) a[q] += c1[q] + c3[q];  // all four rows
        }
#pragma unroll
        for (int q = 0; q < 5; q++) c0[q] += c1[q];  // rows along z
        emit(1, 0, c0);
        if (hy) emit(1, 1, a);
      }
    }
  }
  if (md != CR_NONE) __syncthreads();  // the staging is reused by the next tile
}

template <bool FINAL, int MODE, bool SMALL>
__device__ __forceinline__ void cells_recompose_tiles(const uint32_t* __restrict__ P,
                                                      const LevelDesc& L, const CellGeom& G,
                                                      int E_f, int bl, int k,
                                                      const int64_t* __restrict__ coarse,
                                                      void* __restrict__ dst, CellQ& s_q,
                                                      CellSW& s_sw) {
  for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
    cells_recompose_tile<FINAL, MODE, SMALL>(P, L, G, E_f, bl, k, coarse, dst, tile, s_q, s_sw);
}

template <bool FINAL, bool SMALL>
__device__ __forceinline__ void cells_recompose_modes(const uint32_t* __restrict__ P,
                                                      const LevelDesc& L, const CellGeom& G,
                                                      int E_f, int bl, int k,
                                                      const int64_t* __restrict__ coarse,
                                                      void* __restrict__ dst, CellQ& s_q,
                                                      CellSW& s_sw) {
  switch (cells_mode(bl, k)) {
    case CR_NONE:
      cells_recompose_tiles<FINAL, CR_NONE, SMALL>(P, L, G, E_f, bl, k, coarse, dst, s_q, s_sw);
      break;
    case CR_NARROW:
      cells_recompose_tiles<FINAL, CR_NARROW, SMALL>(P, L, G, E_f, bl, k, coarse, dst, s_q, s_sw);
      break;
    case CR_WIDE3:
      cells_recompose_tiles<FINAL, CR_WIDE3, SMALL>(P, L, G, E_f, bl, k, coarse, dst, s_q, s_sw);
      break;
    default:
      cells_recompose_tiles<FINAL, CR_WIDE, SMALL>(P, L, G, E_f, bl, k, coarse, dst, s_q, s_sw);
  }
}

// FP64 fields (B = 64): q_hat has up to 64 bits, staged as high halves (planes
// 1..32) and low halves (planes 33..64, present only when k > 32); c8 magnitude
// = q_hat >> (64 - bl) (bl <= 63 < B).  The output is FP64 (fixed_to_f64).
struct CellRec64 {
  CellQ q, ql;
  CellSW sw;
};

template <bool FINAL>
__device__ __forceinline__ void cells_recompose_tile64(const uint32_t* __restrict__ P,
                                                       const LevelDesc& L, const CellGeom& G,
                                                       int E_f, int bl, int k,
                                                       const int64_t* __restrict__ coarse,
                                                       void* __restrict__ dst, uint32_t tile,
                                                       CellRec64& S) {
  const uint32_t i = threadIdx.x, per_row = G.XW / 4;
  const uint32_t W = L.W;
  const uint32_t gc1 = L.gc[1], gc2 = L.gc[2];
  uint32_t cz, cy0, x0;
  tile_origin(G, tile, cz, cy0, x0);
  const bool any = k > 0 && bl > 0;  // uniform over the launch
  if (any) {
    if (i < 224) {  // phase words: planes -> q_hat halves per cell
      const int t = i / 32 + 1;
      const uint32_t rw = i % 32, r = rw / G.NW, w = rw % G.NW, cy = cy0 + r;
      if (cy < L.cnt[t][1] && cz < L.cnt[t][0]) {
        const uint32_t word = (L.off[t] + (cz * L.cnt[t][1] + cy) * L.cnt[t][2] + x0) / 32 + w;
        cells_words_top(P, W, word, k < 32 ? k : 32, &S.q[t - 1][rw][0]);
        if (k > 32) cells_words_top(P + (size_t)32 * W, W, word, k - 32, &S.ql[t - 1][rw][0]);
        S.sw[t - 1][rw] = __ldcs(P + word);
      }
    }
    __syncthreads();
  }
  {  // phase cells: one output row (2cz + oz, 2cy + oy) at a time
    const uint32_t r = i / per_row, xl = 4 * (i % per_row), cy = cy0 + r, cx = x0 + xl;
    if (cy < G.c[1]) {
      const bool hz = 2 * cz + 1 < G.g[0], hy = 2 * cy + 1 < G.g[1];
      const uint32_t cz1 = 2 * cz + 2 < G.g[0] ? cz + 1 : cz, cy1 = 2 * cy + 2 < G.g[1] ? cy + 1 : cy;
      const uint32_t xe = 2 * cx + 8 < G.g[2] ? cx + 4 : cx + 3;
      const uint32_t rw = r * G.NW + xl / 32, b0 = xl % 32;
      const bool a32 = (((uintptr_t)dst | (uintptr_t)coarse) & 31u) == 0;
      auto load = [&](uint32_t z, uint32_t y, int64_t c[5]) {
        const int64_t* row = coarse + ((size_t)z * gc1 + y) * gc2;
        if (a32) {
          ld_nc_v4s64(row + cx, c);
        } else {
          const longlong2 p0 = __ldg(reinterpret_cast<const longlong2*>(row + cx));
          const longlong2 p1 = __ldg(reinterpret_cast<const longlong2*>(row + cx) + 1);
          c[0] = p0.x;
          c[1] = p0.y;
          c[2] = p1.x;
          c[3] = p1.y;
        }
        c[4] = __ldg(row + xe);
      };
      auto qof = [&](int t, uint64_t q[4], uint32_t& sg) {
        if (!any) return;
        const uint4 h = *reinterpret_cast<const uint4*>(&S.q[t - 1][rw][b0]);
        uint4 lo = make_uint4(0u, 0u, 0u, 0u);
        if (k > 32) lo = *reinterpret_cast<const uint4*>(&S.ql[t - 1][rw][b0]);
        q[0] = ((uint64_t)h.x << 32) | lo.x;
        q[1] = ((uint64_t)h.y << 32) | lo.y;
        q[2] = ((uint64_t)h.z << 32) | lo.z;
        q[3] = ((uint64_t)h.w << 32) | lo.w;
        sg = S.sw[t - 1][rw] >> b0;
      };
      auto c8at = [&](const uint64_t q[4], uint32_t sg, int kk) -> int64_t {
        if (!any) return 0;
        const uint64_t mag = q[kk] >> (64 - bl);
        const uint64_t neg = 0ull - (uint64_t)((sg >> kk) & 1u);  // all ones if negative
        return (int64_t)((mag ^ neg) - neg);
      };
      // as in the FP32 tile: X = (c8 + S 2^(3-n)) >> 3 for a type with n odd axes
      auto emit = [&](int oz, int oy, const int64_t e[5]) {
        const int te = 2 * oy + 4 * oz, ne = __popc(te), no = ne + 1;
        uint64_t qe[4] = {0, 0, 0, 0}, qo[4] = {0, 0, 0, 0};
        uint32_t se = 0, so = 0;
        if (te != 0) qof(te, qe, se);
        qof(te + 1, qo, so);
        const size_t base = ((size_t)(2 * cz + oz) * G.g[1] + (2 * cy + oy)) * G.g[2] + 2 * cx;
#pragma unroll
        for (int hf = 0; hf < 2; hf++) {
          int64_t V[4];
#pragma unroll
          for (int u = 0; u < 2; u++) {
            const int kk = 2 * hf + u;
            V[2 * u] = te == 0 ? e[kk] : (c8at(qe, se, kk) + e[kk] * (8 >> ne)) >> 3;
            V[2 * u + 1] = (c8at(qo, so, kk) + (e[kk] + e[kk + 1]) * (8 >> no)) >> 3;
          }
          if (FINAL) {
            double o[4];
#pragma unroll
            for (int u = 0; u < 4; u++) o[u] = fixed_to_f64(V[u], E_f);
            double* d = reinterpret_cast<double*>(dst) + base + 4 * hf;
            if (a32) {
              st_v4d(d, o);
            } else {
              reinterpret_cast<double2*>(d)[0] = make_double2(o[0], o[1]);
              reinterpret_cast<double2*>(d)[1] = make_double2(o[2], o[3]);
            }
          } else if (a32) {
            st_v4s64(reinterpret_cast<int64_t*>(dst) + base + 4 * hf, V[0], V[1], V[2], V[3]);
          } else {
            longlong2* d2 = reinterpret_cast<longlong2*>(reinterpret_cast<int64_t*>(dst) + base);
            d2[2 * hf] = make_longlong2(V[0], V[1]);
            d2[2 * hf + 1] = make_longlong2(V[2], V[3]);
          }
        }
      };
      int64_t c0[5], a[5];
      load(cz, cy, c0);
      emit(0, 0, c0);
      if (hy) {
        load(cz, cy1, a);
#pragma unroll
        for (int q = 0; q < 5; q++) a[q] += c0[q];
        emit(0, 1, a);
      }
      if (hz) {
        int64_t c1[5];
        load(cz1, cy, c1);
        if (hy) {
          int64_t c3[5];
          load(cz1, cy1, c3);
#pragma unroll
          for (int q = 0; q < 5; q++) a[q] += c1[q] + c3[q];
        }
#pragma unroll
        for (int q = 0; q < 5; q++) c0[q] += c1[q];
        emit(1, 0, c0);
        if (hy) emit(1, 1, a);
      }
    }
  }
  if (any) __syncthreads();  // the staging is reused by the next tile
}

template <bool FINAL>
__global__ void __launch_bounds__(256, 3) k_cells_recompose64(const uint32_t* __restrict__ planes,
                                                           const FieldMeta* __restrict__ meta,
                                                           const LevelDesc* __restrict__ Lp,
                                                           const int64_t* __restrict__ coarse,
                                                           void* __restrict__ dst) {
  hp::pdl_enter();
  extern __shared__ __align__(16) unsigned char rec64_smem[];
  CellRec64& S = *reinterpret_cast<CellRec64*>(rec64_smem);
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const CellGeom G = cell_geom(L);
  const int E_f = meta->E_f, bl = meta->bl[L.level], k = 4 * meta->cur[L.level];
  const uint32_t* P = planes + L.plane_off / 4;
  for (uint32_t tile = blockIdx.x; tile < G.ntiles; tile += gridDim.x)
    cells_recompose_tile64<FINAL>(P, L, G, E_f, bl, k, coarse, dst, tile, S);
}

// The CTAs that share an SM (blocks b, b + sms, b + 2 sms, ... under the
// block scheduler's round-robin placement) start 0.5 us apart: otherwise they
// run their words phases (integer issue) and their cells phases (memory) in
// step, and neither unit is kept busy while the other phase runs.
template <bool FINAL>
__global__ void __launch_bounds__(256, 4) k_cells_recompose(const uint32_t* __restrict__ planes,
                                                         const FieldMeta* __restrict__ meta,
                                                         const LevelDesc* __restrict__ Lp,
                                                         const int64_t* __restrict__ coarse,
                                                         void* __restrict__ dst, uint32_t sms) {
  hp::pdl_enter();
  __shared__ CellQ s_q;
  __shared__ CellSW s_sw;
  if (const uint32_t slot = blockIdx.x / sms) __nanosleep(500u * slot);
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const CellGeom G = cell_geom(L);
  const int E_f = meta->E_f, bl = meta->bl[L.level], k = 4 * meta->cur[L.level];
  const uint32_t* P = planes + L.plane_off / 4;
  if (FINAL && meta->out_small && E_f - 48 >= -126 && E_f <= 121 &&
      ((uintptr_t)dst & 31u) == 0)
    cells_recompose_modes<FINAL, true>(P, L, G, E_f, bl, k, coarse, dst, s_q, s_sw);
  else
    cells_recompose_modes<FINAL, false>(P, L, G, E_f, bl, k, coarse, dst, s_q, s_sw);
}

void launch_cells_recompose(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* Ld,
                            const LevelDesc& Lh, const int64_t* coarse, void* dst, int final,
                            int B, cstream s) {
  const CellGeom G = cell_geom(Lh);
  if (B == 64) {  // one wave, 3 CTAs per SM (65 KB of staging each)
    uint32_t blocks = G.ntiles, cap = (uint32_t)nsm() * 3;
    if (blocks > cap) blocks = cap;
    if (!blocks) return;
    const size_t sm = sizeof(CellRec64);
    if (final) {
      set_smem_once((const void*)k_cells_recompose64<true>, (int)sm);
      hp::note_launch(), hp::launch_pdl(k_cells_recompose64<true>, blocks, 256, sm, s, planes,
                                        meta, Ld, coarse, dst);
    } else {
      set_smem_once((const void*)k_cells_recompose64<false>, (int)sm);
      hp::note_launch(), hp::launch_pdl(k_cells_recompose64<false>, blocks, 256, sm, s, planes,
                                        meta, Ld, coarse, dst);
    }
    return;
  }
  uint32_t blocks = G.ntiles, cap = (uint32_t)nsm() * 4;  // one wave, 4 CTAs per SM
  if (blocks > cap) blocks = cap;
  if (!blocks) return;
  const uint32_t sms = (uint32_t)nsm();
  if (final)
    hp::note_launch(), hp::launch_pdl(k_cells_recompose<true>, blocks, 256, 0, s, planes, meta, Ld,
                                      coarse, dst, sms);
  else
    hp::note_launch(), hp::launch_pdl(k_cells_recompose<false>, blocks, 256, 0, s, planes, meta, Ld,
                                      coarse, dst, sms);
}

// ------------------------------------------------------------------ batched
uint32_t cell_tiles(const LevelDesc& L) { return cell_geom(L).ntiles; }

// unit = one tile of 1024 cells of one (job, level) entry
// the estimate pass over every (field, cell level) tile, as k_cells_levelmax_est
__global__ void __launch_bounds__(256, 4) kb_cells_levelmax_est(const BatchJob* __restrict__ jobs,
                                                             const LevelRef* __restrict__ refs,
                                                             const uint32_t* __restrict__ unit0,
                                                             uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t e = unit_owner(unit0, nrefs, u);
    const LevelRef R = refs[e];
    const BatchJob& J = jobs[R.job];
    FieldMeta* meta = J.meta;
    if (meta->status) continue;
    const LevelDesc& L = J.levels[R.level];
    const CellGeom G = cell_geom(L);
    float mx = 0.0f;
    uint32_t fl = 0;
    cells_levelmax_est_tile(reinterpret_cast<const float*>(J.f), G, J.dims[1], J.dims[2], L.hlog,
                            meta->E_f, u - unit0[e], mx, fl);
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(HP_FULL, mx, o));
    const unsigned anyfl = __any_sync(HP_FULL, fl != 0);
    if ((threadIdx.x & 31) == 0) {
      if (mx > 0.0f) atomicMax(&meta->m8est[L.level], __float_as_uint(mx));
      if (anyfl) atomicOr(&meta->floored, 1u);
    }
  }
}

// the exact pass, per tile only where the estimate left bl open (FP64: always);
// the first tile of a settled level records it
template <typename T>
__global__ void __launch_bounds__(256, 4) kb_cells_levelmax(const BatchJob* __restrict__ jobs,
                                                         const LevelRef* __restrict__ refs,
                                                         const uint32_t* __restrict__ unit0,
                                                         uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t e = unit_owner(unit0, nrefs, u);
    const LevelRef R = refs[e];
    const BatchJob& J = jobs[R.job];
    FieldMeta* meta = J.meta;
    if (meta->status) continue;
    const LevelDesc& L = J.levels[R.level];
    if (cells_bl_from_estimate(meta, L.level, false)) {
      if (u == unit0[e] && threadIdx.x == 0) cells_bl_from_estimate(meta, L.level, true);
      continue;
    }
    const CellGeom G = cell_geom(L);
    uint64_t mx = 0;
    uint32_t fl = 0;
    cells_levelmax_tile(reinterpret_cast<const T*>(J.f), G, J.dims[1], J.dims[2], L.hlog,
                        meta->E_f, u - unit0[e], mx, fl);
    cells_levelmax_flush(meta, L.level, mx, fl);
  }
}

__global__ void __launch_bounds__(256, 3) kb_cells_encode(const BatchJob* __restrict__ jobs,
                                                       const LevelRef* __restrict__ refs,
                                                       const uint32_t* __restrict__ unit0,
                                                       uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
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
    if (tile == 0) cells_zero_padding(L, 32, P);
    uint64_t low = 0;
    if (meta->E_f >= -78)
      cells_encode_tile<32, true>(reinterpret_cast<const float*>(J.f), G, L, J.dims[1], J.dims[2],
                                  meta->E_f, meta->bl[L.level], P, tile, low, s_q, s_s);
    else
      cells_encode_tile<32, false>(reinterpret_cast<const float*>(J.f), G, L, J.dims[1], J.dims[2],
                                   meta->E_f, meta->bl[L.level], P, tile, low, s_q, s_s);
    cells_lowbits_flush(meta, L.level, low);
  }
}

__global__ void __launch_bounds__(256, 3) kb_cells_encode64(const BatchJob* __restrict__ jobs,
                                                         const LevelRef* __restrict__ refs,
                                                         const uint32_t* __restrict__ unit0,
                                                         uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
  extern __shared__ __align__(16) unsigned char benc64_smem[];
  CellStage64& S = *reinterpret_cast<CellStage64*>(benc64_smem);
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
    if (tile == 0) cells_zero_padding(L, 64, P);
    uint64_t low = 0;
    cells_encode_tile<64, false>(reinterpret_cast<const double*>(J.f), G, L, J.dims[1], J.dims[2],
                                 meta->E_f, meta->bl[L.level], P, tile, low, S.q, S.s, &S.ql);
  }
}

__global__ void __launch_bounds__(256, 3) kb_cells_recompose(const BatchJob* __restrict__ jobs,
                                                          const LevelRef* __restrict__ refs,
                                                          const uint32_t* __restrict__ unit0,
                                                          uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
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
    const uint32_t tile = u - unit0[e];
    if (R.final)
      cells_recompose_tile<true, CR_ANY>(P, L, G, E_f, bl, k, R.coarse, J.out, tile, s_q, s_sw);
    else
      cells_recompose_tile<false, CR_ANY>(P, L, G, E_f, bl, k, R.coarse, R.dst, tile, s_q, s_sw);
  }
}

__global__ void __launch_bounds__(256, 3) kb_cells_recompose64(const BatchJob* __restrict__ jobs,
                                                            const LevelRef* __restrict__ refs,
                                                            const uint32_t* __restrict__ unit0,
                                                            uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
  extern __shared__ __align__(16) unsigned char brec64_smem[];
  CellRec64& S = *reinterpret_cast<CellRec64*>(brec64_smem);
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
    const uint32_t tile = u - unit0[e];
    if (R.final)
      cells_recompose_tile64<true>(P, L, G, E_f, bl, k, R.coarse, J.out, tile, S);
    else
      cells_recompose_tile64<false>(P, L, G, E_f, bl, k, R.coarse, R.dst, tile, S);
  }
}

void launch_b_cells_levelmax(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                             uint32_t nrefs, uint32_t total, uint32_t grid, int dtype, cstream s) {
  if (!total) return;
  if (grid > total) grid = total;
  if (dtype == 0) {
    hp::note_launch(), hp::launch_pdl(kb_cells_levelmax_est, grid, 256, 0, s, jobs, refs, unit0,
                                      nrefs, total);
    hp::note_launch(), hp::launch_pdl(kb_cells_levelmax<float>, grid, 256, 0, s, jobs, refs,
                                      unit0, nrefs, total);
  } else {
    hp::note_launch(), hp::launch_pdl(kb_cells_levelmax<double>, grid, 256, 0, s, jobs, refs,
                                      unit0, nrefs, total);
  }
}

void launch_b_cells_encode(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                           uint32_t nrefs, uint32_t total, uint32_t grid, int dtype, cstream s) {
  if (!total) return;
  if (grid > total) grid = total;
  if (dtype == 0) {
    hp::note_launch(), hp::launch_pdl(kb_cells_encode, grid, 256, 0, s, jobs, refs, unit0, nrefs,
                                      total);
  } else {
    set_smem_once((const void*)kb_cells_encode64, (int)sizeof(CellStage64));
    hp::note_launch(), hp::launch_pdl(kb_cells_encode64, grid, 256, sizeof(CellStage64), s, jobs,
                                      refs, unit0, nrefs, total);
  }
}

void launch_b_cells_recompose(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                              uint32_t nrefs, uint32_t total, uint32_t grid, int dtype,
                              cstream s) {
  if (!total) return;
  if (grid > total) grid = total;
  if (dtype == 0) {
    hp::note_launch(), hp::launch_pdl(kb_cells_recompose, grid, 256, 0, s, jobs, refs, unit0,
                                      nrefs, total);
  } else {
    set_smem_once((const void*)kb_cells_recompose64, (int)sizeof(CellRec64));
    hp::note_launch(), hp::launch_pdl(kb_cells_recompose64, grid, 256, sizeof(CellRec64), s, jobs,
                                      refs, unit0, nrefs, total);
  }
}

}  // namespace hp
