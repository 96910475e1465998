// General-grid cell kernels: decomposition, quantization and recomposition of
// a level of any grid size and either precision, one thread per cell.
//
// A cell (cz, cy, cx) is the coarse node (2cz, 2cy, 2cx) of the level grid
// G_h with the up to seven nodes of parity type t = o_x + 2 o_y + 4 o_z next to
// it (a type exists where 2c + 1 is inside the grid along its odd axes).  Its
// corners are the coarse nodes 2c and 2c + 2 along each odd axis, the right
// one replaced by the left one outside the grid (Sec. 3 decomposer; the same
// coefficients as the tile and fused cell kernels).
//
// The bit transposes are separate passes over a level-linear staging buffer
// (aligned integer and sign per node): quantize (this file) then Algorithm 1
// (the bitplane encoder); on retrieval the bitplane decoder fills the buffer
// and the recomposition reads it.  Consecutive threads take consecutive cells
// along x, so the field reads, the staging reads and writes (type rasters are
// x-fastest) and the output writes are coalesced for every grid size.
#include "dev_common.cuh"

namespace hp {

template <typename T>
struct GView {
  const T* __restrict__ f;
  uint32_t ny, nx;
  int hl, E_f;
};

template <typename T>
__device__ __forceinline__ int64_t gF(const GView<T>& v, uint32_t z, uint32_t y, uint32_t x,
                                      uint32_t& fl) {
  return fixed_point(
      __ldg(v.f + ((size_t)(z << v.hl) * v.ny + (y << v.hl)) * v.nx + ((size_t)x << v.hl)), v.E_f,
      fl);
}

struct CellPos {
  uint32_t cz, cy, cx;
  bool hz, hy, hx;  // the odd neighbour exists along z / y / x
};

// cells in raster order over the coarse grid (gc); dx[0], dy[0] divide by gc
__device__ __forceinline__ CellPos cell_pos(const LevelDesc& L, uint32_t c) {
  CellPos p;
  const uint32_t r = fdiv(c, L.dx[0]);
  p.cx = c - r * L.gc[2];
  p.cz = fdiv(r, L.dy[0]);
  p.cy = r - p.cz * L.gc[1];
  p.hz = 2 * p.cz + 1 < L.g[0];
  p.hy = 2 * p.cy + 1 < L.g[1];
  p.hx = 2 * p.cx + 1 < L.g[2];
  return p;
}

// level-linear index of the type-t node of cell p
__device__ __forceinline__ uint32_t type_index(const LevelDesc& L, int t, const CellPos& p) {
  return L.off[t] + (p.cz * L.cnt[t][1] + p.cy) * L.cnt[t][2] + p.cx;
}

// visit(t, C8) for every existing type of the cell
template <typename T, bool SELF_FLOOR, typename V>
__device__ __forceinline__ void gcell_visit(const GView<T>& v, const LevelDesc& L,
                                            const CellPos& p, uint32_t& fl, V&& visit) {
  uint32_t ign = 0;
  uint32_t& sf = SELF_FLOOR ? fl : ign;
  const uint32_t Z0 = 2 * p.cz, Y0 = 2 * p.cy, X0 = 2 * p.cx;
  const uint32_t Z2 = Z0 + 2 < L.g[0] ? Z0 + 2 : Z0, Y2 = Y0 + 2 < L.g[1] ? Y0 + 2 : Y0;
  const uint32_t X2 = X0 + 2 < L.g[2] ? X0 + 2 : X0;
  const int64_t c000 = gF(v, Z0, Y0, X0, ign);
  int64_t c001 = 0, c010 = 0, c011 = 0;
  if (p.hx) {
    c001 = gF(v, Z0, Y0, X2, ign);
    visit(1, (2 * gF(v, Z0, Y0, X0 + 1, sf) - (c000 + c001)) * 4);
  }
  if (p.hy) {
    c010 = gF(v, Z0, Y2, X0, ign);
    visit(2, (2 * gF(v, Z0, Y0 + 1, X0, sf) - (c000 + c010)) * 4);
    if (p.hx) {
      c011 = gF(v, Z0, Y2, X2, ign);
      visit(3, (4 * gF(v, Z0, Y0 + 1, X0 + 1, sf) - (c000 + c001 + c010 + c011)) * 2);
    }
  }
  if (p.hz) {
    const int64_t c100 = gF(v, Z2, Y0, X0, ign);
    visit(4, (2 * gF(v, Z0 + 1, Y0, X0, sf) - (c000 + c100)) * 4);
    int64_t c101 = 0;
    if (p.hx) {
      c101 = gF(v, Z2, Y0, X2, ign);
      visit(5, (4 * gF(v, Z0 + 1, Y0, X0 + 1, sf) - (c000 + c001 + c100 + c101)) * 2);
    }
    if (p.hy) {
      const int64_t c110 = gF(v, Z2, Y2, X0, ign);
      visit(6, (4 * gF(v, Z0 + 1, Y0 + 1, X0, sf) - (c000 + c010 + c100 + c110)) * 2);
      if (p.hx) {
        const int64_t c111 = gF(v, Z2, Y2, X2, ign);
        visit(7, 8 * gF(v, Z0 + 1, Y0 + 1, X0 + 1, sf) -
                     (c000 + c001 + c010 + c011 + c100 + c101 + c110 + c111));
      }
    }
  }
}

__device__ __forceinline__ uint32_t gcell_count(const LevelDesc& L) {
  return L.gc[0] * L.gc[1] * L.gc[2];
}

// ------------------------------------------------------------ level max
template <typename T>
__device__ __forceinline__ void gcells_levelmax_range(const GView<T>& v, const LevelDesc& L,
                                                      uint32_t c0, uint32_t c1, uint32_t step,
                                                      FieldMeta* meta) {
  uint64_t mx = 0;
  uint32_t fl = 0;
  for (uint32_t c = c0; c < c1; c += step) {
    const CellPos p = cell_pos(L, c);
    gcell_visit<T, true>(v, L, p, fl, [&](int, int64_t c8) {
      const uint64_t m = umag(c8);
      mx = m > mx ? m : mx;
    });
  }
  mx = warp_max_u64(mx);
  const unsigned anyfl = __any_sync(HP_FULL, fl != 0);
  if ((threadIdx.x & 31) == 0) {
    if (mx) atomicMax((unsigned long long*)&meta->m8[L.level], (unsigned long long)mx);
    if (anyfl) atomicOr(&meta->floored, 1u);
  }
}

// FP32 levels: the estimate pass (bound and fallback as for the fused cells,
// k_cells_levelmax_est): each detail f - mean(corners) in FP32, k - 1 roundings
// of partial sums of at most k corners, one rounding of the difference
__device__ __forceinline__ float gFf(const GView<float>& v, uint32_t z, uint32_t y, uint32_t x) {
  return __ldg(v.f + ((size_t)(z << v.hl) * v.ny + (y << v.hl)) * v.nx + ((size_t)x << v.hl));
}

__device__ __forceinline__ void gcells_levelmax_est_range(const GView<float>& v,
                                                          const LevelDesc& L, uint32_t c0,
                                                          uint32_t c1, uint32_t step,
                                                          FieldMeta* meta) {
  float mx = 0.0f;
  uint32_t fl = 0;
  // the floor flag on the floating-point pipes when 2^(48 - E_f) is a normal float
  const bool fp_fl = v.E_f >= -78;
  const float sc = __int_as_float(((fp_fl ? 48 - v.E_f : 0) + 127) << 23);
  auto take = [&](float node, float mean) {
    mx = fmaxf(mx, fabsf(__fsub_rn(node, mean)));
    fl |= fp_fl ? float_floors_fp(node, sc) : float_floors(node, v.E_f);
  };
  for (uint32_t c = c0; c < c1; c += step) {
    const CellPos p = cell_pos(L, c);
    const uint32_t Z0 = 2 * p.cz, Y0 = 2 * p.cy, X0 = 2 * p.cx;
    const uint32_t Z2 = Z0 + 2 < L.g[0] ? Z0 + 2 : Z0, Y2 = Y0 + 2 < L.g[1] ? Y0 + 2 : Y0;
    const uint32_t X2 = X0 + 2 < L.g[2] ? X0 + 2 : X0;
    const float c000 = gFf(v, Z0, Y0, X0);
    float c001 = 0.0f, c010 = 0.0f, c011 = 0.0f, s01 = 0.0f;
    if (p.hx) {
      c001 = gFf(v, Z0, Y0, X2);
      take(gFf(v, Z0, Y0, X0 + 1), __fmul_rn(__fadd_rn(c000, c001), 0.5f));
    }
    if (p.hy) {
      c010 = gFf(v, Z0, Y2, X0);
      take(gFf(v, Z0, Y0 + 1, X0), __fmul_rn(__fadd_rn(c000, c010), 0.5f));
      if (p.hx) {
        c011 = gFf(v, Z0, Y2, X2);
        s01 = __fadd_rn(__fadd_rn(c000, c001), __fadd_rn(c010, c011));
        take(gFf(v, Z0, Y0 + 1, X0 + 1), __fmul_rn(s01, 0.25f));
      }
    }
    if (p.hz) {
      const float c100 = gFf(v, Z2, Y0, X0);
      take(gFf(v, Z0 + 1, Y0, X0), __fmul_rn(__fadd_rn(c000, c100), 0.5f));
      float c101 = 0.0f;
      if (p.hx) {
        c101 = gFf(v, Z2, Y0, X2);
        take(gFf(v, Z0 + 1, Y0, X0 + 1),
             __fmul_rn(__fadd_rn(__fadd_rn(c000, c001), __fadd_rn(c100, c101)), 0.25f));
      }
      if (p.hy) {
        const float c110 = gFf(v, Z2, Y2, X0);
        take(gFf(v, Z0 + 1, Y0 + 1, X0),
             __fmul_rn(__fadd_rn(__fadd_rn(c000, c010), __fadd_rn(c100, c110)), 0.25f));
        if (p.hx) {
          const float c111 = gFf(v, Z2, Y2, X2);
          const float s1 = __fadd_rn(__fadd_rn(c100, c101), __fadd_rn(c110, c111));
          take(gFf(v, Z0 + 1, Y0 + 1, X0 + 1), __fmul_rn(__fadd_rn(s01, s1), 0.125f));
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(HP_FULL, mx, o));
  const unsigned anyfl = __any_sync(HP_FULL, fl != 0);
  if ((threadIdx.x & 31) == 0) {
    if (mx > 0.0f) atomicMax(&meta->m8est[L.level], __float_as_uint(mx));
    if (anyfl) atomicOr(&meta->floored, 1u);
  }
}

__global__ void __launch_bounds__(256) k_gcells_levelmax_est(const float* __restrict__ f,
                                                             uint32_t ny, uint32_t nx,
                                                             const LevelDesc* __restrict__ Lp,
                                                             FieldMeta* meta) {
  hp::pdl_enter();
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const GView<float> v{f, ny, nx, L.hlog, meta->E_f};
  gcells_levelmax_est_range(v, L, blockIdx.x * blockDim.x + threadIdx.x, gcell_count(L),
                            gridDim.x * blockDim.x, meta);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gcells_levelmax(const T* __restrict__ f, uint32_t ny,
                                                         uint32_t nx, const LevelDesc* __restrict__ Lp,
                                                         FieldMeta* meta) {
  hp::pdl_enter();
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  if (sizeof(T) == 4 && cells_bl_from_estimate(meta, L.level, false)) {  // settled
    if (blockIdx.x == 0 && threadIdx.x == 0) cells_bl_from_estimate(meta, L.level, true);
    return;
  }
  const GView<T> v{f, ny, nx, L.hlog, meta->E_f};
  gcells_levelmax_range(v, L, blockIdx.x * blockDim.x + threadIdx.x, gcell_count(L),
                        gridDim.x * blockDim.x, meta);
}

// ------------------------------------------------------------- quantize
// q = |C8| aligned to B bits (sign-magnitude), staged level-linear
template <typename T, int B>
__device__ __forceinline__ void gcells_encode_range(const GView<T>& v, const LevelDesc& L,
                                                    uint32_t c0, uint32_t c1, uint32_t step,
                                                    FieldMeta* meta, void* __restrict__ q,
                                                    uint8_t* __restrict__ sg) {
  const int bl = meta->bl[L.level];
  uint64_t low = 0;
  uint32_t ign = 0;
  for (uint32_t c = c0; c < c1; c += step) {
    const CellPos p = cell_pos(L, c);
    gcell_visit<T, false>(v, L, p, ign, [&](int t, int64_t c8) {
      const uint32_t j = type_index(L, t, p);
      const uint64_t m = umag(c8);
      uint64_t qv;
      if (bl == 0) qv = 0;
      else if (B >= bl) qv = m << (B - bl);
      else {
        qv = m >> (bl - B);
        low |= m & ((1ull << (bl - B)) - 1ull);
      }
      if (B == 32) reinterpret_cast<uint32_t*>(q)[j] = (uint32_t)qv;
      else reinterpret_cast<uint64_t*>(q)[j] = qv;
      sg[j] = c8 < 0 ? 1 : 0;
    });
  }
  low = warp_or_u64(low);
  if ((threadIdx.x & 31) == 0 && low)
    atomicOr((unsigned long long*)&meta->lowbits[L.level], (unsigned long long)low);
}

template <typename T, int B>
__global__ void __launch_bounds__(256) k_gcells_encode(const T* __restrict__ f, uint32_t ny,
                                                       uint32_t nx, const LevelDesc* __restrict__ Lp,
                                                       FieldMeta* meta, void* __restrict__ q,
                                                       uint8_t* __restrict__ sg) {
  hp::pdl_enter();
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  const GView<T> v{f, ny, nx, L.hlog, meta->E_f};
  gcells_encode_range<T, B>(v, L, blockIdx.x * blockDim.x + threadIdx.x, gcell_count(L),
                            gridDim.x * blockDim.x, meta, q, sg);
}

// ---------------------------------------------------------- recompose
template <typename T>
__device__ __forceinline__ T gconvert(int64_t X, int E_f);

template <>
__device__ __forceinline__ float gconvert<float>(int64_t X, int E_f) {
  return fixed_to_f32(X, E_f);
}

template <>
__device__ __forceinline__ double gconvert<double>(int64_t X, int E_f) {
  return fixed_to_f64(X, E_f);
}

// the node's reconstruction X = floor((c8 2^n + 8 S) / 2^(3+n)) = (c8 + S 2^(3-n)) >> 3,
// S the sum of its 2^n corners, written to the level grid or the output
template <typename T, int B>
__device__ __forceinline__ void gcells_recompose_range(const LevelDesc& L, int bl, int E_f,
                                                       const void* __restrict__ q,
                                                       const uint8_t* __restrict__ sg,
                                                       const int64_t* __restrict__ coarse,
                                                       void* __restrict__ dst, bool final,
                                                       uint32_t c0, uint32_t c1, uint32_t step) {
  const uint32_t gc1 = L.gc[1], gc2 = L.gc[2], g1 = L.g[1], g2 = L.g[2];
  for (uint32_t c = c0; c < c1; c += step) {
    const CellPos p = cell_pos(L, c);
    const uint32_t z1 = 2 * p.cz + 2 < L.g[0] ? p.cz + 1 : p.cz;
    const uint32_t y1 = 2 * p.cy + 2 < L.g[1] ? p.cy + 1 : p.cy;
    const uint32_t x1 = 2 * p.cx + 2 < L.g[2] ? p.cx + 1 : p.cx;
    auto C = [&](uint32_t z, uint32_t y, uint32_t x) {
      return __ldg(coarse + ((size_t)z * gc1 + y) * gc2 + x);
    };
    auto c8 = [&](int t) -> int64_t {
      const uint32_t j = type_index(L, t, p);
      const uint64_t qh = B == 32 ? (uint64_t)reinterpret_cast<const uint32_t*>(q)[j]
                                  : reinterpret_cast<const uint64_t*>(q)[j];
      uint64_t mag;
      if (bl == 0) mag = 0;
      else if (B >= bl) mag = qh >> (B - bl);
      else mag = qh << (bl - B);
      return sg[j] ? -(int64_t)mag : (int64_t)mag;
    };
    auto put = [&](uint32_t z, uint32_t y, uint32_t x, int64_t X) {
      const size_t d = ((size_t)z * g1 + y) * g2 + x;
      if (final) reinterpret_cast<T*>(dst)[d] = gconvert<T>(X, E_f);
      else reinterpret_cast<int64_t*>(dst)[d] = X;
    };
    const uint32_t Z0 = 2 * p.cz, Y0 = 2 * p.cy, X0 = 2 * p.cx;
    const int64_t c000 = C(p.cz, p.cy, p.cx);
    put(Z0, Y0, X0, c000);
    int64_t c001 = 0, c010 = 0, c011 = 0;
    if (p.hx) {
      c001 = C(p.cz, p.cy, x1);
      put(Z0, Y0, X0 + 1, (c8(1) + (c000 + c001) * 4) >> 3);
    }
    if (p.hy) {
      c010 = C(p.cz, y1, p.cx);
      put(Z0, Y0 + 1, X0, (c8(2) + (c000 + c010) * 4) >> 3);
      if (p.hx) {
        c011 = C(p.cz, y1, x1);
        put(Z0, Y0 + 1, X0 + 1, (c8(3) + (c000 + c001 + c010 + c011) * 2) >> 3);
      }
    }
    if (p.hz) {
      const int64_t c100 = C(z1, p.cy, p.cx);
      put(Z0 + 1, Y0, X0, (c8(4) + (c000 + c100) * 4) >> 3);
      int64_t c101 = 0;
      if (p.hx) {
        c101 = C(z1, p.cy, x1);
        put(Z0 + 1, Y0, X0 + 1, (c8(5) + (c000 + c001 + c100 + c101) * 2) >> 3);
      }
      if (p.hy) {
        const int64_t c110 = C(z1, y1, p.cx);
        put(Z0 + 1, Y0 + 1, X0, (c8(6) + (c000 + c010 + c100 + c110) * 2) >> 3);
        if (p.hx) {
          const int64_t c111 = C(z1, y1, x1);
          put(Z0 + 1, Y0 + 1, X0 + 1,
              (c8(7) + (c000 + c001 + c010 + c011 + c100 + c101 + c110 + c111)) >> 3);
        }
      }
    }
  }
}

template <typename T, int B>
__global__ void __launch_bounds__(256) k_gcells_recompose(const FieldMeta* __restrict__ meta,
                                                          const LevelDesc* __restrict__ Lp,
                                                          const void* __restrict__ q,
                                                          const uint8_t* __restrict__ sg,
                                                          const int64_t* __restrict__ coarse,
                                                          void* __restrict__ dst, int final) {
  hp::pdl_enter();
  if (meta->status) return;
  const LevelDesc& L = *Lp;
  gcells_recompose_range<T, B>(L, meta->bl[L.level], meta->E_f, q, sg, coarse, dst, final != 0,
                               blockIdx.x * blockDim.x + threadIdx.x, gcell_count(L),
                               gridDim.x * blockDim.x);
}

// ------------------------------------------------------------ launchers
static uint32_t gcell_grid(const LevelDesc& L) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t cells = (uint64_t)L.gc[0] * L.gc[1] * L.gc[2];
  uint64_t blocks = (cells + 255) / 256, cap = (uint64_t)sms * 8;
  return (uint32_t)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

void launch_gcells_levelmax(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* Ld,
                            const LevelDesc& Lh, FieldMeta* meta, cstream s) {
  const uint32_t g = gcell_grid(Lh);
  if (dtype == 0) {
    hp::note_launch(), hp::launch_pdl(k_gcells_levelmax_est, g, 256, 0, s, (const float*)f,
                                      (uint32_t)dims[1], (uint32_t)dims[2], Ld, meta);
    hp::note_launch(), hp::launch_pdl(k_gcells_levelmax<float>, g, 256, 0, s, (const float*)f,
                                      (uint32_t)dims[1], (uint32_t)dims[2], Ld, meta);
  }
  else
    hp::note_launch(), hp::launch_pdl(k_gcells_levelmax<double>, g, 256, 0, s, (const double*)f,
                                      (uint32_t)dims[1], (uint32_t)dims[2], Ld, meta);
}

void launch_gcells_encode(const void* f, int dtype, const uint64_t dims[3], const LevelDesc* Ld,
                          const LevelDesc& Lh, FieldMeta* meta, void* q, uint8_t* sg, cstream s) {
  const uint32_t g = gcell_grid(Lh);
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(k_gcells_encode<float, 32>, g, 256, 0, s, (const float*)f,
                                      (uint32_t)dims[1], (uint32_t)dims[2], Ld, meta, q, sg);
  else
    hp::note_launch(), hp::launch_pdl(k_gcells_encode<double, 64>, g, 256, 0, s, (const double*)f,
                                      (uint32_t)dims[1], (uint32_t)dims[2], Ld, meta, q, sg);
}

void launch_gcells_recompose(const FieldMeta* meta, const LevelDesc* Ld, const LevelDesc& Lh,
                             int dtype, const void* q, const uint8_t* sg, const int64_t* coarse,
                             void* dst, int final, cstream s) {
  const uint32_t g = gcell_grid(Lh);
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(k_gcells_recompose<float, 32>, g, 256, 0, s, meta, Ld, q, sg, coarse, dst,
                                                                       final);
  else
    hp::note_launch(), hp::launch_pdl(k_gcells_recompose<double, 64>, g, 256, 0, s, meta, Ld, q, sg, coarse,
                                                                        dst, final);
}

// ------------------------------------------------------------------ batched
// unit = 256 cells of one (job, level) entry; the staging of entry e starts at
// element R.soff of the job's buffer
template <typename T>
__global__ void __launch_bounds__(256) kb_gcells_levelmax(const BatchJob* __restrict__ jobs,
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
    if (sizeof(T) == 4 && cells_bl_from_estimate(meta, L.level, false)) {  // settled
      if (u == unit0[e] && threadIdx.x == 0) cells_bl_from_estimate(meta, L.level, true);
      continue;
    }
    const GView<T> v{reinterpret_cast<const T*>(J.f), J.dims[1], J.dims[2], L.hlog, meta->E_f};
    const uint32_t c = (u - unit0[e]) * 256 + threadIdx.x, n = gcell_count(L);
    gcells_levelmax_range(v, L, c, c < n ? c + 1 : c, 1, meta);
  }
}

__global__ void __launch_bounds__(256) kb_gcells_levelmax_est(const BatchJob* __restrict__ jobs,
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
    const GView<float> v{reinterpret_cast<const float*>(J.f), J.dims[1], J.dims[2], L.hlog,
                         meta->E_f};
    const uint32_t c = (u - unit0[e]) * 256 + threadIdx.x, n = gcell_count(L);
    gcells_levelmax_est_range(v, L, c, c < n ? c + 1 : c, 1, meta);
  }
}

template <typename T, int B>
__global__ void __launch_bounds__(256) kb_gcells_encode(const BatchJob* __restrict__ jobs,
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
    const GView<T> v{reinterpret_cast<const T*>(J.f), J.dims[1], J.dims[2], L.hlog, meta->E_f};
    const uint32_t c = (u - unit0[e]) * 256 + threadIdx.x, n = gcell_count(L);
    gcells_encode_range<T, B>(v, L, c, c < n ? c + 1 : c, 1, meta,
                              reinterpret_cast<uint8_t*>(J.gq) + R.soff * (B / 8), J.gsg + R.soff);
  }
}

template <typename T, int B>
__global__ void __launch_bounds__(256) kb_gcells_recompose(const BatchJob* __restrict__ jobs,
                                                           const LevelRef* __restrict__ refs,
                                                           const uint32_t* __restrict__ unit0,
                                                           uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t e = unit_owner(unit0, nrefs, u);
    const LevelRef R = refs[e];
    const BatchJob& J = jobs[R.job];
    const FieldMeta* meta = J.meta;
    if (meta->status) continue;
    const LevelDesc& L = J.levels[R.level];
    const uint32_t c = (u - unit0[e]) * 256 + threadIdx.x, n = gcell_count(L);
    gcells_recompose_range<T, B>(L, meta->bl[L.level], meta->E_f,
                                 reinterpret_cast<const uint8_t*>(J.gq) + R.soff * (B / 8),
                                 J.gsg + R.soff, R.coarse, R.final ? J.out : (void*)R.dst,
                                 R.final != 0, c, c < n ? c + 1 : c, 1);
  }
}

static uint32_t cap_units(uint32_t grid, uint32_t total) { return grid < total ? grid : total; }

void launch_b_gcells_levelmax(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                              uint32_t nrefs, uint32_t total, int dtype, uint32_t grid, cstream s) {
  if (!total) return;
  grid = cap_units(grid, total);
  if (dtype == 0) {
    hp::note_launch(), hp::launch_pdl(kb_gcells_levelmax_est, grid, 256, 0, s, jobs, refs, unit0,
                                      nrefs, total);
    hp::note_launch(), hp::launch_pdl(kb_gcells_levelmax<float>, grid, 256, 0, s, jobs, refs, unit0,
                                      nrefs, total);
  }
  else
    hp::note_launch(), hp::launch_pdl(kb_gcells_levelmax<double>, grid, 256, 0, s, jobs, refs,
                                      unit0, nrefs, total);
}

void launch_b_gcells_encode(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                            uint32_t nrefs, uint32_t total, int dtype, uint32_t grid, cstream s) {
  if (!total) return;
  grid = cap_units(grid, total);
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(kb_gcells_encode<float, 32>, grid, 256, 0, s, jobs, refs,
                                      unit0, nrefs, total);
  else
    hp::note_launch(), hp::launch_pdl(kb_gcells_encode<double, 64>, grid, 256, 0, s, jobs, refs,
                                      unit0, nrefs, total);
}

void launch_b_gcells_recompose(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                               uint32_t nrefs, uint32_t total, int dtype, uint32_t grid,
                               cstream s) {
  if (!total) return;
  grid = cap_units(grid, total);
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(kb_gcells_recompose<float, 32>, grid, 256, 0, s, jobs, refs, unit0, nrefs,
                                                                           total);
  else
    hp::note_launch(), hp::launch_pdl(kb_gcells_recompose<double, 64>, grid, 256, 0, s, jobs, refs, unit0, nrefs,
                                                                            total);
}

}  // namespace hp
