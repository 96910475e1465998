// Velocity-magnitude QoI (Sec. 6.2): |v| = sqrt(vx^2 + vy^2 + vz^2) evaluated in
// FP32 with one IEEE rounding per operation (no contraction), so that the
// value and its range are reproducible and the QoI error bound can account
// for the evaluation error.
#include "dev_common.cuh"

namespace hp {

__device__ __forceinline__ float vmag(float x, float y, float z) {
  float s = __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y));
  s = __fadd_rn(s, __fmul_rn(z, z));
  return __fsqrt_rn(s);
}

__global__ void __launch_bounds__(256) k_vmag_range(const float* __restrict__ vx,
                                                    const float* __restrict__ vy,
                                                    const float* __restrict__ vz, uint64_t N,
                                                    unsigned int* qr) {
  hp::pdl_enter();
  uint32_t lo = 0x7f800000u, hi = 0;  // non-negative floats order as their bits
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t q = __float_as_uint(vmag(vx[i], vy[i], vz[i]));
    lo = q < lo ? q : lo;
    hi = q > hi ? q : hi;
  }
  lo = __reduce_min_sync(HP_FULL, lo);
  hi = __reduce_max_sync(HP_FULL, hi);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(qr, lo);
    atomicMax(qr + 1, hi);
  }
}

__global__ void k_vmag_range_init(unsigned int* qr) {
  hp::pdl_enter();
  qr[0] = 0x7f800000u;
  qr[1] = 0;
}

void launch_vmag_range(const float* vx, const float* vy, const float* vz, uint64_t N,
                       float* qrange, cstream s) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t blocks = (N + 255) / 256, cap = (uint64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  hp::note_launch(), hp::launch_pdl(k_vmag_range_init, 1, 1, 0, s, (unsigned int*)qrange);
  hp::note_launch(), hp::launch_pdl(k_vmag_range, (unsigned)blocks, 256, 0, s, vx, vy, vz, N,
                                    (unsigned int*)qrange);
}

__global__ void __launch_bounds__(256) k_vmag(const float* __restrict__ vx, const float* __restrict__ vy,
                                              const float* __restrict__ vz, uint64_t N,
                                              float* __restrict__ out) {
  hp::pdl_enter();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = vmag(vx[i], vy[i], vz[i]);
}

void launch_vmag(const float* vx, const float* vy, const float* vz, uint64_t N, float* out,
                 cstream s) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t blocks = (N + 255) / 256, cap = (uint64_t)sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  hp::note_launch(), hp::launch_pdl(k_vmag, (unsigned)blocks, 256, 0, s, vx, vy, vz, N, out);
}

// ----------------------------------------- total velocity V = vx^2 + vy^2 + vz^2
// Evaluated in FP64 (squares of FP32 values are exact; two additions round),
// every operation an explicit round-to-nearest: the same numbers as the
// pointwise bound of the iterated QoI retrieval (Sec. 6.2, Algorithm 3).
__device__ __forceinline__ double vtotal(float x, float y, float z) {
  const double a = __dmul_rn((double)x, (double)x), b = __dmul_rn((double)y, (double)y);
  const double c = __dmul_rn((double)z, (double)z);
  return __dadd_rn(__dadd_rn(a, b), c);
}

// float(V_hat) without the FP64 pipe where that is provably the same value.
// With |x|, |y|, |z| each 0 or in [2^-32, 2^60], the squares are split exactly
// into FP32 pairs (x^2 = ah + al by one FMA) and summed with two exact
// two-sums: V = s2 + L exactly, L a sum of five terms of at most 3 2^-24 V in
// total, so its FP32 rounding errs by < 2^-44 V.  r = RN32(s2 + L) and the
// residual d ~ V - r (d's own rounding < 2^-25 ulp(r)); the FP64 V_hat is
// within 2^-51 V of V, so V_hat - r = d + err with |err| < 2^-19 ulp(r).  When
// d + err stays strictly inside r's rounding interval (half an ulp above r; half
// or, at a power of two, a quarter of an ulp below) RN32(V_hat) = r; otherwise
// (within 2^-19 ulp of a midpoint, a tie, or the ranges left out) the FP64
// evaluation decides.
__device__ __forceinline__ float vtotal_f32(float x, float y, float z) {
  const float ax = fabsf(x), ay = fabsf(y), az = fabsf(z);
  const bool in = (ax == 0.0f || (ax >= 0x1p-32f && ax <= 0x1p60f)) &&
                  (ay == 0.0f || (ay >= 0x1p-32f && ay <= 0x1p60f)) &&
                  (az == 0.0f || (az >= 0x1p-32f && az <= 0x1p60f));
  if (in) {
    const float ah = __fmul_rn(x, x), al = __fmaf_rn(x, x, -ah);
    const float bh = __fmul_rn(y, y), bl = __fmaf_rn(y, y, -bh);
    const float ch = __fmul_rn(z, z), cl = __fmaf_rn(z, z, -ch);
    const float s1 = __fadd_rn(ah, bh), t1 = __fsub_rn(s1, ah);
    const float e1 = __fadd_rn(__fsub_rn(ah, __fsub_rn(s1, t1)), __fsub_rn(bh, t1));
    const float s2 = __fadd_rn(s1, ch), t2 = __fsub_rn(s2, s1);
    const float e2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, t2)), __fsub_rn(ch, t2));
    if (s2 == 0.0f) return 0.0f;  // all three zero
    const float L = __fadd_rn(__fadd_rn(__fadd_rn(al, bl), __fadd_rn(cl, e1)), e2);
    const float r = __fadd_rn(s2, L);
    const float d = __fadd_rn(__fsub_rn(s2, r), L);  // s2 - r is exact
    const uint32_t rb = __float_as_uint(r);
    const float u = __uint_as_float(((rb >> 23) - 23u) << 23);  // ulp(r); r >= 2^-64
    const float m = d >= 0.0f ? __fmul_rn(u, 0.5f - 0x1p-19f)
                              : __fmul_rn(u, ((rb & 0x7fffffu) ? 0.5f : 0.25f) - 0x1p-19f);
    if (fabsf(d) < m) return r;
  }
  return __double2float_rn(vtotal(x, y, z));
}

// bound on |float(V_hat) - V| at one point for |x_hat_i - x_i| <= e_i:
// sum of 2 |x_hat| e + e^2, the FP32 rounding of V_hat (relative 2^-24, 2^-150
// absolute below the normal range, infinite past the FP32 range) and the FP64
// additions forming V_hat (2^-50 V_hat)
__device__ __forceinline__ double vtotal_point_bound(float x, float y, float z, double e0,
                                                     double e1, double e2) {
  const float xs[3] = {x, y, z};
  const double es[3] = {e0, e1, e2};
  double b = 0.0;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    double t = __dmul_rn(2.0, fabs((double)xs[i]));
    t = __dmul_rn(t, es[i]);
    const double u = __dmul_rn(es[i], es[i]);
    t = __dadd_rn(t, u);
    b = __dadd_rn(b, t);
  }
  const double v = vtotal(x, y, z);
  if (v > 0x1.fffffep127) return __longlong_as_double(0x7ff0000000000000ll);  // +inf
  b = __dadd_rn(b, __dmul_rn(v, 0x1p-24));
  if (v != 0.0) b = __dadd_rn(b, 0x1p-150);
  b = __dadd_rn(b, __dmul_rn(v, 0x1p-50));
  return b;
}

// V range: non-negative doubles order as their bits
__global__ void __launch_bounds__(256) k_vtotal_range(const float* __restrict__ vx,
                                                      const float* __restrict__ vy,
                                                      const float* __restrict__ vz, uint64_t N,
                                                      unsigned long long* vr) {
  hp::pdl_enter();
  unsigned long long lo = 0x7ff0000000000000ull, hi = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long q = (unsigned long long)__double_as_longlong(vtotal(vx[i], vy[i], vz[i]));
    lo = q < lo ? q : lo;
    hi = q > hi ? q : hi;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(HP_FULL, lo, o), b = __shfl_xor_sync(HP_FULL, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(vr, lo);
    atomicMax(vr + 1, hi);
  }
}

__global__ void k_vtotal_range_init(unsigned long long* vr) {
  hp::pdl_enter();
  vr[0] = 0x7ff0000000000000ull;
  vr[1] = 0;
}

static uint32_t qoi_grid(uint64_t N, uint32_t per_sm) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t blocks = (N + 255) / 256, cap = (uint64_t)sms * per_sm;
  if (blocks > cap) blocks = cap;
  return blocks ? (uint32_t)blocks : 1u;
}

void launch_vtotal_range(const float* vx, const float* vy, const float* vz, uint64_t N,
                         double* vrange, cstream s) {
  unsigned long long* vr = reinterpret_cast<unsigned long long*>(vrange);
  hp::note_launch(), hp::launch_pdl(k_vtotal_range_init, 1, 1, 0, s, vr);
  hp::note_launch(), hp::launch_pdl(k_vtotal_range, qoi_grid(N, 8), 256, 0, s, vx, vy, vz, N, vr);
}

// The largest pointwise bound only decides the iteration, so the FP64 bound is
// evaluated only where it can be the largest.  A bracket lo <= b <= hi of the
// FP64 bound b (vtotal_point_bound) in FP32 with directed rounding: the same
// terms over the real numbers, with e_i rounded down (up), widened by 2^-20
// relative (the FP64 evaluation rounds a dozen times, each within 2^-53) and by
// the smallest FP32 subnormal (underflow, the 2^-150 term).  Overflow gives
// hi = +inf (a candidate) and lo <= FLT_MAX, below b = +inf.  Pass 1 writes
// V_hat and each block's largest lo; pass 2 takes T = max lo <= max b and
// evaluates b exactly at the points with hi >= T, which include every point
// whose b equals max b.  An FP64 V_hat above FLT_MAX (b = +inf) needs V within
// 2^-52 relative of FLT_MAX, so hi is +inf from V >= 0x1.fffp127 on.
__device__ __forceinline__ float vtotal_bound_lo(float x, float y, float z, const float el[3]) {
  const float xs[3] = {x, y, z};
  float b = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    const float t = __fmul_rd(__fmul_rd(2.0f, fabsf(xs[i])), el[i]);
    b = __fadd_rd(b, __fadd_rd(t, __fmul_rd(el[i], el[i])));
  }
  const float v = __fadd_rd(__fadd_rd(__fmul_rd(x, x), __fmul_rd(y, y)), __fmul_rd(z, z));
  b = __fadd_rd(b, __fmul_rd(v, 0x1p-24f));
  b = __fadd_rd(b, __fmul_rd(v, 0x1p-50f));
  b = __fsub_rd(__fmul_rd(b, 1.0f - 0x1p-20f), 0x1p-149f);
  return b > 0.0f ? b : 0.0f;  // (a NaN gives 0)
}

__device__ __forceinline__ float vtotal_bound_hi(float x, float y, float z, const float eh[3]) {
  const float xs[3] = {x, y, z};
  float b = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    const float t = __fmul_ru(__fmul_ru(2.0f, fabsf(xs[i])), eh[i]);
    b = __fadd_ru(b, __fadd_ru(t, __fmul_ru(eh[i], eh[i])));
  }
  const float v = __fadd_ru(__fadd_ru(__fmul_ru(x, x), __fmul_ru(y, y)), __fmul_ru(z, z));
  // the FP64 V_hat can round past FLT_MAX (b = +inf) from just below it
  if (v > 0x1.fffp127f) return __int_as_float(0x7f800000);
  b = __fadd_ru(b, __fmul_ru(v, 0x1p-24f));
  b = __fadd_ru(b, 0x1p-149f);
  b = __fadd_ru(b, __fmul_ru(v, 0x1p-50f));
  return __fadd_ru(__fmul_ru(b, 1.0f + 0x1p-20f), 0x1p-149f);
}

// A thread's points in ascending order: four consecutive points per step with
// 16-byte loads when the arrays allow it, then the tail one at a time.
// f(i, x, y, z) per point.
template <typename F>
__device__ __forceinline__ void vtotal_points(const float* __restrict__ vx,
                                              const float* __restrict__ vy,
                                              const float* __restrict__ vz, uint64_t N,
                                              bool vec, F&& f) {
  const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t st = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n4 = vec ? N / 4 : 0;
  for (uint64_t g = t0; g < n4; g += st) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(vx) + g);
    const float4 b = __ldg(reinterpret_cast<const float4*>(vy) + g);
    const float4 c = __ldg(reinterpret_cast<const float4*>(vz) + g);
    f(4 * g, a.x, b.x, c.x);
    f(4 * g + 1, a.y, b.y, c.y);
    f(4 * g + 2, a.z, b.z, c.z);
    f(4 * g + 3, a.w, b.w, c.w);
  }
  for (uint64_t i = 4 * n4 + t0; i < N; i += st) f(i, vx[i], vy[i], vz[i]);
}

__device__ __forceinline__ bool aligned16(const void* a, const void* b, const void* c,
                                          const void* d) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
           reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(d)) & 15u) == 0;
}

// pass 1: V_hat into out, lo_part[block] = the block's largest lo
__global__ void __launch_bounds__(256) k_vtotal_value(const float* __restrict__ vx,
                                                      const float* __restrict__ vy,
                                                      const float* __restrict__ vz, uint64_t N,
                                                      const double* e0p, const double* e1p,
                                                      const double* e2p, float* __restrict__ out,
                                                      float* __restrict__ lo_part) {
  hp::pdl_enter();
  __shared__ float s_lo[8];
  const double e0 = *e0p, e1 = *e1p, e2 = *e2p;
  const float el[3] = {__double2float_rd(e0), __double2float_rd(e1), __double2float_rd(e2)};
  float lo = 0.0f;
  const bool vec = aligned16(vx, vy, vz, out);
  vtotal_points(vx, vy, vz, N, vec, [&](uint64_t i, float x, float y, float z) {
    out[i] = vtotal_f32(x, y, z);
    lo = fmaxf(lo, vtotal_bound_lo(x, y, z, el));
  });
#pragma unroll
  for (int o = 16; o; o >>= 1) lo = fmaxf(lo, __shfl_xor_sync(HP_FULL, lo, o));
  if ((threadIdx.x & 31) == 0) s_lo[threadIdx.x >> 5] = lo;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < 8; k++) lo = fmaxf(lo, s_lo[k]);
    lo_part[blockIdx.x] = lo;
  }
}

// (b, i) beats (bb, bi): a valid point with a larger bound, or the same bound at
// an earlier point (bounds are >= 0, so their bits order them)
__device__ __forceinline__ bool vtotal_better(unsigned long long b, unsigned long long i,
                                              unsigned long long bb, unsigned long long bi) {
  return i != ~0ull && (bi == ~0ull || b > bb || (b == bb && i < bi));
}

__device__ __forceinline__ void vtotal_warp_best(unsigned long long& bb, unsigned long long& bi) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(HP_FULL, bb, o), oi = __shfl_xor_sync(HP_FULL, bi, o);
    if (vtotal_better(ob, oi, bb, bi)) bb = ob, bi = oi;
  }
}

// pass 2: per block the largest FP64 pointwise bound among the candidates, with
// its first point (best[2 block] = bound bits, best[2 block + 1] = point)
__global__ void __launch_bounds__(256) k_vtotal_bound(const float* __restrict__ vx,
                                                      const float* __restrict__ vy,
                                                      const float* __restrict__ vz, uint64_t N,
                                                      const double* e0p, const double* e1p,
                                                      const double* e2p,
                                                      const float* __restrict__ lo_part,
                                                      uint32_t nparts,
                                                      unsigned long long* __restrict__ best) {
  hp::pdl_enter();
  const double e0 = *e0p, e1 = *e1p, e2 = *e2p;
  __shared__ unsigned long long s_b[8], s_i[8];
  __shared__ float s_t[8];
  float T = 0.0f;
  for (uint32_t k = threadIdx.x; k < nparts; k += blockDim.x) T = fmaxf(T, lo_part[k]);
#pragma unroll
  for (int o = 16; o; o >>= 1) T = fmaxf(T, __shfl_xor_sync(HP_FULL, T, o));
  if ((threadIdx.x & 31) == 0) s_t[threadIdx.x >> 5] = T;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 8; k++) T = fmaxf(T, s_t[k]);
  const float eh[3] = {__double2float_ru(e0), __double2float_ru(e1), __double2float_ru(e2)};
  unsigned long long bb = 0, bi = ~0ull;
  const bool vec = aligned16(vx, vy, vz, nullptr);
  vtotal_points(vx, vy, vz, N, vec, [&](uint64_t i, float x, float y, float z) {
    if (!(vtotal_bound_hi(x, y, z, eh) < T)) {  // a candidate (a NaN bracket too)
      const unsigned long long b =
          (unsigned long long)__double_as_longlong(vtotal_point_bound(x, y, z, e0, e1, e2));
      if (bi == ~0ull || b > bb) bb = b, bi = i;  // a thread's points ascend: keep the first
    }
  });
  vtotal_warp_best(bb, bi);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) s_b[w] = bb, s_i[w] = bi;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < 8; k++)
      if (vtotal_better(s_b[k], s_i[k], bb, bi)) bb = s_b[k], bi = s_i[k];
    best[2 * blockIdx.x] = bb;
    best[2 * blockIdx.x + 1] = bi;
  }
}

// the blocks' results -> best[0], best[1] (one block of 256 threads)
__global__ void __launch_bounds__(256) k_vtotal_bound_final(unsigned long long* best,
                                                            uint32_t nblocks) {
  hp::pdl_enter();
  __shared__ unsigned long long s_b[8], s_i[8];
  unsigned long long bb = 0, bi = ~0ull;
  for (uint32_t k = threadIdx.x; k < nblocks; k += blockDim.x)
    if (vtotal_better(best[2 * k], best[2 * k + 1], bb, bi)) bb = best[2 * k], bi = best[2 * k + 1];
  vtotal_warp_best(bb, bi);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) s_b[w] = bb, s_i[w] = bi;
  __syncthreads();  // every read of best[] is done before it is overwritten
  if (threadIdx.x == 0) {
    for (int k = 1; k < 8; k++)
      if (vtotal_better(s_b[k], s_i[k], bb, bi)) bb = s_b[k], bi = s_i[k];
    best[0] = bb;
    best[1] = bi;
  }
}

uint32_t vtotal_bound_blocks(uint64_t N) { return qoi_grid(N, 4); }

// best[2 g] (u64), the blocks' lower bounds lo_part[g] (float), then 32 bytes
// for a caller's copy of e[3] (vtotal_bound_e)
uint64_t vtotal_bound_scratch(uint64_t N) { return 24ull * vtotal_bound_blocks(N) + 32; }

double* vtotal_bound_e(unsigned long long* best, uint64_t N) {
  return reinterpret_cast<double*>(reinterpret_cast<uint8_t*>(best) + 24ull * vtotal_bound_blocks(N));
}

void launch_vtotal_bound(const float* vx, const float* vy, const float* vz, uint64_t N,
                         const double* const e[3], float* out, unsigned long long* best,
                         cstream s) {
  const uint32_t g = vtotal_bound_blocks(N);
  float* lo_part = reinterpret_cast<float*>(best + 2 * (size_t)g);
  hp::note_launch(), hp::launch_pdl(k_vtotal_value, g, 256, 0, s, vx, vy, vz, N, e[0], e[1], e[2],
                                    out, lo_part);
  hp::note_launch(), hp::launch_pdl(k_vtotal_bound, g, 256, 0, s, vx, vy, vz, N, e[0], e[1], e[2],
                                    (const float*)lo_part, g, best);
  hp::note_launch(), hp::launch_pdl(k_vtotal_bound_final, 1, 256, 0, s, best, g);
}

}  // namespace hp
