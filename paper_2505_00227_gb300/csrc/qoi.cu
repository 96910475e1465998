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

// V_hat into out, and per block the largest pointwise bound with its first
// point (best[2 block] = bound bits, best[2 block + 1] = point)
__global__ void __launch_bounds__(256) k_vtotal_bound(const float* __restrict__ vx,
                                                      const float* __restrict__ vy,
                                                      const float* __restrict__ vz, uint64_t N,
                                                      double e0, double e1, double e2,
                                                      float* __restrict__ out,
                                                      unsigned long long* __restrict__ best) {
  hp::pdl_enter();
  __shared__ unsigned long long s_b[8], s_i[8];
  unsigned long long bb = 0, bi = ~0ull;  // bounds are >= 0: their bits order them
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float x = vx[i], y = vy[i], z = vz[i];
    out[i] = __double2float_rn(vtotal(x, y, z));
    const unsigned long long b =
        (unsigned long long)__double_as_longlong(vtotal_point_bound(x, y, z, e0, e1, e2));
    if (bi == ~0ull || b > bb) bb = b, bi = i;  // a thread's points ascend: keep the first
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(HP_FULL, bb, o), oi = __shfl_xor_sync(HP_FULL, bi, o);
    if (oi != ~0ull && (bi == ~0ull || ob > bb || (ob == bb && oi < bi))) bb = ob, bi = oi;
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) s_b[w] = bb, s_i[w] = bi;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < 8; k++)
      if (s_i[k] != ~0ull && (bi == ~0ull || s_b[k] > bb || (s_b[k] == bb && s_i[k] < bi)))
        bb = s_b[k], bi = s_i[k];
    best[2 * blockIdx.x] = bb;
    best[2 * blockIdx.x + 1] = bi;
  }
}

__global__ void k_vtotal_bound_final(unsigned long long* best, uint32_t nblocks) {
  hp::pdl_enter();
  unsigned long long bb = 0, bi = ~0ull;
  for (uint32_t k = 0; k < nblocks; k++)
    if (best[2 * k + 1] != ~0ull && (bi == ~0ull || best[2 * k] > bb ||
                                     (best[2 * k] == bb && best[2 * k + 1] < bi)))
      bb = best[2 * k], bi = best[2 * k + 1];
  best[0] = bb;
  best[1] = bi;
}

uint32_t vtotal_bound_blocks(uint64_t N) { return qoi_grid(N, 4); }

void launch_vtotal_bound(const float* vx, const float* vy, const float* vz, uint64_t N,
                         const double e[3], float* out, unsigned long long* best, cstream s) {
  const uint32_t g = vtotal_bound_blocks(N);
  hp::note_launch(), hp::launch_pdl(k_vtotal_bound, g, 256, 0, s, vx, vy, vz, N, e[0], e[1], e[2],
                                    out, best);
  hp::note_launch(), hp::launch_pdl(k_vtotal_bound_final, 1, 1, 0, s, best, g);
}

}  // namespace hp
