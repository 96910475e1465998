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
  hp::note_launch(), k_vmag_range_init<<<1, 1, 0, s>>>((unsigned int*)qrange);
  hp::note_launch(), k_vmag_range<<<(unsigned)blocks, 256, 0, s>>>(vx, vy, vz, N, (unsigned int*)qrange);
}

__global__ void __launch_bounds__(256) k_vmag(const float* __restrict__ vx, const float* __restrict__ vy,
                                              const float* __restrict__ vz, uint64_t N,
                                              float* __restrict__ out) {
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
  hp::note_launch(), k_vmag<<<(unsigned)blocks, 256, 0, s>>>(vx, vy, vz, N, out);
}

}  // namespace hp
