// Field statistics: max|f|, min f, max f in one streaming pass, then the
// exponent E_f that fixes the alignment unit U = 2^(E_f-48) (Sec. 4, the
// "AlignExponent" step of Algorithm 1 needs the maximum exponent first).
#include <algorithm>
#include <type_traits>

#include "dev_common.cuh"

namespace hp {

__global__ void k_meta_init(FieldMeta* meta, int dtype, int B, int nlev, int ngroups) {
  hp::pdl_enter();
  meta->status = 0;
  meta->dtype = dtype;
  meta->B = B;
  meta->nlev = nlev;
  meta->ngroups = ngroups;
  meta->key_absmax = 0;
  meta->key_min = ~0ull;
  meta->key_max = 0;
  meta->floored = 0;
  meta->lsb_min = 0x7fffffff;
  for (int l = 0; l < HP_MAX_LEVELS; l++) {
    meta->m8[l] = 0;
    meta->lowbits[l] = 0;
    meta->m8est[l] = 0;
    meta->bl[l] = 0;
    meta->exact[l] = 1;
    meta->fetched[l] = 0;
    meta->cur[l] = 0;
  }
  meta->seq_len = 0;
}

void launch_meta_init(FieldMeta* meta, int dtype, int B, int nlev, int ngroups, cstream s) {
  hp::note_launch(), hp::launch_pdl(k_meta_init, 1, 1, 0, s, meta, dtype, B, nlev, ngroups);
}

// Small device -> page-locked host copies written by a kernel (stores through
// the mapped host pointer): they do not queue on the copy engines behind large
// transfers of other streams.  Two ranges per launch, each in 16-byte units
// when both ends allow it, else in words; a few CTAs so that every thread has
// one or two stores in flight.
__device__ __forceinline__ void to_host_range(const uint32_t* __restrict__ a, uint32_t* b,
                                              uint32_t nw) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, T = gridDim.x * blockDim.x;
  if (((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0) {
    const uint4* a4 = reinterpret_cast<const uint4*>(a);
    uint4* b4 = reinterpret_cast<uint4*>(b);
    for (uint32_t i = t; i < nw / 4; i += T) b4[i] = a4[i];
    for (uint32_t i = nw / 4 * 4 + t; i < nw; i += T) b[i] = a[i];
  } else {
    for (uint32_t i = t; i < nw; i += T) b[i] = a[i];
  }
}

__global__ void __launch_bounds__(256) k_to_host(const uint32_t* __restrict__ a, uint32_t* b,
                                                 uint32_t na, const uint32_t* __restrict__ c,
                                                 uint32_t* d, uint32_t nc) {
  hp::pdl_enter();
  to_host_range(a, b, na);
  to_host_range(c, d, nc);
}

void launch_to_host(const void* a, void* b, size_t na_bytes, const void* c, void* d,
                    size_t nc_bytes, cstream s) {
  const size_t units = (na_bytes + nc_bytes) / 16 + 1;
  const unsigned blocks = (unsigned)std::min<size_t>(16, (units + 255) / 256);
  hp::note_launch(), hp::launch_pdl(k_to_host, blocks, 256, 0, s, (const uint32_t*)a, (uint32_t*)b,
                                                      (uint32_t)(na_bytes / 4), (const uint32_t*)c,
                                                      (uint32_t*)d, (uint32_t)(nc_bytes / 4));
}

// 128-bit vector loads over the bulk (four in flight per thread), scalar loads
// for the tail; FP32 keys are compared as 32-bit integers.
template <typename T>
__global__ void __launch_bounds__(256) k_stats(const T* __restrict__ f, uint64_t N,
                                               int aligned, FieldMeta* meta) {
  hp::pdl_enter();
  constexpr int VEC = 16 / sizeof(T), UN = 4;
  typedef typename std::conditional<sizeof(T) == 4, uint32_t, uint64_t>::type K;
  K am = 0, kn = (K)~(K)0, kx = 0;
  auto visit = [&](T v) {
    const K a = (K)abs_key(v), o = (K)order_key(v);
    am = a > am ? a : am;
    kn = o < kn ? o : kn;
    kx = o > kx ? o : kx;
  };
  const uint64_t nvec = aligned ? N / VEC : 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint4* fv = reinterpret_cast<const uint4*>(f);
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (UN - 1) * stride < nvec; i += UN * stride) {
    uint4 w[UN];
#pragma unroll
    for (int u = 0; u < UN; u++) w[u] = __ldcs(fv + i + u * stride);
#pragma unroll
    for (int u = 0; u < UN; u++) {
      T v[VEC];
      memcpy(v, &w[u], 16);
#pragma unroll
      for (int k = 0; k < VEC; k++) visit(v[k]);
    }
  }
  for (; i < nvec; i += stride) {
    const uint4 w = __ldcs(fv + i);
    T v[VEC];
    memcpy(v, &w, 16);
#pragma unroll
    for (int k = 0; k < VEC; k++) visit(v[k]);
  }
  for (uint64_t t = nvec * VEC + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += stride)
    visit(f[t]);
  uint64_t amax = am, kmin = kn == (K)~(K)0 ? ~0ull : (uint64_t)kn, kmax = kx;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    uint64_t a = __shfl_xor_sync(HP_FULL, amax, o);
    uint64_t b = __shfl_xor_sync(HP_FULL, kmin, o);
    uint64_t c = __shfl_xor_sync(HP_FULL, kmax, o);
    amax = a > amax ? a : amax;
    kmin = b < kmin ? b : kmin;
    kmax = c > kmax ? c : kmax;
  }
  __shared__ uint64_t sa[8], sb[8], sc[8];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sa[w] = amax;
    sb[w] = kmin;
    sc[w] = kmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); k++) {
      amax = sa[k] > amax ? sa[k] : amax;
      kmin = sb[k] < kmin ? sb[k] : kmin;
      kmax = sc[k] > kmax ? sc[k] : kmax;
    }
    atomicMax((unsigned long long*)&meta->key_absmax, (unsigned long long)amax);
    atomicMin((unsigned long long*)&meta->key_min, (unsigned long long)kmin);
    atomicMax((unsigned long long*)&meta->key_max, (unsigned long long)kmax);
  }
}

void launch_stats(const void* f, uint64_t N, int dtype, FieldMeta* meta, cstream s) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t per = dtype == 0 ? 4 : 2;
  uint64_t want = (N / per + 255) / 256;
  uint64_t grid = (uint64_t)sms * 8;
  if (want < grid) grid = want ? want : 1;
  int aligned = ((uintptr_t)f & 15) == 0;
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(k_stats<float>, (unsigned)grid, 256, 0, s, (const float*)f, N,
                                      aligned, meta);
  else
    hp::note_launch(), hp::launch_pdl(k_stats<double>, (unsigned)grid, 256, 0, s, (const double*)f,
                                      N, aligned, meta);
}

__device__ double key_to_double(uint64_t k, int dtype) {
  if (dtype == 0) {
    uint32_t u = (uint32_t)k;
    u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    return (double)__uint_as_float(u);
  }
  uint64_t u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)u);
}

// E_f = smallest integer with max|f| < 2^E_f (0 for an all-zero field);
// rejects non-finite values and magnitudes outside the supported range.
__device__ void stats_finalize(FieldMeta* meta) {
  int dtype = meta->dtype;
  uint64_t a = meta->key_absmax;
  int E = 0;
  bool bad = false;
  if (dtype == 0) {
    uint32_t u = (uint32_t)a;
    bad = u >= 0x7f800000u;
    uint32_t e = u >> 23, m = u & 0x7fffffu;
    if (u == 0) E = 0;
    else if (e == 0) E = (32 - __clz((int)m)) - 149;
    else E = (int)e - 126;
    if (E > 121) bad = true;
    meta->maxabs = (double)__uint_as_float(u);
  } else {
    bad = a >= 0x7ff0000000000000ull;
    uint32_t e = (uint32_t)(a >> 52);
    uint64_t m = a & 0xfffffffffffffull;
    if (a == 0) E = 0;
    else if (e == 0) E = bitlen64(m) - 1074;
    else E = (int)e - 1022;
    if (E > 1017 || (a != 0 && E < -1000)) bad = true;
    meta->maxabs = __longlong_as_double((long long)a);
  }
  meta->E_f = E;
  meta->vmin = key_to_double(meta->key_min, dtype);
  meta->vmax = key_to_double(meta->key_max, dtype);
  meta->range = __dsub_rn(meta->vmax, meta->vmin);
  if (bad) meta->status = -1;  // HPMDR_ERR_ARG
}

__global__ void k_stats_finalize(FieldMeta* meta) {
  hp::pdl_enter();
  stats_finalize(meta);
}

void launch_stats_finalize(FieldMeta* meta, cstream s) {
  hp::note_launch(), hp::launch_pdl(k_stats_finalize, 1, 1, 0, s, meta);
}

// ------------------------------------------------------------------ batched
// 16-byte copy of n bytes (both 16-byte aligned, n a multiple of 16)
__device__ __forceinline__ void block_copy16(void* dst, const void* src, size_t n) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (size_t i = threadIdx.x; i < n / 16; i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ void block_zero16(void* dst, size_t n) {
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (size_t i = threadIdx.x; i < n / 16; i += blockDim.x) d[i] = make_uint4(0, 0, 0, 0);
}

static_assert(sizeof(FieldMeta) % 16 == 0, "FieldMeta is copied in 16-byte words");
static_assert(sizeof(RetrieveDev) % 16 == 0, "RetrieveDev is copied in 16-byte words");

// one CTA per job: the plan's initial metadata, zeroed histograms and RLE sizes
__global__ void __launch_bounds__(256) kb_init(const BatchJob* __restrict__ jobs) {
  hp::pdl_enter();
  const BatchJob& J = jobs[blockIdx.x];
  block_copy16(J.meta, J.meta0, sizeof(FieldMeta));
  block_zero16(J.hist, 1024ull * J.ngt);
  for (uint32_t g = threadIdx.x; g < J.ngt; g += blockDim.x) J.gcost[g] = 0ull;
}

void launch_b_init(const BatchJob* jobs, uint32_t njobs, cstream s) {
  if (njobs) hp::note_launch(), hp::launch_pdl(kb_init, njobs, 256, 0, s, jobs);
}

// unit = `seg` consecutive values of one field (seg a multiple of 256 * 16 bytes)
template <typename T>
__global__ void __launch_bounds__(256) kb_stats(const BatchJob* __restrict__ jobs,
                                                const uint32_t* __restrict__ unit0, uint32_t njobs,
                                                uint32_t total, uint32_t seg) {
  hp::pdl_enter();
  constexpr int VEC = 16 / sizeof(T);
  __shared__ uint64_t sa[8], sb[8], sc[8];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t j = unit_owner(unit0, njobs, u);
    const BatchJob& J = jobs[j];
    const uint64_t a = (uint64_t)(u - unit0[j]) * seg, b = min(J.N, a + seg);
    const T* f = reinterpret_cast<const T*>(J.f);
    uint64_t amax = 0, kmin = ~0ull, kmax = 0;
    const uint64_t va = a / VEC, vb = b / VEC;
    const uint4* fv = reinterpret_cast<const uint4*>(f);
    for (uint64_t i = va + threadIdx.x; i < vb; i += blockDim.x) {
      uint4 x = __ldcs(fv + i);
      T v[VEC];
      memcpy(v, &x, 16);
#pragma unroll
      for (int k = 0; k < VEC; k++) {
        uint64_t p = abs_key(v[k]), o = order_key(v[k]);
        amax = p > amax ? p : amax;
        kmin = o < kmin ? o : kmin;
        kmax = o > kmax ? o : kmax;
      }
    }
    for (uint64_t i = vb * VEC + threadIdx.x; i < b; i += blockDim.x) {
      T v = f[i];
      uint64_t p = abs_key(v), o = order_key(v);
      amax = p > amax ? p : amax;
      kmin = o < kmin ? o : kmin;
      kmax = o > kmax ? o : kmax;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      uint64_t x = __shfl_xor_sync(HP_FULL, amax, o);
      uint64_t y = __shfl_xor_sync(HP_FULL, kmin, o);
      uint64_t z = __shfl_xor_sync(HP_FULL, kmax, o);
      amax = x > amax ? x : amax;
      kmin = y < kmin ? y : kmin;
      kmax = z > kmax ? z : kmax;
    }
    if (lane == 0) {
      sa[w] = amax;
      sb[w] = kmin;
      sc[w] = kmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 1; k < (int)(blockDim.x >> 5); k++) {
        amax = sa[k] > amax ? sa[k] : amax;
        kmin = sb[k] < kmin ? sb[k] : kmin;
        kmax = sc[k] > kmax ? sc[k] : kmax;
      }
      atomicMax((unsigned long long*)&J.meta->key_absmax, (unsigned long long)amax);
      atomicMin((unsigned long long*)&J.meta->key_min, (unsigned long long)kmin);
      atomicMax((unsigned long long*)&J.meta->key_max, (unsigned long long)kmax);
    }
    __syncthreads();
  }
}

void launch_b_stats(const BatchJob* jobs, const uint32_t* unit0, uint32_t njobs, uint32_t total,
                    uint32_t seg, int dtype, uint32_t grid, cstream s) {
  if (!total) return;
  if (grid > total) grid = total;
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(kb_stats<float>, grid, 256, 0, s, jobs, unit0, njobs, total,
                                      seg);
  else
    hp::note_launch(), hp::launch_pdl(kb_stats<double>, grid, 256, 0, s, jobs, unit0, njobs, total,
                                      seg);
}

__global__ void kb_finalize(const BatchJob* __restrict__ jobs, uint32_t njobs) {
  hp::pdl_enter();
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < njobs) stats_finalize(jobs[j].meta);
}

void launch_b_finalize(const BatchJob* jobs, uint32_t njobs, cstream s) {
  if (njobs) hp::note_launch(), hp::launch_pdl(kb_finalize, (njobs + 63) / 64, 64, 0, s, jobs,
                                               njobs);
}

__global__ void __launch_bounds__(256) kb_gather(const BatchJob* __restrict__ jobs,
                                                 FieldMeta* metas, RetrieveDev* rds,
                                                 int32_t* statuses) {
  hp::pdl_enter();
  const BatchJob& J = jobs[blockIdx.x];
  if (metas) block_copy16(metas + blockIdx.x, J.meta, sizeof(FieldMeta));
  if (rds) block_copy16(rds + blockIdx.x, J.rd, sizeof(RetrieveDev));
  if (statuses && threadIdx.x == 0) statuses[blockIdx.x] = J.meta->status;
}

void launch_b_gather(const BatchJob* jobs, uint32_t njobs, FieldMeta* metas, RetrieveDev* rds,
                     int32_t* statuses, cstream s) {
  if (njobs) hp::note_launch(), hp::launch_pdl(kb_gather, njobs, 256, 0, s, jobs, metas, rds,
                                               statuses);
}

}  // namespace hp
