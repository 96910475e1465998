// Device helpers shared by the sm_103a kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

#define HP_FULL 0xffffffffu

namespace hp {

// ------------------------------------------------- programmatic dependent launch
// Every kernel is launched with programmatic stream serialization and starts by
// waiting for the grid before it in the stream (griddepcontrol.wait: that grid
// has completed and its writes are visible).  No kernel signals its dependents
// early, so the next kernel is launched as this one's CTAs exit, and its launch
// and CTA scheduling overlap the end of this grid instead of following its
// completion; its CTAs only begin work after this grid has completed, so the
// stream order of every read and write is that of ordinary launches.  (Signals
// at kernel start were measured slower: waiting CTAs of the next kernel then
// hold SM resources while this one's last wave runs.)
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------- division
__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) l++;
  f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s = l;  // shifts derived from l: s1 = min(l,1), s2 = max(l-1,0)
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  uint32_t t = __umulhi(f.m, n);
  uint32_t s1 = f.s ? 1u : 0u, s2 = f.s ? f.s - 1u : 0u;
  return (t + ((n - t) >> s1)) >> s2;
}

// --------------------------------------------------------- bit transposition
// In-register 32x32 bit-matrix transpose: on return a[c] bit r = old a[r] bit c.
// Recursive off-diagonal block swap at scales 16, 8, 4, 2, 1.
__device__ __forceinline__ void transpose32(uint32_t a[32]) {
#define HP_TSTAGE(S, M)                                            \
  _Pragma("unroll") for (int i = 0; i < 32; i++) {                \
    if ((i & S) == 0) {                                            \
      uint32_t t = ((a[i] >> S) ^ a[i + S]) & (M);                 \
      a[i + S] ^= t;                                               \
      a[i] ^= t << S;                                              \
    }                                                              \
  }
  // the 16- and 8-bit stages move whole bytes: one byte permute per word
#pragma unroll
  for (int i = 0; i < 16; i++) {
    const uint32_t x = a[i], y = a[i + 16];
    a[i] = __byte_perm(x, y, 0x5410);       // low halves of x, y
    a[i + 16] = __byte_perm(x, y, 0x7632);  // high halves of x, y
  }
#pragma unroll
  for (int i = 0; i < 32; i++) {
    if ((i & 8) == 0) {
      const uint32_t x = a[i], y = a[i + 8];
      a[i] = __byte_perm(x, y, 0x6240);      // bytes 0, 2 of x, y interleaved
      a[i + 8] = __byte_perm(x, y, 0x7351);  // bytes 1, 3 of x, y interleaved
    }
  }
  HP_TSTAGE(4, 0x0F0F0F0Fu)
  HP_TSTAGE(2, 0x33333333u)
  HP_TSTAGE(1, 0x55555555u)
#undef HP_TSTAGE
}

// Two 16x16 bit-matrix transposes side by side, one in each 16-bit half of
// r[0..15]: on return r[c] bit i = old r[i] bit c and r[c] bit (16 + i) = old
// r[i] bit (16 + c), for i, c < 16.  With at most 16 planes (the top rows of a
// 32x32 transpose, the others zero) this gives the same result as transpose32
// at about half the cost: out[c] = r[c] << 16 (c < 16), r[c - 16] & 0xffff0000.
__device__ __forceinline__ void transpose16x2(uint32_t r[16]) {
#pragma unroll
  for (int i = 0; i < 8; i++) {  // the 8-bit stage moves whole bytes
    const uint32_t x = r[i], y = r[i + 8];
    r[i] = __byte_perm(x, y, 0x6240);
    r[i + 8] = __byte_perm(x, y, 0x7351);
  }
#define HP_T16STAGE(S, M)                                          \
  _Pragma("unroll") for (int i = 0; i < 16; i++) {                \
    if ((i & S) == 0) {                                            \
      uint32_t t = ((r[i] >> S) ^ r[i + S]) & (M);                 \
      r[i + S] ^= t;                                               \
      r[i] ^= t << S;                                              \
    }                                                              \
  }
  HP_T16STAGE(4, 0x0F0F0F0Fu)
  HP_T16STAGE(2, 0x33333333u)
  HP_T16STAGE(1, 0x55555555u)
#undef HP_T16STAGE
}

// Four 8x8 bit-matrix transposes side by side, one in each byte of r[0..7]:
// on return byte b of r[c] holds, in bit i, old r[i] bit (8 b + c).  With at
// most 8 planes the 32x32 transpose reduces to this: out[c] = byte (c >> 3) of
// r[c & 7], shifted to the top byte.
__device__ __forceinline__ void transpose8x4(uint32_t r[8]) {
#define HP_T8STAGE(S, M)                                           \
  _Pragma("unroll") for (int i = 0; i < 8; i++) {                 \
    if ((i & S) == 0) {                                            \
      uint32_t t = ((r[i] >> S) ^ r[i + S]) & (M);                 \
      r[i + S] ^= t;                                               \
      r[i] ^= t << S;                                              \
    }                                                              \
  }
  HP_T8STAGE(4, 0x0F0F0F0Fu)
  HP_T8STAGE(2, 0x33333333u)
  HP_T8STAGE(1, 0x55555555u)
#undef HP_T8STAGE
}

// ---------------------------------------------------- 32-byte accesses
// One 256-bit global access per thread (addresses 32-byte aligned): a warp's
// 32 threads then cover whole 32-byte sectors, where two 16-byte accesses at a
// 32-byte stride would touch every sector twice, half of it each time.
__device__ __forceinline__ void ld_nc_v8f(const float* p, float v[8]) {
  asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                 "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}
__device__ __forceinline__ void ld_nc_v4s64(const int64_t* p, int64_t v[4]) {
  long long a, b, c, d;
  asm volatile("ld.global.nc.v4.s64 {%0,%1,%2,%3}, [%4];"
               : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
               : "l"(p));
  v[0] = a;
  v[1] = b;
  v[2] = c;
  v[3] = d;
}
__device__ __forceinline__ void ld_nc_v4d(const double* p, double v[4]) {
  asm volatile("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
               : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
               : "l"(p));
}
__device__ __forceinline__ void st_v4d(double* p, const double v[4]) {
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]),
               "d"(v[3])
               : "memory");
}
__device__ __forceinline__ void st_v8f(float* p, const float v[8]) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void st_v4s64(int64_t* p, int64_t a, int64_t b, int64_t c, int64_t d) {
  asm volatile("st.global.v4.s64 [%0], {%1,%2,%3,%4};" ::"l"(p), "l"((long long)a),
               "l"((long long)b), "l"((long long)c), "l"((long long)d)
               : "memory");
}

// ------------------------------------------------------------- fixed point
// F = sign(v) * floor(|v| / 2^(E_f-48)), exactly, from the IEEE fields.
__device__ __forceinline__ int64_t fixed_point(float v, int E_f, uint32_t& floored) {
  uint32_t u = __float_as_uint(v);
  uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  int ee = e ? (int)e : 1;
  if (e) m |= 0x800000u;
  int s = ee - 102 - E_f;
  uint64_t mag;
  if (s >= 0) {
    mag = (uint64_t)m << s;
  } else {
    int r = -s;
    if (r >= 32) {
      mag = 0;
      floored |= (m != 0);
    } else {
      mag = m >> r;
      floored |= ((m & ((1u << r) - 1u)) != 0);
    }
  }
  return (u >> 31) ? -(int64_t)mag : (int64_t)mag;
}

// The same F for an FP32 value without the floor flag, on the floating-point
// pipes: with sc = 2^(48 - E_f) (a normal float, so -78 <= E_f), x = v sc is
// exact (|x| < 2^48; a value whose product underflows has |x| < 1 and F = 0),
// t = trunc(x / 2^24) is an integer of at most 24 bits, r = x - t 2^24 is exact
// (|r| < 2^24, the sign of x or zero) and F = trunc(x) = t 2^24 + trunc(r).
__device__ __forceinline__ int64_t fixed_point_fp(float v, float sc) {
  const float x = __fmul_rn(v, sc);
  const float t = truncf(__fmul_rn(x, 0x1p-24f));
  const float r = __fmaf_rn(t, -0x1p24f, x);
  return (int64_t)__float2int_rz(t) * 16777216ll + (int64_t)__float2int_rz(r);
}

__device__ __forceinline__ int64_t fixed_point(double v, int E_f, uint32_t& floored) {
  uint64_t u = (uint64_t)__double_as_longlong(v);
  uint32_t e = (uint32_t)((u >> 52) & 0x7ffu);
  uint64_t m = u & 0xfffffffffffffull;
  int ee = e ? (int)e : 1;
  if (e) m |= 0x10000000000000ull;
  int s = ee - 1027 - E_f;
  uint64_t mag;
  if (s >= 0) {
    mag = m << s;
  } else {
    int r = -s;
    if (r >= 64) {
      mag = 0;
      floored |= (m != 0);
    } else {
      mag = m >> r;
      floored |= ((m & ((1ull << r) - 1ull)) != 0);
    }
  }
  return (u >> 63) ? -(int64_t)mag : (int64_t)mag;
}

// ------------------------------------------------------- output conversion
// The last step of recomposition: f = RN(X) * 2^(E_f - 48), X the fixed-point
// reconstruction, RN the IEEE 754 round-to-nearest-even conversion to the
// output type followed by an exact power-of-two scale.  On this GPU the 64-bit
// integer conversions run on the narrow FP64 pipe, so the common cases are
// built without them.
//
// FP32, |X| < 2^48: X = h 2^24 + l with h = floor(X / 2^24), |h| <= 2^24, and
// 0 <= l < 2^24, both exact in FP32 by 32-bit conversions; one fused
// multiply-add rounds h 2^(24+e) + l 2^e once, and with the result normal
// (e >= -126 and X != 0) that equals RN(X) 2^e.
// (s24, s0) = (2^(24+e), 2^e); the caller has checked |X| < 2^48, e >= -126
// and E_f <= 121
__device__ __forceinline__ float fixed_to_f32_small(int64_t X, float s24, float s0) {
  const float hf = __int2float_rn((int32_t)(X >> 24));
  const float lf = __uint2float_rn((uint32_t)X & 0xffffffu);
  return __fmaf_rn(hf, s24, __fmul_rn(lf, s0));
}

__device__ __forceinline__ float fixed_to_f32(int64_t X, int E_f) {
  const int e = E_f - 48;
  if (e >= -126 && E_f <= 121) {
    const uint32_t t = (uint32_t)((uint64_t)X >> 32);
    if (t + 65536u < 131072u)  // -2^48 <= X < 2^48
      return fixed_to_f32_small(X, __int_as_float((e + 24 + 127) << 23),
                                __int_as_float((e + 127) << 23));
    return __fmul_rn(__ll2float_rn(X), __int_as_float((e + 127) << 23));
  }
  const double d = __dmul_rn(__ll2double_rn(X), __longlong_as_double((long long)(e + 1023) << 52));
  return __double2float_rn(d);
}

// FP64, |X| < 2^53 and a finite normal result: exact, so the IEEE fields are
// written directly (leading one at bit 52 of the shifted magnitude, exponent
// carried by the addition); anything else takes the conversion instructions.
__device__ __forceinline__ double fixed_to_f64(int64_t X, int E_f) {
  const int e = E_f - 48;
  const uint64_t sg = (uint64_t)(X >> 63);
  const uint64_t M = ((uint64_t)X ^ sg) - sg;
  const int lz = __clzll((long long)M);
  if (M < (1ull << 53) && e >= -1022 && 63 - lz + e <= 1023) {
    if (M == 0) return 0.0;
    const uint64_t m53 = (M << lz) >> 11;  // bit 52 set, nothing lost
    const uint64_t bits = ((uint64_t)(63 - lz + e + 1022) << 52) + m53;
    return __longlong_as_double((long long)(bits | (sg << 63)));
  }
  const double x = __ll2double_rn(X);
  if (e >= -1022) return __dmul_rn(x, __longlong_as_double((long long)(e + 1023) << 52));
  const double y = __dmul_rn(x, __longlong_as_double((long long)(-500 + 1023) << 52));
  return __dmul_rn(y, __longlong_as_double((long long)(e + 500 + 1023) << 52));
}

// ---------------------------------------------- level maximum by estimate
// (FP32 levels) a pass in FP32 bounds every detail to within 2^31 + 16 units of
// U/8 (the error analysis is beside k_cells_levelmax_est); these helpers give
// the exact floor flag of a value and turn the estimate into bl when its
// interval holds one bit length.
__device__ __forceinline__ uint32_t float_floors(float v, int E_f) {
  const uint32_t u = __float_as_uint(v), e = (u >> 23) & 0xffu;
  uint32_t m = u & 0x7fffffu;
  if (e) m |= 0x800000u;
  const int r = 102 + E_f - (int)(e ? e : 1u);  // bits of m below the unit
  if (r <= 0 || m == 0) return 0u;
  return r >= 32 ? 1u : ((m & ((1u << r) - 1u)) != 0u);
}

// The same flag on the floating-point pipes, for sc = 2^(48 - E_f) a normal
// float: x = v sc is exact unless it underflows (then |x| < 1 and v != 0 loses
// everything), and v loses bits exactly when x is not an integer.
__device__ __forceinline__ uint32_t float_floors_fp(float v, float sc) {
  const float x = __fmul_rn(v, sc);
  return (x != truncf(x) || (x == 0.0f && v != 0.0f)) ? 1u : 0u;
}

// bl from the estimate when it is unambiguous (then m8 = 2^(bl-1)); false:
// the exact pass must run
__device__ __forceinline__ bool cells_bl_from_estimate(FieldMeta* meta, int level, bool write) {
  const int E_f = meta->E_f;
  const uint32_t bits = meta->m8est[level];
  if (E_f < -90 || bits == 0u) return false;
  const double M = (double)__uint_as_float(bits) * __longlong_as_double((long long)(51 - E_f + 1023) << 52);
  const double lo = M - 0x1p33, hi = M + 0x1p33;
  if (!(lo >= 1.0)) return false;
  int el, eh;
  frexp(lo, &el);
  frexp(hi, &eh);
  if (el != eh) return false;  // the interval holds a power of two
  if (write) meta->m8[level] = 1ull << (el - 1);  // bitlen el
  return true;
}

__device__ __forceinline__ uint64_t umag(int64_t c) {
  return c < 0 ? (uint64_t)(-c) : (uint64_t)c;
}

__device__ __forceinline__ int bitlen64(uint64_t v) { return 64 - __clzll((long long)v); }

// floor(a / 2^s) for signed a (arithmetic shift is floor division on two's complement)
__device__ __forceinline__ int64_t floor_shift(int64_t a, int s) { return a >> s; }

// --------------------------------------------------------- warp reductions
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    uint64_t w = __shfl_xor_sync(HP_FULL, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__device__ __forceinline__ uint64_t warp_or_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v |= __shfl_xor_sync(HP_FULL, v, o);
  return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(HP_FULL, v, o);
  return v;
}

// ------------------------------------------------------ level node geometry
// Node j of a level: parity type t (1..7), and its coordinates in the level grid.
struct NodePos {
  int t;
  uint32_t gz, gy, gx;  // coordinates in G_h
};

__device__ __forceinline__ NodePos node_pos(const LevelDesc& L, uint32_t j) {
  NodePos p;
  int t = 1;
#pragma unroll
  for (int k = 2; k <= 7; k++) t += (j >= L.off[k]) ? 1 : 0;
  uint32_t local = j - L.off[t];
  uint32_t r = fdiv(local, L.dx[t]);
  uint32_t x = local - r * L.cnt[t][2];
  uint32_t z = fdiv(r, L.dy[t]);
  uint32_t y = r - z * L.cnt[t][1];
  p.t = t;
  p.gx = 2 * x + (t & 1);
  p.gy = 2 * y + ((t >> 1) & 1);
  p.gz = 2 * z + ((t >> 2) & 1);
  return p;
}

// lo/hi neighbour along one axis at grid coordinate c (odd), grid size G
__device__ __forceinline__ void axis_nb(uint32_t c, uint32_t G, uint32_t& lo, uint32_t& hi) {
  lo = c - 1;
  hi = (c + 1 < G) ? c + 1 : c - 1;
}

// --------------------------------------------------- ordered float keys
__device__ __forceinline__ uint64_t order_key(float v) {
  uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? (uint64_t)(~u) : (uint64_t)(u | 0x80000000u);
}
__device__ __forceinline__ uint64_t order_key(double v) {
  uint64_t u = (uint64_t)__double_as_longlong(v);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ uint64_t abs_key(float v) { return __float_as_uint(v) & 0x7fffffffu; }
__device__ __forceinline__ uint64_t abs_key(double v) {
  return (uint64_t)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// Batched launches: the job (or level entry) owning work unit u is the last
// j with unit0[j] <= u (unit0 ascending; jobs without units repeat a value)
__device__ __forceinline__ uint32_t unit_owner(const uint32_t* __restrict__ unit0, uint32_t n,
                                               uint32_t u) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(unit0 + mid) <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

}  // namespace hp
