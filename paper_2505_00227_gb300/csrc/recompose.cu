// Recomposition from the fetched bitplanes (Sec. 3 reverse path; Algorithm 3
// `recompose`).  Coarse to fine, level by level: the top k = 4 g_l magnitude
// planes (and the sign plane) give q_hat by the inverse register-block
// transpose, c8_hat = +-(q_hat aligned back by the level exponent), and a node
// of parity type t with odd axes O becomes
//   X_hat = floor((c8_hat * 2^|O| + 8 * sum of its 2^|O| coarse corners) / 2^(3+|O|))
// in exact int64 (units of U = 2^(E_f-48)).  The finest level writes the
// output, f_hat = round-to-nearest(X_hat) * U in the field's type.
#include "dev_common.cuh"

namespace hp {

template <typename T>
__device__ __forceinline__ T convert_out(int64_t X, int E_f);

template <>
__device__ __forceinline__ float convert_out<float>(int64_t X, int E_f) {
  return fixed_to_f32(X, E_f);
}

template <>
__device__ __forceinline__ double convert_out<double>(int64_t X, int E_f) {
  return fixed_to_f64(X, E_f);
}

__device__ __forceinline__ int64_t dequant(uint64_t qh, bool neg, int B, int bl) {
  uint64_t a;
  if (bl == 0) a = 0;
  else if (B >= bl) a = qh >> (B - bl);
  else a = qh << (bl - B);
  return neg ? -(int64_t)a : (int64_t)a;
}

// root: X_root = floor(c8_hat / 8)
template <typename T>
__global__ void k_recompose_root(const uint32_t* __restrict__ planes, const FieldMeta* __restrict__ m,
                                 const LevelDesc* __restrict__ L0, int64_t* xroot, T* out) {
  hp::pdl_enter();
  if (m->status) return;
  const int B = m->B, k = 4 * m->cur[0];
  const uint32_t* P = planes + L0->plane_off / 4;
  const uint32_t W = L0->W;
  uint64_t q = 0;
  for (int p = 0; p < k; p++) q |= (uint64_t)(P[(size_t)(1 + p) * W] & 1u) << (B - 1 - p);
  const bool neg = k > 0 && (P[0] & 1u);
  const int64_t X = dequant(q, neg, B, m->bl[0]) >> 3;
  if (xroot) *xroot = X;
  if (out) *out = convert_out<T>(X, m->E_f);
}

void launch_recompose_root(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* L0,
                           int64_t* xroot, void* out, int dtype, cstream s) {
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(k_recompose_root<float>, 1, 1, 0, s, planes, meta, L0, xroot,
                                      (float*)out);
  else
    hp::note_launch(), hp::launch_pdl(k_recompose_root<double>, 1, 1, 0, s, planes, meta, L0, xroot,
                                      (double*)out);
}

// coarse nodes (all coordinates even in G_h) are copied from G_2h
template <typename T, bool FINAL>
__global__ void __launch_bounds__(256) k_recompose_copy(const LevelDesc* __restrict__ Lp,
                                                        const int64_t* __restrict__ coarse,
                                                        void* __restrict__ dst,
                                                        const FieldMeta* __restrict__ m) {
  hp::pdl_enter();
  const LevelDesc& L = *Lp;
  const uint32_t cz = L.gc[0], cy = L.gc[1], cx = L.gc[2];
  const uint64_t total = (uint64_t)cz * cy * cx;
  const int E_f = m->E_f;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = (uint32_t)(i % cx);
    const uint64_t r = i / cx;
    const uint32_t y = (uint32_t)(r % cy), z = (uint32_t)(r / cy);
    const size_t d = ((size_t)(2 * z) * L.g[1] + 2 * y) * L.g[2] + 2 * x;
    const int64_t X = coarse[i];
    if (FINAL) reinterpret_cast<T*>(dst)[d] = convert_out<T>(X, E_f);
    else reinterpret_cast<int64_t*>(dst)[d] = X;
  }
}

// detail nodes of one level, one warp tile of 1024 level-linear nodes starting
// at node `base`.  Words: lane = word, the inverse transpose of the top k
// planes into the tile's shared rows (hi, lo) and sign words (sgn).
template <int B>
__device__ __forceinline__ void recompose_words(const uint32_t* __restrict__ P, const LevelDesc& L,
                                                uint32_t base, int k, uint32_t* hi, uint32_t* lo,
                                                uint32_t* sgn) {
  const int lane = threadIdx.x & 31;
  const uint32_t W = L.W;
  const uint32_t wi = base / 32 + lane;
  if (wi < W) {
    uint32_t a[32];
#pragma unroll
    for (int p = 0; p < 32; p++) a[31 - p] = (p < k) ? P[(size_t)(1 + p) * W + wi] : 0u;
    if (k) transpose32(a);
#pragma unroll
    for (int b = 0; b < 32; b++) hi[lane * 33 + b] = a[b];
    if (B == 64) {
#pragma unroll
      for (int p = 0; p < 32; p++) a[31 - p] = (32 + p < k) ? P[(size_t)(33 + p) * W + wi] : 0u;
      if (k > 32) transpose32(a);
#pragma unroll
      for (int b = 0; b < 32; b++) lo[lane * 33 + b] = a[b];
    }
    sgn[lane] = k > 0 ? P[wi] : 0u;
  }
}

// row r of the tile (lane = node): dequantize, add the corners, store
template <typename T, int B, bool FINAL>
__device__ __forceinline__ void recompose_row(const LevelDesc& L, uint32_t base, int r, int bl,
                                              int E_f, const int64_t* __restrict__ coarse,
                                              void* __restrict__ dst, const uint32_t* hi,
                                              const uint32_t* lo, const uint32_t* sgn) {
  const int lane = threadIdx.x & 31;
  const uint32_t j = base + r * 32 + lane;
  if (j >= L.n) return;
  const uint64_t qh = B == 64 ? (((uint64_t)hi[r * 33 + lane] << 32) | lo[r * 33 + lane])
                              : (uint64_t)hi[r * 33 + lane];
  const bool neg = (sgn[r] >> lane) & 1u;
  const int64_t c8 = dequant(qh, neg, B, bl);
  const NodePos p = node_pos(L, j);
  uint32_t zs[2], ys[2], xs[2];
  int nz = 1, ny = 1, nx = 1;
  zs[0] = zs[1] = p.gz >> 1;
  ys[0] = ys[1] = p.gy >> 1;
  xs[0] = xs[1] = p.gx >> 1;
  if (p.t & 4) {
    uint32_t a, b;
    axis_nb(p.gz, L.g[0], a, b);
    zs[0] = a >> 1; zs[1] = b >> 1; nz = 2;
  }
  if (p.t & 2) {
    uint32_t a, b;
    axis_nb(p.gy, L.g[1], a, b);
    ys[0] = a >> 1; ys[1] = b >> 1; ny = 2;
  }
  if (p.t & 1) {
    uint32_t a, b;
    axis_nb(p.gx, L.g[2], a, b);
    xs[0] = a >> 1; xs[1] = b >> 1; nx = 2;
  }
  int64_t sum = 0;
  for (int a = 0; a < nz; a++)
    for (int b = 0; b < ny; b++)
      for (int c = 0; c < nx; c++)
        sum += coarse[((size_t)zs[a] * L.gc[1] + ys[b]) * L.gc[2] + xs[c]];
  const int nodd = __popc(p.t);
  const int64_t X = floor_shift(c8 * ((int64_t)1 << nodd) + 8 * sum, 3 + nodd);
  const size_t d = ((size_t)p.gz * L.g[1] + p.gy) * L.g[2] + p.gx;
  if (FINAL) reinterpret_cast<T*>(dst)[d] = convert_out<T>(X, E_f);
  else reinterpret_cast<int64_t*>(dst)[d] = X;
}

template <typename T, int B, bool FINAL>
__device__ __forceinline__ void recompose_tile(const uint32_t* __restrict__ P, const LevelDesc& L,
                                               uint32_t base, int k, int bl, int E_f,
                                               const int64_t* __restrict__ coarse,
                                               void* __restrict__ dst, uint32_t* hi, uint32_t* lo,
                                               uint32_t* sgn) {
  recompose_words<B>(P, L, base, k, hi, lo, sgn);
  __syncwarp();
  // rows are independent: unrolled so that the coarse loads of several rows
  // are in flight together
#pragma unroll 4
  for (int r = 0; r < 32; r++)
    recompose_row<T, B, FINAL>(L, base, r, bl, E_f, coarse, dst, hi, lo, sgn);
  __syncwarp();
}

template <typename T, int B, bool FINAL>
__global__ void __launch_bounds__(B == 32 ? 256 : 128)
    k_recompose_level(const uint32_t* __restrict__ planes, const FieldMeta* __restrict__ m,
                      const LevelDesc* __restrict__ Lp, const uint32_t* __restrict__ perm,
                      const int64_t* __restrict__ coarse, void* __restrict__ dst) {
  hp::pdl_enter();
  constexpr int WPB = B == 32 ? 8 : 4;
  __shared__ uint32_t s_hi[WPB][32 * 33];
  __shared__ uint32_t s_lo[B == 64 ? WPB : 1][B == 64 ? 32 * 33 : 1];
  __shared__ uint32_t s_sign[WPB][32];
  if (m->status) return;
  const LevelDesc& L = *Lp;
  const int w = threadIdx.x >> 5;
  const int k = 4 * m->cur[L.level], bl = m->bl[L.level], E_f = m->E_f;
  const uint32_t* P = planes + L.plane_off / 4;
  for (uint32_t slot = blockIdx.x * WPB + w; slot < L.ntiles; slot += gridDim.x * WPB)
    recompose_tile<T, B, FINAL>(P, L, perm[L.tile0 + slot] * HP_TILE, k, bl, E_f, coarse, dst,
                                s_hi[w], s_lo[B == 64 ? w : 0], s_sign[w]);
}

// The root and a run of small levels 1..l_end in one CTA (levels are
// sequential: each needs the whole coarser grid): X_root, then per level the
// coarse-node copy and the detail tiles, separated by block barriers.  Grids
// alternate between the two scratch buffers as in the per-level path.
// With prefetch, the descriptors, coefficient counts and bit lengths of levels
// 0..l_end and the plane words they use are first copied to shared memory in
// one round of independent loads (after the staging: descriptors, k[], bl[],
// then the words of each level packed in level order), so that the levels'
// chain of dependent reads runs on shared memory.
template <typename T, int B>
__device__ __forceinline__ void recompose_small_body(const uint32_t* __restrict__ planes,
                                                     const FieldMeta* __restrict__ m,
                                                     const LevelDesc* __restrict__ levels,
                                                     int l_end, int nlev, int64_t* xroot,
                                                     int64_t* xa, int64_t* xb,
                                                     void* __restrict__ out, uint32_t* sm,
                                                     bool prefetch,
                                                     const int32_t* hcur = nullptr) {
  constexpr int WPB = 16;
  uint32_t* s_hi = sm;                                      // [WPB][32*33]
  uint32_t* s_lo = sm + WPB * 32 * 33;                      // [WPB][32*33] (B = 64)
  uint32_t* s_sign = sm + (B == 64 ? 2 : 1) * WPB * 32 * 33;  // [WPB][32]
  // (the word offset of s_desc is even: 8-byte aligned)
  LevelDesc* s_desc = reinterpret_cast<LevelDesc*>(s_sign + WPB * 32);  // [l_end + 1]
  int* s_k = reinterpret_cast<int*>(s_desc + (l_end + 1));              // [l_end + 1]
  int* s_bl = s_k + (l_end + 1);                                        // [l_end + 1]
  uint32_t* s_pl = reinterpret_cast<uint32_t*>(
      (reinterpret_cast<uintptr_t>(s_bl + (l_end + 1)) + 15) & ~(uintptr_t)15);
  if (m->status) return;
  if (prefetch) {
    const uint32_t nd = (uint32_t)(l_end + 1) * (uint32_t)(sizeof(LevelDesc) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(levels);
    for (uint32_t i = threadIdx.x; i < nd; i += blockDim.x) reinterpret_cast<uint32_t*>(s_desc)[i] = src[i];
    if (threadIdx.x <= (unsigned)l_end) {
      s_k[threadIdx.x] = 4 * (hcur ? hcur[threadIdx.x] : m->cur[threadIdx.x]);
      s_bl[threadIdx.x] = m->bl[threadIdx.x];
    }
    __syncthreads();
    uint32_t tot = 0;
    for (int l = 0; l <= l_end; l++) tot += (1u + (uint32_t)s_k[l]) * s_desc[l].W;
    constexpr int U = 8;  // loads in flight per thread
    for (uint32_t f0 = 0; f0 < tot; f0 += U * blockDim.x) {
      uint32_t v[U], at[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint32_t f = f0 + u * blockDim.x + threadIdx.x;
        at[u] = 0xffffffffu;
        if (f < tot) {
          uint32_t l = 0, acc = 0;
          while (f >= acc + (1u + (uint32_t)s_k[l]) * s_desc[l].W) {
            acc += (1u + (uint32_t)s_k[l]) * s_desc[l].W;
            l++;
          }
          v[u] = planes[s_desc[l].plane_off / 4 + (f - acc)];
          at[u] = f;
        }
      }
#pragma unroll
      for (int u = 0; u < U; u++)
        if (at[u] != 0xffffffffu) s_pl[at[u]] = v[u];
    }
    __syncthreads();
  }
  const LevelDesc* Ls = prefetch ? s_desc : levels;
  uint32_t acc_pl = 0;  // prefetched words of the levels before the current one
  auto level_planes = [&](int l) -> const uint32_t* {
    return prefetch ? s_pl + acc_pl : planes + Ls[l].plane_off / 4;
  };
  auto level_k = [&](int l) { return prefetch ? s_k[l] : 4 * (hcur ? hcur[l] : m->cur[l]); };
  const int L = nlev - 1, w = threadIdx.x >> 5, E_f = m->E_f;
  if (threadIdx.x < 32) {  // the root: lane p reads plane p, a ballot gathers q
    const int lane = threadIdx.x;
    const LevelDesc& D = Ls[0];
    const uint32_t* P = level_planes(0);
    const int k = level_k(0);
    uint64_t q = 0;
#pragma unroll
    for (int r = 0; r < B / 32; r++) {
      const int p = 32 * r + lane;  // plane p holds bit B - 1 - p
      const bool b = p < k && (P[(size_t)(1 + p) * D.W] & 1u);
      q |= (uint64_t)__brev(__ballot_sync(HP_FULL, b)) << (B - 32 - 32 * r);
    }
    if (lane == 0) {
      const bool neg = k > 0 && (P[0] & 1u);
      const int64_t X = dequant(q, neg, B, prefetch ? s_bl[0] : m->bl[0]) >> 3;
      *xroot = X;
      if (L == 0) *reinterpret_cast<T*>(out) = convert_out<T>(X, E_f);
    }
  }
  __syncthreads();
  if (prefetch) acc_pl += (1u + (uint32_t)s_k[0]) * s_desc[0].W;
  const int64_t* coarse = xroot;
  for (int l = 1; l <= l_end; l++) {
    const LevelDesc& D = Ls[l];
    const bool final = l == L;
    void* dst = final ? out : (void*)(((L - l) % 2 == 1) ? xa : xb);
    // coarse nodes of G_h come from G_2h
    const uint32_t cz = D.gc[0], cy = D.gc[1], cx = D.gc[2];
    const uint32_t total = cz * cy * cx;
    for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
      const uint32_t x = i % cx, r = i / cx, y = r % cy, z = r / cy;
      const size_t d = ((size_t)(2 * z) * D.g[1] + 2 * y) * D.g[2] + 2 * x;
      if (final) reinterpret_cast<T*>(dst)[d] = convert_out<T>(coarse[i], E_f);
      else reinterpret_cast<int64_t*>(dst)[d] = coarse[i];
    }
    const int k = level_k(l), bl = prefetch ? s_bl[l] : m->bl[l];
    const uint32_t* P = level_planes(l);
    if (prefetch) acc_pl += (1u + (uint32_t)k) * D.W;
    // the level's tiles, WPB at a time: each unpacked by one warp, then their
    // 32 rows spread over all warps
    const uint32_t nt = D.ntiles;
    for (uint32_t t0 = 0; t0 < nt; t0 += WPB) {
      const uint32_t nr = nt - t0 < (uint32_t)WPB ? nt - t0 : (uint32_t)WPB;
      if ((uint32_t)w < nr)
        recompose_words<B>(P, D, (t0 + w) * HP_TILE, k, s_hi + w * 32 * 33,
                           s_lo + (B == 64 ? w * 32 * 33 : 0), s_sign + w * 32);
      __syncthreads();
      for (uint32_t q = w; q < nr * 32; q += WPB) {
        const uint32_t tl = q / 32;
        const int r = (int)(q % 32);
        if (final)
          recompose_row<T, B, true>(D, (t0 + tl) * HP_TILE, r, bl, E_f, coarse, dst,
                                    s_hi + tl * 32 * 33, s_lo + (B == 64 ? tl * 32 * 33 : 0),
                                    s_sign + tl * 32);
        else
          recompose_row<T, B, false>(D, (t0 + tl) * HP_TILE, r, bl, E_f, coarse, dst,
                                     s_hi + tl * 32 * 33, s_lo + (B == 64 ? tl * 32 * 33 : 0),
                                     s_sign + tl * 32);
      }
      __syncthreads();
    }
    coarse = (const int64_t*)dst;
  }
}

template <typename T, int B>
__global__ void __launch_bounds__(512)
    k_recompose_small(const uint32_t* __restrict__ planes, const FieldMeta* __restrict__ m,
                      const LevelDesc* __restrict__ levels, int l_end, int nlev,
                      int64_t* xroot, int64_t* xa, int64_t* xb, void* __restrict__ out,
                      bool prefetch, SmallSel hs) {
  hp::pdl_enter();
  extern __shared__ __align__(16) uint32_t sm[];
  recompose_small_body<T, B>(planes, m, levels, l_end, nlev, xroot, xa, xb, out, sm, prefetch,
                             hs.l_end >= 0 ? hs.cur : nullptr);
}

static int sms() {
  int dev = 0, n = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

// the output conversion alone, over a plain array of fixed-point values
template <typename T>
__global__ void k_convert_fixed(const int64_t* __restrict__ X, uint64_t n, int E_f,
                                T* __restrict__ out) {
  hp::pdl_enter();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = convert_out<T>(X[i], E_f);
}

void launch_convert_fixed(const int64_t* X, uint64_t n, int E_f, int dtype, void* out, cstream s) {
  if (!n) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 152ull * 8) blocks = 152ull * 8;
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(k_convert_fixed<float>, (unsigned)blocks, 256, 0, s, X, n,
                                      E_f, (float*)out);
  else
    hp::note_launch(), hp::launch_pdl(k_convert_fixed<double>, (unsigned)blocks, 256, 0, s, X, n,
                                      E_f, (double*)out);
}

void launch_recompose_copy(const LevelDesc* Lh, const LevelDesc& Lh_host, const int64_t* coarse,
                           void* dst, int final_dtype, const FieldMeta* meta, cstream s) {
  uint64_t total = (uint64_t)Lh_host.gc[0] * Lh_host.gc[1] * Lh_host.gc[2];
  uint64_t blocks = (total + 255) / 256, cap = (uint64_t)sms() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  if (final_dtype < 0)
    hp::note_launch(), hp::launch_pdl(k_recompose_copy<float, false>, (unsigned)blocks, 256, 0, s,
                                      Lh, coarse, dst, meta);
  else if (final_dtype == 0)
    hp::note_launch(), hp::launch_pdl(k_recompose_copy<float, true>, (unsigned)blocks, 256, 0, s,
                                      Lh, coarse, dst, meta);
  else
    hp::note_launch(), hp::launch_pdl(k_recompose_copy<double, true>, (unsigned)blocks, 256, 0, s,
                                      Lh, coarse, dst, meta);
}

// shared memory for the prefetched plane words (every plane of every small level)
constexpr size_t kSmallPrefetchBytes = 48 * 1024;

void launch_recompose_small(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* levels,
                            const LevelDesc* levels_host, int l_end, int nlev, int64_t* xroot,
                            int64_t* xa, int64_t* xb, void* out, int dtype, cstream s,
                            const SmallSel* hs) {
  SmallSel h;
  h.l_end = -1;
  if (hs) h = *hs;
  const int B = dtype == 0 ? 32 : 64;
  const size_t base = (size_t)((dtype == 0 ? 1 : 2) * 16 * 32 * 33 + 16 * 32) * 4;
  const size_t meta_bytes = (size_t)(l_end + 1) * (sizeof(LevelDesc) + 8) + 16;
  const size_t meta_max = (size_t)HP_MAX_LEVELS * (sizeof(LevelDesc) + 8) + 16;
  uint64_t words = 0;
  for (int l = 0; l <= l_end; l++) words += (uint64_t)(B + 1) * levels_host[l].W;
  const bool prefetch = words * 4 <= kSmallPrefetchBytes;
  const size_t smem = base + (prefetch ? meta_bytes + words * 4 : 0);
  const int most = (int)(base + meta_max + kSmallPrefetchBytes);
  if (dtype == 0) {
    set_smem_once((const void*)k_recompose_small<float, 32>, most);
    hp::note_launch(), hp::launch_pdl(k_recompose_small<float, 32>, 1, 512, smem, s, planes, meta,
                                      levels, l_end, nlev, xroot, xa, xb, out, prefetch, h);
  } else {
    set_smem_once((const void*)k_recompose_small<double, 64>, most);
    hp::note_launch(), hp::launch_pdl(k_recompose_small<double, 64>, 1, 512, smem, s, planes, meta,
                                      levels, l_end, nlev, xroot, xa, xb, out, prefetch, h);
  }
}

void launch_recompose_level(const uint32_t* planes, const FieldMeta* meta, const LevelDesc* Lh,
                            const LevelDesc& Lh_host, const uint32_t* perm, const int64_t* coarse,
                            void* dst, int B, int final_dtype, cstream s) {
  const uint32_t wpb = B == 32 ? 8 : 4;
  uint32_t blocks = (Lh_host.ntiles + wpb - 1) / wpb, cap = (uint32_t)sms() * (B == 32 ? 8 : 16);
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  const int thr = B == 32 ? 256 : 128;
  if (B == 32) {
    if (final_dtype < 0)
      hp::note_launch(), hp::launch_pdl(k_recompose_level<float, 32, false>, blocks, thr, 0, s,
                                        planes, meta, Lh, perm, coarse, dst);
    else
      hp::note_launch(), hp::launch_pdl(k_recompose_level<float, 32, true>, blocks, thr, 0, s,
                                        planes, meta, Lh, perm, coarse, dst);
  } else {
    if (final_dtype < 0)
      hp::note_launch(), hp::launch_pdl(k_recompose_level<double, 64, false>, blocks, thr, 0, s,
                                        planes, meta, Lh, perm, coarse, dst);
    else
      hp::note_launch(), hp::launch_pdl(k_recompose_level<double, 64, true>, blocks, thr, 0, s,
                                        planes, meta, Lh, perm, coarse, dst);
  }
}

// ------------------------------------------------------------------ batched
template <typename T, int B>
__global__ void __launch_bounds__(512) kb_recompose_small(const BatchJob* __restrict__ jobs) {
  hp::pdl_enter();
  extern __shared__ uint32_t sm[];
  const BatchJob& J = jobs[blockIdx.x];
  recompose_small_body<T, B>(reinterpret_cast<const uint32_t*>(J.planes), J.meta, J.levels,
                             J.small_end, (int)J.nlev, J.xroot, J.xa, J.xb, J.out, sm, false);
}

void launch_b_recompose_small(const BatchJob* jobs, uint32_t njobs, int dtype, cstream s) {
  if (!njobs) return;
  const size_t smem = (size_t)((dtype == 0 ? 1 : 2) * 16 * 32 * 33 + 16 * 32) * 4;
  if (dtype == 0) {
    set_smem_once((const void*)kb_recompose_small<float, 32>, (int)smem);
    hp::note_launch(), hp::launch_pdl(kb_recompose_small<float, 32>, njobs, 512, smem, s, jobs);
  } else {
    set_smem_once((const void*)kb_recompose_small<double, 64>, (int)smem);
    hp::note_launch(), hp::launch_pdl(kb_recompose_small<double, 64>, njobs, 512, smem, s, jobs);
  }
}

// unit = 256 coarse nodes of one (job, level) entry
template <typename T>
__global__ void __launch_bounds__(256) kb_recompose_copy(const BatchJob* __restrict__ jobs,
                                                         const LevelRef* __restrict__ refs,
                                                         const uint32_t* __restrict__ unit0,
                                                         uint32_t nrefs, uint32_t total) {
  hp::pdl_enter();
  for (uint32_t u = blockIdx.x; u < total; u += gridDim.x) {
    const uint32_t e = unit_owner(unit0, nrefs, u);
    const LevelRef R = refs[e];
    const BatchJob& J = jobs[R.job];
    const LevelDesc& L = J.levels[R.level];
    const uint32_t cz = L.gc[0], cy = L.gc[1], cx = L.gc[2];
    const uint64_t n = (uint64_t)cz * cy * cx;
    const uint64_t i = (uint64_t)(u - unit0[e]) * 256 + threadIdx.x;
    if (i >= n) continue;
    const uint32_t x = (uint32_t)(i % cx);
    const uint64_t r = i / cx;
    const uint32_t y = (uint32_t)(r % cy), z = (uint32_t)(r / cy);
    const size_t d = ((size_t)(2 * z) * L.g[1] + 2 * y) * L.g[2] + 2 * x;
    const int64_t X = R.coarse[i];
    if (R.final) reinterpret_cast<T*>(J.out)[d] = convert_out<T>(X, J.meta->E_f);
    else R.dst[d] = X;
  }
}

template <typename T, int B>
__global__ void __launch_bounds__(B == 32 ? 256 : 128)
    kb_recompose_level(const BatchJob* __restrict__ jobs, const LevelRef* __restrict__ refs,
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
    const FieldMeta* m = J.meta;
    if (m->status) continue;
    const LevelDesc& L = J.levels[R.level];
    const int k = 4 * m->cur[L.level], bl = m->bl[L.level], E_f = m->E_f;
    const uint32_t* P = reinterpret_cast<const uint32_t*>(J.planes) + L.plane_off / 4;
    const uint32_t base = J.perm[L.tile0 + (u - unit0[e])] * HP_TILE;
    if (R.final)
      recompose_tile<T, B, true>(P, L, base, k, bl, E_f, R.coarse, J.out, s_hi[w],
                                 s_lo[B == 64 ? w : 0], s_sign[w]);
    else
      recompose_tile<T, B, false>(P, L, base, k, bl, E_f, R.coarse, R.dst, s_hi[w],
                                  s_lo[B == 64 ? w : 0], s_sign[w]);
  }
}

void launch_b_recompose_copy(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                             uint32_t nrefs, uint32_t total, int dtype, uint32_t grid, cstream s) {
  if (!total) return;
  if (grid > total) grid = total;
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(kb_recompose_copy<float>, grid, 256, 0, s, jobs, refs, unit0,
                                      nrefs, total);
  else
    hp::note_launch(), hp::launch_pdl(kb_recompose_copy<double>, grid, 256, 0, s, jobs, refs, unit0,
                                      nrefs, total);
}

void launch_b_recompose_level(const BatchJob* jobs, const LevelRef* refs, const uint32_t* unit0,
                              uint32_t nrefs, uint32_t total, int dtype, uint32_t grid, cstream s) {
  if (!total) return;
  const uint32_t wpb = dtype == 0 ? 8 : 4, need = (total + wpb - 1) / wpb;
  if (grid > need) grid = need;
  if (dtype == 0)
    hp::note_launch(), hp::launch_pdl(kb_recompose_level<float, 32>, grid, 256, 0, s, jobs, refs,
                                      unit0, nrefs, total);
  else
    hp::note_launch(), hp::launch_pdl(kb_recompose_level<double, 64>, grid, 128, 0, s, jobs, refs,
                                      unit0, nrefs, total);
}

}  // namespace hp
