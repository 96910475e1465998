// Error-bound-driven selection of bitplane groups (Sec. 3 error control;
// Algorithm 3's copy_to_device(S, eps)).
//
// Estimator: with k magnitude planes of level l fetched, every coefficient is
// off by less than 2^(bl_l-k) units of U/8, i.e. delta_l = 2^(bl_l-k-3) U (zero
// for an all-zero level, when k >= bl_l, and at k = B when the alignment
// dropped no nonzero bit).  Recomposition adds each coefficient to a convex
// combination of coarser values, so |x_hat - x| <= sum_l delta_l, plus one U per
// level for the floors (when some delta > 0), plus U for the fixed-point floor
// of the input (when it lost bits), plus half an ulp of the output type.  The
// estimate is an exact 128-bit integer in units of 2^(E_f-51-B).
//
// Greedy order (independent of the bound): repeatedly fetch the next group of
// the level with the largest 2^(bl-k) / stored bytes, ties to the smaller
// level.  A retrieval uses the shortest prefix whose estimate meets the bound,
// so incremental and from-scratch retrievals agree.
#include "dev_common.cuh"

namespace hp {

typedef unsigned __int128 u128;

__host__ __device__ __forceinline__ u128 p2(int e) {
  if (e < 0) return 0;
  if (e > 127) e = 127;
  return (u128)1 << e;
}

__host__ __device__ __forceinline__ int bitlen64_hd(uint64_t v) {
#ifdef __CUDA_ARCH__
  return 64 - __clzll((long long)v);
#else
  return v ? 64 - __builtin_clzll(v) : 0;
#endif
}

__device__ __forceinline__ u128 sat_add(u128 a, u128 b) {
  u128 s = a + b;
  return s < a ? ~(u128)0 : s;
}

// The metadata the greedy sequence reads, staged in shared memory so that
// its steps make no global loads.
struct SeqView {
  int B, nlev, ngroups, dtype, E_f, input_exact;
  int bl[HP_MAX_LEVELS], exact[HP_MAX_LEVELS];
  int lim[HP_MAX_LEVELS];  // groups of the level that still reduce its error
  // stored bytes per unit of error removed, len / 2^(bl - 4g), as the bits of
  // the (exact, positive, normal) double: comparing the bits as unsigned
  // integers is comparing the greedy ratios 2^(bl-4g) / len exactly
  uint64_t key[HP_MAX_LEVELS][HP_MAX_GROUPS];
};

// the IEEE bits of len * 2^-s for 1 <= len < 2^53, |s| < 900
__device__ __forceinline__ uint64_t ratio_key(uint64_t len, int s) {
  const int lz = __clzll((long long)len);
  const uint64_t frac = (len << lz << 1) >> 12;  // bits below the leading one
  return ((uint64_t)(1023 + 63 - lz - s) << 52) | frac;
}

template <class M>
__device__ u128 level_delta(const M* m, int l, int k) {
  const int bl = m->bl[l];
  if (bl == 0 || k >= bl) return 0;
  if (k >= m->B && m->exact[l]) return 0;
  return p2(bl - k + m->B);
}

// E from the sum of the per-level truncation errors (same terms as estimate())
template <class M>
__device__ u128 finish_estimate(const M* m, u128 sum_delta) {
  u128 E = sum_delta;
  const u128 U = p2(m->B + 3);
  if (sum_delta) E = sat_add(E, (u128)m->nlev * U);
  if (!m->input_exact) E = sat_add(E, U);
  if (E == 0) return 0;
  u128 eps;
  if (E < p2(m->B + 51)) {
    int e1 = m->dtype == 0 ? m->B + 27 : m->B - 2;
    int e2 = m->dtype == 0 ? m->B - 99 - m->E_f : m->B - 1024 - m->E_f;
    eps = p2(e1 > e2 ? e1 : e2);
  } else {
    eps = E;
  }
  return sat_add(E, eps);
}

// One warp: lane l evaluates levels l and l + 32; the best level of each step
// is a warp-wide reduction with the greedy comparison.  The estimate after
// each step is updated from the chosen level's change only.
__device__ __forceinline__ void sequence_warp(FieldMeta* m, int* g) {
  __shared__ SeqView V;
  const int lane = threadIdx.x;
  if (m->status) return;
  const int nlev = m->nlev, ng = m->ngroups;
  for (int l = lane; l < 64; l += 32) {
    g[l] = 0;
    if (l < nlev) {
      const int ex = m->lowbits[l] == 0 ? 1 : 0;
      m->exact[l] = ex;
      V.exact[l] = ex;
      V.bl[l] = m->bl[l];
    }
  }
  if (lane == 0) {
    V.B = m->B;
    V.nlev = nlev;
    V.ngroups = ng;
    V.dtype = m->dtype;
    V.E_f = m->E_f;
    V.input_exact = m->input_exact;
  }
  __syncwarp();
  for (int i = lane; i < nlev * ng; i += 32) {
    const int l = i / ng, q = i % ng;
    const uint64_t len = m->grp[l][q].stored_len;
    V.key[l][q] = len ? ratio_key(len, V.bl[l] - 4 * q) : 0;
  }
  const SeqView* v = &V;
  for (int l = lane; l < nlev; l += 32) {
    int q = 0;
    while (q < ng && level_delta(v, l, 4 * q) != 0) q++;
    V.lim[l] = q;
  }
  __syncwarp();
  // 1. the sequence: repeatedly the level with the smallest key (ties to the
  // smaller level) among those with a group left that reduces the error.  Lane
  // j owns levels j and j + 32 (their group counts in registers); a step is
  // three warp minimum reductions: key high word, key low word, level.
  __shared__ uint8_t s_seq[HP_SEQ_MAX], s_gq[HP_SEQ_MAX];
  int ga = 0, gb = 0;  // groups taken of levels lane, lane + 32
  int n = 0;
  while (n < HP_SEQ_MAX) {
    uint64_t bk = ~0ull;
    int best = 255;
    if (lane < nlev && ga < V.lim[lane]) bk = V.key[lane][ga], best = lane;
    if (lane + 32 < nlev && gb < V.lim[lane + 32]) {
      const uint64_t k2 = V.key[lane + 32][gb];
      if (k2 < bk) bk = k2, best = lane + 32;
    }
    const uint32_t hi = (uint32_t)(bk >> 32), lo = (uint32_t)bk;
    const uint32_t mh = __reduce_min_sync(HP_FULL, hi);
    if (mh == 0xffffffffu) break;  // no level has a useful group left
    const uint32_t ml = __reduce_min_sync(HP_FULL, hi == mh ? lo : 0xffffffffu);
    const uint32_t win = __reduce_min_sync(HP_FULL, (hi == mh && lo == ml) ? (uint32_t)best : 255u);
    if ((int)win == best) {  // the owner records the step
      const int q = best == lane ? ga++ : gb++;
      s_seq[n] = (uint8_t)best;
      s_gq[n] = (uint8_t)q;
    }
    n++;
  }
  g[lane] = ga;
  g[lane + 32] = gb;
  __syncwarp();
  // 2. the estimate after every prefix: sum_n = S0 - (r_0 + ... + r_{n-1}),
  // r_i = delta(l_i, 4 g_i) - delta(l_i, 4 g_i + 4) >= 0, an exact 128-bit
  // prefix sum (lane = block of consecutive steps, then a warp scan)
  u128 S0 = 0;
  for (int l = 0; l < nlev; l++) S0 += level_delta(v, l, 0);
  auto r_of = [&](int i) {
    const int l = s_seq[i], q = s_gq[i];
    return level_delta(v, l, 4 * q) - level_delta(v, l, 4 * q + 4);
  };
  const int per = (n + 31) / 32, i0 = lane * per, i1 = min(n, i0 + per);
  u128 tot = 0;
  for (int i = i0; i < i1; i++) tot += r_of(i);
  u128 incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t hi = __shfl_up_sync(HP_FULL, (unsigned long long)(incl >> 64), o);
    const uint64_t lo = __shfl_up_sync(HP_FULL, (unsigned long long)incl, o);
    if (lane >= o) incl += ((u128)hi << 64) | lo;
  }
  u128 run = incl - tot;  // before this lane's block
  for (int i = i0; i < i1; i++) {
    run += r_of(i);
    const u128 E = finish_estimate(v, S0 - run);
    m->seq[i] = s_seq[i];
    m->E_hi[i + 1] = (uint64_t)(E >> 64);
    m->E_lo[i + 1] = (uint64_t)E;
  }
  if (lane == 0) {
    const u128 E = finish_estimate(v, S0);
    m->E_hi[0] = (uint64_t)(E >> 64);
    m->E_lo[0] = (uint64_t)E;
    m->seq_len = n;
  }
}

__global__ void k_sequence(FieldMeta* m) {
  hp::pdl_enter();
  __shared__ int g[64];
  sequence_warp(m, g);
}

void launch_sequence(FieldMeta* meta, cstream s) {
  hp::note_launch(), hp::launch_pdl(k_sequence, 1, 32, 0, s, meta);
}

// floor(tau * 2^(51+B-E_f)) from the IEEE fields of tau, saturating at 2^127
// (integer work only: the host computes the same value)
__host__ __device__ u128 tau_units(double tau, int E_f, int B) {
  uint64_t u;
  memcpy(&u, &tau, 8);
  if (u >> 63) return 0;                       // negative (or -0)
  const uint32_t e = (uint32_t)(u >> 52);
  if (e == 0x7ff) return (u & 0xfffffffffffffull) ? 0 : p2(127);  // NaN -> 0, inf -> max
  uint64_t m = u & 0xfffffffffffffull;
  int ex;
  if (e == 0) ex = -1074;
  else {
    m |= 0x10000000000000ull;
    ex = (int)e - 1075;
  }
  if (m == 0) return 0;
  const int s = ex + 51 + B - E_f;             // tau = m 2^ex, scaled: m 2^s
  if (s >= 0) {
    if (bitlen64_hd(m) + s > 127) return p2(127);
    return (u128)m << s;
  }
  if (-s >= 64) return 0;
  return (u128)(m >> (-s));
}

// One warp: the prefix by binary search (lane 0), the groups per level by
// counting the prefix's entries (all lanes), the per-level bytes by lane =
// level, and the list of chunks to decode in (level, group) order (lane 0).
// m: the metadata read (a shared-memory copy, or the field's own); mw: the
// field's metadata, where the fetched state is updated.
__device__ void select_prefix(const FieldMeta* m, FieldMeta* mw, double tau, int tau_is_abs,
                              RetrieveDev* rd, const SmallSel* hs = nullptr) {
  __shared__ int s_g[HP_MAX_LEVELS + 1];
  __shared__ int s_c;
  const int lane = threadIdx.x & 31;
  const int mst = m->status;
  if (mst) {  // nothing to decode or recompose
    if (lane == 0) {
      rd->status = mst;
      rd->n_new = 0;
      rd->items = 0;
    }
    return;
  }
  const double tau_abs = tau_is_abs ? tau : __dmul_rn(tau, m->range);
  const int n = m->seq_len, nlev = m->nlev, ng = m->ngroups;
  {
    // the estimates never increase along the sequence: the shortest prefix
    // whose estimate meets the bound is the number of prefixes that do not.
    // Lanes test 32 prefixes at a time (a stride search, then a fine one).
    const u128 T = tau_units(tau_abs, m->E_f, m->B);
    auto fails = [&](int i) {  // prefix i does not meet the bound
      if (i > n) return false;
      const u128 E = ((u128)m->E_hi[i] << 64) | m->E_lo[i];
      return E > T;
    };
    const int stride = (n + 1 + 31) / 32;  // prefixes 0..n
    const unsigned coarse = __ballot_sync(HP_FULL, fails(lane * stride));
    const int first_ok = coarse == HP_FULL ? 32 : __ffs(~coarse) - 1;  // first chunk start that meets
    // the answer lies in ((first_ok - 1) * stride, first_ok * stride]
    const int base = first_ok == 0 ? 0 : (first_ok - 1) * stride + 1;
    int c = first_ok * stride;  // no prefix meets it: c > n after the clamp below
    for (int b0 = base; b0 < first_ok * stride && b0 <= n; b0 += 32) {
      const unsigned fine = __ballot_sync(HP_FULL, b0 + lane < first_ok * stride && fails(b0 + lane));
      if (fine != HP_FULL) {
        c = b0 + __ffs(~fine) - 1;
        break;
      }
    }
    if (first_ok == 0) c = 0;
    if (lane == 0) s_c = c > n ? n + 1 : c;
  }
  for (int l = lane; l <= HP_MAX_LEVELS; l += 32) s_g[l] = 0;
  __syncwarp();
  int c = s_c, status = 0;
  if (c > n) {
    c = n;
    status = -5;  // HPMDR_ERR_UNATTAINABLE: best reconstruction, estimate reported
  }
  for (int i = lane; i < c; i += 32) atomicAdd(&s_g[m->seq[i]], 1);
  __syncwarp();
  // the small levels were recomposed with the host's selection (host_select_small):
  // it must be this one
  if (hs && hs->l_end >= 0 &&
      __any_sync(HP_FULL, lane <= hs->l_end && s_g[lane] != hs->cur[lane]))
    status = -4;  // HPMDR_ERR_CORRUPT
  uint64_t bnew = 0, btot = 0;
  for (int l = lane; l < nlev; l += 32) {
    const int gl = s_g[l], f0 = m->fetched[l], fe = gl > f0 ? gl : f0;
#pragma unroll
    for (int q = 0; q < HP_MAX_GROUPS; q++) {  // unrolled: the loads issue together
      if (q < fe) {
        const uint64_t len = m->grp[l][q].stored_len;
        btot += len;
        if (q >= f0 && q < gl) bnew += len;
      }
    }
  }
  bnew = warp_sum_u64(bnew);
  btot = warp_sum_u64(btot);
  // the newly fetched groups to decode, in (level, group) order: lane = group
  // of a run of 32 flat indices, ranks by ballot, chunk offsets by a warp scan
  uint32_t n_new = 0, items = 0;
  const int compact = m->compact;
  for (int b0 = 0; b0 < nlev * ng; b0 += 32) {
    const int i = b0 + lane;
    bool take = false;
    uint32_t nc = 0;
    if (i < nlev * ng) {
      const int l = i / ng, q = i % ng;
      if (q >= m->fetched[l] && q < s_g[l]) {
        const GroupMeta& gm = m->grp[l][q];
        if (gm.method != 0 || compact) {  // compact handles copy DC groups too
          take = true;
          nc = gm.nchunks;
        }
      }
    }
    const unsigned bal = __ballot_sync(HP_FULL, take);
    uint32_t incl = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(HP_FULL, incl, o);
      if (lane >= o) incl += y;
    }
    if (take) {
      const uint32_t r = n_new + __popc(bal & ((1u << lane) - 1u));
      rd->new_gi[r] = (uint32_t)i;
      rd->new_pref[r] = items + incl - nc;
    }
    n_new += __popc(bal);
    items += __shfl_sync(HP_FULL, incl, 31);
  }
  if (lane == 0) {
    rd->new_pref[n_new] = items;
    rd->n_new = n_new;
    rd->items = items;
    rd->bytes_new = bnew;
    rd->bytes_total = btot;
    rd->nsel = c;
    rd->status = status;
    rd->E_hi = m->E_hi[c];
    rd->E_lo = m->E_lo[c];
    double v = __dadd_rn(__dmul_rn(__ull2double_rn(m->E_hi[c]), 18446744073709551616.0),
                         __ull2double_rn(m->E_lo[c]));
    rd->E_abs = ldexp(v, m->E_f - 51 - m->B);
    rd->tau_abs = tau_abs;
    // every reconstructed value is within E of its input value, itself at most
    // max|f| in magnitude: |X| U <= max|f| + E.  Below 2^E_f (= 2^48 U), with a
    // margin for the roundings of this test, |X| < 2^48
    const double bound = __dmul_rn(__dadd_rn(m->maxabs, rd->E_abs), 1.0 + 0x1p-40);
    mw->out_small = bound < ldexp(1.0, m->E_f) ? 1 : 0;
  }
  __syncwarp();
  for (int l = lane; l < nlev; l += 32) {  // after lane 0 has read the old state
    const int gl = s_g[l];
    if (gl > m->fetched[l]) mw->fetched[l] = gl;
    mw->cur[l] = gl;
    rd->g[l] = gl;
  }
}

// The field's metadata is first copied to shared memory by the whole CTA (16-byte
// units, 8 loads in flight per thread), so that the warp's chain of dependent
// reads (estimates, sequence, fetched state, group sizes) runs on shared memory.
__global__ void __launch_bounds__(256) k_select(FieldMeta* m, double tau, int tau_is_abs,
                                                RetrieveDev* rd, SmallSel hs) {
  hp::pdl_enter();
  extern __shared__ __align__(16) unsigned char sel_smem[];
  FieldMeta* sm = reinterpret_cast<FieldMeta*>(sel_smem);
  constexpr uint32_t N16 = sizeof(FieldMeta) / 16;
  static_assert(sizeof(FieldMeta) % 16 == 0, "the copy moves whole 16-byte units");
  const uint4* src = reinterpret_cast<const uint4*>(m);
  uint4* dst = reinterpret_cast<uint4*>(sm);
  for (uint32_t i0 = 0; i0 < N16; i0 += 8 * blockDim.x) {
    uint4 v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint32_t i = i0 + u * blockDim.x + threadIdx.x;
      if (i < N16) v[u] = src[i];
    }
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint32_t i = i0 + u * blockDim.x + threadIdx.x;
      if (i < N16) dst[i] = v[u];
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) select_prefix(sm, m, tau, tau_is_abs, rd, &hs);
}

void launch_select(FieldMeta* meta, double tau, int tau_is_abs, RetrieveDev* rd, cstream s,
                   const SmallSel* hs) {
  SmallSel h;
  h.l_end = -1;
  if (hs) h = *hs;
  set_smem_once((const void*)k_select, (int)sizeof(FieldMeta));
  hp::note_launch(), hp::launch_pdl(k_select, 1, 256, sizeof(FieldMeta), s, meta, tau, tau_is_abs,
                                    rd, h);
}

// The groups per level l <= l_end that k_select will choose for tau, from the
// host copy of the metadata (the greedy sequence and its estimates): the
// shortest prefix whose estimate is at most tau in the same 128-bit units (the
// estimates never increase along the sequence), all of it when none is.
void host_select_small(const FieldMeta& m, double tau, int tau_is_abs, int l_end, SmallSel* out) {
  const double tau_abs = tau_is_abs ? tau : tau * m.range;
  const u128 T = tau_units(tau_abs, m.E_f, m.B);
  const int n = m.seq_len;
  int c = n;
  for (int i = 0; i <= n; i++) {
    const u128 E = ((u128)m.E_hi[i] << 64) | m.E_lo[i];
    if (!(E > T)) {
      c = i;
      break;
    }
  }
  out->l_end = l_end;
  for (int l = 0; l < HP_MAX_LEVELS; l++) out->cur[l] = 0;
  for (int i = 0; i < c; i++)
    if (m.seq[i] <= l_end) out->cur[m.seq[i]]++;
}

// ------------------------------------------------------------------ batched
__global__ void kb_sequence(const BatchJob* __restrict__ jobs) {
  hp::pdl_enter();
  __shared__ int g[64];
  sequence_warp(jobs[blockIdx.x].meta, g);
}

void launch_b_sequence(const BatchJob* jobs, uint32_t njobs, cstream s) {
  if (njobs) hp::note_launch(), hp::launch_pdl(kb_sequence, njobs, 32, 0, s, jobs);
}

__global__ void kb_select(const BatchJob* __restrict__ jobs) {
  hp::pdl_enter();
  const BatchJob& J = jobs[blockIdx.x];
  select_prefix(J.meta, J.meta, J.tau, 0, J.rd);
}

void launch_b_select(const BatchJob* jobs, uint32_t njobs, cstream s) {
  if (njobs) hp::note_launch(), hp::launch_pdl(kb_select, njobs, 32, 0, s, jobs);
}

}  // namespace hp
