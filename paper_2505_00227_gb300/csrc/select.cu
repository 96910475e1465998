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

__device__ __forceinline__ u128 p2(int e) {
  if (e < 0) return 0;
  if (e > 127) e = 127;
  return (u128)1 << e;
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
  uint64_t len[HP_MAX_LEVELS][HP_MAX_GROUPS];
};

__device__ __forceinline__ uint64_t stored_len(const SeqView* m, int l, int g) { return m->len[l][g]; }

template <class M>
__device__ u128 level_delta(const M* m, int l, int k) {
  const int bl = m->bl[l];
  if (bl == 0 || k >= bl) return 0;
  if (k >= m->B && m->exact[l]) return 0;
  return p2(bl - k + m->B);
}

// 2^(bl_a-k_a) * bytes_b > 2^(bl_b-k_b) * bytes_a, ties to the smaller level
template <class M>
__device__ bool better(const M* m, const int* g, int a, int b) {
  const int sa = m->bl[a] - 4 * g[a], sb = m->bl[b] - 4 * g[b];
  const u128 ba = stored_len(m, a, g[a]), bb = stored_len(m, b, g[b]);
  const int lo = sa < sb ? sa : sb;
  const u128 left = bb << (sa - lo), right = ba << (sb - lo);
  if (left != right) return left > right;
  return a < b;
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
  for (int i = lane; i < nlev * ng; i += 32) V.len[i / ng][i % ng] = m->grp[i / ng][i % ng].stored_len;
  if (lane == 0) {
    V.B = m->B;
    V.nlev = nlev;
    V.ngroups = ng;
    V.dtype = m->dtype;
    V.E_f = m->E_f;
    V.input_exact = m->input_exact;
  }
  __syncwarp();
  const SeqView* v = &V;
  u128 sum = 0;
  if (lane == 0) {
    for (int l = 0; l < nlev; l++) sum += level_delta(v, l, 0);
    const u128 E = finish_estimate(v, sum);
    m->E_hi[0] = (uint64_t)(E >> 64);
    m->E_lo[0] = (uint64_t)E;
  }
  int n = 0;
  while (n < HP_SEQ_MAX) {
    int best = -1;
    for (int l = lane; l < nlev; l += 32) {
      if (g[l] >= ng || level_delta(v, l, 4 * g[l]) == 0) continue;
      if (best < 0 || better(v, g, l, best)) best = l;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const int other = __shfl_xor_sync(HP_FULL, best, o);
      if (other >= 0 && (best < 0 || better(v, g, other, best))) best = other;
    }
    if (best < 0) break;
    if (lane == 0) {
      sum -= level_delta(v, best, 4 * g[best]);
      g[best]++;
      sum += level_delta(v, best, 4 * g[best]);
      m->seq[n] = (uint8_t)best;
      const u128 E = finish_estimate(v, sum);
      m->E_hi[n + 1] = (uint64_t)(E >> 64);
      m->E_lo[n + 1] = (uint64_t)E;
    }
    n++;
    __syncwarp();
  }
  if (lane == 0) m->seq_len = n;
}

__global__ void k_sequence(FieldMeta* m) {
  __shared__ int g[64];
  sequence_warp(m, g);
}

void launch_sequence(FieldMeta* meta, cstream s) { hp::note_launch(), k_sequence<<<1, 32, 0, s>>>(meta); }

// floor(tau * 2^(51+B-E_f)) from the IEEE fields of tau, saturating at 2^127
__device__ u128 tau_units(double tau, int E_f, int B) {
  const uint64_t u = (uint64_t)__double_as_longlong(tau);
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
    if (bitlen64(m) + s > 127) return p2(127);
    return (u128)m << s;
  }
  if (-s >= 64) return 0;
  return (u128)(m >> (-s));
}

// One warp: the prefix by binary search (lane 0), the groups per level by
// counting the prefix's entries (all lanes), the per-level bytes by lane =
// level, and the list of chunks to decode in (level, group) order (lane 0).
__device__ void select_prefix(FieldMeta* m, double tau, int tau_is_abs, RetrieveDev* rd) {
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
  if (lane == 0) {
    const u128 T = tau_units(tau_abs, m->E_f, m->B);
    // the estimates never increase along the sequence: binary search for the
    // shortest prefix whose estimate meets the bound
    int lo = 0, hi = n + 1;  // answer in [lo, hi]; hi = n + 1 means none
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      const u128 E = ((u128)m->E_hi[mid] << 64) | m->E_lo[mid];
      if (E <= T) hi = mid;
      else lo = mid + 1;
    }
    s_c = lo;
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
  uint64_t bnew = 0, btot = 0;
  for (int l = lane; l < nlev; l += 32) {
    const int gl = s_g[l], f0 = m->fetched[l], fe = gl > f0 ? gl : f0;
    for (int q = f0; q < gl; q++) bnew += m->grp[l][q].stored_len;
    for (int q = 0; q < fe; q++) btot += m->grp[l][q].stored_len;
  }
  bnew = warp_sum_u64(bnew);
  btot = warp_sum_u64(btot);
  if (lane == 0) {
    uint32_t n_new = 0, items = 0;
    for (int l = 0; l < nlev; l++)
      for (int q = m->fetched[l]; q < s_g[l]; q++) {
        const GroupMeta& gm = m->grp[l][q];
        if (gm.method != 0 || m->compact) {  // compact handles copy DC groups too
          rd->new_gi[n_new] = (uint32_t)(l * ng + q);
          rd->new_pref[n_new] = items;
          items += gm.nchunks;
          n_new++;
        }
      }
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
  }
  __syncwarp();
  for (int l = lane; l < nlev; l += 32) {  // after lane 0 has read the old state
    const int gl = s_g[l];
    if (gl > m->fetched[l]) m->fetched[l] = gl;
    m->cur[l] = gl;
    rd->g[l] = gl;
  }
}

__global__ void k_select(FieldMeta* m, double tau, int tau_is_abs, RetrieveDev* rd) {
  select_prefix(m, tau, tau_is_abs, rd);
}

void launch_select(FieldMeta* meta, double tau, int tau_is_abs, RetrieveDev* rd, cstream s) {
  hp::note_launch(), k_select<<<1, 32, 0, s>>>(meta, tau, tau_is_abs, rd);
}

// ------------------------------------------------------------------ batched
__global__ void kb_sequence(const BatchJob* __restrict__ jobs) {
  __shared__ int g[64];
  sequence_warp(jobs[blockIdx.x].meta, g);
}

void launch_b_sequence(const BatchJob* jobs, uint32_t njobs, cstream s) {
  if (njobs) hp::note_launch(), kb_sequence<<<njobs, 32, 0, s>>>(jobs);
}

__global__ void kb_select(const BatchJob* __restrict__ jobs) {
  const BatchJob& J = jobs[blockIdx.x];
  select_prefix(J.meta, J.tau, 0, J.rd);
}

void launch_b_select(const BatchJob* jobs, uint32_t njobs, cstream s) {
  if (njobs) hp::note_launch(), kb_select<<<njobs, 32, 0, s>>>(jobs);
}

}  // namespace hp
