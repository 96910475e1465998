/*
 * Oracle: L-infinity error estimator and greedy bitplane-group selection for
 * error-controlled retrieval.  TEST INFRASTRUCTURE ONLY (see hpmdr_oracle.h).
 *
 * The paper fetches "the necessary bitplanes" for a data error bound
 * (Sec. 3; Algorithm 3, copy_to_device(S, eps)) following MDR/PMGARD without
 * spelling the estimator or the selection out.  Readings used:
 *   - with k magnitude planes of a level fetched, |C8 - c8_hat| < 2^(bl-k)
 *     (units U/8), so delta_l(k) = 2^(bl-k-3) U; delta = 0 for an all-zero
 *     level, when k >= bl (every bit of C8 fetched), and for k = B on a level
 *     whose dropped low bits are all zero;
 *   - recomposition is a convex combination plus the coefficient, so the
 *     reconstruction error is at most sum_l delta_l, plus one unit U for each
 *     floor (one per level, only when some delta > 0), plus U when the input
 *     was floored to the fixed point, plus the final round-to-nearest
 *     conversion (half an ulp of the output type at |x| < 2^(E_f+1));
 *   - E is kept exactly as a 128-bit integer in units of 2^(E_f-51-B);
 *   - greedy: start from nothing, repeatedly add the next group of the level
 *     with the largest 2^(bl-k) / bytes (exact cross-multiplied comparison,
 *     ties to the smaller level), skipping all-zero and exhausted levels; the
 *     selection for tau is the shortest prefix of that tau-independent
 *     sequence with E <= tau.
 */
#include <math.h>
#include <string.h>

#include "hpmdr_oracle.h"

typedef unsigned __int128 u128;

static u128 pow2_sat(int e) { /* 2^e for e in [0, 127], saturating above */
  if (e < 0) return 0;
  if (e > 127) e = 127;
  return (u128)1 << e;
}

static u128 add_sat(u128 a, u128 b) {
  u128 s = a + b;
  return s < a ? ~(u128)0 : s;
}

/* delta_l(k) in units of 2^(E_f-51-B) */
static u128 level_delta(const or_sel_meta* m, int l, int k) {
  int bl = m->bl[l];
  if (bl == 0 || k >= bl) return 0;
  if (k >= m->B && m->exact[l]) return 0;
  return pow2_sat(bl - k + m->B);
}

static u128 estimate(const or_sel_meta* m, const int* g) {
  u128 E = 0;
  int any = 0;
  for (int l = 0; l < m->nlev; l++) {
    u128 d = level_delta(m, l, 4 * g[l]);
    if (d) any = 1;
    E = add_sat(E, d);
  }
  u128 unitU = pow2_sat(m->B + 3);
  if (any) E = add_sat(E, (u128)(m->nlev) * unitU);   /* one floor per level */
  if (!m->input_exact) E = add_sat(E, unitU);         /* fixed-point floor of f */
  if (E == 0) return 0;                               /* exact reconstruction */
  /* final rounding of X*U to the output type */
  u128 eps;
  if (E < pow2_sat(m->B + 51)) {
    int e1, e2;
    if (m->dtype == OR_F32) {
      e1 = m->B + 27;            /* 2^(E_f-24) */
      e2 = m->B - 99 - m->E_f;   /* 2^-150 */
    } else {
      e1 = m->B - 2;             /* 2^(E_f-53) */
      e2 = m->B - 1024 - m->E_f; /* 2^-1075 */
    }
    eps = pow2_sat(e1 > e2 ? e1 : e2);
  } else {
    eps = E;                     /* |x_hat| may exceed 2^(E_f+1): generous */
  }
  return add_sat(E, eps);
}

void or_estimate(const or_sel_meta* m, const int* g, uint64_t* E_hi, uint64_t* E_lo) {
  u128 E = estimate(m, g);
  *E_hi = (uint64_t)(E >> 64);
  *E_lo = (uint64_t)E;
}

/* a before b: 2^(bl_a-k_a) * bytes_b > 2^(bl_b-k_b) * bytes_a, ties to smaller l */
static int better(const or_sel_meta* m, const int* g, int a, int b) {
  int sa = m->bl[a] - 4 * g[a], sb = m->bl[b] - 4 * g[b];
  u128 ba = m->group_bytes[a][g[a]], bb = m->group_bytes[b][g[b]];
  int lo = sa < sb ? sa : sb;
  u128 left = bb << (sa - lo), right = ba << (sb - lo);
  if (left != right) return left > right;
  return a < b;
}

int or_greedy_sequence(const or_sel_meta* m, int* seq, int cap) {
  int g[OR_MAX_LEVELS], n = 0;
  memset(g, 0, sizeof(g));
  for (;;) {
    int best = -1;
    for (int l = 0; l < m->nlev; l++) {
      if (g[l] >= m->ngroups[l]) continue;          /* exhausted */
      if (level_delta(m, l, 4 * g[l]) == 0) continue; /* nothing left to gain */
      if (best < 0 || better(m, g, l, best)) best = l;
    }
    if (best < 0) break;
    if (n < cap) seq[n] = best;
    n++;
    g[best]++;
  }
  return n;
}

void or_tau_units(double tau_abs, int E_f, int B, uint64_t* hi, uint64_t* lo) {
  u128 t;
  double x = ldexp(tau_abs, 51 + B - E_f);
  if (!(x >= 1.0)) t = 0;                        /* also catches NaN */
  else if (x >= ldexp(1.0, 127)) t = (u128)1 << 127;
  else {
    int e;
    double fr = frexp(x, &e);                    /* x = fr * 2^e, fr in [0.5,1) */
    uint64_t mant = (uint64_t)ldexp(fr, 53);     /* exact 53-bit integer */
    if (e >= 53) t = (u128)mant << (e - 53);
    else t = (u128)(mant >> (53 - e));           /* floor */
  }
  *hi = (uint64_t)(t >> 64);
  *lo = (uint64_t)t;
}

double or_units_to_abs(uint64_t hi, uint64_t lo, int E_f, int B) {
  double v = ldexp((double)hi, 64) + (double)lo;
  return ldexp(v, E_f - 51 - B);
}

int or_select(const or_sel_meta* m, double tau_abs, int* g, double* E_abs, uint64_t* E_hi,
              uint64_t* E_lo) {
  int seq[OR_MAX_LEVELS * 16];
  int n = or_greedy_sequence(m, seq, OR_MAX_LEVELS * 16);
  uint64_t th, tl;
  or_tau_units(tau_abs, m->E_f, m->B, &th, &tl);
  u128 tau = ((u128)th << 64) | tl;
  int status = OR_ERR_UNATTAINABLE;
  memset(g, 0, sizeof(int) * (size_t)m->nlev);
  u128 E = estimate(m, g);
  if (E <= tau) status = OR_OK;
  for (int i = 0; i < n && status != OR_OK; i++) {
    g[seq[i]]++;
    E = estimate(m, g);
    if (E <= tau) status = OR_OK;
  }
  *E_hi = (uint64_t)(E >> 64);
  *E_lo = (uint64_t)E;
  *E_abs = or_units_to_abs(*E_hi, *E_lo, m->E_f, m->B);
  return status;
}
