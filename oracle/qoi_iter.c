/*
 * Oracle: progressive retrieval with QoI error control, iterated (Sec. 6.2,
 * Algorithm 3), for the total velocity QoI V = vx^2 + vy^2 + vz^2 of three
 * FP32 fields.  TEST INFRASTRUCTURE ONLY (see hpmdr_oracle.h).
 *
 * One iteration: retrieve every variable to its data bound eps_i (estimate
 * E_i <= eps_i), bound the QoI error of the reconstruction pointwise, take
 * the maximum tau'; stop when tau' <= tau, else choose the next data bounds:
 *   MA   (minimal augmentation): one more group of each variable's sequence;
 *   MAPE (MA with proportional estimation): p = tau'/tau; if p > c every
 *        bound becomes E_i / p, else MA;
 *   CP   (CPU porting): at the point of the largest bound, halve all bounds
 *        until that point's bound meets tau (reconstruction held fixed).
 * Initial bounds: eps_i = (tau / max V) * (max v_i - min v_i), the relative
 * QoI tolerance carried over to each variable's range.
 *
 * Pointwise bound: |x_hat^2 - x^2| <= 2 |x_hat| e + e^2 for |x_hat - x| <= e,
 * summed over the three variables, plus the output rounding of V_hat to FP32
 * (2^-24 V_hat, and 2^-150 in the subnormal range; infinite if V_hat exceeds
 * the FP32 range) and the two FP64 additions that form V_hat (2^-50 V_hat,
 * generous); the maximum over points is scaled by (1 + 2^-40) to absorb the
 * roundings of the bound's own evaluation.  Every operation is one FP64
 * operation in a fixed order (-ffp-contract=off), so the GPU, evaluating the
 * same operations, obtains the same numbers.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "hpmdr_oracle.h"

double or_vtotal(float x, float y, float z) {
  double a = (double)x * (double)x, b = (double)y * (double)y, c = (double)z * (double)z;
  double s = a + b;
  return s + c;
}

void or_vtotal_range(const float* vx, const float* vy, const float* vz, uint64_t N, double* vmin,
                     double* vmax) {
  double lo = 0.0, hi = 0.0;
  for (uint64_t i = 0; i < N; i++) {
    double v = or_vtotal(vx[i], vy[i], vz[i]);
    if (i == 0 || v < lo) lo = v;
    if (i == 0 || v > hi) hi = v;
  }
  *vmin = lo;
  *vmax = hi;
}

double or_vtotal_point_bound(float x, float y, float z, const double e[3]) {
  const float xs[3] = {x, y, z};
  double b = 0.0;
  for (int i = 0; i < 3; i++) {
    double t = 2.0 * fabs((double)xs[i]);
    t = t * e[i];
    double u = e[i] * e[i];
    t = t + u;
    b = b + t;
  }
  double v = or_vtotal(x, y, z);
  if (v > 0x1.fffffep127) return INFINITY;  /* V_hat does not fit FP32 */
  b = b + v * 0x1p-24;
  if (v != 0.0) b = b + 0x1p-150;  /* rounding into the FP32 subnormal range */
  b = b + v * 0x1p-50;
  return b;
}

double or_vtotal_bound(const float* x, const float* y, const float* z, uint64_t N,
                       const double e[3], uint64_t* arg) {
  double best = 0.0;
  uint64_t at = 0;
  for (uint64_t i = 0; i < N; i++) {
    double b = or_vtotal_point_bound(x[i], y[i], z[i], e);
    if (i == 0 || b > best) {
      best = b;
      at = i;
    }
  }
  if (arg) *arg = at;
  return best * (1.0 + 0x1p-40);
}

/* absolute estimate after the first k steps of the field's greedy sequence */
double or_field_prefix_estimate(const or_field* F, int k) {
  int seq[OR_MAX_LEVELS * 16], g[OR_MAX_LEVELS] = {0};
  int n = or_field_sequence(F, seq, OR_MAX_LEVELS * 16);
  if (k > n) k = n;
  for (int i = 0; i < k; i++) g[seq[i]]++;
  double E = 0.0;
  or_field_estimate(F, g, &E);
  return E;
}

int or_qoi_vtotal(const or_field* const F[3], uint64_t N, double vt_min, double vt_max,
                  double tau_rel, int estimator, double c, float* out[3], float* qoi,
                  or_qoi_report* rep) {
  memset(rep, 0, sizeof(*rep));
  const double tau = tau_rel * (vt_max - vt_min);
  rep->tau_abs = tau;
  double eps[3], E[3];
  int nseq[3];
  for (int i = 0; i < 3; i++) {
    int nlev, E_f, ie;
    double st[4];
    or_field_info(F[i], &nlev, &E_f, &ie, st);
    eps[i] = vt_max > 0.0 ? (tau / vt_max) * st[3] : 0.0;
    int seq[OR_MAX_LEVELS * 16];
    nseq[i] = or_field_sequence(F[i], seq, OR_MAX_LEVELS * 16);
  }
  int status = OR_ERR_UNATTAINABLE;
  for (int it = 1; it <= OR_QOI_MAX_ITERATIONS; it++) {
    int full = 1;
    for (int i = 0; i < 3; i++) {
      uint64_t hi, lo;
      or_field_select(F[i], eps[i], rep->g[i], &E[i], &hi, &lo);
      int k = 0;
      for (int l = 0; l < OR_MAX_LEVELS; l++) k += rep->g[i][l];
      rep->prefix[i] = k;
      if (k < nseq[i]) full = 0;
      or_reconstruct(F[i], rep->g[i], out[i]);
    }
    uint64_t arg = 0;
    const double bound = or_vtotal_bound(out[0], out[1], out[2], N, E, &arg);
    rep->iterations = it;
    rep->est = bound;
    for (int i = 0; i < 3; i++) rep->eps[i] = E[i];
    if (bound <= tau) {
      status = OR_OK;
      break;
    }
    if (full) break;
    int ma = estimator == OR_EST_MA;
    if (estimator == OR_EST_MAPE) {
      const double p = bound / tau;
      if (p > c) {
        for (int i = 0; i < 3; i++) eps[i] = E[i] / p;
      } else {
        ma = 1;
      }
    } else if (estimator == OR_EST_CP) {
      const float xs = out[0][arg], ys = out[1][arg], zs = out[2][arg];
      double e[3] = {E[0], E[1], E[2]};
      for (int k = 0; k < OR_QOI_MAX_HALVINGS; k++) {
        for (int i = 0; i < 3; i++) e[i] = e[i] * 0.5;
        if (or_vtotal_point_bound(xs, ys, zs, e) * (1.0 + 0x1p-40) <= tau) break;
      }
      for (int i = 0; i < 3; i++) eps[i] = e[i];
    }
    if (ma)
      for (int i = 0; i < 3; i++)
        if (rep->prefix[i] < nseq[i]) eps[i] = or_field_prefix_estimate(F[i], rep->prefix[i] + 1);
  }
  for (uint64_t p = 0; p < N; p++) qoi[p] = (float)or_vtotal(out[0][p], out[1][p], out[2][p]);
  rep->status = status;
  return status;
}
