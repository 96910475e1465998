/*
 * Oracle: QoI error control for the velocity magnitude |v| = sqrt(vx^2 +
 * vy^2 + vz^2).  TEST INFRASTRUCTURE ONLY (see hpmdr_oracle.h).
 *
 * Sec. 6.2 / Algorithm 3 retrieve every variable to a data bound eps_i, bound
 * the QoI error, and tighten until it meets tau.  For |v| a closed form ends
 * the loop after one pass: by the reverse triangle inequality
 * | |v_hat| - |v| | <= |v_hat - v|_2 <= sqrt(sum eps_i^2).  |v| is evaluated in
 * FP32 with one rounding per operation (three products, two sums, a square
 * root: relative error below 3 * 2^-24 for each side), so each component is
 * asked for eps = (tau - slack) / sqrt(3) with slack = 7 * 2^-24 * (max|v| + tau),
 * and the reported bound is r + 7 * 2^-24 * (max|v| + r), r = sqrt(sum E_i^2).
 */
#include <math.h>

#include "hpmdr_oracle.h"

float or_vmag(float x, float y, float z) {
  float xx = x * x, yy = y * y, zz = z * z; /* -ffp-contract=off: no FMA */
  float s = xx + yy;
  s = s + zz;
  return sqrtf(s);
}

void or_vmag_field(const float* vx, const float* vy, const float* vz, uint64_t N, float* out,
                   float* qmin, float* qmax) {
  float lo = 0.0f, hi = 0.0f;
  for (uint64_t i = 0; i < N; i++) {
    float q = or_vmag(vx[i], vy[i], vz[i]);
    if (out) out[i] = q;
    if (i == 0 || q < lo) lo = q;
    if (i == 0 || q > hi) hi = q;
  }
  if (qmin) *qmin = lo;
  if (qmax) *qmax = hi;
}

double or_qoi_component_bound(double tau_q_abs, double qmax) {
  double slack = 7.0 * ldexp(1.0, -24) * (qmax + tau_q_abs);
  double eps = (tau_q_abs - slack) / sqrt(3.0);
  eps = eps * (1.0 - ldexp(1.0, -50)); /* absorb the roundings of this line */
  return eps > 0.0 ? eps : 0.0;
}

double or_qoi_estimate(double Ex, double Ey, double Ez, double qmax) {
  double r = sqrt(Ex * Ex + Ey * Ey + Ez * Ez);
  return (r + 7.0 * ldexp(1.0, -24) * (qmax + r)) * (1.0 + ldexp(1.0, -50));
}
