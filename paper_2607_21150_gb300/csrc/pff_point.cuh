// Device helpers of the pointwise kernels (principal-stress format, App. A):
// Voigt indices, cyclic Jacobi eigen-decomposition, stable divided differences.
#pragma once
#include <cmath>

#include "pff_df.cuh"
#include "pff_internal.h"

namespace pff {

static __device__ __forceinline__ void vo_idx(int v, int& r, int& c) {
  const int I[6] = {0, 1, 2, 1, 0, 0};
  const int J[6] = {0, 1, 2, 2, 2, 1};
  r = I[v]; c = J[v];
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (in place).
// On exit w = eigenvalues, V columns = eigenvectors.  Returns 0 when the
// off-diagonal part vanished within the sweep cap.  Each rotation annihilates
// A[p][q] with tan(phi) = t the smaller root of t^2 + 2 theta t - 1 = 0,
// theta = (A_qq - A_pp) / (2 A_pq), written as
//   t = sgn 2 |A_pq| / (|A_qq - A_pp| + sqrt((A_qq - A_pp)^2 + 4 A_pq^2)),
// c = 1 / sqrt(1 + t^2), s = t c: one division, one square root and one
// reciprocal square root per rotation (the FP64 pipe is the binding unit).
static __device__ inline int jacobi3(double A[3][3], double V[3][3], double w[3]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) V[r][c] = (r == c) ? 1.0 : 0.0;
  int ok = 0;
  for (int sweep = 0; sweep < 20; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-36 * dia || off < 1e-300) { ok = 1; break; }
    for (int pr = 0; pr < 3; ++pr) {
      const int p = (pr == 2) ? 1 : 0;
      const int q = (pr == 0) ? 1 : 2;
      const double apq = A[p][q];
      if (apq == 0.0) continue;
      const double diff = A[q][q] - A[p][p];
      const double sgn = ((diff >= 0.0) == (apq > 0.0) || diff == 0.0) ? 1.0 : -1.0;
      const double t = sgn * 2.0 * fabs(apq) / (fabs(diff) + sqrt(diff * diff + 4.0 * apq * apq));
      const double c = rsqrt(fma(t, t, 1.0));
      const double s = t * c;
      A[p][p] -= t * apq;
      A[q][q] += t * apq;
      A[p][q] = A[q][p] = 0.0;
      const int r = 3 - p - q;
      const double arp = A[r][p], arq = A[r][q];
      A[r][p] = A[p][r] = c * arp - s * arq;
      A[r][q] = A[q][r] = s * arp + c * arq;
      for (int k = 0; k < 3; ++k) {
        const double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
  w[0] = A[0][0]; w[1] = A[1][1]; w[2] = A[2][2];
  return ok;
}

// Yield stress of the Prandtl branch and its slope H = d sigma_y / d ep (Eq.
// plasticity-strain-hardening-law: linear + Voce).
static __device__ __forceinline__ double yield_stress(const PhaseDev& ph, double ep) {
  if (!ph.hard) return ph.sig0;
  return ph.sig0 + ph.Hlin * ep + (ph.sinf - ph.sig0) * (1.0 - exp(-ph.beta * ep));
}
static __device__ __forceinline__ double yield_slope(const PhaseDev& ph, double ep) {
  if (!ph.hard) return 0.0;
  return ph.Hlin + (ph.sinf - ph.sig0) * ph.beta * exp(-ph.beta * ep);
}

// Plastic step of Box 2 with the degraded trial stress: the root dgam of
//   g q_tr - 3 g mu dgam - sigma_y(ep_n + dgam) = 0
// by Newton from the linearised step; perfect plasticity is the first step.
// Sets *ok = 0 when 50 iterations leave |f| > 1e-14 max(sigma_y, g q_tr).
static __device__ inline double return_map(const PhaseDev& ph, double g, double mu, double qtr, double epn, int* ok) {
  const double f0 = g * qtr - yield_stress(ph, epn);
  double dg = f0 / (3.0 * g * mu + yield_slope(ph, epn));
  *ok = 1;
  if (!ph.hard) return dg;
  for (int it = 0; it < 50; ++it) {
    const double sy = yield_stress(ph, epn + dg);
    const double f = g * qtr - 3.0 * g * mu * dg - sy;
    if (fabs(f) <= 1e-14 * fmax(sy, g * qtr)) return dg;
    dg += f / (3.0 * g * mu + yield_slope(ph, epn + dg));
  }
  *ok = 0;
  return dg;
}

// (ln b_p - ln b_q) / (b_p - b_q) from the eigenvalues x = b - 1:
// log1p(y) / (y b_q) with y = (b_p - b_q) / b_q.  For |y| < 1/64 the Taylor
// series of log1p(y) / y to y^8 (remainder below y^9 / 10 < 2e-17) replaces the
// logarithm and the division.
static __device__ __forceinline__ double log_ratio(double xp, double xq) {
  const double rb = 1.0 / (1.0 + xq);
  const double y = (xp - xq) * rb;
  double l1;
  if (fabs(y) < 0.015625) {
    l1 = 1.0 / 9.0;
    l1 = fma(l1, -y, 1.0 / 8.0);
    l1 = fma(l1, -y, 1.0 / 7.0);
    l1 = fma(l1, -y, 1.0 / 6.0);
    l1 = fma(l1, -y, 1.0 / 5.0);
    l1 = fma(l1, -y, 1.0 / 4.0);
    l1 = fma(l1, -y, 1.0 / 3.0);
    l1 = fma(l1, -y, 1.0 / 2.0);
    l1 = fma(l1, -y, 1.0);
  } else {
    l1 = log1p(y) / y;
  }
  return l1 * rb;
}

// log_ratio for the tangent, in double-float on the FP32 pipes: 1 / b_q by one
// double-float Newton step from the FP32 reciprocal, the Taylor series in
// double-float; |y| >= 1/64 (eigenvalues 1.6 % apart or more) takes the FP64
// function.  About 2^-46 relative.
static __device__ __forceinline__ df64 df_rcp(df64 b) {
  const df64 r0 = df_make(__frcp_rn(b.hi), 0.0f);
  const df64 e = df_sub(df_make(1.0f, 0.0f), df_mul(b, r0));
  return df_madd(r0, r0, e);
}
static __device__ __forceinline__ df64 log_ratio_df(double xp, double xq) {
  const df64 rb = df_rcp(df_add(df_make(1.0f, 0.0f), df_split(xq)));
  const df64 y = df_mul(df_split(xp - xq), rb);
  if (!(fabsf(y.hi) < 0.015625f)) return df_split(log_ratio(xp, xq));
  const df64 ny = df_neg(y);
  df64 l1 = df_split(1.0 / 9.0);
  l1 = df_madd(df_split(1.0 / 8.0), l1, ny);
  l1 = df_madd(df_split(1.0 / 7.0), l1, ny);
  l1 = df_madd(df_split(1.0 / 6.0), l1, ny);
  l1 = df_madd(df_split(1.0 / 5.0), l1, ny);
  l1 = df_madd(df_split(1.0 / 4.0), l1, ny);
  l1 = df_madd(df_split(1.0 / 3.0), l1, ny);
  l1 = df_madd(df_split(1.0 / 2.0), l1, ny);
  l1 = df_madd(df_make(1.0f, 0.0f), l1, ny);
  return df_mul(l1, rb);
}


}  // namespace pff
