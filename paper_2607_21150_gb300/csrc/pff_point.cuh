// Device helpers of the pointwise kernels (principal-stress format, App. A):
// Voigt indices, cyclic Jacobi eigen-decomposition, stable divided differences.
#pragma once
#include <cmath>

#include "pff_internal.h"

namespace pff {

static __device__ __forceinline__ void vo_idx(int v, int& r, int& c) {
  const int I[6] = {0, 1, 2, 1, 0, 0};
  const int J[6] = {0, 1, 2, 2, 2, 1};
  r = I[v]; c = J[v];
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (in place).
// On exit w = eigenvalues, V columns = eigenvectors.  Returns 0 when the
// off-diagonal part vanished within the sweep cap.
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
      double apq = A[p][q];
      if (apq == 0.0) continue;
      double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
      double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0);
      double s = t * c;
      double tau = s / (1.0 + c);
      A[p][p] -= t * apq;
      A[q][q] += t * apq;
      A[p][q] = A[q][p] = 0.0;
      const int r = 3 - p - q;
      double arp = A[r][p], arq = A[r][q];
      A[r][p] = A[p][r] = arp - s * (arq + tau * arp);
      A[r][q] = A[q][r] = arq + s * (arp - tau * arq);
      for (int k = 0; k < 3; ++k) {
        double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = vkp - s * (vkq + tau * vkp);
        V[k][q] = vkq + s * (vkp - tau * vkq);
      }
    }
  }
  w[0] = A[0][0]; w[1] = A[1][1]; w[2] = A[2][2];
  return ok;
}

// (ln b_p - ln b_q) / (b_p - b_q) from the eigenvalues x = b - 1.
static __device__ __forceinline__ double log_ratio(double xp, double xq) {
  double bq = 1.0 + xq;
  double y = (xp - xq) / bq;
  double l1;
  if (fabs(y) < 1e-4) l1 = 1.0 - y * (0.5 - y * (1.0 / 3.0 - 0.25 * y));
  else l1 = log1p(y) / y;
  return l1 / bq;
}


}  // namespace pff
