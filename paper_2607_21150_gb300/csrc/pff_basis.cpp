// One-dimensional bases of the tensor-product elements (Sec. 4: B_I, B_xi).
//
// Gauss-Lobatto-Legendre nodes by the Newton iteration on x P_p(x) - P_{p-1}(x)
// started from Chebyshev-Gauss-Lobatto points; Gauss-Legendre points by Newton
// on P_Q; Lagrange polynomials in barycentric form.
#include <cmath>
#include <vector>

#include "pff_internal.h"

namespace pff {

// Legendre polynomials P_0..P_n at x into out[0..n].
static void legendre_all(int n, double x, double* out) {
  out[0] = 1.0;
  if (n >= 1) out[1] = x;
  for (int k = 2; k <= n; ++k) out[k] = ((2 * k - 1) * x * out[k - 1] - (k - 1) * out[k - 2]) / k;
}

void gll_nodes(int p, double* x) {
  std::vector<double> L(p + 2);
  for (int i = 0; i <= p; ++i) {
    double xi = std::cos(M_PI * (double)(p - i) / (double)p);  // ascending
    for (int it = 0; it < 200; ++it) {
      legendre_all(p, xi, L.data());
      double Pp = L[p], Pm = (p >= 1) ? L[p - 1] : 0.0;
      double dx = (xi * Pp - Pm) / ((p + 1) * Pp);
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[i] = xi;
  }
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 0; i <= p / 2; ++i) {  // exact symmetry
    double s = 0.5 * (x[p - i] - x[i]);
    x[i] = -s;
    x[p - i] = s;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
}

void gauss_rule(int Q, double* x, double* w) {
  std::vector<double> L(Q + 1);
  for (int i = 0; i < Q; ++i) {
    double xi = -std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * Q + 2.0));
    double dP = 0.0;
    for (int it = 0; it < 200; ++it) {
      legendre_all(Q, xi, L.data());
      dP = Q * (xi * L[Q] - L[Q - 1]) / (xi * xi - 1.0);
      double dx = L[Q] / dP;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    legendre_all(Q, xi, L.data());
    dP = Q * (xi * L[Q] - L[Q - 1]) / (xi * xi - 1.0);
    x[i] = xi;
    w[i] = 2.0 / ((1.0 - xi * xi) * dP * dP);
  }
  for (int i = 0; i < Q / 2; ++i) {
    double s = 0.5 * (x[Q - 1 - i] - x[i]);
    double ws = 0.5 * (w[i] + w[Q - 1 - i]);
    x[i] = -s; x[Q - 1 - i] = s;
    w[i] = ws; w[Q - 1 - i] = ws;
  }
  if (Q % 2 == 1) x[Q / 2] = 0.0;
}

static double bary_weight(const double* nodes, int n, int a) {
  double prod = 1.0;
  for (int b = 0; b < n; ++b)
    if (b != a) prod *= (nodes[a] - nodes[b]);
  return 1.0 / prod;
}

double lagrange(const double* nodes, int n, int a, double t) {
  for (int b = 0; b < n; ++b)
    if (t == nodes[b]) return (a == b) ? 1.0 : 0.0;
  double num = bary_weight(nodes, n, a) / (t - nodes[a]);
  double den = 0.0;
  for (int b = 0; b < n; ++b) den += bary_weight(nodes, n, b) / (t - nodes[b]);
  return num / den;
}

double lagrange_deriv(const double* nodes, int n, int a, double t) {
  for (int c = 0; c < n; ++c) {
    if (t != nodes[c]) continue;
    if (c == a) {
      double s = 0.0;
      for (int b = 0; b < n; ++b)
        if (b != a) s += 1.0 / (nodes[a] - nodes[b]);
      return s;
    }
    return bary_weight(nodes, n, a) / (bary_weight(nodes, n, c) * (nodes[c] - nodes[a]));
  }
  double s = 0.0;
  for (int b = 0; b < n; ++b)
    if (b != a) s += 1.0 / (t - nodes[b]);
  return lagrange(nodes, n, a, t) * s;
}

}  // namespace pff
