// Plain FP64 CPU oracle for the matrix-free phase-field fracture operator.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file; only the tests, the package smoke check and the CPU
// baseline leg of the benchmark do.  It shares no code, header, table or
// constant generator with the CUDA library.
//
// What it computes (paper: "Matrix-free phase-field modeling of fracture in
// micromechanical testing simulations of inelastic materials"):
//   * the pointwise Peric-Dettmer update of Box 1 with the Hooke, Maxwell and
//     Prandtl branches, the last perfectly plastic or hardening (linear +
//     Voce, Eq. plasticity-strain-hardening-law, Box 2 local Newton carried
//     in dual numbers) (Sec. 2.3, Eqs. hencky-tau-current,
//     viscoelasticity-deviatoric-strain-update-hencky,
//     plasticity-deviatoric-strain-update-perfect), degraded in series by the
//     fracture element of Sec. 3 (Eqs. linear-Psi-plus,
//     linear-degraded-stress, degraded-trial-stress,
//     principal-directions-format-1, degr-funct, L-viscous);
//   * the weak-form integrands of Sec. 4 (Eq. physical-residual-integrands),
//     pulled back to the reference frame with the identities of
//     Eqs. mechanical-gradient-transformation and
//     phase-gradient-transformation;
//   * element residuals and element matrices by FULL quadrature (every 3D
//     basis function evaluated at every Gauss point, no sum factorisation),
//     assembled into CSR (Eqs. matrix-free-residual-compact and
//     matrix-free-jacobian written as plain sums over elements and points).
//
// Deliberately a different route from the GPU path:
//   * Hencky strains as MATRIX functions (log of I + X by a power series,
//     with inverse scaling and squaring when |X| > 1/4) instead of the
//     principal-stress format of Appendix A;
//   * the consistent tangent by forward-mode dual numbers with 13 seed
//     directions (grad u: 9, phi: 1, grad phi: 3) instead of the closed forms
//     of Appendix B / Box A1 and Appendix C.  Branch decisions (yield, history
//     activity, sign of the volumetric strain) are taken on primal values and
//     frozen, exactly as the linearisation of Appendix C does.
//
// Readings of points the paper leaves open:
//   R1  theta = ln J is the volumetric strain of every branch and decides the
//       Amor split; each branch's deviator uses its own trace.
//   R4  the history is active iff psi+ > H_n (strict).
//   R5  theta >= 0 selects the tensile case.  R6: g q_tr - sigma0 <= 0 is
//       elastic.  phi_dot = (phi - phi_n) / dt (backward Euler).
//   Commit: eps_e = a * dev(eps_tr) + theta/3 I, C_in^-1 = F^-1 exp(2 eps_e) F^-T.
//
// Conventions (the same numbers the CUDA library documents in its header):
//   box mesh nx*ny*nz elements of size hx,hy,hz, order p (P = p+1 GLL nodes
//   per direction), Q Gauss points per direction; node (I,J,K) has id
//   I + nnx*(J + nny*K), nnx = p*nx+1; DoF vector SoA [4][N_n] (ux,uy,uz,phi);
//   element e = ex + nx*(ey + ny*ez); quadrature point q = e*Q^3 + i + Q*(j + Q*k);
//   history SoA [15][N_q]: C_M (Voigt 11,22,33,23,13,12), C_P (Voigt),
//   eps_p_bar, H, phi_n.  Flags: bit0 Prandtl yield, bit1 history active,
//   bit2 theta >= 0.
//
// Parity pins for every function here live in tests/test_oracle_*.py.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ----------------------------------------------------------------------------
// Forward-mode dual numbers
// ----------------------------------------------------------------------------
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
};
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r;
}
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r; r.v = a.v * b; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b; return r;
}
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r; r.v = std::sqrt(a.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v); return r;
}
template <int N> inline Dual<N> exp(const Dual<N>& a) {
  Dual<N> r; r.v = std::exp(a.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * r.v; return r;
}
template <int N> inline Dual<N> log1p(const Dual<N>& a) {
  Dual<N> r; r.v = std::log1p(a.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (1.0 + a.v); return r;
}
inline double val(double x) { return x; }
template <int N> inline double val(const Dual<N>& x) { return x.v; }
using std::sqrt;
using std::log1p;
using std::exp;

// ----------------------------------------------------------------------------
// 3x3 matrices
// ----------------------------------------------------------------------------
template <typename T> struct M3 { T a[3][3]; };
template <typename T> M3<T> zero3() { M3<T> m; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) m.a[i][j] = T(0.0); return m; }
template <typename T> M3<T> eye3() { M3<T> m = zero3<T>(); for (int i = 0; i < 3; ++i) m.a[i][i] = T(1.0); return m; }
template <typename T> M3<T> mul(const M3<T>& A, const M3<T>& B) {
  M3<T> C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = A.a[i][0] * B.a[0][j];
      s = s + A.a[i][1] * B.a[1][j];
      s = s + A.a[i][2] * B.a[2][j];
      C.a[i][j] = s;
    }
  return C;
}
template <typename T> M3<T> transpose(const M3<T>& A) {
  M3<T> C; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) C.a[i][j] = A.a[j][i]; return C;
}
template <typename T> M3<T> add(const M3<T>& A, const M3<T>& B) {
  M3<T> C; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) C.a[i][j] = A.a[i][j] + B.a[i][j]; return C;
}
template <typename T> M3<T> sub(const M3<T>& A, const M3<T>& B) {
  M3<T> C; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) C.a[i][j] = A.a[i][j] - B.a[i][j]; return C;
}
template <typename T, typename S> M3<T> scale(const M3<T>& A, const S& s) {
  M3<T> C; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) C.a[i][j] = A.a[i][j] * s; return C;
}
template <typename T> T trace(const M3<T>& A) { return A.a[0][0] + A.a[1][1] + A.a[2][2]; }
template <typename T> T ddot(const M3<T>& A, const M3<T>& B) {
  T s = T(0.0); for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) s = s + A.a[i][j] * B.a[i][j]; return s;
}
template <typename T> T det3(const M3<T>& A) {
  return A.a[0][0] * (A.a[1][1] * A.a[2][2] - A.a[1][2] * A.a[2][1])
       - A.a[0][1] * (A.a[1][0] * A.a[2][2] - A.a[1][2] * A.a[2][0])
       + A.a[0][2] * (A.a[1][0] * A.a[2][1] - A.a[1][1] * A.a[2][0]);
}
// Inverse by the adjugate (cofactor transpose) divided by the determinant.
template <typename T> M3<T> inverse(const M3<T>& A, const T& det) {
  M3<T> C;
  C.a[0][0] = (A.a[1][1] * A.a[2][2] - A.a[1][2] * A.a[2][1]) / det;
  C.a[0][1] = (A.a[0][2] * A.a[2][1] - A.a[0][1] * A.a[2][2]) / det;
  C.a[0][2] = (A.a[0][1] * A.a[1][2] - A.a[0][2] * A.a[1][1]) / det;
  C.a[1][0] = (A.a[1][2] * A.a[2][0] - A.a[1][0] * A.a[2][2]) / det;
  C.a[1][1] = (A.a[0][0] * A.a[2][2] - A.a[0][2] * A.a[2][0]) / det;
  C.a[1][2] = (A.a[0][2] * A.a[1][0] - A.a[0][0] * A.a[1][2]) / det;
  C.a[2][0] = (A.a[1][0] * A.a[2][1] - A.a[1][1] * A.a[2][0]) / det;
  C.a[2][1] = (A.a[0][1] * A.a[2][0] - A.a[0][0] * A.a[2][1]) / det;
  C.a[2][2] = (A.a[0][0] * A.a[1][1] - A.a[0][1] * A.a[1][0]) / det;
  return C;
}
template <typename T> double frob_val(const M3<T>& A) {
  double s = 0.0; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) s += val(A.a[i][j]) * val(A.a[i][j]); return std::sqrt(s);
}

// log(I + X) for |X|_F <= 1/4 by the power series sum_k (-1)^(k+1) X^k / k
// (the Hencky strain eps = log(b)/2 of Sec. 2.2 with b = I + X, taken as a
// matrix function; X is formed without b, the log1p form of Sec. 2.2).
// The number of terms makes |X|^(k-1) < 1e-19 so that both the value and its
// first derivative are converged to below FP64 rounding.
template <typename T> M3<T> log1p_series(const M3<T>& X) {
  double r = frob_val(X);
  int kmax = 1;
  if (r > 0.0) {
    kmax = (int)std::ceil(std::log(1e-19) / std::log(r)) + 1;
    if (kmax < 2) kmax = 2;
    if (kmax > 200) kmax = 200;
  }
  M3<T> S = X, Pk = X;
  for (int k = 2; k <= kmax; ++k) {
    Pk = mul(Pk, X);
    double c = ((k % 2) ? 1.0 : -1.0) / (double)k;
    S = add(S, scale(Pk, c));
  }
  return S;
}
// Principal square root by the Denman-Beavers iteration (Y -> A^(1/2)).
template <typename T> M3<T> sqrtm_db(const M3<T>& A) {
  M3<T> Y = A, Z = eye3<T>();
  for (int it = 0; it < 60; ++it) {
    M3<T> Yi = inverse(Y, det3(Y));
    M3<T> Zi = inverse(Z, det3(Z));
    M3<T> Yn = scale(add(Y, Zi), 0.5);
    M3<T> Zn = scale(add(Z, Yi), 0.5);
    double dy = frob_val(sub(Yn, Y));
    Y = Yn; Z = Zn;
    if (dy < 1e-17 * frob_val(Y) && it > 3) {
      // two extra sweeps so that the derivative parts settle as well
      for (int e = 0; e < 2; ++e) {
        M3<T> Yi2 = inverse(Y, det3(Y));
        M3<T> Zi2 = inverse(Z, det3(Z));
        M3<T> Y2 = scale(add(Y, Zi2), 0.5);
        M3<T> Z2 = scale(add(Z, Yi2), 0.5);
        Y = Y2; Z = Z2;
      }
      break;
    }
  }
  return Y;
}
// log(I + X) (Sec. 2.2): the series when small, else inverse scaling and squaring
// (square roots until the argument is within 1/4 of I, then 2^s times the series).
template <typename T> M3<T> logm_1p(const M3<T>& X) {
  if (frob_val(X) <= 0.25) return log1p_series(X);
  M3<T> A = add(eye3<T>(), X);
  int s = 0;
  M3<T> Xs = X;
  while (frob_val(Xs) > 0.25 && s < 60) {
    A = sqrtm_db(A);
    Xs = sub(A, eye3<T>());
    ++s;
  }
  return scale(log1p_series(Xs), std::ldexp(1.0, s));
}
// exp(A) by scaling and squaring of the Taylor series (primal only): the
// exponential map of the history commit, Box 1 step 4.
M3<double> expm(const M3<double>& A) {
  double r = frob_val(A);
  int s = 0;
  while (r > 0.25) { r *= 0.5; ++s; }
  M3<double> As = scale(A, std::ldexp(1.0, -s));
  M3<double> S = eye3<double>(), term = eye3<double>();
  for (int k = 1; k < 40; ++k) {
    term = scale(mul(term, As), 1.0 / (double)k);
    S = add(S, term);
    if (frob_val(term) < 1e-22) break;
  }
  for (int i = 0; i < s; ++i) S = mul(S, S);
  return S;
}

// ----------------------------------------------------------------------------
// Material description
// ----------------------------------------------------------------------------
// Phase parameters, kPhaseWords = 15 doubles: Gc, l0, E_inf, nu_inf, hasM, E1,
// nu1, eta_d, hasP, E2, nu2, sigma0, H_lin, sigma_inf, beta (units mm, MPa, s;
// eta_d = +inf allowed).  The last three are the linear + Voce hardening law of
// the Prandtl branch (Eq. plasticity-strain-hardening-law); H_lin = 0,
// sigma_inf = sigma0 is perfect plasticity.
static const int kPhaseWords = 15;
template <typename T>
struct PhaseT {
  T Gc, l0, E0, nu0;
  int hasM; T E1, nu1, eta; bool eta_inf;
  int hasP; T E2, nu2, sig0;
  T Hlin, sinf, beta;
};
typedef PhaseT<double> Phase;
// Global parameters, 5 doubles: AT (1 or 2), eta (residual stiffness),
// zeta (damage viscosity), dt, s_phi.
struct Glob { int at; double eta_res, zeta, dt, s_phi; };

static Phase read_phase(const double* p) {
  Phase ph;
  ph.Gc = p[0]; ph.l0 = p[1]; ph.E0 = p[2]; ph.nu0 = p[3];
  ph.hasM = p[4] != 0.0; ph.E1 = p[5]; ph.nu1 = p[6]; ph.eta = p[7]; ph.eta_inf = !std::isfinite(p[7]);
  ph.hasP = p[8] != 0.0; ph.E2 = p[9]; ph.nu2 = p[10]; ph.sig0 = p[11];
  ph.Hlin = p[12]; ph.sinf = p[13]; ph.beta = p[14];
  return ph;
}
template <typename T> PhaseT<T> lift(const Phase& p) {
  PhaseT<T> q;
  q.Gc = T(p.Gc); q.l0 = T(p.l0); q.E0 = T(p.E0); q.nu0 = T(p.nu0);
  q.hasM = p.hasM; q.E1 = T(p.E1); q.nu1 = T(p.nu1); q.eta = T(p.eta_inf ? 1.0 : p.eta); q.eta_inf = p.eta_inf;
  q.hasP = p.hasP; q.E2 = T(p.E2); q.nu2 = T(p.nu2); q.sig0 = T(p.sig0);
  q.Hlin = T(p.Hlin); q.sinf = T(p.sinf); q.beta = T(p.beta);
  return q;
}

// Yield stress of the hardening law (Eq. plasticity-strain-hardening-law) and
// its slope H = d sigma_y / d eps_p.
template <typename T>
T yield_stress(const PhaseT<T>& ph, const T& ep) {
  return ph.sig0 + ph.Hlin * ep + (ph.sinf - ph.sig0) * (1.0 - exp(-ph.beta * ep));
}
template <typename T>
T yield_slope(const PhaseT<T>& ph, const T& ep) {
  return ph.Hlin + (ph.sinf - ph.sig0) * ph.beta * exp(-ph.beta * ep);
}
static Glob read_glob(const double* g) {
  Glob gl; gl.at = (int)g[0]; gl.eta_res = g[1]; gl.zeta = g[2]; gl.dt = g[3]; gl.s_phi = g[4];
  return gl;
}

static const int VOIGT_I[6] = {0, 1, 2, 1, 0, 0};
static const int VOIGT_J[6] = {0, 1, 2, 2, 2, 1};

// exp(A) by scaling and squaring of the Taylor series (term count and scaling
// decided on primal values, so that dual parts follow the same expression);
// the exponential map of Box 1 step 4 inside the differentiated path.
template <typename T> M3<T> expm_t(const M3<T>& A) {
  double r = frob_val(A);
  int s = 0;
  while (r > 0.25) { r *= 0.5; ++s; }
  M3<T> As = scale(A, std::ldexp(1.0, -s));
  M3<T> S = eye3<T>(), term = eye3<T>();
  for (int k = 1; k < 40; ++k) {
    term = scale(mul(term, As), 1.0 / (double)k);
    S = add(S, term);
    if (frob_val(term) < 1e-22) break;
  }
  for (int i = 0; i < s; ++i) S = mul(S, S);
  return S;
}

template <typename T>
struct PointResult {
  T f0[4];
  T f1[4][3];
  T hist_new[15];
  uint8_t flags;
  double psi_plus, margin_yield, margin_hist, theta;
};

// Pointwise update at one quadrature point.  G = grad_X u (G[i][A] = du_i/dX_A),
// phi, gphi = grad_X phi; hist = committed history (15 words); ph = the
// point's phase parameters; commit = also produce the trial history of Box 1
// step 4.  Every input may carry dual parts (history and parameters included),
// so the same function gives the tangent and the adjoint's local partials.
template <typename T>
void pointwise(const T G[3][3], const T& phi, const T gphi[3], const T* hist,
               const PhaseT<T>& ph, const Glob& gl, bool commit, PointResult<T>& out) {
  M3<T> Gm;
  for (int i = 0; i < 3; ++i) for (int A = 0; A < 3; ++A) Gm.a[i][A] = G[i][A];
  M3<T> F = add(eye3<T>(), Gm);
  // J - 1 = tr G + I2(G) + det G (principal invariants, no cancellation)
  T trG = trace(Gm);
  T I2 = 0.5 * (trG * trG - trace(mul(Gm, Gm)));
  T Jm1 = trG + I2 + det3(Gm);
  T theta = log1p(Jm1);
  T J = 1.0 + Jm1;
  M3<T> Finv = inverse(F, J);
  M3<T> GGt = add(add(Gm, transpose(Gm)), mul(Gm, transpose(Gm)));  // F F^T - I

  // degradation function g = (1-phi)^2 + eta (Eq. degr-funct)
  T omp = 1.0 - phi;
  T g = omp * omp + gl.eta_res;
  T gp = -2.0 * omp;

  M3<T> taud = zero3<T>();
  T psid = T(0.0);
  T kap_tot = T(0.0);
  out.flags = 0;
  out.margin_yield = INFINITY;  // no yield decision without a Prandtl branch
  T dgam = T(0.0);
  M3<T> epsE_M = zero3<T>(), epsE_P = zero3<T>();

  for (int br = 0; br < 3; ++br) {
    T E, nu;
    const T* Ch = nullptr;
    if (br == 0) { E = ph.E0; nu = ph.nu0; }
    else if (br == 1) { if (!ph.hasM) continue; E = ph.E1; nu = ph.nu1; Ch = hist + 0; }
    else { if (!ph.hasP) continue; E = ph.E2; nu = ph.nu2; Ch = hist + 6; }
    T mu = E / (2.0 * (1.0 + nu));
    T kap = E / (3.0 * (1.0 - 2.0 * nu));
    kap_tot = kap_tot + kap;
    // Elastic predictor (Box 1 step 1): b_tr - I = F (C - I) F^T + (F F^T - I)
    M3<T> X = GGt;
    if (Ch) {
      M3<T> CmI;
      for (int v = 0; v < 6; ++v) {
        T c = Ch[v] - (v < 3 ? 1.0 : 0.0);
        CmI.a[VOIGT_I[v]][VOIGT_J[v]] = c;
        CmI.a[VOIGT_J[v]][VOIGT_I[v]] = c;
      }
      X = add(X, mul(mul(F, CmI), transpose(F)));
    }
    // Hencky trial strain eps_tr = 1/2 log(b_tr) as a matrix function
    M3<T> Etr = scale(logm_1p(X), 0.5);
    T trE = trace(Etr);
    M3<T> Ed = sub(Etr, scale(eye3<T>(), trE / 3.0));
    T s = ddot(Ed, Ed);
    // Correction step (Box 1 step 2) with degradation inside the branch (Sec. 3)
    T a = T(1.0);
    if (br == 1) {
      if (!ph.eta_inf) a = 1.0 / (1.0 + g * (mu * gl.dt / ph.eta));
    } else if (br == 2) {
      // Box 2 with the degraded trial stress (reading: g multiplies q_tr and the
      // 3 mu dgam term, not sigma_y): admissible iff g q_tr - sigma_y(eps_p,n) <= 0
      const T& epn = hist[12];
      double qv = 2.0 * val(mu) * std::sqrt(1.5 * val(s));
      double sy0 = val(yield_stress(ph, epn));
      double fv = val(g) * qv - sy0;
      out.margin_yield = fv / sy0;
      if (fv > 0.0) {
        T q = 2.0 * mu * sqrt(1.5 * s);
        // plastic step: Newton on f(dgam) = g q_tr - 3 g mu dgam - sigma_y(eps_p,n + dgam),
        // from dgam = 0, to |f| <= 1e-14 sigma_y, then two more iterations so that
        // the dual parts (implicit derivatives) converge with the value
        T dg = T(0.0);
        int extra = 0;
        for (int it = 0; it < 60; ++it) {
          T f = g * q - 3.0 * g * mu * dg - yield_stress(ph, epn + dg);
          T den = -3.0 * g * mu - yield_slope(ph, epn + dg);
          dg = dg - f / den;
          if (std::fabs(val(f)) <= 1e-14 * sy0 && ++extra > 2) break;
        }
        dgam = dg;
        a = 1.0 - 3.0 * mu * dg / q;
        out.flags |= 1;
      }
    }
    taud = add(taud, scale(Ed, 2.0 * mu * a));
    psid = psid + mu * a * a * s;
    if (commit && Ch) {
      M3<T> e = add(scale(Ed, a), scale(eye3<T>(), theta / 3.0));
      if (br == 1) epsE_M = e; else epsE_P = e;
    }
  }
  // volumetric part (R1): tau_v = kappa theta I, psi_v = kappa theta^2 / 2
  T tauv = kap_tot * theta;
  T psiv = 0.5 * kap_tot * theta * theta;
  bool tens = val(theta) >= 0.0;
  if (tens) out.flags |= 4;
  T psip;
  M3<T> taudeg;
  if (tens) {  // Eqs. linear-Psi-plus and linear-degraded-stress, tr >= 0
    psip = psid + psiv;
    taudeg = scale(add(taud, scale(eye3<T>(), tauv)), g);
  } else {
    psip = psid;
    taudeg = add(scale(taud, g), scale(eye3<T>(), tauv));
  }
  // Miehe history field (Sec. 3.3), strict activity (R4)
  const T& Hn = hist[13];
  bool active = val(psip) > val(Hn);
  if (active) out.flags |= 2;
  T H = active ? psip : Hn;
  double denom = std::max(std::fabs(val(Hn)), std::fabs(val(psip)));
  out.margin_hist = denom > 0 ? (val(psip) - val(Hn)) / denom : 0.0;
  // local phase-field residual L (Eq. L-viscous)
  double c0 = (gl.at == 1) ? 8.0 / 3.0 : 2.0;
  T alphap = (gl.at == 1) ? T(1.0) : 2.0 * phi;
  T L = gp * H + (ph.Gc / (c0 * ph.l0)) * alphap + gl.zeta * (phi - hist[14]) / gl.dt;
  // integrands in the reference frame: P = tau_degr F^-T, s_phi L, s_phi k grad_X phi
  for (int i = 0; i < 3; ++i) out.f0[i] = T(0.0);
  out.f0[3] = gl.s_phi * L;
  for (int i = 0; i < 3; ++i)
    for (int A = 0; A < 3; ++A) {
      T s = taudeg.a[i][0] * Finv.a[A][0];
      s = s + taudeg.a[i][1] * Finv.a[A][1];
      s = s + taudeg.a[i][2] * Finv.a[A][2];
      out.f1[i][A] = s;
    }
  T kphi = gl.s_phi * 2.0 * ph.Gc * ph.l0 / c0;
  for (int A = 0; A < 3; ++A) out.f1[3][A] = kphi * gphi[A];
  out.psi_plus = val(psip);
  out.theta = val(theta);

  if (commit) {
    // Box 1 step 4: C_in^-1 = F^-1 exp(2 eps_e) F^-T, plus eps_p, H, phi_n
    for (int v = 0; v < 15; ++v) out.hist_new[v] = hist[v];
    M3<T> FiT = transpose(Finv);
    if (ph.hasM) {
      M3<T> C = mul(mul(Finv, expm_t(scale(epsE_M, 2.0))), FiT);
      for (int v = 0; v < 6; ++v) out.hist_new[v] = C.a[VOIGT_I[v]][VOIGT_J[v]];
    }
    if (ph.hasP) {
      M3<T> C = mul(mul(Finv, expm_t(scale(epsE_P, 2.0))), FiT);
      for (int v = 0; v < 6; ++v) out.hist_new[6 + v] = C.a[VOIGT_I[v]][VOIGT_J[v]];
      out.hist_new[12] = hist[12] + dgam;
    }
    out.hist_new[13] = H;
    out.hist_new[14] = phi;
  }
}

// ----------------------------------------------------------------------------
// 1D bases: Gauss-Legendre and Gauss-Lobatto-Legendre points, Lagrange
// polynomials (Sec. 4: B_I and B_xi are tensor products of these)
// ----------------------------------------------------------------------------
// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
static void legendre(int n, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = p2;
  }
  P = p1;
  dP = (std::fabs(x) < 1.0) ? n * (x * p1 - p0) / (x * x - 1.0) : 0.5 * x * n * (n + 1) * std::pow(x, n + 1);
}
// Gauss points (the quadrature of Sec. 4): roots of P_Q by Newton from
// Chebyshev guesses; w = 2/((1-x^2) P'^2).
static void gauss(int Q, double* x, double* w) {
  for (int i = 0; i < Q; ++i) {
    double xi = -std::cos(M_PI * (i + 0.75) / (Q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP; legendre(Q, xi, P, dP);
      double dx = P / dP; xi -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    double P, dP; legendre(Q, xi, P, dP);
    x[i] = xi; w[i] = 2.0 / ((1.0 - xi * xi) * dP * dP);
  }
  std::sort(x, x + Q);
  for (int i = 0; i < Q; ++i) { double P, dP; legendre(Q, x[i], P, dP); w[i] = 2.0 / ((1.0 - x[i] * x[i]) * dP * dP); }
}
// GLL points (the nodes of the Sec. 4 elements): -1, +1 and the roots of P_p'
// (Newton with P'' from Legendre's equation).
static void gll(int p, double* x) {
  x[0] = -1.0; x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double xi = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP; legendre(p, xi, P, dP);
      double d2P = (2.0 * xi * dP - p * (p + 1.0) * P) / (1.0 - xi * xi);
      double dx = dP / d2P; xi -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    x[i] = xi;
  }
  std::sort(x, x + p + 1);
  if (p % 2 == 0) x[p / 2] = 0.0;
}
// Lagrange basis l_a(t) on nodes xn[0..P-1] (product formula) and l_a'(t)
// (sum over the dropped factor of the remaining products): the 1D factors of
// the tensor-product basis B_I, B_xi of Sec. 4.
static double lagr(const double* xn, int P, int a, double t) {
  double r = 1.0;
  for (int b = 0; b < P; ++b) if (b != a) r *= (t - xn[b]) / (xn[a] - xn[b]);
  return r;
}
static double dlagr(const double* xn, int P, int a, double t) {
  double s = 0.0;
  for (int c = 0; c < P; ++c) {
    if (c == a) continue;
    double r = 1.0 / (xn[a] - xn[c]);
    for (int b = 0; b < P; ++b) if (b != a && b != c) r *= (t - xn[b]) / (xn[a] - xn[b]);
    s += r;
  }
  return s;
}

struct Mesh {
  int nx, ny, nz, p, Q;
  double hx, hy, hz;
  int nnx, nny, nnz;
  long long nn;
  std::vector<double> xg, xq, wq;     // GLL nodes, Gauss nodes and weights
  std::vector<double> Bt, Dt;         // [Q][P] values and derivatives at Gauss points
};
static Mesh make_mesh(const int* dims, const double* h) {
  Mesh m;
  m.nx = dims[0]; m.ny = dims[1]; m.nz = dims[2]; m.p = dims[3]; m.Q = dims[4];
  m.hx = h[0]; m.hy = h[1]; m.hz = h[2];
  m.nnx = m.p * m.nx + 1; m.nny = m.p * m.ny + 1; m.nnz = m.p * m.nz + 1;
  m.nn = (long long)m.nnx * m.nny * m.nnz;
  int P = m.p + 1;
  m.xg.resize(P); m.xq.resize(m.Q); m.wq.resize(m.Q);
  gll(m.p, m.xg.data()); gauss(m.Q, m.xq.data(), m.wq.data());
  m.Bt.resize(m.Q * P); m.Dt.resize(m.Q * P);
  for (int i = 0; i < m.Q; ++i)
    for (int a = 0; a < P; ++a) {
      m.Bt[i * P + a] = lagr(m.xg.data(), P, a, m.xq[i]);
      m.Dt[i * P + a] = dlagr(m.xg.data(), P, a, m.xq[i]);
    }
  return m;
}
static inline long long node_id(const Mesh& m, int I, int J, int K) { return I + (long long)m.nnx * (J + (long long)m.nny * K); }
static void elem_nodes(const Mesh& m, long long e, long long* nodes) {
  int ex = e % m.nx, ey = (e / m.nx) % m.ny, ez = e / ((long long)m.nx * m.ny);
  int P = m.p + 1;
  for (int c = 0; c < P; ++c) for (int b = 0; b < P; ++b) for (int a = 0; a < P; ++a)
    nodes[a + P * (b + P * c)] = node_id(m, m.p * ex + a, m.p * ey + b, m.p * ez + c);
}

// Per-point data of one element: basis values, reference-frame gradients
// and w * det J, evaluated for every (3D basis function, 3D Gauss point) pair.
struct ElemBasis {
  int P3, Q3;
  std::vector<double> N, dN, wdet;  // N[q*P3+a], dN[(q*P3+a)*3+A]
};
static ElemBasis elem_basis(const Mesh& m) {
  ElemBasis eb;
  int P = m.p + 1, Q = m.Q;
  eb.P3 = P * P * P; eb.Q3 = Q * Q * Q;
  eb.N.resize(eb.Q3 * eb.P3); eb.dN.resize(eb.Q3 * eb.P3 * 3); eb.wdet.resize(eb.Q3);
  double s[3] = {2.0 / m.hx, 2.0 / m.hy, 2.0 / m.hz};
  double detJ = m.hx * m.hy * m.hz / 8.0;
  for (int k = 0; k < Q; ++k) for (int j = 0; j < Q; ++j) for (int i = 0; i < Q; ++i) {
    int q = i + Q * (j + Q * k);
    eb.wdet[q] = m.wq[i] * m.wq[j] * m.wq[k] * detJ;
    double xi[3] = {m.xq[i], m.xq[j], m.xq[k]};
    for (int c = 0; c < P; ++c) for (int b = 0; b < P; ++b) for (int a = 0; a < P; ++a) {
      int A = a + P * (b + P * c);
      double l0 = lagr(m.xg.data(), P, a, xi[0]), l1 = lagr(m.xg.data(), P, b, xi[1]), l2 = lagr(m.xg.data(), P, c, xi[2]);
      double d0 = dlagr(m.xg.data(), P, a, xi[0]), d1 = dlagr(m.xg.data(), P, b, xi[1]), d2 = dlagr(m.xg.data(), P, c, xi[2]);
      eb.N[q * eb.P3 + A] = l0 * l1 * l2;
      eb.dN[(q * eb.P3 + A) * 3 + 0] = s[0] * d0 * l1 * l2;
      eb.dN[(q * eb.P3 + A) * 3 + 1] = s[1] * l0 * d1 * l2;
      eb.dN[(q * eb.P3 + A) * 3 + 2] = s[2] * l0 * l1 * d2;
    }
  }
  return eb;
}

// The same for element e of a mapped mesh with nodal coordinates X [3][nn]
// (isoparametric: X(xi) = sum_a X_a N_a(xi)): J = dX/dxi = sum_a X_a (x) grad_xi N_a,
// reference gradients grad_X N_a = J^-T grad_xi N_a, weight w_q det J.
static ElemBasis elem_basis_geo(const Mesh& m, const double* X, long long e) {
  ElemBasis eb;
  int P = m.p + 1, Q = m.Q;
  eb.P3 = P * P * P; eb.Q3 = Q * Q * Q;
  eb.N.resize(eb.Q3 * eb.P3); eb.dN.resize(eb.Q3 * eb.P3 * 3); eb.wdet.resize(eb.Q3);
  std::vector<long long> nodes(eb.P3);
  elem_nodes(m, e, nodes.data());
  std::vector<double> dxi(eb.P3 * 3);
  for (int k = 0; k < Q; ++k) for (int j = 0; j < Q; ++j) for (int i = 0; i < Q; ++i) {
    int q = i + Q * (j + Q * k);
    double xi[3] = {m.xq[i], m.xq[j], m.xq[k]};
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int c = 0; c < P; ++c) for (int b = 0; b < P; ++b) for (int a = 0; a < P; ++a) {
      int A = a + P * (b + P * c);
      double l0 = lagr(m.xg.data(), P, a, xi[0]), l1 = lagr(m.xg.data(), P, b, xi[1]), l2 = lagr(m.xg.data(), P, c, xi[2]);
      double d0 = dlagr(m.xg.data(), P, a, xi[0]), d1 = dlagr(m.xg.data(), P, b, xi[1]), d2 = dlagr(m.xg.data(), P, c, xi[2]);
      eb.N[q * eb.P3 + A] = l0 * l1 * l2;
      dxi[A * 3 + 0] = d0 * l1 * l2;
      dxi[A * 3 + 1] = l0 * d1 * l2;
      dxi[A * 3 + 2] = l0 * l1 * d2;
      for (int d = 0; d < 3; ++d)
        for (int al = 0; al < 3; ++al) J[d][al] += X[d * m.nn + nodes[A]] * dxi[A * 3 + al];
    }
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double G[3][3];  // G = J^-1 (d xi / dX), by cofactors
    G[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    G[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    G[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    G[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    G[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    G[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    G[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    G[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    G[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    eb.wdet[q] = m.wq[i] * m.wq[j] * m.wq[k] * det;
    for (int A = 0; A < eb.P3; ++A)
      for (int d = 0; d < 3; ++d)
        eb.dN[(q * eb.P3 + A) * 3 + d] = dxi[A * 3 + 0] * G[0][d] + dxi[A * 3 + 1] * G[1][d] + dxi[A * 3 + 2] * G[2][d];
  }
  return eb;
}

typedef Dual<13> D13;

struct Problem {
  Mesh m;
  ElemBasis eb;
  std::vector<Phase> phases;
  Glob gl;
  const double* z;        // [4][nn]
  const double* hist;     // [15][nq]
  const uint8_t* phase;   // [nq]
  long long nq;
  const double* X;        // nodal coordinates [3][nn] of a mapped mesh, or null (box)
};
static ElemBasis basis_of(const Problem& pr, long long e) {
  return pr.X ? elem_basis_geo(pr.m, pr.X, e) : pr.eb;
}

// One element: residual r_e[f*P3+a] (Eq. matrix-free-residual-compact, full
// quadrature: every 3D basis function at every Gauss point), optionally the
// pointwise tangents Dh[q][16][16] (rows: f0 (4), f1 (12); cols: values (4),
// gradients (12); Eq. matrix-free-jacobian, by dual numbers), trial history
// (Box 1 step 4) and flags.
static void element_eval(const Problem& pr, const ElemBasis& eb, long long e, double* re, double* Dh,
                         double* hist_new, uint8_t* flags, double* margins) {
  const Mesh& m = pr.m;
  int P3 = eb.P3, Q3 = eb.Q3;
  std::vector<long long> nodes(P3);
  elem_nodes(m, e, nodes.data());
  std::vector<double> ze(4 * P3);
  for (int f = 0; f < 4; ++f)
    for (int a = 0; a < P3; ++a) ze[f * P3 + a] = pr.z[f * m.nn + nodes[a]];
  if (re) for (int i = 0; i < 4 * P3; ++i) re[i] = 0.0;
  for (int q = 0; q < Q3; ++q) {
    long long gq = e * Q3 + q;
    double hq[15];
    for (int v = 0; v < 15; ++v) hq[v] = pr.hist[v * pr.nq + gq];
    const Phase& ph = pr.phases[pr.phase[gq]];
    double G[3][3] = {{0}}, phi = 0.0, gphi[3] = {0, 0, 0};
    for (int a = 0; a < P3; ++a) {
      double Na = eb.N[q * P3 + a];
      const double* dNa = &eb.dN[(q * P3 + a) * 3];
      for (int i = 0; i < 3; ++i) for (int A = 0; A < 3; ++A) G[i][A] += ze[i * P3 + a] * dNa[A];
      phi += ze[3 * P3 + a] * Na;
      for (int A = 0; A < 3; ++A) gphi[A] += ze[3 * P3 + a] * dNa[A];
    }
    double f0[4], f1[4][3];
    if (Dh) {
      D13 Gd[3][3], phid(phi), gphid[3];
      for (int i = 0; i < 3; ++i) for (int A = 0; A < 3; ++A) { Gd[i][A] = D13(G[i][A]); Gd[i][A].d[3 * i + A] = 1.0; }
      phid.d[9] = 1.0;
      for (int A = 0; A < 3; ++A) { gphid[A] = D13(gphi[A]); gphid[A].d[10 + A] = 1.0; }
      PointResult<D13> pt;
      D13 hqd[15];
      for (int v = 0; v < 15; ++v) hqd[v] = D13(hq[v]);
      pointwise<D13>(Gd, phid, gphid, hqd, lift<D13>(ph), pr.gl, false, pt);
      double* D = Dh + (size_t)q * 256;
      for (int i = 0; i < 256; ++i) D[i] = 0.0;
      // seed -> input column: grad u_iA -> 4+3i+A, phi -> 3, grad phi_A -> 13+A
      int colOf[13];
      for (int s = 0; s < 9; ++s) colOf[s] = 4 + s;
      colOf[9] = 3;
      for (int A = 0; A < 3; ++A) colOf[10 + A] = 13 + A;
      for (int s = 0; s < 13; ++s) {
        for (int f = 0; f < 4; ++f) D[f * 16 + colOf[s]] = pt.f0[f].d[s];
        for (int f = 0; f < 4; ++f) for (int A = 0; A < 3; ++A) D[(4 + 3 * f + A) * 16 + colOf[s]] = pt.f1[f][A].d[s];
      }
      for (int f = 0; f < 4; ++f) { f0[f] = pt.f0[f].v; for (int A = 0; A < 3; ++A) f1[f][A] = pt.f1[f][A].v; }
    }
    PointResult<double> pd;
    pointwise<double>(G, phi, gphi, hq, ph, pr.gl, hist_new != nullptr, pd);
    if (!Dh) { for (int f = 0; f < 4; ++f) { f0[f] = pd.f0[f]; for (int A = 0; A < 3; ++A) f1[f][A] = pd.f1[f][A]; } }
    if (hist_new) for (int v = 0; v < 15; ++v) hist_new[v * Q3 + q] = pd.hist_new[v];
    if (flags) flags[q] = pd.flags;
    if (margins) { margins[q * 3 + 0] = pd.margin_yield; margins[q * 3 + 1] = pd.margin_hist; margins[q * 3 + 2] = pd.theta; }
    if (re) {
      double w = eb.wdet[q];
      for (int f = 0; f < 4; ++f)
        for (int a = 0; a < P3; ++a) {
          const double* dNa = &eb.dN[(q * P3 + a) * 3];
          re[f * P3 + a] += w * (f0[f] * eb.N[q * P3 + a] + f1[f][0] * dNa[0] + f1[f][1] * dNa[1] + f1[f][2] * dNa[2]);
        }
    }
  }
}

// Element matrix K_e[(f,a),(g,b)] = sum_q w_q det J  B_q^T Dh_q B_q, where
// row r of B_q is a value (N_a) or a reference gradient component (dN_a/dX_A).
static void element_matrix(const ElemBasis& eb, const double* Dh, double* Ke) {
  int P3 = eb.P3, Q3 = eb.Q3, n = 4 * P3;
  for (int i = 0; i < n * n; ++i) Ke[i] = 0.0;
  std::vector<double> Bv(16 * P3);  // Bv[r*P3+a] for rows r of one field pattern
  std::vector<double> M(4 * P3);
  for (int q = 0; q < Q3; ++q) {
    const double* D = Dh + (size_t)q * 256;
    double w = eb.wdet[q];
    for (int f = 0; f < 4; ++f)
      for (int g = 0; g < 4; ++g) {
        int rows[4] = {f, 4 + 3 * f, 5 + 3 * f, 6 + 3 * f};
        int cols[4] = {g, 4 + 3 * g, 5 + 3 * g, 6 + 3 * g};
        // M[r][b] = sum_c Dh[row r][col c] * basis_c(b)
        for (int r = 0; r < 4; ++r)
          for (int b = 0; b < P3; ++b) {
            double s = D[rows[r] * 16 + cols[0]] * eb.N[q * P3 + b];
            for (int A = 0; A < 3; ++A) s += D[rows[r] * 16 + cols[1 + A]] * eb.dN[(q * P3 + b) * 3 + A];
            M[r * P3 + b] = s;
          }
        for (int a = 0; a < P3; ++a) {
          double ba[4] = {eb.N[q * P3 + a], eb.dN[(q * P3 + a) * 3 + 0], eb.dN[(q * P3 + a) * 3 + 1], eb.dN[(q * P3 + a) * 3 + 2]};
          double* Krow = Ke + (size_t)(f * P3 + a) * n + g * P3;
          for (int b = 0; b < P3; ++b)
            Krow[b] += w * (ba[0] * M[0 * P3 + b] + ba[1] * M[1 * P3 + b] + ba[2] * M[2 * P3 + b] + ba[3] * M[3 * P3 + b]);
        }
      }
  }
}

static Problem make_problem(const int* dims, const double* h, const double* phase_params, int nphase,
                            const double* glob, const double* z, const double* hist, const uint8_t* phase,
                            const double* X) {
  Problem pr;
  pr.X = X;
  pr.m = make_mesh(dims, h);
  pr.eb = elem_basis(pr.m);
  for (int i = 0; i < nphase; ++i) pr.phases.push_back(read_phase(phase_params + kPhaseWords * i));
  pr.gl = read_glob(glob);
  pr.z = z; pr.hist = hist; pr.phase = phase;
  pr.nq = (long long)pr.m.nx * pr.m.ny * pr.m.nz * pr.eb.Q3;
  return pr;
}

struct CSR {
  long long nrows;
  std::vector<long long> indptr;
  std::vector<long long> indices;
  std::vector<double> data;
};

}  // namespace orc

using namespace orc;

extern "C" {

int orc_version() { return 1; }

// 1D basis data: xg[P], xq[Q], wq[Q], B[Q*P], D[Q*P] (Lagrange values and
// derivatives on the GLL nodes, evaluated at the Gauss points).
int orc_basis(int p, int Q, double* xg, double* xq, double* wq, double* B, double* D) {
  int P = p + 1;
  std::vector<double> x(P), g(Q), w(Q);
  gll(p, x.data()); gauss(Q, g.data(), w.data());
  for (int a = 0; a < P; ++a) xg[a] = x[a];
  for (int i = 0; i < Q; ++i) { xq[i] = g[i]; wq[i] = w[i]; }
  for (int i = 0; i < Q; ++i) for (int a = 0; a < P; ++a) {
    B[i * P + a] = lagr(x.data(), P, a, g[i]);
    D[i * P + a] = dlagr(x.data(), P, a, g[i]);
  }
  return 0;
}
// Lagrange basis on the GLL nodes of order p evaluated at arbitrary points.
int orc_lagrange_eval(int p, int n, const double* t, double* L, double* dL) {
  int P = p + 1;
  std::vector<double> x(P);
  gll(p, x.data());
  for (int k = 0; k < n; ++k) for (int a = 0; a < P; ++a) {
    L[k * P + a] = lagr(x.data(), P, a, t[k]);
    dL[k * P + a] = dlagr(x.data(), P, a, t[k]);
  }
  return 0;
}

// Batched pointwise evaluation.  inputs[n][13] = grad u (row-major 9), phi,
// grad phi (3); hist[n][15] (point-major here); phase[n].  Outputs: f0[n][4],
// f1[n][12], tangent Dh[n][16][16] (may be NULL), hist_new[n][15] (may be
// NULL), flags[n], aux[n][4] = psi+, margin_yield, margin_hist, theta.
int orc_pointwise(int n, const double* inputs, const double* hist, const uint8_t* phase,
                  const double* phase_params, int nphase, const double* glob,
                  double* f0, double* f1, double* Dh, double* hist_new, uint8_t* flags, double* aux) {
  std::vector<Phase> phases;
  for (int i = 0; i < nphase; ++i) phases.push_back(read_phase(phase_params + kPhaseWords * i));
  Glob gl = read_glob(glob);
#pragma omp parallel for schedule(dynamic, 64)
  for (int k = 0; k < n; ++k) {
    const double* in = inputs + 13 * (size_t)k;
    double G[3][3];
    for (int i = 0; i < 3; ++i) for (int A = 0; A < 3; ++A) G[i][A] = in[3 * i + A];
    double gphi[3] = {in[10], in[11], in[12]};
    const Phase& ph = phases[phase[k]];
    PointResult<double> pd;
    pointwise<double>(G, in[9], gphi, hist + 15 * (size_t)k, ph, gl, hist_new != nullptr, pd);
    for (int f = 0; f < 4; ++f) f0[4 * (size_t)k + f] = pd.f0[f];
    for (int f = 0; f < 4; ++f) for (int A = 0; A < 3; ++A) f1[12 * (size_t)k + 3 * f + A] = pd.f1[f][A];
    if (hist_new) for (int v = 0; v < 15; ++v) hist_new[15 * (size_t)k + v] = pd.hist_new[v];
    flags[k] = pd.flags;
    aux[4 * (size_t)k + 0] = pd.psi_plus; aux[4 * (size_t)k + 1] = pd.margin_yield;
    aux[4 * (size_t)k + 2] = pd.margin_hist; aux[4 * (size_t)k + 3] = pd.theta;
    if (Dh) {
      D13 Gd[3][3], phid(in[9]), gphid[3];
      for (int i = 0; i < 3; ++i) for (int A = 0; A < 3; ++A) { Gd[i][A] = D13(G[i][A]); Gd[i][A].d[3 * i + A] = 1.0; }
      phid.d[9] = 1.0;
      for (int A = 0; A < 3; ++A) { gphid[A] = D13(gphi[A]); gphid[A].d[10 + A] = 1.0; }
      PointResult<D13> pt;
      D13 hqd[15];
      for (int v = 0; v < 15; ++v) hqd[v] = D13(hist[15 * (size_t)k + v]);
      pointwise<D13>(Gd, phid, gphid, hqd, lift<D13>(ph), gl, false, pt);
      double* D = Dh + 256 * (size_t)k;
      for (int i = 0; i < 256; ++i) D[i] = 0.0;
      int colOf[13];
      for (int s = 0; s < 9; ++s) colOf[s] = 4 + s;
      colOf[9] = 3;
      for (int A = 0; A < 3; ++A) colOf[10 + A] = 13 + A;
      for (int s = 0; s < 13; ++s) {
        for (int f = 0; f < 4; ++f) D[f * 16 + colOf[s]] = pt.f0[f].d[s];
        for (int f = 0; f < 4; ++f) for (int A = 0; A < 3; ++A) D[(4 + 3 * f + A) * 16 + colOf[s]] = pt.f1[f][A].d[s];
      }
    }
  }
  return 0;
}

// Matrix logarithm and exponential of single 3x3 matrices (row-major), for pins.
int orc_logm1p(const double* X, double* L) {
  M3<double> m; for (int i = 0; i < 9; ++i) m.a[i / 3][i % 3] = X[i];
  M3<double> r = logm_1p(m);
  for (int i = 0; i < 9; ++i) L[i] = r.a[i / 3][i % 3];
  return 0;
}
int orc_expm(const double* A, double* E) {
  M3<double> m; for (int i = 0; i < 9; ++i) m.a[i / 3][i % 3] = A[i];
  M3<double> r = expm(m);
  for (int i = 0; i < 9; ++i) E[i] = r.a[i / 3][i % 3];
  return 0;
}

// Global assembly (Sec. 4: the element operators summed with E^T P^T; here
// explicitly into CSR).  dims = {nx,ny,nz,p,Q}; h = {hx,hy,hz}; z [4][nn];
// hist [15][nq] (SoA); phase [nq]; mask [4][nn] (uint8, may be NULL);
// dvals [4][nn] Dirichlet values (may be NULL).  Produces the residual
// r [4][nn] (masked rows r = z - ubar), trial history [15][nq], flags [nq],
// margins [nq][3]; if want_matrix, builds the CSR Jacobian with masked rows
// and columns replaced by the identity and returns a handle.
void* orc_assemble(const int* dims, const double* h, const double* phase_params, int nphase,
                   const double* glob, const double* z, const double* hist, const uint8_t* phase,
                   const uint8_t* mask, const double* dvals, int want_matrix,
                   double* r, double* hist_new, uint8_t* flags, double* margins, const double* X) {
  Problem pr = make_problem(dims, h, phase_params, nphase, glob, z, hist, phase, X);
  const Mesh& m = pr.m;
  int P3 = pr.eb.P3, Q3 = pr.eb.Q3, ne = 4 * P3;
  long long nel = (long long)m.nx * m.ny * m.nz;
  long long nd = 4 * m.nn;
  for (long long i = 0; i < nd; ++i) r[i] = 0.0;
  CSR* csr = nullptr;
  std::vector<std::vector<long long>> nbr;
  if (want_matrix) {
    csr = new CSR();
    csr->nrows = nd;
    // sparsity: nodes sharing an element
    nbr.resize(m.nn);
    std::vector<long long> nodes(P3);
    for (long long e = 0; e < nel; ++e) {
      elem_nodes(m, e, nodes.data());
      for (int a = 0; a < P3; ++a) for (int b = 0; b < P3; ++b) nbr[nodes[a]].push_back(nodes[b]);
    }
    for (long long n = 0; n < m.nn; ++n) {
      std::sort(nbr[n].begin(), nbr[n].end());
      nbr[n].erase(std::unique(nbr[n].begin(), nbr[n].end()), nbr[n].end());
    }
    csr->indptr.resize(nd + 1);
    csr->indptr[0] = 0;
    for (int f = 0; f < 4; ++f)
      for (long long n = 0; n < m.nn; ++n) {
        long long row = f * m.nn + n;
        csr->indptr[row + 1] = csr->indptr[row] + 4 * (long long)nbr[n].size();
      }
    csr->indices.resize(csr->indptr[nd]);
    csr->data.assign(csr->indptr[nd], 0.0);
    for (int f = 0; f < 4; ++f)
      for (long long n = 0; n < m.nn; ++n) {
        long long k = csr->indptr[f * m.nn + n];
        for (int g = 0; g < 4; ++g)
          for (long long c : nbr[n]) csr->indices[k++] = g * m.nn + c;
      }
  }
  // elements in chunks: evaluate in parallel, accumulate serially
  const long long chunk = 256;
  std::vector<double> reb, Dhb, Keb, hnb;
  std::vector<uint8_t> flb;
  std::vector<double> mgb;
  for (long long e0 = 0; e0 < nel; e0 += chunk) {
    long long e1 = std::min(nel, e0 + chunk), nc = e1 - e0;
    reb.assign(nc * ne, 0.0);
    hnb.assign(nc * 15 * Q3, 0.0);
    flb.assign(nc * Q3, 0);
    mgb.assign(nc * Q3 * 3, 0.0);
    if (want_matrix) { Dhb.assign(nc * Q3 * 256, 0.0); Keb.assign(nc * (size_t)ne * ne, 0.0); }
#pragma omp parallel for schedule(dynamic, 1)
    for (long long c = 0; c < nc; ++c) {
      const ElemBasis eb = basis_of(pr, e0 + c);
      element_eval(pr, eb, e0 + c, &reb[c * ne], want_matrix ? &Dhb[c * Q3 * 256] : nullptr,
                   &hnb[c * 15 * Q3], &flb[c * Q3], &mgb[c * Q3 * 3]);
      if (want_matrix) element_matrix(eb, &Dhb[c * Q3 * 256], &Keb[c * (size_t)ne * ne]);
    }
    std::vector<long long> nodes(P3);
    for (long long c = 0; c < nc; ++c) {
      long long e = e0 + c;
      elem_nodes(m, e, nodes.data());
      for (int f = 0; f < 4; ++f) for (int a = 0; a < P3; ++a) r[f * m.nn + nodes[a]] += reb[c * ne + f * P3 + a];
      for (int q = 0; q < Q3; ++q) {
        for (int v = 0; v < 15; ++v) hist_new[v * pr.nq + e * Q3 + q] = hnb[c * 15 * Q3 + v * Q3 + q];
        flags[e * Q3 + q] = flb[c * Q3 + q];
        for (int t = 0; t < 3; ++t) margins[(e * Q3 + q) * 3 + t] = mgb[(c * Q3 + q) * 3 + t];
      }
      if (want_matrix) {
        const double* Ke = &Keb[c * (size_t)ne * ne];
        for (int f = 0; f < 4; ++f) for (int a = 0; a < P3; ++a) {
          long long row = f * m.nn + nodes[a];
          long long k0 = csr->indptr[row], k1 = csr->indptr[row + 1];
          for (int g = 0; g < 4; ++g) for (int b = 0; b < P3; ++b) {
            long long col = g * m.nn + nodes[b];
            long long k = std::lower_bound(csr->indices.begin() + k0, csr->indices.begin() + k1, col) - csr->indices.begin();
            csr->data[k] += Ke[(size_t)(f * P3 + a) * ne + g * P3 + b];
          }
        }
      }
    }
  }
  if (mask) {
    for (long long i = 0; i < nd; ++i) if (mask[i]) r[i] = z[i] - (dvals ? dvals[i] : 0.0);
    if (want_matrix) {
      for (long long row = 0; row < nd; ++row)
        for (long long k = csr->indptr[row]; k < csr->indptr[row + 1]; ++k) {
          long long col = csr->indices[k];
          if (mask[row] || mask[col]) csr->data[k] = (row == col) ? 1.0 : 0.0;
        }
    }
  }
  return csr;
}
long long orc_csr_nnz(void* h) { return ((CSR*)h)->indptr.back(); }
int orc_csr_get(void* h, long long* indptr, long long* indices, double* data) {
  CSR* c = (CSR*)h;
  std::memcpy(indptr, c->indptr.data(), sizeof(long long) * c->indptr.size());
  std::memcpy(indices, c->indices.data(), sizeof(long long) * c->indices.size());
  std::memcpy(data, c->data.data(), sizeof(double) * c->data.size());
  return 0;
}
void orc_csr_free(void* h) { delete (CSR*)h; }

// Sampled rows for meshes too large to assemble: for each requested global
// DoF i, the residual r_i, (J x)_i and (J^T x)_i and the diagonal J_ii, each
// from the element matrices of the elements around the DoF's node (full
// quadrature).  Dirichlet handling as in orc_assemble.
int orc_sample_rows(const int* dims, const double* h, const double* phase_params, int nphase,
                    const double* glob, const double* z, const double* hist, const uint8_t* phase,
                    const uint8_t* mask, const double* dvals, const double* x,
                    int ns, const long long* dofs, double* r_out, double* jx_out, double* jtx_out, double* diag_out,
                    const double* X) {
  Problem pr = make_problem(dims, h, phase_params, nphase, glob, z, hist, phase, X);
  const Mesh& m = pr.m;
  int P3 = pr.eb.P3, Q3 = pr.eb.Q3, ne = 4 * P3;
  // collect the elements needed
  std::vector<long long> need;
  for (int s = 0; s < ns; ++s) {
    long long n = dofs[s] % m.nn;
    int I = n % m.nnx, J = (n / m.nnx) % m.nny, K = n / ((long long)m.nnx * m.nny);
    // elements whose closure holds the node: one or two per direction
    int exs[2], eys[2], ezs[2], nxs = 0, nys = 0, nzs = 0;
    auto cand = [](int Ic, int p, int ne_, int* out, int& cnt) {
      int e1 = Ic / p;
      if (Ic % p == 0) { if (e1 - 1 >= 0) out[cnt++] = e1 - 1; if (e1 < ne_) out[cnt++] = e1; }
      else out[cnt++] = e1;
    };
    cand(I, m.p, m.nx, exs, nxs); cand(J, m.p, m.ny, eys, nys); cand(K, m.p, m.nz, ezs, nzs);
    for (int a = 0; a < nxs; ++a) for (int b = 0; b < nys; ++b) for (int c = 0; c < nzs; ++c)
      need.push_back(exs[a] + (long long)m.nx * (eys[b] + (long long)m.ny * ezs[c]));
  }
  std::sort(need.begin(), need.end());
  need.erase(std::unique(need.begin(), need.end()), need.end());
  std::vector<double> Ke_all(need.size() * (size_t)ne * ne), re_all(need.size() * ne);
#pragma omp parallel for schedule(dynamic, 1)
  for (long long t = 0; t < (long long)need.size(); ++t) {
    std::vector<double> Dh(Q3 * 256), hn(15 * Q3), mg(3 * Q3);
    std::vector<uint8_t> fl(Q3);
    const ElemBasis eb = basis_of(pr, need[t]);
    element_eval(pr, eb, need[t], &re_all[t * ne], Dh.data(), hn.data(), fl.data(), mg.data());
    element_matrix(eb, Dh.data(), &Ke_all[t * (size_t)ne * ne]);
  }
  std::vector<long long> nodes(P3);
  for (int s = 0; s < ns; ++s) {
    long long dof = dofs[s];
    int f = dof / m.nn;
    long long n = dof % m.nn;
    double rr = 0.0, jx = 0.0, jtx = 0.0, dg = 0.0;
    for (size_t t = 0; t < need.size(); ++t) {
      elem_nodes(m, need[t], nodes.data());
      int aloc = -1;
      for (int a = 0; a < P3; ++a) if (nodes[a] == n) aloc = a;
      if (aloc < 0) continue;
      const double* Ke = &Ke_all[t * (size_t)ne * ne];
      int i = f * P3 + aloc;
      rr += re_all[t * ne + i];
      dg += Ke[(size_t)i * ne + i];
      for (int g = 0; g < 4; ++g) for (int b = 0; b < P3; ++b) {
        long long col = g * m.nn + nodes[b];
        double xv = (mask && mask[col]) ? 0.0 : x[col];
        int j = g * P3 + b;
        jx += Ke[(size_t)i * ne + j] * xv;
        jtx += Ke[(size_t)j * ne + i] * xv;
      }
    }
    if (mask && mask[dof]) {
      rr = z[dof] - (dvals ? dvals[dof] : 0.0);
      jx = x[dof]; jtx = x[dof]; dg = 1.0;
    }
    r_out[s] = rr; jx_out[s] = jx; jtx_out[s] = jtx; diag_out[s] = dg;
  }
  return 0;
}

// p-prolongation of the multigrid of Sec. 5 from order pc to order pf on the
// same element grid: entry
// P[fine node, coarse node] = coarse Lagrange basis at the fine GLL node.
// Returns the number of entries written as COO (rows, cols, vals), per field
// block 0 (the 4 fields repeat the same block).  Call with rows == NULL to size.
long long orc_prolong_coo(const int* dims, int pc, int pf, long long* rows, long long* cols, double* vals) {
  int nx = dims[0], ny = dims[1], nz = dims[2];
  int Pc = pc + 1, Pf = pf + 1;
  std::vector<double> xc(Pc), xf(Pf);
  gll(pc, xc.data()); gll(pf, xf.data());
  long long fnx = (long long)pf * nx + 1, fny = (long long)pf * ny + 1, fnz = (long long)pf * nz + 1;
  long long cnx = (long long)pc * nx + 1, cny = (long long)pc * ny + 1;
  long long cnt = 0;
  for (long long K = 0; K < fnz; ++K) for (long long J = 0; J < fny; ++J) for (long long I = 0; I < fnx; ++I) {
    long long idx[3] = {I, J, K};
    int ne_[3] = {nx, ny, nz};
    int el[3]; double t[3];
    for (int d = 0; d < 3; ++d) {
      int e = (int)(idx[d] / pf);
      if (e >= ne_[d]) e = ne_[d] - 1;
      el[d] = e;
      t[d] = xf[idx[d] - (long long)pf * e];
    }
    long long frow = I + fnx * (J + fny * K);
    for (int c = 0; c < Pc; ++c) for (int b = 0; b < Pc; ++b) for (int a = 0; a < Pc; ++a) {
      double v = lagr(xc.data(), Pc, a, t[0]) * lagr(xc.data(), Pc, b, t[1]) * lagr(xc.data(), Pc, c, t[2]);
      if (v == 0.0) continue;
      if (rows) {
        long long ccol = ((long long)pc * el[0] + a) + cnx * (((long long)pc * el[1] + b) + cny * ((long long)pc * el[2] + c));
        rows[cnt] = frow; cols[cnt] = ccol; vals[cnt] = v;
      }
      ++cnt;
    }
  }
  return cnt;
}

// ---------------------------------------------------------------------------
// Adjoint building blocks
// ---------------------------------------------------------------------------
typedef Dual<34> D34;

// Per point: values out_vals[n][28] = (P_iA (9), s_phi L, f1_phi (3), trial
// history (15)) and partials out_J[n][28][34] with respect to (grad u (9), phi,
// grad phi (3), committed history (15), own-phase parameters E_inf, nu_inf,
// sigma0, eta_d, Gc, l0), all by dual numbers through the same pointwise code.
int orc_point_partials(int n, const double* inputs, const double* hist, const uint8_t* phase,
                       const double* phase_params, int nphase, const double* glob, double* out_vals,
                       double* out_J) {
  std::vector<Phase> phases;
  for (int i = 0; i < nphase; ++i) phases.push_back(read_phase(phase_params + kPhaseWords * i));
  Glob gl = read_glob(glob);
#pragma omp parallel for schedule(dynamic, 16)
  for (int k = 0; k < n; ++k) {
    const double* in = inputs + 13 * (size_t)k;
    D34 Gd[3][3], phid, gphid[3], hd[15];
    for (int i = 0; i < 3; ++i) for (int A = 0; A < 3; ++A) { Gd[i][A] = D34(in[3 * i + A]); Gd[i][A].d[3 * i + A] = 1.0; }
    phid = D34(in[9]); phid.d[9] = 1.0;
    for (int A = 0; A < 3; ++A) { gphid[A] = D34(in[10 + A]); gphid[A].d[10 + A] = 1.0; }
    for (int v = 0; v < 15; ++v) { hd[v] = D34(hist[15 * (size_t)k + v]); hd[v].d[13 + v] = 1.0; }
    const Phase& ph = phases[phase[k]];
    PhaseT<D34> pd = lift<D34>(ph);
    pd.E0.d[28] = 1.0; pd.nu0.d[29] = 1.0;
    if (ph.hasP) pd.sig0.d[30] = 1.0;
    if (ph.hasM && !ph.eta_inf) pd.eta.d[31] = 1.0;
    pd.Gc.d[32] = 1.0; pd.l0.d[33] = 1.0;
    PointResult<D34> pt;
    pointwise<D34>(Gd, phid, gphid, hd, pd, gl, true, pt);
    const D34* outs[28];
    for (int i = 0; i < 3; ++i) for (int A = 0; A < 3; ++A) outs[3 * i + A] = &pt.f1[i][A];
    outs[9] = &pt.f0[3];
    for (int A = 0; A < 3; ++A) outs[10 + A] = &pt.f1[3][A];
    for (int v = 0; v < 15; ++v) outs[13 + v] = &pt.hist_new[v];
    for (int r = 0; r < 28; ++r) {
      out_vals[28 * (size_t)k + r] = outs[r]->v;
      for (int c = 0; c < 34; ++c) out_J[(28 * (size_t)k + r) * 34 + c] = outs[r]->d[c];
    }
  }
  return 0;
}

// Interpolation of a nodal field y [4][nn] to every quadrature point:
// out[nq][14] = (grad_X y_u (9), y_phi, grad_X y_phi (3), w_q det J).
int orc_qpoint_inputs(const int* dims, const double* h, const double* y, double* out, const double* X) {
  Mesh m = make_mesh(dims, h);
  const ElemBasis ebox = elem_basis(m);
  long long nel = (long long)m.nx * m.ny * m.nz;
  int P3 = ebox.P3, Q3 = ebox.Q3;
#pragma omp parallel for schedule(static)
  for (long long e = 0; e < nel; ++e) {
    const ElemBasis eb = X ? elem_basis_geo(m, X, e) : ebox;
    std::vector<long long> nodes(P3);
    elem_nodes(m, e, nodes.data());
    for (int q = 0; q < Q3; ++q) {
      double* o = out + 14 * (size_t)(e * Q3 + q);
      for (int c = 0; c < 13; ++c) o[c] = 0.0;
      for (int a = 0; a < P3; ++a) {
        const double* dNa = &eb.dN[(q * P3 + a) * 3];
        for (int i = 0; i < 3; ++i) for (int A = 0; A < 3; ++A) o[3 * i + A] += y[i * m.nn + nodes[a]] * dNa[A];
        o[9] += y[3 * m.nn + nodes[a]] * eb.N[q * P3 + a];
        for (int A = 0; A < 3; ++A) o[10 + A] += y[3 * m.nn + nodes[a]] * dNa[A];
      }
      o[13] = eb.wdet[q];
    }
  }
  return 0;
}

// out [4][nn] = sum_q B_q^T pseudo_q (optionally times w_q det J): the
// transpose of orc_qpoint_inputs, with pseudo[nq][13] in the same layout.
int orc_apply_bt(const int* dims, const double* h, const double* pseudo, int weighted, double* out,
                 const double* X) {
  Mesh m = make_mesh(dims, h);
  const ElemBasis ebox = elem_basis(m);
  long long nel = (long long)m.nx * m.ny * m.nz;
  int P3 = ebox.P3, Q3 = ebox.Q3;
  for (long long i = 0; i < 4 * m.nn; ++i) out[i] = 0.0;
  std::vector<long long> nodes(P3);
  for (long long e = 0; e < nel; ++e) {
    const ElemBasis eb = X ? elem_basis_geo(m, X, e) : ebox;
    elem_nodes(m, e, nodes.data());
    for (int q = 0; q < Q3; ++q) {
      const double* p = pseudo + 13 * (size_t)(e * Q3 + q);
      double w = weighted ? eb.wdet[q] : 1.0;
      for (int a = 0; a < P3; ++a) {
        const double* dNa = &eb.dN[(q * P3 + a) * 3];
        for (int i = 0; i < 3; ++i)
          out[i * m.nn + nodes[a]] += w * (p[3 * i] * dNa[0] + p[3 * i + 1] * dNa[1] + p[3 * i + 2] * dNa[2]);
        out[3 * m.nn + nodes[a]] += w * (p[9] * eb.N[q * P3 + a] + p[10] * dNa[0] + p[11] * dNa[1] + p[12] * dNa[2]);
      }
    }
  }
  return 0;
}

// y = A x for a CSR matrix (plain row loop, OpenMP over rows): the oracle's
// Jacobian action once the Jacobian is assembled.
int orc_csr_spmv(long long nrows, const long long* indptr, const long long* indices, const double* data,
                 const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < nrows; ++i) {
    double s = 0.0;
    for (long long k = indptr[i]; k < indptr[i + 1]; ++k) s += data[k] * x[indices[k]];
    y[i] = s;
  }
  return 0;
}

int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Threads of the following parallel loops (timing with one core and with all).
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

}  // extern "C"
