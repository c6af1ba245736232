// Newton-Krylov solver with p-multigrid preconditioning (Sec. 5: Newton,
// GMRES with adaptive classical Gram-Schmidt refinement, p-multigrid with
// Chebyshev smoothing), host-driven, every vector operation a device kernel.
//
// * Outer: Newton on the FP64 residual with a backtracking line search; each
//   linear solve is FGMRES(m) with FP64 vectors and inner products, its
//   operator the FP64 or the double-float fine action (outer_prec), right-
//   preconditioned by one V-cycle (flexible because the coarse solve and the
//   mixed-precision cycle are not exactly linear in FP64).
// * V-cycle: Chebyshev(k) pre- and post-smoothing on D^-1 J of every
//   matrix-free level (FP64, or FP32 in the mixed variant), p-restriction /
//   prolongation between levels, and on an order-1 coarsest level an FP64
//   solve with the assembled Q1 Galerkin operator: Chebyshev-Jacobi,
//   Jacobi-GMRES, or GMRES preconditioned by a geometric h-multigrid V-cycle
//   on the structured Q1 grid (the paper's algebraic coarse solver replaced
//   by geometric coarsening, which the structured box allows).
// * Eigenvalue bounds: lambda_max of D^-1 J per level (and per h-level) as the
//   spectral radius of the Hessenberg matrix of a few Arnoldi steps from a
//   seeded random-sign vector, re-estimated every eig_every Newton iterations
//   (0: only on the first); smoothing interval [lo, hi] * lambda_max.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pff_handles.h"

using namespace pff;

namespace {

int sfail(int code, const std::string& msg) { return set_last_error(code, msg.c_str()); }

#define S_CK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return sfail(PFF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define S_RC(call)            \
  do {                        \
    int r_ = (call);          \
    if (r_ != PFF_OK) return r_; \
  } while (0)

struct LevelWork {
  pff_level* L = nullptr;
  int p = 0;
  int prec = PFF_F64;
  size_t esz = 8;
  long long n = 0;
  void *diag = nullptr, *b = nullptr, *x = nullptr, *tmp = nullptr, *work = nullptr;
  double lmax = 1.0;
};

// One level of the geometric h-hierarchy below the assembled Q1 level (level 0
// aliases the Q1 level's operator, diagonal, element matrices and mask).
struct HLevel {
  MeshDev mesh;
  long long n = 0;
  double *Ke = nullptr, *A = nullptr, *diag = nullptr;
  float* A32 = nullptr;  // mixed solver: FP32 copy of A for the preconditioner's products
  const uint8_t* mask = nullptr;
  uint8_t* own_mask = nullptr;
  double *b = nullptr, *x = nullptr, *r = nullptr, *work = nullptr;
  double lmax = 1.0;
  bool owns = false;
};

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct pff_solver {
  pff_op* op = nullptr;
  pff_solver_params prm;
  std::vector<LevelWork> lv;
  bool assembled = false;
  double *A = nullptr, *cdiag = nullptr, *cb = nullptr, *cx = nullptr, *cwork = nullptr;
  float* A32 = nullptr;                 // mixed solver: FP32 copy of the coarse stencil
  double *cV = nullptr, *cZ = nullptr;  // coarse GMRES basis
  double* Ke = nullptr;                 // coarse element matrices [nel][32][32]
  std::vector<HLevel> hl;               // geometric h-hierarchy (coarse_solver 2)
  long long coarse_iters = 0;
  double clmax = 1.0;
  long long n = 0;
  double *V = nullptr, *Z = nullptr, *r = nullptr, *dz = nullptr, *zold = nullptr;
  double *partial = nullptr, *dots = nullptr, *hdev = nullptr;
  double* pw64 = nullptr;  // power-iteration start vector (FP64, fine size)
  float* pw32 = nullptr;
  int transpose = 0;       // 1 while solving with J^T (adjoint)
  // adjoint work space (allocated on the first pff_adjoint_step)
  double *a_in = nullptr, *pbuf = nullptr, *qa = nullptr, *ag = nullptr, *alam = nullptr, *av = nullptr, *gth = nullptr;
};

namespace {

int dev_dots(pff_solver* s, const double* V, long long ldv, int k, const double* w, long long n, double* host,
             cudaStream_t st) {
  S_CK((launch_mdot<double, double>(V, ldv, k, w, n, s->partial, s->dots, st)));
  S_CK(cudaMemcpyAsync(host, s->dots, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  S_CK(cudaStreamSynchronize(st));
  return PFF_OK;
}

int norm_level(pff_solver* s, const LevelWork& w, const void* v, double* out, cudaStream_t st) {
  if (w.prec == PFF_F64) S_CK((launch_mdot<double, double>((const double*)v, 0, 1, (const double*)v, w.n, s->partial, s->dots, st)));
  else S_CK((launch_mdot<float, float>((const float*)v, 0, 1, (const float*)v, w.n, s->partial, s->dots, st)));
  double h = 0.0;
  S_CK(cudaMemcpyAsync(&h, s->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
  S_CK(cudaStreamSynchronize(st));
  *out = std::sqrt(h);
  return PFF_OK;
}

int axpby_level(const LevelWork& w, void* y, const void* x, double a, double b, cudaStream_t st) {
  if (w.prec == PFF_F64) S_CK(launch_axpby<double>((double*)y, (const double*)x, a, b, w.n, st));
  else S_CK(launch_axpby<float>((float*)y, (const float*)x, a, b, w.n, st));
  return PFF_OK;
}

int coarse_gmres(pff_solver* s, cudaStream_t st);

int level_apply(pff_solver* s, const LevelWork& w, const void* x, void* y, cudaStream_t st) {
  if (s->transpose) return pff_jacobian_transpose_apply(w.L, (pff_prec)w.prec, x, y, st);
  return pff_jacobian_apply(w.L, (pff_prec)w.prec, x, y, st);
}

// Chebyshev smoothing (Saad, Alg. 12.1) of J x = b or, in transposed mode,
// J^T x = b (same eigenvalue bounds: D^-1 J^T and D^-1 J have the same spectrum).
int cheb_level(pff_solver* s, LevelWork& w, int degree, double lmin, double lmax, cudaStream_t st) {
  const long long n = w.n;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  char* base = (char*)w.work;
  void* r = base;
  void* d = base + w.esz * n;
  void* Ad = base + 2 * w.esz * n;
  S_RC(level_apply(s, w, w.x, Ad, st));
  if (w.prec == PFF_F64)
    S_CK(launch_cheb_init<double>(n, (const double*)w.b, (const double*)Ad, (const double*)w.diag, (double*)r, (double*)d, 1.0 / theta, st));
  else
    S_CK(launch_cheb_init<float>(n, (const float*)w.b, (const float*)Ad, (const float*)w.diag, (float*)r, (float*)d, 1.0 / theta, st));
  for (int k = 0; k < degree; ++k) {
    const bool last = (k == degree - 1);
    double cd = 0.0, cr = 0.0;
    if (!last) {
      S_RC(level_apply(s, w, d, Ad, st));
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      cd = rho_new * rho;
      cr = 2.0 * rho_new / delta;
      rho = rho_new;
    }
    if (w.prec == PFF_F64)
      S_CK(launch_cheb_step<double>(n, (double*)w.x, (double*)d, (double*)r, (const double*)Ad, (const double*)w.diag, cd, cr, last, st));
    else
      S_CK(launch_cheb_step<float>(n, (float*)w.x, (float*)d, (float*)r, (const float*)Ad, (const float*)w.diag, cd, cr, last, st));
  }
  return PFF_OK;
}

// Products with the assembled coarse level: FP64, or with the mixed solver
// the FP32 copy of the stencil (the coarse level only preconditions; the
// transposed product of the adjoint stays FP64).
int coarse_spmv(pff_solver* s, const MeshDev& mc, const double* x, double* y, cudaStream_t st) {
  if (s->transpose) S_CK(launch_q1_spmv_t(mc, s->A, x, y, st));
  else if (s->A32) S_CK(launch_q1_spmv32(mc, s->A32, x, y, st));
  else S_CK(launch_q1_spmv(mc, s->A, x, y, st));
  return PFF_OK;
}

int coarse_cheb(pff_solver* s, cudaStream_t st) {
  if (s->prm.coarse_solver >= 1) return coarse_gmres(s, st);
  // FP64 Chebyshev-Jacobi on the assembled coarse operator, from x = 0.
  LevelWork& c = s->lv.back();
  const MeshDev& mc = c.L->mesh;
  const long long n = c.n;
  double* r = s->cwork;
  double* d = s->cwork + n;
  double* Ad = s->cwork + 2 * n;
  if (c.prec == PFF_F64) S_CK(cudaMemcpyAsync(s->cb, c.b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  else S_CK(launch_f2d(s->cb, (const float*)c.b, n, st));
  S_CK(cudaMemsetAsync(s->cx, 0, sizeof(double) * n, st));
  const double lmax = s->clmax * s->prm.cheb_hi, lmin = s->clmax * s->prm.coarse_lo;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  S_CK(cudaMemsetAsync(Ad, 0, sizeof(double) * n, st));
  S_CK(launch_cheb_init<double>(n, s->cb, Ad, s->cdiag, r, d, 1.0 / theta, st));
  const int deg = s->prm.coarse_degree;
  for (int k = 0; k < deg; ++k) {
    if (k == deg - 1) {
      S_CK(launch_cheb_step<double>(n, s->cx, d, r, Ad, s->cdiag, 0.0, 0.0, 1, st));
      break;
    }
    S_RC(coarse_spmv(s, mc, d, Ad, st));
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    S_CK(launch_cheb_step<double>(n, s->cx, d, r, Ad, s->cdiag, rho_new * rho, 2.0 * rho_new / delta, 0, st));
    rho = rho_new;
  }
  if (c.prec == PFF_F64) S_CK(cudaMemcpyAsync(c.x, s->cx, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  else S_CK(launch_d2f((float*)c.x, s->cx, n, st));
  return PFF_OK;
}

int vcycle(pff_solver* s, int l, cudaStream_t st) {
  LevelWork& w = s->lv[l];
  const bool coarsest = (l + 1 == (int)s->lv.size());
  if (coarsest && s->assembled) return coarse_cheb(s, st);
  S_CK(cudaMemsetAsync(w.x, 0, w.esz * w.n, st));
  const int deg = coarsest ? s->prm.coarse_degree : s->prm.cheb_degree;
  const double lo = coarsest ? s->prm.coarse_lo : s->prm.cheb_lo;
  S_RC(cheb_level(s, w, deg, lo * w.lmax, s->prm.cheb_hi * w.lmax, st));
  if (coarsest) return PFF_OK;
  // residual, restriction, coarse correction, prolongation
  S_RC(level_apply(s, w, w.x, w.tmp, st));
  if (w.prec == PFF_F64) S_CK(launch_bminus<double>((double*)w.tmp, (const double*)w.b, w.n, st));
  else S_CK(launch_bminus<float>((float*)w.tmp, (const float*)w.b, w.n, st));
  LevelWork& c = s->lv[l + 1];
  S_RC(pff_restrict(c.L, w.L, (pff_prec)w.prec, w.tmp, c.b, st));
  S_RC(vcycle(s, l + 1, st));
  S_RC(pff_prolong(c.L, w.L, (pff_prec)w.prec, c.x, w.tmp, st));
  S_RC(axpby_level(w, w.x, w.tmp, 1.0, 1.0, st));
  S_RC(cheb_level(s, w, s->prm.cheb_degree, s->prm.cheb_lo * w.lmax, s->prm.cheb_hi * w.lmax, st));
  return PFF_OK;
}

// ---- geometric h-multigrid on the assembled order-1 grid ------------------
int h_spmv(pff_solver* s, const HLevel& h, const double* x, double* y, cudaStream_t st) {
  if (s->transpose) S_CK(launch_q1_spmv_t(h.mesh, h.A, x, y, st));
  else if (h.A32) S_CK(launch_q1_spmv32(h.mesh, h.A32, x, y, st));
  else S_CK(launch_q1_spmv(h.mesh, h.A, x, y, st));
  return PFF_OK;
}

// Chebyshev-Jacobi (Saad, Alg. 12.1) on an assembled level, from x = 0 or from
// the given x.
int h_cheb(pff_solver* s, HLevel& h, int degree, double lmin, double lmax, bool zero_init, cudaStream_t st) {
  const long long n = h.n;
  double* r = h.work;
  double* d = h.work + n;
  double* Ad = h.work + 2 * n;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (zero_init) {
    S_CK(cudaMemsetAsync(h.x, 0, sizeof(double) * n, st));
    S_CK(cudaMemsetAsync(Ad, 0, sizeof(double) * n, st));
  } else {
    S_RC(h_spmv(s, h, h.x, Ad, st));
  }
  S_CK(launch_cheb_init<double>(n, h.b, Ad, h.diag, r, d, 1.0 / theta, st));
  for (int k = 0; k < degree; ++k) {
    if (k == degree - 1) {
      S_CK(launch_cheb_step<double>(n, h.x, d, r, Ad, h.diag, 0.0, 0.0, 1, st));
      break;
    }
    S_RC(h_spmv(s, h, d, Ad, st));
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    S_CK(launch_cheb_step<double>(n, h.x, d, r, Ad, h.diag, rho_new * rho, 2.0 * rho_new / delta, 0, st));
    rho = rho_new;
  }
  return PFF_OK;
}

// V-cycle on h-level l for A_l x = b_l (x from zero): Chebyshev pre- and
// post-smoothing, residual restriction by P^T, coarse correction, trilinear
// prolongation; the coarsest grid takes Chebyshev(coarse_degree).
int hcycle(pff_solver* s, int l, cudaStream_t st) {
  HLevel& h = s->hl[l];
  const pff_solver_params& p = s->prm;
  if (l + 1 == (int)s->hl.size())
    return h_cheb(s, h, p.coarse_degree, p.coarse_lo * h.lmax, p.cheb_hi * h.lmax, true, st);
  S_RC(h_cheb(s, h, p.cheb_degree, p.cheb_lo * h.lmax, p.cheb_hi * h.lmax, true, st));
  S_RC(h_spmv(s, h, h.x, h.r, st));
  S_CK(launch_bminus<double>(h.r, h.b, h.n, st));
  HLevel& c = s->hl[l + 1];
  S_CK(launch_hrestrict(c.mesh, h.mesh, h.r, c.b, c.mask, h.mask, st));
  S_RC(hcycle(s, l + 1, st));
  S_CK(launch_hprolong_add(c.mesh, h.mesh, c.x, h.x, c.mask, h.mask, st));
  return h_cheb(s, h, p.cheb_degree, p.cheb_lo * h.lmax, p.cheb_hi * h.lmax, false, st);
}

// Spectral radius of a small dense matrix (row-major k x k) by power iteration
// on the host, with the growth rate averaged over the last iterations so that a
// dominant complex pair is measured too.
double small_spectral_radius(const std::vector<double>& H, int k) {
  std::vector<double> v(k, 1.0), y(k);
  for (int i = 0; i < k; ++i) v[i] = 1.0 + 0.01 * i;
  double logsum = 0.0;
  int counted = 0;
  for (int it = 0; it < 2000; ++it) {
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += H[i * k + j] * v[j];
      y[i] = s;
      nrm += s * s;
    }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return 0.0;
    for (int i = 0; i < k; ++i) v[i] = y[i] / nrm;
    if (it >= 1000) { logsum += std::log(nrm); ++counted; }
  }
  return std::exp(logsum / counted);
}

// lambda_max of D^-1 A: k Arnoldi steps (Gram-Schmidt twice, FP64 basis in the
// FGMRES storage) from a seeded random-sign vector; the estimate is the spectral
// radius of the k x k Hessenberg block (the reading of the eigenvalue bound of
// a Chebyshev smoother: a few Arnoldi/Lanczos steps).  op(v, w) sets
// w = D^-1 A v on FP64 vectors of length n.
template <typename Op>
int arnoldi_lmax(pff_solver* s, long long n, Op&& op, double* out, cudaStream_t st) {
  const int k = std::min(s->prm.power_iters, s->prm.krylov_restart);
  double* V = s->V;  // (restart + 1) fine vectors >= (k + 1) level vectors
  S_CK(cudaMemcpyAsync(V, s->pw64, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  double h0;
  S_RC(dev_dots(s, V, 0, 1, V, n, &h0, st));
  S_CK(launch_axpby<double>(V, V, 1.0 / std::sqrt(h0), 0.0, n, st));
  std::vector<double> H((k + 1) * k, 0.0), h(k + 2);
  int kk = k;
  for (int j = 0; j < k; ++j) {
    double* vj = V + (long long)j * n;
    double* wv = V + (long long)(j + 1) * n;
    S_RC(op(vj, wv));
    // classical Gram-Schmidt with the second pass only when the first removed
    // more than half of ||w||^2 (the criterion of the outer FGMRES); the dots
    // include w . w itself (wv is V_{j+1})
    double ww2 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      S_RC(dev_dots(s, V, n, j + 2, wv, n, h.data(), st));
      const double ww = h[j + 1];
      S_CK(cudaMemcpyAsync(s->hdev, h.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st));
      S_CK(launch_maxpy(wv, V, n, j + 1, s->hdev, -1.0, n, st));
      double hsq = 0.0;
      for (int i = 0; i <= j; ++i) {
        H[i * k + j] += h[i];
        hsq += h[i] * h[i];
      }
      ww2 = std::max(ww - hsq, 0.0);
      if (ww2 >= 0.5 * ww) break;
    }
    const double hn = std::sqrt(ww2);
    if (!std::isfinite(hn)) return sfail(PFF_ERR_DEVICE, "Arnoldi eigenvalue estimate: non-finite vector");
    H[(j + 1) * k + j] = hn;
    if (hn <= 1e-14 * std::fabs(H[j * k + j]) + 1e-300) { kk = j + 1; break; }
    S_CK(launch_axpby<double>(wv, wv, 1.0 / hn, 0.0, n, st));
  }
  std::vector<double> Hk(kk * kk);
  for (int i = 0; i < kk; ++i)
    for (int j = 0; j < kk; ++j) Hk[i * kk + j] = H[i * k + j];
  const double lam = small_spectral_radius(Hk, kk);
  if (!(lam > 0.0) || !std::isfinite(lam)) return sfail(PFF_ERR_DEVICE, "Arnoldi eigenvalue estimate failed");
  *out = lam;
  return PFF_OK;
}

int arnoldi_level(pff_solver* s, LevelWork& w, cudaStream_t st) {
  const long long n = w.n;
  auto op = [&](const double* vj, double* wv) -> int {
    if (w.prec == PFF_F64) {
      S_RC(pff_jacobian_apply(w.L, PFF_F64, vj, wv, st));
      S_CK(launch_dscale<double>(wv, wv, (const double*)w.diag, n, st));
    } else {
      S_CK(launch_d2f((float*)w.x, vj, n, st));
      S_RC(pff_jacobian_apply(w.L, (pff_prec)w.prec, w.x, w.tmp, st));
      S_CK(launch_dscale<float>((float*)w.tmp, (const float*)w.tmp, (const float*)w.diag, n, st));
      S_CK(launch_f2d(wv, (const float*)w.tmp, n, st));
    }
    return PFF_OK;
  };
  return arnoldi_lmax(s, n, op, &w.lmax, st);
}

int arnoldi_hlevel(pff_solver* s, HLevel& h, cudaStream_t st) {
  auto op = [&](const double* vj, double* wv) -> int {
    S_RC(h_spmv(s, h, vj, wv, st));
    S_CK(launch_dscale<double>(wv, wv, h.diag, h.n, st));
    return PFF_OK;
  };
  return arnoldi_lmax(s, h.n, op, &h.lmax, st);
}

int power_coarse(pff_solver* s, cudaStream_t st) {
  LevelWork& c = s->lv.back();
  const long long n = c.n;
  double* v = s->cx;
  double* y = s->cb;
  S_CK(cudaMemcpyAsync(v, s->pw64, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  double h;
  S_RC(dev_dots(s, v, 0, 1, v, n, &h, st));
  S_CK(launch_axpby<double>(v, v, 1.0 / std::sqrt(h), 0.0, n, st));
  double lam = 1.0;
  for (int it = 0; it < s->prm.power_iters; ++it) {
    S_RC(coarse_spmv(s, c.L->mesh, v, y, st));
    S_CK(launch_dscale<double>(y, y, s->cdiag, n, st));
    S_RC(dev_dots(s, y, 0, 1, y, n, &h, st));
    lam = std::sqrt(h);
    if (!(lam > 0.0) || !std::isfinite(lam)) return sfail(PFF_ERR_DEVICE, "coarse power iteration failed");
    S_CK(launch_axpby<double>(v, y, 1.0 / lam, 0.0, n, st));
  }
  s->clmax = lam;
  return PFF_OK;
}

// Flexible GMRES(m), right preconditioned (Saad, Alg. 9.6), FP64; classical
// Gram-Schmidt with a second pass when the first one loses accuracy (the
// adaptive CGS refinement of Sec. 5).  V: (m+1) n, Z: m n device doubles.
struct Krylov {
  long long n = 0;
  int m = 0;
  double *V = nullptr, *Z = nullptr;
};

template <typename ApplyA, typename ApplyM>
int gmres_flex(pff_solver* s, const Krylov& kw, ApplyA&& applyA, ApplyM&& applyM, const double* b, double* x,
               double rtol, int maxit, int* iters, double* relres, cudaStream_t st) {
  const long long n = kw.n;
  const int m = kw.m;
  std::vector<double> H((m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0), h(m + 2), y(m);
  S_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
  double beta0 = -1.0, res = 0.0;
  int total = 0;
  bool first = true;
  while (true) {
    double* v0 = kw.V;
    if (first) {
      S_CK(cudaMemcpyAsync(v0, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    } else {
      S_RC(applyA(x, v0));
      S_CK(launch_bminus<double>(v0, b, n, st));
    }
    double bb;
    S_RC(dev_dots(s, v0, 0, 1, v0, n, &bb, st));
    double beta = std::sqrt(bb);
    if (beta0 < 0) beta0 = beta;
    if (beta == 0.0 || beta0 == 0.0) { res = 0.0; break; }
    res = beta;
    if (beta <= rtol * beta0 || total >= maxit) break;
    S_CK(launch_axpby<double>(v0, v0, 1.0 / beta, 0.0, n, st));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < m && total < maxit; ++j) {
      double* vj = kw.V + (long long)j * n;
      double* zj = kw.Z + (long long)j * n;
      double* w = kw.V + (long long)(j + 1) * n;
      S_RC(applyM(vj, zj));
      S_RC(applyA(zj, w));
      S_RC(dev_dots(s, kw.V, n, j + 2, w, n, h.data(), st));
      double ww = h[j + 1];
      S_CK(cudaMemcpyAsync(s->hdev, h.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st));
      S_CK(launch_maxpy(w, kw.V, n, j + 1, s->hdev, -1.0, n, st));
      double hsq = 0.0;
      for (int i = 0; i <= j; ++i) hsq += h[i] * h[i];
      std::vector<double> hcol(h.begin(), h.begin() + j + 1);
      // ||w||^2 after the projection is ww - hsq; a second pass only when the
      // first one removed more than half of ||w||^2 (cancellation has cost
      // accuracy: Daniel-Gragg-Kaufman-Stewart criterion), otherwise the
      // estimate is accurate to a few rounding errors and no further
      // reduction is needed
      double ww2 = ww - hsq;
      if (ww2 < 0.5 * ww) {
        S_RC(dev_dots(s, kw.V, n, j + 2, w, n, h.data(), st));
        ww2 = h[j + 1];
        double h2sq = 0.0;
        for (int i = 0; i <= j; ++i) h2sq += h[i] * h[i];
        S_CK(cudaMemcpyAsync(s->hdev, h.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st));
        S_CK(launch_maxpy(w, kw.V, n, j + 1, s->hdev, -1.0, n, st));
        for (int i = 0; i <= j; ++i) hcol[i] += h[i];
        ww2 = std::max(ww2 - h2sq, 0.0);
      }
      double hn = std::sqrt(std::max(ww2, 0.0));
      for (int i = 0; i <= j; ++i) H[i * m + j] = hcol[i];
      H[(j + 1) * m + j] = hn;
      if (hn > 0.0) S_CK(launch_axpby<double>(w, w, 1.0 / hn, 0.0, n, st));
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double den = std::hypot(a, c);
      cs[j] = den > 0 ? a / den : 1.0;
      sn[j] = den > 0 ? c / den : 0.0;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      jend = j + 1;
      res = std::fabs(g[j + 1]);
      if (res <= rtol * beta0 || hn == 0.0) break;
    }
    for (int i = jend - 1; i >= 0; --i) {
      double sum = g[i];
      for (int k = i + 1; k < jend; ++k) sum -= H[i * m + k] * y[k];
      y[i] = sum / H[i * m + i];
    }
    S_CK(cudaMemcpyAsync(s->hdev, y.data(), sizeof(double) * jend, cudaMemcpyHostToDevice, st));
    S_CK(launch_maxpy(x, kw.Z, n, jend, s->hdev, 1.0, n, st));
    S_CK(cudaStreamSynchronize(st));
    first = false;
    if (res <= rtol * beta0 || total >= maxit) break;
  }
  *iters = total;
  *relres = beta0 > 0 ? res / beta0 : 0.0;
  return PFF_OK;
}

int precondition(pff_solver* s, const double* v, double* z, cudaStream_t st);

int fgmres(pff_solver* s, const double* b, double* x, double rtol, int maxit, int* iters, double* relres,
           cudaStream_t st) {
  pff_level* F = s->lv[0].L;
  Krylov kw;
  kw.n = s->n;
  kw.m = s->prm.krylov_restart;
  kw.V = s->V;
  kw.Z = s->Z;
  const pff_prec outer = (pff_prec)s->prm.outer_prec;
  auto A = [&](const double* in, double* out) {
    if (s->transpose) return pff_jacobian_transpose_apply(F, outer, in, out, st);
    return pff_jacobian_apply(F, outer, in, out, st);
  };
  auto M = [&](const double* in, double* out) { return precondition(s, in, out, st); };
  return gmres_flex(s, kw, A, M, b, x, rtol, maxit, iters, relres, st);
}

// z = M^-1 v on FP64 fine vectors: one V-cycle (FP32 levels in the mixed variant).
int precondition(pff_solver* s, const double* v, double* z, cudaStream_t st) {
  LevelWork& f = s->lv[0];
  const long long n = s->n;
  if (f.prec == PFF_F64) S_CK(cudaMemcpyAsync(f.b, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  else S_CK(launch_d2f((float*)f.b, v, n, st));
  S_RC(vcycle(s, 0, st));
  if (f.prec == PFF_F64) S_CK(cudaMemcpyAsync(z, f.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  else S_CK(launch_f2d(z, (const float*)f.x, n, st));
  return PFF_OK;
}

// Coarsest level: GMRES on the assembled FP64 operator to coarse_rtol (at most
// coarse_maxit iterations), from x = 0, preconditioned by Jacobi
// (coarse_solver 1) or by one h-multigrid V-cycle (coarse_solver 2).
int coarse_gmres(pff_solver* s, cudaStream_t st) {
  LevelWork& c = s->lv.back();
  const MeshDev& mc = c.L->mesh;
  const long long n = c.n;
  if (c.prec == PFF_F64) S_CK(cudaMemcpyAsync(s->cb, c.b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  else S_CK(launch_f2d(s->cb, (const float*)c.b, n, st));
  Krylov kw;
  kw.n = n;
  kw.m = s->prm.krylov_restart;
  kw.V = s->cV;
  kw.Z = s->cZ;
  auto A = [&](const double* in, double* out) -> int { return coarse_spmv(s, mc, in, out, st); };
  auto M = [&](const double* in, double* out) -> int {
    if (s->prm.coarse_solver == 2) {  // one h-multigrid V-cycle
      HLevel& h0 = s->hl[0];
      S_CK(cudaMemcpyAsync(h0.b, in, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      S_RC(hcycle(s, 0, st));
      S_CK(cudaMemcpyAsync(out, h0.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      return PFF_OK;
    }
    S_CK(launch_dscale<double>(out, in, s->cdiag, n, st));
    return PFF_OK;
  };
  int its = 0;
  double rel = 0.0;
  S_RC(gmres_flex(s, kw, A, M, s->cb, s->cx, s->prm.coarse_rtol, s->prm.coarse_maxit, &its, &rel, st));
  s->coarse_iters += its;
  if (c.prec == PFF_F64) S_CK(cudaMemcpyAsync(c.x, s->cx, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  else S_CK(launch_d2f((float*)c.x, s->cx, n, st));
  return PFF_OK;
}

// Diagonals, coarse operators and eigenvalue bounds for the current stored
// linearisation.  `eig` = false keeps the previous lambda_max estimates (the
// eig_every option of a Newton solve).
int setup(pff_solver* s, cudaStream_t st, bool eig = true) {
  const int L = (int)s->lv.size();
  for (int l = 0; l < L; ++l) {
    LevelWork& w = s->lv[l];
    if (l + 1 == L && s->assembled) continue;
    S_RC(pff_assemble_diagonal(w.L, (pff_prec)w.prec, w.diag, st));
  }
  if (s->assembled) {
    LevelWork& c = s->lv.back();
    pff_op* op = s->op;
    // the mixed solver assembles its (preconditioning) coarse level from the
    // FP32 words in FP32 arithmetic, the FP64 solver from the FP64 words
    S_CK(launch_q1_assemble_sf(c.L->mesh, op->Q, op->lin64, s->prm.mixed ? op->lin32 : nullptr, c.L->tab.B64,
                               c.L->tab.Dt64, c.L->mask, s->Ke, s->A,
                               op->geo != nullptr, st));
    S_CK(launch_q1_diag(c.L->mesh, s->A, s->cdiag, st));
    if (s->A32) S_CK(launch_d2f(s->A32, s->A, 27LL * 16 * c.L->mesh.nn, st));
    if (s->prm.coarse_solver == 0 && eig) S_RC(power_coarse(s, st));
    if (s->prm.coarse_solver == 2) {
      for (size_t l = 1; l < s->hl.size(); ++l) {
        HLevel& f = s->hl[l - 1];
        HLevel& h = s->hl[l];
        S_CK(launch_hmask(f.mesh, h.mesh, f.mask, h.own_mask, st));
        S_CK(launch_q1_coarsen(f.mesh, h.mesh, f.mask, f.Ke, h.Ke, s->prm.mixed != 0, st));
        S_CK(launch_q1_gather(h.mesh, h.Ke, h.mask, h.A, st));
        S_CK(launch_q1_diag(h.mesh, h.A, h.diag, st));
        if (h.A32) S_CK(launch_d2f(h.A32, h.A, 27LL * 16 * h.mesh.nn, st));
      }
      if (eig)
        for (HLevel& h : s->hl) S_RC(arnoldi_hlevel(s, h, st));
    }
  }
  for (int l = 0; l < L && eig; ++l) {
    if (l + 1 == L && s->assembled) continue;
    S_RC(arnoldi_level(s, s->lv[l], st));
  }
  return PFF_OK;
}

void free_solver(pff_solver* s) {
  for (auto& w : s->lv) {
    cudaFree(w.diag); cudaFree(w.b); cudaFree(w.x); cudaFree(w.tmp); cudaFree(w.work);
  }
  cudaFree(s->A); cudaFree(s->A32); cudaFree(s->cdiag); cudaFree(s->cb); cudaFree(s->cx); cudaFree(s->cwork);
  cudaFree(s->cV); cudaFree(s->cZ); cudaFree(s->Ke);
  for (HLevel& h : s->hl) {
    if (h.owns) { cudaFree(h.Ke); cudaFree(h.A); cudaFree(h.A32); cudaFree(h.diag); cudaFree(h.own_mask); }
    cudaFree(h.b); cudaFree(h.x); cudaFree(h.r); cudaFree(h.work);
  }
  cudaFree(s->V); cudaFree(s->Z); cudaFree(s->r); cudaFree(s->dz); cudaFree(s->zold);
  cudaFree(s->partial); cudaFree(s->dots); cudaFree(s->hdev);
  cudaFree(s->pw64); cudaFree(s->pw32);
  cudaFree(s->a_in); cudaFree(s->pbuf); cudaFree(s->qa); cudaFree(s->ag); cudaFree(s->alam); cudaFree(s->av);
  cudaFree(s->gth);
}

}  // namespace

extern "C" {

int pff_solver_default_params(pff_solver_params* p) {
  if (!p) return sfail(PFF_ERR_INVALID, "pff_solver_default_params: null");
  p->mixed = 1;
  p->cheb_degree = 3;
  p->cheb_lo = 0.1;
  p->cheb_hi = 1.1;
  p->coarse_degree = 16;
  p->coarse_lo = 0.02;
  p->power_iters = 10;
  p->krylov_restart = 30;
  p->krylov_maxit = 200;
  p->krylov_rtol = 1e-3;
  p->newton_maxit = 20;
  p->newton_rtol = 1e-8;
  p->line_search_max = 8;
  p->coarse_solver = 2;
  p->coarse_rtol = 1e-2;
  p->coarse_maxit = 200;
  p->verbose = 0;
  p->outer_prec = PFF_F64;
  p->newton_stall = 0;
  p->eig_every = 1;
  p->level_words = 32;
  return PFF_OK;
}

int pff_create_solver(pff_op* op, int nlevels, pff_level* const* levels, const pff_solver_params* prm,
                      pff_solver** out) {
  if (!op || !levels || !prm || !out || nlevels < 1) return sfail(PFF_ERR_INVALID, "pff_create_solver: bad argument");
  if (prm->krylov_restart < 1 || prm->krylov_restart > 60) return sfail(PFF_ERR_INVALID, "pff_create_solver: 1 <= restart <= 60");
  if (prm->cheb_degree < 1 || prm->coarse_degree < 1) return sfail(PFF_ERR_INVALID, "pff_create_solver: degrees >= 1");
  if (!(prm->cheb_hi > prm->cheb_lo && prm->cheb_lo > 0 && prm->coarse_lo > 0 && prm->coarse_lo < prm->cheb_hi))
    return sfail(PFF_ERR_INVALID, "pff_create_solver: need 0 < lo < hi");
  if (levels[0]->op != op || !levels[0]->is_fine) return sfail(PFF_ERR_INVALID, "pff_create_solver: levels[0] must be the fine level of op");
  for (int l = 1; l < nlevels; ++l)
    if (levels[l]->op != op || levels[l]->p >= levels[l - 1]->p)
      return sfail(PFF_ERR_INVALID, "pff_create_solver: levels must share op with decreasing order");
  if (prm->mixed && !op->lin32) return sfail(PFF_ERR_INVALID, "pff_create_solver: mixed precision needs pff_op_enable_f32");
  if (prm->coarse_solver < 0 || prm->coarse_solver > 2)
    return sfail(PFF_ERR_INVALID, "pff_create_solver: coarse_solver must be 0, 1 or 2");
  if (prm->outer_prec != PFF_F64 && prm->outer_prec != PFF_DF64)
    return sfail(PFF_ERR_INVALID, "pff_create_solver: outer_prec must be PFF_F64 or PFF_DF64");
  if (prm->outer_prec == PFF_DF64 && !op->df)
    return sfail(PFF_ERR_INVALID, "pff_create_solver: outer_prec PFF_DF64 needs pff_op_enable_df");
  if (prm->level_words != 32 && prm->level_words != 16)
    return sfail(PFF_ERR_INVALID, "pff_create_solver: level_words must be 32 or 16");
  if (prm->mixed && prm->level_words == 16 && !(op->bf16 && op->lin16))
    return sfail(PFF_ERR_INVALID, "pff_create_solver: level_words 16 needs pff_op_enable_bf16");
  pff_solver* s = new pff_solver();
  s->op = op;
  s->prm = *prm;
  s->n = 4 * op->mesh.nn;
  s->assembled = (levels[nlevels - 1]->p == 1 && nlevels > 1);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < nlevels; ++l) {
    LevelWork w;
    w.L = levels[l];
    w.p = levels[l]->p;
    w.prec = prm->mixed ? (prm->level_words == 16 ? PFF_F32_BF16 : PFF_F32) : PFF_F64;
    w.esz = (w.prec == PFF_F64) ? 8 : 4;
    w.n = 4 * levels[l]->mesh.nn;
    if (e == cudaSuccess) e = cudaMalloc(&w.diag, w.esz * w.n);
    if (e == cudaSuccess) e = cudaMalloc(&w.b, w.esz * w.n);
    if (e == cudaSuccess) e = cudaMalloc(&w.x, w.esz * w.n);
    if (e == cudaSuccess) e = cudaMalloc(&w.tmp, w.esz * w.n);
    if (e == cudaSuccess) e = cudaMalloc(&w.work, 3 * w.esz * w.n);
    s->lv.push_back(w);
  }
  if (s->assembled) {
    const long long nc = s->lv.back().n;
    if (e == cudaSuccess) e = cudaMalloc(&s->A, sizeof(double) * 27 * 16 * (nc / 4));
    if (e == cudaSuccess && prm->mixed) e = cudaMalloc(&s->A32, sizeof(float) * 27 * 16 * (nc / 4));
    if (e == cudaSuccess) e = cudaMalloc(&s->cdiag, sizeof(double) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&s->cb, sizeof(double) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&s->cx, sizeof(double) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&s->cwork, sizeof(double) * 3 * nc);
    if (e == cudaSuccess) e = cudaMalloc(&s->Ke, sizeof(double) * 1024 * (size_t)op->nel);
    if (e == cudaSuccess && prm->coarse_solver >= 1) e = cudaMalloc(&s->cV, sizeof(double) * (prm->krylov_restart + 1) * nc);
    if (e == cudaSuccess && prm->coarse_solver >= 1) e = cudaMalloc(&s->cZ, sizeof(double) * prm->krylov_restart * nc);
    if (prm->coarse_solver == 2) {
      // h-levels: the Q1 level, then full coarsening while every direction has
      // an even number of elements and keeps at least two
      pff_level* Lc = s->lv.back().L;
      HLevel h0;
      h0.mesh = Lc->mesh;
      h0.n = nc;
      h0.Ke = s->Ke;
      h0.A = s->A;
      h0.A32 = s->A32;
      h0.diag = s->cdiag;
      h0.mask = Lc->is_fine ? op->mask : Lc->mask;
      s->hl.push_back(h0);
      while (true) {
        const MeshDev& mf = s->hl.back().mesh;
        if (mf.nx % 2 || mf.ny % 2 || mf.nz % 2 || mf.nx < 4 || mf.ny < 4 || mf.nz < 4) break;
        HLevel h;
        h.mesh = mf;
        h.mesh.nx = mf.nx / 2; h.mesh.ny = mf.ny / 2; h.mesh.nz = mf.nz / 2;
        h.mesh.nel = h.mesh.nx * h.mesh.ny * h.mesh.nz;
        h.mesh.nnx = h.mesh.nx + 1; h.mesh.nny = h.mesh.ny + 1;
        h.mesh.nn = (long long)h.mesh.nnx * h.mesh.nny * (h.mesh.nz + 1);
        h.mesh.offsets = nullptr;
        h.n = 4 * h.mesh.nn;
        h.owns = true;
        if (e == cudaSuccess) e = cudaMalloc(&h.Ke, sizeof(double) * 1024 * (size_t)h.mesh.nel);
        if (e == cudaSuccess) e = cudaMalloc(&h.A, sizeof(double) * 27 * 16 * (size_t)h.mesh.nn);
        if (e == cudaSuccess && prm->mixed) e = cudaMalloc(&h.A32, sizeof(float) * 27 * 16 * (size_t)h.mesh.nn);
        if (e == cudaSuccess) e = cudaMalloc(&h.diag, sizeof(double) * h.n);
        if (e == cudaSuccess) e = cudaMalloc(&h.own_mask, h.n);
        h.mask = h.own_mask;
        s->hl.push_back(h);
        if (e != cudaSuccess) break;
      }
      for (HLevel& h : s->hl) {
        if (e == cudaSuccess) e = cudaMalloc(&h.b, sizeof(double) * h.n);
        if (e == cudaSuccess) e = cudaMalloc(&h.x, sizeof(double) * h.n);
        if (e == cudaSuccess) e = cudaMalloc(&h.r, sizeof(double) * h.n);
        if (e == cudaSuccess) e = cudaMalloc(&h.work, sizeof(double) * 3 * h.n);
      }
    }
  }
  const int m = prm->krylov_restart;
  if (e == cudaSuccess) e = cudaMalloc(&s->V, sizeof(double) * (m + 1) * s->n);
  if (e == cudaSuccess) e = cudaMalloc(&s->Z, sizeof(double) * m * s->n);
  if (e == cudaSuccess) e = cudaMalloc(&s->r, sizeof(double) * s->n);
  if (e == cudaSuccess) e = cudaMalloc(&s->dz, sizeof(double) * s->n);
  if (e == cudaSuccess) e = cudaMalloc(&s->zold, sizeof(double) * s->n);
  if (e == cudaSuccess) e = cudaMalloc(&s->partial, sizeof(double) * 64 * kReduceBlocks);
  if (e == cudaSuccess) e = cudaMalloc(&s->dots, sizeof(double) * 64);
  if (e == cudaSuccess) e = cudaMalloc(&s->hdev, sizeof(double) * 64);
  if (e == cudaSuccess) e = cudaMalloc(&s->pw64, sizeof(double) * s->n);
  if (e == cudaSuccess) e = cudaMalloc(&s->pw32, sizeof(float) * s->n);
  if (e == cudaSuccess) {
    // seeded start vector of the eigenvalue estimates (xorshift64*, random signs)
    std::vector<double> h(s->n);
    std::vector<float> hf(s->n);
    unsigned long long st = 0x9E3779B97F4A7C15ull;
    for (long long i = 0; i < s->n; ++i) {
      st ^= st >> 12; st ^= st << 25; st ^= st >> 27;
      double u = (double)((st * 0x2545F4914F6CDD1Dull) >> 11) * (1.0 / 9007199254740992.0);
      h[i] = (u < 0.5) ? -1.0 : 1.0;
      hf[i] = (float)h[i];
    }
    e = cudaMemcpy(s->pw64, h.data(), sizeof(double) * s->n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->pw32, hf.data(), sizeof(float) * s->n, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    free_solver(s);
    delete s;
    return sfail(PFF_ERR_CUDA, std::string("pff_create_solver: ") + cudaGetErrorString(e));
  }
  *out = s;
  return PFF_OK;
}

int pff_vec_axpby(pff_prec prec, int64_t n, double a, const void* x, double b, void* y, void* stream) {
  if (!x || !y || n < 0) return sfail(PFF_ERR_INVALID, "pff_vec_axpby: bad argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (prec == PFF_F64) S_CK(launch_axpby<double>((double*)y, (const double*)x, a, b, n, st));
  else if (prec == PFF_F32) S_CK(launch_axpby<float>((float*)y, (const float*)x, a, b, n, st));
  else return sfail(PFF_ERR_INVALID, "pff_vec_axpby: unknown precision");
  return PFF_OK;
}

int pff_destroy_solver(pff_solver* s) {
  if (!s) return PFF_OK;
  free_solver(s);
  delete s;
  return PFF_OK;
}

int pff_solver_setup(pff_solver* s, void* stream) {
  if (!s) return sfail(PFF_ERR_INVALID, "pff_solver_setup: null solver");
  return setup(s, reinterpret_cast<cudaStream_t>(stream));
}

int pff_solver_level_lambda(const pff_solver* s, int level, double* lmax) {
  if (!s || !lmax || level < 0 || level >= (int)s->lv.size()) return sfail(PFF_ERR_INVALID, "pff_solver_level_lambda: bad argument");
  *lmax = (level + 1 == (int)s->lv.size() && s->assembled) ? s->clmax : s->lv[level].lmax;
  return PFF_OK;
}

int pff_solver_vcycle(pff_solver* s, const double* r, double* z, void* stream) {
  if (!s || !r || !z) return sfail(PFF_ERR_INVALID, "pff_solver_vcycle: null argument");
  return precondition(s, r, z, reinterpret_cast<cudaStream_t>(stream));
}

int pff_solver_coarse_apply(pff_solver* s, const double* x, double* y, void* stream) {
  if (!s || !x || !y || !s->assembled) return sfail(PFF_ERR_INVALID, "pff_solver_coarse_apply: needs an assembled coarse level");
  S_CK(launch_q1_spmv(s->lv.back().L->mesh, s->A, x, y, reinterpret_cast<cudaStream_t>(stream)));
  return PFF_OK;
}

int pff_solver_num_hlevels(const pff_solver* s) { return s ? (int)s->hl.size() : 0; }

int pff_solver_hlevel_info(const pff_solver* s, int level, int* dims, double* lmax) {
  if (!s || !dims || !lmax || level < 0 || level >= (int)s->hl.size())
    return sfail(PFF_ERR_INVALID, "pff_solver_hlevel_info: bad argument");
  const HLevel& h = s->hl[level];
  dims[0] = h.mesh.nx; dims[1] = h.mesh.ny; dims[2] = h.mesh.nz;
  *lmax = h.lmax;
  return PFF_OK;
}

int pff_solver_hlevel_apply(pff_solver* s, int level, const double* x, double* y, void* stream) {
  if (!s || !x || !y || level < 0 || level >= (int)s->hl.size())
    return sfail(PFF_ERR_INVALID, "pff_solver_hlevel_apply: bad argument");
  S_CK(launch_q1_spmv(s->hl[level].mesh, s->hl[level].A, x, y, reinterpret_cast<cudaStream_t>(stream)));
  return PFF_OK;
}

int pff_solver_hcycle(pff_solver* s, const double* b, double* x, void* stream) {
  if (!s || !b || !x || s->hl.empty()) return sfail(PFF_ERR_INVALID, "pff_solver_hcycle: needs coarse_solver 2");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  HLevel& h0 = s->hl[0];
  S_CK(cudaMemcpyAsync(h0.b, b, sizeof(double) * h0.n, cudaMemcpyDeviceToDevice, st));
  S_RC(hcycle(s, 0, st));
  S_CK(cudaMemcpyAsync(x, h0.x, sizeof(double) * h0.n, cudaMemcpyDeviceToDevice, st));
  return PFF_OK;
}

int pff_solver_krylov(pff_solver* s, const double* b, double* x, double rtol, int maxit, int* iters, double* relres,
                      void* stream) {
  if (!s || !b || !x || !iters || !relres) return sfail(PFF_ERR_INVALID, "pff_solver_krylov: null argument");
  return fgmres(s, b, x, rtol, maxit, iters, relres, reinterpret_cast<cudaStream_t>(stream));
}

int pff_newton_solve(pff_solver* s, double* z, pff_newton_stats* stats, void* stream) {
  if (!s || !z || !stats) return sfail(PFF_ERR_INVALID, "pff_newton_solve: null argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::memset(stats, 0, sizeof(*stats));
  s->coarse_iters = 0;
  const long long n = s->n;
  double r0 = -1.0;
  for (int it = 0;; ++it) {
    double t0 = now();
    if (it == 0 || s->prm.line_search_max == 0) {
      S_RC(pff_residual(s->op, z, s->r, st));
      int status = 0;
      S_RC(pff_get_status(s->op, stream, &status));
      if (status) {
        stats->status = status;
        return sfail(PFF_ERR_DEVICE, "pff_newton_solve: residual kernel status " + std::to_string(status));
      }
    }
    double rr;
    S_RC(dev_dots(s, s->r, 0, 1, s->r, n, &rr, st));
    double rn = std::sqrt(rr);
    stats->t_residual += now() - t0;
    if (r0 < 0) r0 = rn;
    if (it < 64) stats->res_history[it] = rn;
    stats->res0 = r0;
    stats->res = rn;
    if (rn <= s->prm.newton_rtol * r0 || rn == 0.0) { stats->converged = 1; break; }
    if (it >= s->prm.newton_maxit) break;
    const int k = s->prm.newton_stall;
    if (k > 0 && it >= k && it - k < 64 && rn > 0.5 * stats->res_history[it - k]) break;  // stagnation
    t0 = now();
    const int ev = s->prm.eig_every;
    S_RC(setup(s, st, ev > 0 ? (it % ev == 0) : (it == 0)));
    S_CK(cudaStreamSynchronize(st));
    stats->t_setup += now() - t0;
    t0 = now();
    int its = 0;
    double rel = 0.0;
    S_RC(fgmres(s, s->r, s->dz, s->prm.krylov_rtol, s->prm.krylov_maxit, &its, &rel, st));
    S_CK(cudaStreamSynchronize(st));
    stats->t_krylov += now() - t0;
    stats->krylov_iterations += its;
    stats->newton_iterations = it + 1;
    stats->last_krylov_relres = rel;
    stats->coarse_iterations = (int)s->coarse_iters;
    if (s->prm.verbose)
      std::fprintf(stderr, "[pff newton] it %d |r| %.6e |r|/|r0| %.3e krylov %d (rel %.2e) coarse its %lld t_res %.3f t_setup %.3f t_krylov %.3f\n",
                   it, rn, rn / r0, its, rel, s->coarse_iters, stats->t_residual, stats->t_setup, stats->t_krylov);
    // backtracking line search (Sec. 5): accept z - alpha dz once the residual is
    // finite, every det F > 0 and ||r|| <= (1 - 1e-4 alpha) ||r_prev||; halve alpha
    // otherwise.  The residual of the accepted point is the next iteration's.
    t0 = now();
    S_CK(cudaMemcpyAsync(s->zold, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double alpha = 1.0;
    bool accepted = false;
    for (int ls = 0; ls <= s->prm.line_search_max; ++ls) {
      S_CK(cudaMemcpyAsync(z, s->zold, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      S_CK(launch_axpby<double>(z, s->dz, -alpha, 1.0, n, st));
      if (s->prm.line_search_max == 0) { accepted = true; break; }
      S_RC(pff_residual(s->op, z, s->r, st));
      int lst = 0;
      S_RC(pff_get_status(s->op, stream, &lst));
      double r2 = 0.0;
      if (!lst) S_RC(dev_dots(s, s->r, 0, 1, s->r, n, &r2, st));
      const double rt = std::sqrt(r2);
      if (!lst && std::isfinite(rt) && rt <= (1.0 - 1e-4 * alpha) * rn) { accepted = true; break; }
      if (!lst && std::isfinite(rt) && ls == s->prm.line_search_max) { accepted = true; break; }
      alpha *= 0.5;
      stats->line_search_cuts += 1;
    }
    stats->t_residual += now() - t0;
    if (!accepted) {
      S_CK(cudaMemcpyAsync(z, s->zold, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      return sfail(PFF_ERR_DEVICE, "pff_newton_solve: line search found no admissible step");
    }
  }
  return PFF_OK;
}

}  // extern "C"

namespace {

template <typename T>
cudaError_t elem_launch(int Q, int P, int mode, const ElemArgs<T>& a, cudaStream_t st) {
  switch (Q) {
    case 2: return launch_elem_q2<T>(P, mode, a, st);
    case 3: return launch_elem_q3<T>(P, mode, a, st);
    case 4: return launch_elem_q4<T>(P, mode, a, st);
    case 5: return launch_elem_q5<T>(P, mode, a, st);
  }
  return cudaErrorInvalidValue;
}

ElemArgs<double> fine_args(pff_op* op) {
  ElemArgs<double> a;
  std::memset(&a, 0, sizeof(a));
  a.mesh = op->mesh;
  a.B = op->tab.B64;
  a.Dc = op->tab.Dc64;
  a.Dt = op->tab.Dt64;
  a.lin = op->lin64;
  a.nq = op->nq;
  a.geo = op->geo;
  a.kx = op->geo != nullptr;
  for (int d = 0; d < 3; ++d) a.s[d] = op->geom.s[d];
  return a;
}

AdjArgs adj_args(pff_op* op) {
  AdjArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int i = 0; i < op->ctx->nphase; ++i) a.phase[i] = op->ctx->phase[i];
  a.glob = op->ctx->glob;
  a.geom = op->geom;
  a.Q = op->Q;
  a.nphase = op->ctx->nphase;
  a.nq = op->nq;
  a.hist = op->hist_c;
  a.phase_id = op->phase;
  a.status = op->status;
  a.geo = op->geo;
  return a;
}

}  // namespace

extern "C" int pff_adjoint_step(pff_solver* s, const double* z, const double* hist_prev, const uint8_t* sel,
                                double wF, const double* hbar_n, double* hbar_prev, double* grad, double rtol,
                                int maxit, int* iters, void* stream) {
  if (!s || !z || !hist_prev || !sel || !hbar_prev || !grad || !iters)
    return sfail(PFF_ERR_INVALID, "pff_adjoint_step: null argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  pff_op* op = s->op;
  const long long nq = op->nq, n = s->n;
  cudaError_t e = cudaSuccess;
  if (!s->a_in) {
    if (e == cudaSuccess) e = cudaMalloc(&s->a_in, sizeof(double) * 13 * nq);
    if (e == cudaSuccess) e = cudaMalloc(&s->pbuf, sizeof(double) * 13 * nq);
    if (e == cudaSuccess) e = cudaMalloc(&s->qa, sizeof(double) * 13 * nq);
    if (e == cudaSuccess) e = cudaMalloc(&s->ag, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&s->alam, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&s->av, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&s->gth, sizeof(double) * kMaxPhase * 6);
    if (e != cudaSuccess) return sfail(PFF_ERR_CUDA, std::string("pff_adjoint_step: ") + cudaGetErrorString(e));
  }
  // 1. linearisation at (z_n, h_{n-1}): recomputed from the checkpoint
  S_CK(cudaMemcpyAsync(op->hist_c, hist_prev, sizeof(double) * 15 * nq, cudaMemcpyDeviceToDevice, st));
  S_RC(pff_residual(op, z, s->r, st));
  int status = 0;
  S_RC(pff_get_status(op, stream, &status));
  if (status) return sfail(PFF_ERR_DEVICE, "pff_adjoint_step: residual kernel status " + std::to_string(status));
  S_RC(setup(s, st));
  // point inputs a(q)
  ElemArgs<double> ea = fine_args(op);
  ea.x = z;
  ea.scratch = s->a_in;
  S_CK(elem_launch<double>(op->Q, op->p + 1, kEval, ea, st));
  // 2. right-hand side g = wF J_int^T sel + B^T [(dPhi/da)^T hbar_n], zero on Dirichlet DoFs
  S_CK(cudaMemsetAsync(s->ag, 0, sizeof(double) * n, st));
  if (hbar_n) {
    AdjArgs aa = adj_args(op);
    aa.mode = 0;
    aa.a_in = s->a_in;
    aa.hbar = hbar_n;
    aa.qa_out = s->qa;
    S_CK(launch_adjoint_point(aa, st));
    ElemArgs<double> eb = fine_args(op);
    eb.y = s->ag;
    eb.scratch = s->qa;
    S_CK(elem_launch<double>(op->Q, op->p + 1, kBack, eb, st));
  }
  S_CK(launch_sel_scale(s->av, sel, wF, n, st));
  {
    ElemArgs<double> et = fine_args(op);
    const long long stride = (long long)op->Q * op->Q * op->Q * elems_per_block(op->Q);
    et.x = s->av;
    et.y = s->ag;
    et.linP = op->lin64 + kWC * stride;
    et.linC = op->lin64 + kWP * stride;
    et.transpose = 1;
    S_CK(elem_launch<double>(op->Q, op->p + 1, kApply, et, st));
  }
  S_CK(launch_zero_masked(s->ag, op->mask, n, st));
  // 3. adjoint solve J_n^T lam = g (Dirichlet rows/columns identity, g = 0 there)
  s->transpose = 1;
  double rel = 0.0;
  int rc = fgmres(s, s->ag, s->alam, rtol, maxit, iters, &rel, st);
  s->transpose = 0;
  if (rc) return rc;
  // 4. pull-back p = interpolation of (wF sel - lam) to the Gauss points
  S_CK(launch_axpby<double>(s->av, s->alam, -1.0, 1.0, n, st));
  ElemArgs<double> ep = fine_args(op);
  ep.x = s->av;
  ep.scratch = s->pbuf;
  S_CK(elem_launch<double>(op->Q, op->p + 1, kEval, ep, st));
  // 5. history adjoint of the previous step and parameter gradient
  S_CK(cudaMemsetAsync(s->gth, 0, sizeof(double) * kMaxPhase * 6, st));
  AdjArgs ab = adj_args(op);
  ab.mode = 1;
  ab.a_in = s->a_in;
  ab.p = s->pbuf;
  ab.hbar = hbar_n;
  ab.hbar_out = hbar_prev;
  ab.gtheta = s->gth;
  S_CK(launch_adjoint_point(ab, st));
  std::vector<double> h(kMaxPhase * 6);
  S_CK(cudaMemcpyAsync(h.data(), s->gth, sizeof(double) * kMaxPhase * 6, cudaMemcpyDeviceToHost, st));
  S_CK(cudaStreamSynchronize(st));
  for (int i = 0; i < op->ctx->nphase * 6; ++i) grad[i] += h[i];
  S_RC(pff_get_status(op, stream, &status));
  if (status) return sfail(PFF_ERR_DEVICE, "pff_adjoint_step: adjoint kernel status " + std::to_string(status));
  return PFF_OK;
}
