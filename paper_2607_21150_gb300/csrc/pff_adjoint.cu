// Adjoint of the pointwise update: directional derivatives of the residual
// integrands f and of the trial history Phi (Box 1 step 4) with respect to the
// point inputs a = (grad_X u, phi, grad_X phi), the committed history h and the
// point's own phase parameters (E_inf, nu_inf, sigma0, eta_d, Gc, l0), each
// contracted with the adjoint weights of the load-step recursion.
//
// The paper linearises only in (u, phi) (Appendix B/C).  The derivatives here
// extend the same principal-frame construction: for a perturbation db of the
// trial b of a branch (db = ell b + b ell^T + F dC F^T, ell = dF F^-1), the
// eigenvalue terms follow Box A1 and the eigenvector terms the divided
// differences (t_i - t_j)/(b_i - b_j) = mu a log1p(x)/(x b_j) for the stress
// and (g_i - g_j)/(b_i - b_j) = g_j/b_j expm1(a log1p(x))/x for the committed
// b^e = N diag(g) N^T, g_i = exp(2 (a eps_d,i + theta/3)) = K b_i^a; both stay
// smooth where eigenvalues coincide.
#include <cmath>

#include "pff_internal.h"
#include "pff_point.cuh"

namespace pff {

namespace {

struct Branch {
  bool has, plastic;
  double mu, af, s2, q, c;  // c: Maxwell mu dt / eta_d
  double dgam, H, esig0;    // Prandtl: plastic increment, slope of sigma_y, d sigma_y / d sigma0 at ep_n + dgam
  double N[3][3], x[3], b[3], ed[3], ghat[3];
  double rho[3], gam[3];    // pairs (0,1), (0,2), (1,2)
  double Be[3][3];          // N diag(ghat) N^T
};

__device__ __forceinline__ int pair_of(int p, int q) { return (p + q) - 1 + (p == 0 && q == 0); }

// (b_p^a - b_q^a) / (b_p - b_q) * K with K b_q^a = ghat_q, from x = b - 1.
__device__ double power_ratio(double a, double xp, double xq, double gq) {
  const double bq = 1.0 + xq;
  const double y = (xp - xq) / bq;
  double r;
  if (fabs(y) < 1e-4) r = a * (1.0 + 0.5 * (a - 1.0) * y * (1.0 + (a - 2.0) * y / 3.0));
  else r = expm1(a * log1p(y)) / y;
  return gq / bq * r;
}

}  // namespace

__global__ void __launch_bounds__(128) k_adjoint_point(const AdjArgs a) {
  __shared__ double red[kMaxPhase * 6];
  if (a.mode == 1) {
    for (int i = threadIdx.x; i < kMaxPhase * 6; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
  }
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool live = q < a.nq;
  if (live) {
    const long long nq = a.nq;
    const int Q = a.Q, Q2 = Q * Q, Q3 = Q2 * Q;
    const int lq = (int)(q % Q3);
    const int qi = lq % Q, qj = (lq / Q) % Q, qk = lq / Q2;
    const double wdet = a.geo ? a.geo[9 * nq + q] : a.geom.wq[qi] * a.geom.wq[qj] * a.geom.wq[qk] * a.geom.detJ;
    double hvs[9];  // mapped mesh, mode 0: reference-frame components, transformed after the loop
    int pid = a.phase_id[q];
    int status = 0;
    if (pid >= a.nphase) { status |= 8; pid = 0; }
    const PhaseDev ph = a.phase[pid];
    const GlobDev gl = a.glob;

    // ---------------- primal
    double Hm[3][3], F[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        Hm[r][c] = a.a_in[(3 * r + c) * nq + q];
        F[r][c] = Hm[r][c] + (r == c ? 1.0 : 0.0);
      }
    const double phi = a.a_in[9 * nq + q];
    const double gphi[3] = {a.a_in[10 * nq + q], a.a_in[11 * nq + q], a.a_in[12 * nq + q]};
    const double trH = Hm[0][0] + Hm[1][1] + Hm[2][2];
    double trHH = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) trHH += Hm[r][c] * Hm[c][r];
    const double detH = Hm[0][0] * (Hm[1][1] * Hm[2][2] - Hm[1][2] * Hm[2][1]) -
                        Hm[0][1] * (Hm[1][0] * Hm[2][2] - Hm[1][2] * Hm[2][0]) +
                        Hm[0][2] * (Hm[1][0] * Hm[2][1] - Hm[1][1] * Hm[2][0]);
    const double Jm1 = trH + 0.5 * (trH * trH - trHH) + detH;
    if (!(Jm1 > -1.0)) status |= 2;
    const double theta = log1p(Jm1);
    const double J = 1.0 + Jm1;
    double Fi[3][3];
    Fi[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) / J;
    Fi[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) / J;
    Fi[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) / J;
    Fi[1][0] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) / J;
    Fi[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) / J;
    Fi[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) / J;
    Fi[2][0] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) / J;
    Fi[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) / J;
    Fi[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) / J;
    double GG[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double s = Hm[r][c] + Hm[c][r];
        for (int k = 0; k < 3; ++k) s += Hm[r][k] * Hm[c][k];
        GG[r][c] = s;
      }
    const double omp = 1.0 - phi;
    const double g = omp * omp + gl.eta;
    const double gp = -2.0 * omp;
    double hist[15];
    for (int v = 0; v < 15; ++v) hist[v] = a.hist[v * nq + q];

    Branch Bs[3];
    double taud[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double psid = 0.0;
    for (int br = 0; br < 3; ++br) {
      Branch& B = Bs[br];
      B.has = ph.has[br] != 0;
      B.plastic = false;
      if (!B.has) continue;
      B.mu = ph.mu[br];
      double X[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) X[r][c] = GG[r][c];
      if (br > 0) {
        const int off = (br == 1) ? 0 : 6;
        double M[3][3];
        for (int v = 0; v < 6; ++v) {
          int r, c;
          vo_idx(v, r, c);
          const double m = hist[off + v] - (v < 3 ? 1.0 : 0.0);
          M[r][c] = m; M[c][r] = m;
        }
        for (int r = 0; r < 3; ++r)
          for (int c = r; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k)
              for (int l = 0; l < 3; ++l) s += F[r][k] * M[k][l] * F[c][l];
            X[r][c] += s;
            if (c != r) X[c][r] += s;
          }
      }
      if (!jacobi3(X, B.N, B.x)) status |= 1;
      double eps[3];
      for (int p = 0; p < 3; ++p) {
        B.b[p] = 1.0 + B.x[p];
        eps[p] = 0.5 * log1p(B.x[p]);
      }
      const double tr = eps[0] + eps[1] + eps[2];
      for (int p = 0; p < 3; ++p) B.ed[p] = eps[p] - tr / 3.0;
      B.s2 = B.ed[0] * B.ed[0] + B.ed[1] * B.ed[1] + B.ed[2] * B.ed[2];
      B.af = 1.0;
      B.c = 0.0;
      B.q = 0.0;
      if (br == 1) {
        B.c = ph.cmax;
        B.af = 1.0 / (1.0 + B.c * g);
      } else if (br == 2) {
        B.q = 2.0 * B.mu * sqrt(1.5 * B.s2);
        if (g * B.q - yield_stress(ph, hist[12]) > 0.0) {
          int ok;
          B.dgam = return_map(ph, g, B.mu, B.q, hist[12], &ok);
          if (!ok) status |= 16;
          B.H = yield_slope(ph, hist[12] + B.dgam);
          B.esig0 = ph.hard ? exp(-ph.beta * (hist[12] + B.dgam)) : 1.0;
          B.af = 1.0 - 3.0 * B.mu * B.dgam / B.q;
          B.plastic = true;
        }
      }
      B.rho[0] = log_ratio(B.x[0], B.x[1]);
      B.rho[1] = log_ratio(B.x[0], B.x[2]);
      B.rho[2] = log_ratio(B.x[1], B.x[2]);
      for (int p = 0; p < 3; ++p) B.ghat[p] = exp(2.0 * (B.af * B.ed[p] + theta / 3.0));
      B.gam[0] = power_ratio(B.af, B.x[0], B.x[1], B.ghat[1]);
      B.gam[1] = power_ratio(B.af, B.x[0], B.x[2], B.ghat[2]);
      B.gam[2] = power_ratio(B.af, B.x[1], B.x[2], B.ghat[2]);
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          B.Be[r][c] = B.N[r][0] * B.ghat[0] * B.N[c][0] + B.N[r][1] * B.ghat[1] * B.N[c][1] +
                       B.N[r][2] * B.ghat[2] * B.N[c][2];
          taud[r][c] += 2.0 * B.mu * B.af *
                        (B.N[r][0] * B.ed[0] * B.N[c][0] + B.N[r][1] * B.ed[1] * B.N[c][1] + B.N[r][2] * B.ed[2] * B.N[c][2]);
        }
      psid += B.mu * B.af * B.af * B.s2;
    }
    const double tv = ph.kap_tot * theta;
    const double psiv = 0.5 * ph.kap_tot * theta * theta;
    const bool tens = theta >= 0.0;
    double tdeg[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        tdeg[r][c] = tens ? g * (taud[r][c] + (r == c ? tv : 0.0)) : g * taud[r][c] + (r == c ? tv : 0.0);
    const double psip = tens ? psid + psiv : psid;
    const bool active = psip > hist[13];
    const double Hh = active ? psip : hist[13];
    const double alphap = (gl.at == 1) ? 1.0 : 2.0 * phi;

    // ---------------- directional derivative of (f, Phi)
    // dirs: mode 0 -> 0..9 (grad u components, phi); mode 1 -> 15 history words, 6 parameters
    const int ndir = (a.mode == 0) ? 10 : 21;
    double hb[15];
    for (int v = 0; v < 15; ++v) hb[v] = a.hbar ? a.hbar[v * nq + q] : 0.0;
    double pw[13];
    if (a.mode == 1)
      for (int m = 0; m < 13; ++m) pw[m] = wdet * a.p[m * nq + q];
    for (int d = 0; d < ndir; ++d) {
      double dF[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      double dphi = 0.0, dh[15], dpar[6] = {0, 0, 0, 0, 0, 0};
      for (int v = 0; v < 15; ++v) dh[v] = 0.0;
      if (a.mode == 0) {
        if (d < 9) dF[d / 3][d % 3] = 1.0;
        else dphi = 1.0;
      } else {
        if (d < 15) dh[d] = 1.0;
        else dpar[d - 15] = 1.0;
      }
      // kinematics
      double ell[3][3], dFi[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) ell[r][c] = dF[r][0] * Fi[0][c] + dF[r][1] * Fi[1][c] + dF[r][2] * Fi[2][c];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) dFi[r][c] = -(Fi[r][0] * ell[0][c] + Fi[r][1] * ell[1][c] + Fi[r][2] * ell[2][c]);
      const double dth = ell[0][0] + ell[1][1] + ell[2][2];
      const double dg = gp * dphi, dgp = 2.0 * dphi;
      const double onu = 1.0 + ph.nu0, tnu = 1.0 - 2.0 * ph.nu0;
      const double dmu0 = dpar[0] / (2.0 * onu) - ph.E0 * dpar[1] / (2.0 * onu * onu);
      const double dkap0 = dpar[0] / (3.0 * tnu) + 2.0 * ph.E0 * dpar[1] / (3.0 * tnu * tnu);
      double dtaud[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      double dpsid = 0.0, dgam = 0.0;
      double dPhi[15];
      for (int v = 0; v < 15; ++v) dPhi[v] = dh[v];  // pass-through for absent branches
      for (int br = 0; br < 3; ++br) {
        const Branch& B = Bs[br];
        if (!B.has) continue;
        const int off = (br == 1) ? 0 : 6;
        // db in the eigenframe: ell_hat b + b ell_hat^T + N^T F dC F^T N
        double lh[3][3];
        for (int p = 0; p < 3; ++p)
          for (int r = 0; r < 3; ++r) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i)
              for (int j = 0; j < 3; ++j) s += B.N[i][p] * ell[i][j] * B.N[j][r];
            lh[p][r] = s;
          }
        double dbh[3][3];
        for (int p = 0; p < 3; ++p)
          for (int r = 0; r < 3; ++r) dbh[p][r] = lh[p][r] * B.b[r] + B.b[p] * lh[r][p];
        if (br > 0) {
          bool any = false;
          for (int v = 0; v < 6; ++v) any = any || dh[off + v] != 0.0;
          if (any) {
            double dC[3][3], W[3][3];
            for (int v = 0; v < 6; ++v) {
              int r, c;
              vo_idx(v, r, c);
              dC[r][c] = dh[off + v]; dC[c][r] = dh[off + v];
            }
            for (int r = 0; r < 3; ++r)  // W = F^T N
              for (int p = 0; p < 3; ++p) W[r][p] = F[0][r] * B.N[0][p] + F[1][r] * B.N[1][p] + F[2][r] * B.N[2][p];
            for (int p = 0; p < 3; ++p)
              for (int r = 0; r < 3; ++r) {
                double s = 0.0;
                for (int i = 0; i < 3; ++i)
                  for (int j = 0; j < 3; ++j) s += W[i][p] * dC[i][j] * W[j][r];
                dbh[p][r] += s;
              }
          }
        }
        double deps[3], dtr = 0.0, edde = 0.0;
        for (int p = 0; p < 3; ++p) {
          deps[p] = dbh[p][p] / (2.0 * B.b[p]);
          dtr += deps[p];
          edde += B.ed[p] * deps[p];
        }
        double ded[3];
        for (int p = 0; p < 3; ++p) ded[p] = deps[p] - dtr / 3.0;
        const double ds2 = 2.0 * edde;
        const double dmu = (br == 0) ? dmu0 : 0.0;
        double da = 0.0, dq = 0.0, ddgam = 0.0;
        if (br == 1) {
          if (B.c != 0.0) {
            const double dc = -B.c * dpar[3] / ph.eta_d;
            da = -B.af * B.af * (dc * g + B.c * dg);
          }
        } else if (br == 2 && B.plastic) {
          // implicit derivative of the degraded consistency condition
          // g q - 3 g mu dgam - sigma_y(ep_n + dgam; sigma0) = 0
          dq = B.q * edde / B.s2;
          ddgam = (g * dq + (B.q - 3.0 * B.mu * B.dgam) * dg - B.esig0 * dpar[2] - B.H * dh[12]) /
                  (3.0 * g * B.mu + B.H);
          da = -3.0 * B.mu * ddgam / B.q + 3.0 * B.mu * B.dgam * dq / (B.q * B.q);
        }
        double dth_[3][3];
        for (int p = 0; p < 3; ++p) dth_[p][p] = 2.0 * (dmu * B.af * B.ed[p] + B.mu * da * B.ed[p] + B.mu * B.af * ded[p]);
        for (int p = 0; p < 3; ++p)
          for (int r = p + 1; r < 3; ++r) {
            const double v = B.mu * B.af * B.rho[pair_of(p, r)] * dbh[p][r];
            dth_[p][r] = v; dth_[r][p] = v;
          }
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int p = 0; p < 3; ++p)
              for (int t = 0; t < 3; ++t) s += B.N[r][p] * dth_[p][t] * B.N[c][t];
            dtaud[r][c] += s;
          }
        dpsid += dmu * B.af * B.af * B.s2 + 2.0 * B.mu * B.af * da * B.s2 + B.mu * B.af * B.af * ds2;
        if (br > 0) {  // trial C_in^-1 = F^-1 N diag(ghat) N^T F^-T
          double dgh[3][3];
          for (int p = 0; p < 3; ++p) dgh[p][p] = 2.0 * B.ghat[p] * (da * B.ed[p] + B.af * ded[p] + dth / 3.0);
          for (int p = 0; p < 3; ++p)
            for (int r = p + 1; r < 3; ++r) {
              const double v = B.gam[pair_of(p, r)] * dbh[p][r];
              dgh[p][r] = v; dgh[r][p] = v;
            }
          double dBe[3][3];
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
              double s = 0.0;
              for (int p = 0; p < 3; ++p)
                for (int t = 0; t < 3; ++t) s += B.N[r][p] * dgh[p][t] * B.N[c][t];
              dBe[r][c] = s;
            }
          for (int v = 0; v < 6; ++v) {
            int r, c;
            vo_idx(v, r, c);
            double s = 0.0;
            for (int i = 0; i < 3; ++i)
              for (int j = 0; j < 3; ++j)
                s += dFi[r][i] * B.Be[i][j] * Fi[c][j] + Fi[r][i] * dBe[i][j] * Fi[c][j] + Fi[r][i] * B.Be[i][j] * dFi[c][j];
            dPhi[off + v] = s;
          }
        }
        if (br == 2 && B.plastic) dgam = ddgam;
      }
      const double dtv = dkap0 * theta + ph.kap_tot * dth;
      const double dpsiv = 0.5 * dkap0 * theta * theta + ph.kap_tot * theta * dth;
      double dtdeg[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          const double dI = (r == c) ? 1.0 : 0.0;
          if (tens) dtdeg[r][c] = dg * (taud[r][c] + dI * tv) + g * (dtaud[r][c] + dI * dtv);
          else dtdeg[r][c] = dg * taud[r][c] + g * dtaud[r][c] + dI * dtv;
        }
      const double dpsip = tens ? dpsid + dpsiv : dpsid;
      const double dH = active ? dpsip : dh[13];
      const double c0 = ph.c0;
      const double dgc = (dpar[4] / ph.l0 - ph.Gc * dpar[5] / (ph.l0 * ph.l0)) / c0;
      const double dalphap = (gl.at == 1) ? 0.0 : 2.0 * dphi;
      const double dL = dgp * Hh + gp * dH + dgc * alphap + ph.gc_c0l0 * dalphap + gl.zeta * (dphi - dh[14]) / gl.dt;
      const double dkphi = gl.s_phi * 2.0 * (dpar[4] * ph.l0 + ph.Gc * dpar[5]) / c0;
      double df[13];
      for (int r = 0; r < 3; ++r)
        for (int A = 0; A < 3; ++A) {
          double s = 0.0;
          for (int j = 0; j < 3; ++j) s += dtdeg[r][j] * Fi[A][j] + tdeg[r][j] * dFi[A][j];
          df[3 * r + A] = s;
        }
      df[9] = gl.s_phi * dL;
      for (int A = 0; A < 3; ++A) df[10 + A] = dkphi * gphi[A];
      dPhi[12] = dh[12] + dgam;
      dPhi[13] = dH;
      dPhi[14] = dphi;
      double hv = 0.0;
      for (int v = 0; v < 15; ++v) hv += hb[v] * dPhi[v];
      if (a.mode == 0) {
        // parent-frame pseudo-integrand for the transposed basis (no weight)
        if (a.geo && d < 9) {
          hvs[d] = hv;
        } else {
          const double val = (d < 9) ? hv * a.geom.s[d % 3] : hv;
          a.qa_out[d * nq + q] = val;
        }
      } else {
        double pv = 0.0;
        for (int m = 0; m < 13; ++m) pv += pw[m] * df[m];
        if (d < 15) a.hbar_out[d * nq + q] = pv + hv;
        else atomicAdd(&red[pid * 6 + (d - 15)], pv + hv);
      }
    }
    if (a.mode == 0 && a.geo)  // parent component al of field f: sum_A (d xi_al / dX_A) hv_(f, A)
      for (int f = 0; f < 3; ++f)
        for (int al = 0; al < 3; ++al)
          a.qa_out[(3 * f + al) * nq + q] = a.geo[(3 * al) * nq + q] * hvs[3 * f] +
                                            a.geo[(3 * al + 1) * nq + q] * hvs[3 * f + 1] +
                                            a.geo[(3 * al + 2) * nq + q] * hvs[3 * f + 2];
    if (a.mode == 0)
      for (int m = 10; m < 13; ++m) a.qa_out[m * nq + q] = 0.0;
    if (status) atomicOr(a.status, status);
  }
  if (a.mode == 1) {
    __syncthreads();
    for (int i = threadIdx.x; i < a.nphase * 6; i += blockDim.x)
      if (red[i] != 0.0) atomicAdd(a.gtheta + i, red[i]);
  }
}

cudaError_t launch_adjoint_point(const AdjArgs& a, cudaStream_t st) {
  if (a.nq == 0) return cudaSuccess;
  k_adjoint_point<<<(unsigned)((a.nq + 127) / 128), 128, 0, st>>>(a); note_launch();
  return cudaGetLastError();
}

}  // namespace pff
