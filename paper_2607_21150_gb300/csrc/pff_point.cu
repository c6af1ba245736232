// Pointwise Peric-Dettmer update with the series fracture element, one thread
// per quadrature point, FP64.
//
// Principal-stress format (Appendix A): every branch k spectrally decomposes
// X_k = b_k^tr - I = F (C_k - I) F^T + (F F^T - I) (Eq. inelasticity-be-update),
// takes eps_i = log1p(x_i) / 2 (the log1p form of Sec. 2.2), corrects the
// deviatoric principal strains with the branch factor a_k (Box 1 step 2 and
// Eq. principal-directions-format-1 with the degraded mu and q_tr of Sec. 3),
// and rebuilds tau_d,k = N diag(2 mu a eps_d) N^T.  The Maxwell and Prandtl
// branches are diagonalised in the Hooke branch's principal frame (their b_tr
// differ from it by the inelastic strains, so Jacobi starts nearly
// converged).  The volumetric strain
// theta = ln J is shared by all branches and decides the Amor split
// (Eqs. linear-Psi-plus, linear-degraded-stress).
//
// The consistent tangent follows Appendix B (d b = ell b + b ell^T with
// ell = dF F^-1, d eps_i = d b_i / (2 b_i), Box A1 per branch, Eq.
// hencky-stress-linearization) with the eigenvector term written as the
// divided difference (tau_i - tau_j)/(b_i - b_j) = mu a log1p(x)/(x b_j),
// x = (b_i - b_j)/b_j, which is exact at distinct eigenvalues and smooth where
// they coincide; and Appendix C for the phase-field coupling
// (Eqs. linear-degraded-stress-linearization, maxwell-dtau-dphi,
// prandtl-dtau-dphi, linearized-local-damage-residual,
// history-field-linearization, energy-displacement-linearization,
// maxwell-energy-dphi, prandtl-energy-dphi).  The reference-frame tangent
// dP = (d tau_degr - tau_degr ell^T) F^-T is evaluated for the nine unit
// directions of F together: with ell = e_a (x) F^-T e_B the principal-frame
// increment is n_a v_B^T (rows of N and of V = F^-1 N), so every Voigt
// component v of d tau is the 3x3 product (N M_v V^T)[a][B] with a small
// coefficient matrix M_v per branch; then the direction phi.  The words are
// scaled by the quadrature weight and the parent-to-reference factors (mapped
// meshes: transformed to the parent frame with d xi / dX) and stored in the
// tiled layout of kLinWords words.  The tangent's
// products and sums run in double-float on the FP32 pipes (about 2^-46
// relative per operation), converted to and from FP64 by integer operations:
// on GB300 the FP64 pipe, not memory, bounds this kernel.
#include <cmath>

#include "pff_df.cuh"
#include "pff_internal.h"
#include "pff_point.cuh"

namespace pff {

__global__ void __launch_bounds__(128) k_pointwise(const PointArgs a) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= a.nq) return;
  const int Q = a.Q, Q2 = Q * Q, Q3 = Q2 * Q;
  const long long nq = a.nq;
  const int lq = (int)(q % Q3);
  const int qi = lq % Q, qj = (lq / Q) % Q, qk = lq / Q2;
  const long long e = q / Q3;
  const bool mapped = a.geo != nullptr;
  const double wdet = mapped ? a.geo[9 * nq + q] : a.geom.wq[qi] * a.geom.wq[qj] * a.geom.wq[qk] * a.geom.detJ;
  const double* sg = a.geom.s;
  double Gx[3][3];  // mapped mesh: d xi_al / dX_A
  if (mapped)
    for (int al = 0; al < 3; ++al)
      for (int A = 0; A < 3; ++A) Gx[al][A] = a.geo[(3 * al + A) * nq + q];

  double Hm[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Hm[r][c] = a.io[(3 * r + c) * nq + q];
  const double phi = a.io[9 * nq + q];
  double gphi[3] = {a.io[10 * nq + q], a.io[11 * nq + q], a.io[12 * nq + q]};
  int status = 0;
  int pid = a.phase_id[q];
  if (pid >= a.nphase) {
    status |= 8;
    pid = 0;
  }
  const PhaseDev ph = a.phase[pid];
  const GlobDev gl = a.glob;

  // kinematics
  double F[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) F[r][c] = Hm[r][c] + (r == c ? 1.0 : 0.0);
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
  const double rJ = 1.0 / J;
  Fi[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) * rJ;
  Fi[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * rJ;
  Fi[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * rJ;
  Fi[1][0] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) * rJ;
  Fi[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * rJ;
  Fi[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * rJ;
  Fi[2][0] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) * rJ;
  Fi[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * rJ;
  Fi[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * rJ;
  double GG[3][3];  // F F^T - I
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = Hm[r][c] + Hm[c][r];
      for (int k = 0; k < 3; ++k) s += Hm[r][k] * Hm[c][k];
      GG[r][c] = s;
    }

  // degradation g = (1 - phi)^2 + eta (Eq. degr-funct)
  const double omp = 1.0 - phi;
  const double g = omp * omp + gl.eta;
  const double gp = -2.0 * omp;

  double tau6[6] = {0, 0, 0, 0, 0, 0};  // deviatoric Kirchhoff stress of all branches, Voigt order
  double psid = 0.0;
  // the tangent's products and sums run in double-float on the FP32 pipes
  // (the FP64 pipe is this kernel's bound), converted by integer operations
  df64 dtau[10][6];
  df64 dpsi[10];
  df64 Fid[3][3];
  const df64 dz = df_make(0.0f, 0.0f);
  for (int d = 0; d < 10; ++d) {
    dpsi[d] = dz;
    for (int v = 0; v < 6; ++v) dtau[d][v] = dz;
  }
  if (a.want_tangent)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Fid[r][c] = df_split(Fi[r][c]);
  uint8_t flag = 0;
  double dgam = 0.0;
  double hist_new[12];
  for (int v = 0; v < 12; ++v) hist_new[v] = a.hist[v * nq + q];

  double N0[3][3];  // principal frame of the Hooke branch (always present): warm start of the others
  for (int br = 0; br < 3; ++br) {
    if (!ph.has[br]) continue;
    const double mu = ph.mu[br];
    double X[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) X[r][c] = GG[r][c];
    if (br > 0) {
      const int off = (br == 1) ? 0 : 6;
      double M[3][3];
      for (int v = 0; v < 6; ++v) {
        int r, c;
        vo_idx(v, r, c);
        double m = a.hist[(off + v) * nq + q] - (v < 3 ? 1.0 : 0.0);
        M[r][c] = m; M[c][r] = m;
      }
      double FM[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) FM[r][c] = F[r][0] * M[0][c] + F[r][1] * M[1][c] + F[r][2] * M[2][c];
      for (int r = 0; r < 3; ++r)
        for (int c = r; c < 3; ++c) {
          double s = FM[r][0] * F[c][0] + FM[r][1] * F[c][1] + FM[r][2] * F[c][2];
          X[r][c] += s;
          if (c != r) X[c][r] += s;
        }
    }
    double N[3][3], x[3];
    if (br == 0) {
      if (!jacobi3(X, N, x)) status |= 1;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) N0[r][c] = N[r][c];
    } else {
      // the inelastic branches' b_tr differ from the elastic one by the
      // (small) inelastic strains, so in the Hooke frame X is nearly
      // diagonal: Jacobi on N0^T X N0 needs fewer sweeps, N = N0 N~
      double T1[3][3], Xt[3][3], Nt[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) T1[r][c] = X[r][0] * N0[0][c] + X[r][1] * N0[1][c] + X[r][2] * N0[2][c];
      for (int r = 0; r < 3; ++r)
        for (int c = r; c < 3; ++c) {
          const double v = N0[0][r] * T1[0][c] + N0[1][r] * T1[1][c] + N0[2][r] * T1[2][c];
          Xt[r][c] = v;
          Xt[c][r] = v;
        }
      if (!jacobi3(Xt, Nt, x)) status |= 1;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) N[r][c] = N0[r][0] * Nt[0][c] + N0[r][1] * Nt[1][c] + N0[r][2] * Nt[2][c];
    }
    double eps[3], ed[3];
    for (int p = 0; p < 3; ++p) eps[p] = 0.5 * log1p(x[p]);
    const double tr = eps[0] + eps[1] + eps[2];
    for (int p = 0; p < 3; ++p) ed[p] = eps[p] - tr * (1.0 / 3.0);
    const double s2 = ed[0] * ed[0] + ed[1] * ed[1] + ed[2] * ed[2];
    double af = 1.0, da_dphi = 0.0, cq = 0.0;
    bool plastic = false;
    if (br == 1) {
      af = 1.0 / (1.0 + ph.cmax * g);
      da_dphi = -af * af * ph.cmax * gp;
    } else if (br == 2) {
      // Box 2, degraded: admissible iff g q_tr <= sigma_y(ep_n); else the local Newton
      const double qtr = 2.0 * mu * sqrt(1.5 * s2);
      const double epn = a.hist[12 * nq + q];
      if (g * qtr - yield_stress(ph, epn) > 0.0) {
        int ok;
        dgam = return_map(ph, g, mu, qtr, epn, &ok);
        if (!ok) status |= 16;
        const double Hs = yield_slope(ph, epn + dgam);
        af = 1.0 - 3.0 * mu * dgam / qtr;
        // implicit derivatives of dgam: d a = cq dq / q + da_dphi dphi
        // (Eq. plasticity-dtau-vonMises with the degraded consistency condition)
        const double den = 1.0 / (3.0 * g * mu + Hs);
        cq = (1.0 - af) - 3.0 * g * mu * den;
        da_dphi = -3.0 * mu * af * gp * den;
        plastic = true;
        flag |= 1;
      }
    }
    // tau_d += N diag(ti) N^T: the six entries of the symmetric sum (Voigt order)
    const double tma = 2.0 * mu * af;
    double Nt[3][3];  // N diag(ti), ti = 2 mu a ed
    for (int r = 0; r < 3; ++r)
      for (int p = 0; p < 3; ++p) Nt[r][p] = N[r][p] * (tma * ed[p]);
    for (int v = 0; v < 6; ++v) {
      int r, c;
      vo_idx(v, r, c);
      tau6[v] += Nt[r][0] * N[c][0] + Nt[r][1] * N[c][1] + Nt[r][2] * N[c][2];
    }
    psid += mu * af * af * s2;

    if (br > 0) {  // trial history: C = F^-1 N diag(exp(2 eps_e)) N^T F^-T
      double ee[3];
      for (int p = 0; p < 3; ++p) ee[p] = exp(2.0 * (af * ed[p] + theta / 3.0));
      double W[3][3];  // F^-1 N
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) W[r][c] = Fi[r][0] * N[0][c] + Fi[r][1] * N[1][c] + Fi[r][2] * N[2][c];
      const int off = (br == 1) ? 0 : 6;
      double We[3][3];  // W diag(ee)
      for (int r = 0; r < 3; ++r)
        for (int p = 0; p < 3; ++p) We[r][p] = W[r][p] * ee[p];
      for (int v = 0; v < 6; ++v) {
        int r, c;
        vo_idx(v, r, c);
        hist_new[off + v] = We[r][0] * W[c][0] + We[r][1] * W[c][1] + We[r][2] * W[c][2];
      }
    }

    if (a.want_tangent) {
      df64 Nd[3][3], Vd[3][3];  // N and V = F^-1 N: ell_hat for ell = e_a (x) F^-T e_B is N[a][p] V[B][q]
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Nd[r][c] = df_split(N[r][c]);
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
          Vd[r][c] = df_madd(df_madd(df_mul(Fid[r][0], Nd[0][c]), Fid[r][1], Nd[1][c]), Fid[r][2], Nd[2][c]);
      const df64 rho01 = log_ratio_df(x[0], x[1]);
      const df64 rho02 = log_ratio_df(x[0], x[2]);
      const df64 rho12 = log_ratio_df(x[1], x[2]);
      const df64 one = df_make(1.0f, 0.0f);
      df64 bd[3], edd[3];
      for (int p = 0; p < 3; ++p) {
        bd[p] = df_add(one, df_split(x[p]));
        edd[p] = df_split(ed[p]);
      }
      // symmetric basis of the principal frame in Voigt order: N dh N^T =
      // sum_p dh_pp n_p n_p^T + sum_{p<t} dh_pt (n_p n_t^T + n_t n_p^T)
      df64 E[6][6];
      for (int v = 0; v < 6; ++v) {
        int r, c;
        vo_idx(v, r, c);
        E[0][v] = df_mul(Nd[r][0], Nd[c][0]);
        E[1][v] = df_mul(Nd[r][1], Nd[c][1]);
        E[2][v] = df_mul(Nd[r][2], Nd[c][2]);
        E[3][v] = df_madd(df_mul(Nd[r][1], Nd[c][2]), Nd[r][2], Nd[c][1]);
        E[4][v] = df_madd(df_mul(Nd[r][0], Nd[c][2]), Nd[r][2], Nd[c][0]);
        E[5][v] = df_madd(df_mul(Nd[r][0], Nd[c][1]), Nd[r][1], Nd[c][0]);
      }
      const df64 mud = df_split(mu), afd = df_split(af);
      const df64 mua = df_mul(mud, afd);
      const df64 k01 = df_mul(mua, rho01), k02 = df_mul(mua, rho02), k12 = df_mul(mua, rho12);
      // off-diagonal coefficients of M_v per unit E entry
      const df64 c12 = df_mul(k12, bd[2]), c21 = df_mul(k12, bd[1]), c02 = df_mul(k02, bd[2]),
                 c20 = df_mul(k02, bd[0]), c01 = df_mul(k01, bd[1]), c10 = df_mul(k01, bd[0]);
      const double cq_s2 = plastic ? cq / s2 : 0.0;  // d a / d(eps_d . d eps_d) = cq / s2 (dq / q = edde / s2)
      // The nine F-directions ell = e_a (x) F^-T e_B have ell_hat = n_a v_B^T
      // (rows of N and V), and every term of the branch tangent is bilinear in
      // (n_a, v_B): dtau_v(a, B) = (N M_v V^T)[a][B] with the 3x3 coefficient
      // matrices M_v of the principal-frame map ell_hat -> dh (Box A1, the
      // divided differences off the diagonal), and dpsi(a, B) = c (N diag(ed) V^T)[a][B].
      //   dh_q (diagonal) = sum_p ell_pp [2 mu a (delta_qp - 1/3) + 2 mu cq_s2 ed_q ed_p]
      //   dh_12 = k12 (b_2 ell_12 + b_1 ell_21), dh_02, dh_01 alike.
      const df64 two_mua = df_add(mua, mua);
      const df64 c2 = df_mul(df_add(mud, mud), df_split(cq_s2));
      const df64 third = df_split(1.0 / 3.0);
      df64 cdiag[3][3];  // cdiag[q][p]: coefficient of ell_pp in dh_q
      for (int qq = 0; qq < 3; ++qq)
        for (int p = 0; p < 3; ++p) {
          const df64 dq = qq == p ? df_sub(one, third) : df_neg(third);
          cdiag[qq][p] = df_madd(df_mul(two_mua, dq), df_mul(c2, edd[qq]), edd[p]);
        }
      const df64 cphi = df_mul(df_add(mud, mud), df_split(da_dphi));  // phi direction: dh_q = 2 mu da_dphi ed_q
#pragma unroll 1
      for (int v = 0; v < 6; ++v) {
        df64 M[3][3];
        for (int p = 0; p < 3; ++p)
          M[p][p] = df_madd(df_madd(df_mul(cdiag[0][p], E[0][v]), cdiag[1][p], E[1][v]), cdiag[2][p], E[2][v]);
        M[1][2] = df_mul(c12, E[3][v]);
        M[2][1] = df_mul(c21, E[3][v]);
        M[0][2] = df_mul(c02, E[4][v]);
        M[2][0] = df_mul(c20, E[4][v]);
        M[0][1] = df_mul(c01, E[5][v]);
        M[1][0] = df_mul(c10, E[5][v]);
        df64 T[3][3];  // N M
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c)
            T[r][c] = df_madd(df_madd(df_mul(Nd[r][0], M[0][c]), Nd[r][1], M[1][c]), Nd[r][2], M[2][c]);
        for (int aa = 0; aa < 3; ++aa)
          for (int BB = 0; BB < 3; ++BB) {
            df64 acc = dtau[3 * aa + BB][v];
            acc = df_madd(acc, T[aa][0], Vd[BB][0]);
            acc = df_madd(acc, T[aa][1], Vd[BB][1]);
            dtau[3 * aa + BB][v] = df_madd(acc, T[aa][2], Vd[BB][2]);
          }
        const df64 edE = df_madd(df_madd(df_mul(edd[0], E[0][v]), edd[1], E[1][v]), edd[2], E[2][v]);
        dtau[9][v] = df_madd(dtau[9][v], cphi, edE);
      }
      // energy: dpsi = 2 mu a^2 edde + 2 mu a s2 da = 2 mu a (a + cq) edde in the F-directions
      const df64 cpsi = df_mul(two_mua, df_add(afd, df_split(plastic ? cq : 0.0)));
      df64 Ne[3][3];  // N diag(ed)
      for (int r = 0; r < 3; ++r)
        for (int p = 0; p < 3; ++p) Ne[r][p] = df_mul(Nd[r][p], edd[p]);
      for (int aa = 0; aa < 3; ++aa)
        for (int BB = 0; BB < 3; ++BB) {
          const df64 t = df_madd(df_madd(df_mul(Ne[aa][0], Vd[BB][0]), Ne[aa][1], Vd[BB][1]), Ne[aa][2], Vd[BB][2]);
          dpsi[3 * aa + BB] = df_madd(dpsi[3 * aa + BB], cpsi, t);
        }
      dpsi[9] = df_madd(dpsi[9], df_mul(two_mua, df_split(s2)), df_split(da_dphi));
    }
  }

  double taud[3][3];
  for (int v = 0; v < 6; ++v) {
    int r, c;
    vo_idx(v, r, c);
    taud[r][c] = tau6[v];
    taud[c][r] = tau6[v];
  }

  // volumetric part and the Amor split
  const double tv = ph.kap_tot * theta;
  const double psiv = 0.5 * ph.kap_tot * theta * theta;
  const bool tens = theta >= 0.0;
  double tdeg[3][3];
  double psip;
  if (tens) {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) tdeg[r][c] = g * (taud[r][c] + (r == c ? tv : 0.0));
    psip = psid + psiv;
    flag |= 4;
  } else {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) tdeg[r][c] = g * taud[r][c] + (r == c ? tv : 0.0);
    psip = psid;
  }
  const double Hn = a.hist[13 * nq + q];
  const bool active = psip > Hn;
  if (active) flag |= 2;
  const double Hh = active ? psip : Hn;
  const double alphap = (gl.at == 1) ? 1.0 : 2.0 * phi;
  const double phin = a.hist[14 * nq + q];
  const double L = gp * Hh + ph.gc_c0l0 * alphap + gl.zeta * (phi - phin) / gl.dt;

  // residual integrands, parent frame with the weight folded in
  double Pm[3][3];
  for (int r = 0; r < 3; ++r)
    for (int A = 0; A < 3; ++A) Pm[r][A] = tdeg[r][0] * Fi[A][0] + tdeg[r][1] * Fi[A][1] + tdeg[r][2] * Fi[A][2];
  double outv[13];
  if (mapped) {
    for (int r = 0; r < 3; ++r)
      for (int al = 0; al < 3; ++al)
        outv[3 * r + al] = wdet * (Gx[al][0] * Pm[r][0] + Gx[al][1] * Pm[r][1] + Gx[al][2] * Pm[r][2]);
    for (int al = 0; al < 3; ++al)
      outv[10 + al] = wdet * ph.kphi * (Gx[al][0] * gphi[0] + Gx[al][1] * gphi[1] + Gx[al][2] * gphi[2]);
  } else {
    for (int r = 0; r < 3; ++r)
      for (int A = 0; A < 3; ++A) outv[3 * r + A] = wdet * sg[A] * Pm[r][A];
    for (int A = 0; A < 3; ++A) outv[10 + A] = wdet * sg[A] * ph.kphi * gphi[A];
  }
  outv[9] = wdet * gl.s_phi * L;
  for (int v = 0; v < 13; ++v) {
    if (!isfinite(outv[v])) status |= 4;
    a.io[v * nq + q] = outv[v];
  }

  // trial history and flags
  for (int v = 0; v < 12; ++v) a.hist_trial[v * nq + q] = hist_new[v];
  a.hist_trial[12 * nq + q] = a.hist[12 * nq + q] + dgam;
  a.hist_trial[13 * nq + q] = Hh;
  a.hist_trial[14 * nq + q] = phi;
  a.flags[q] = flag;

  if (a.want_tangent) {
    const int EB = elems_per_block(Q);
    const long long stride = (long long)Q3 * EB;
    const long long blk = e / EB;
    const int el = (int)(e % EB);
    double* lin = a.lin + blk * (long long)kLinWords * stride + (long long)qk * Q2 * EB + el * Q2 + qj * Q + qi;
    const double app = (gl.at == 1) ? 0.0 : 2.0;
    const double cL = 2.0 * Hh + ph.gc_c0l0 * app + gl.zeta / gl.dt;
    // mapped mesh: reference-frame columns kept, transformed to the parent frame below
    double Dm[9][9], Pv[9], Lv[9], Lphi = 0.0;
    // double-float copies of the point's scalars and matrices
    const df64 gd = df_split(g), gpd = df_split(gp), tvd = df_split(tv), kapd = df_split(ph.kap_tot);
    const df64 kth = df_mul(kapd, df_split(theta)), cLd = df_split(cL);
    df64 taudd[6];
    for (int v = 0; v < 6; ++v) {
      int r, c;
      vo_idx(v, r, c);
      taudd[v] = df_split(taud[r][c]);
    }
    df64 TF[3][3];  // tau_degr F^-T: the geometric term of direction (aa, BB) is column BB, placed in column aa
    {
      df64 td[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) td[r][c] = df_split(tdeg[r][c]);
      for (int r = 0; r < 3; ++r)
        for (int B = 0; B < 3; ++B)
          TF[r][B] = df_madd(df_madd(df_mul(td[r][0], Fid[B][0]), td[r][1], Fid[B][1]), td[r][2], Fid[B][2]);
    }
    // scale of the stored words: w det J, d xi / dX per direction, s_phi
    df64 wsc[3], wsc2[3][3];
    const df64 wd = df_split(wdet), sphi = df_split(gl.s_phi);
    for (int A = 0; A < 3; ++A) wsc[A] = df_mul(wd, df_split(sg[A]));
    for (int A = 0; A < 3; ++A)
      for (int B = 0; B < 3; ++B) wsc2[A][B] = df_mul(wsc[A], df_split(sg[B]));
    for (int d = 0; d < 10; ++d) {
      const bool dphi = d == 9;
      const int aa = (d < 9) ? d / 3 : 0, BB = (d < 9) ? d % 3 : 0;
      const df64 trl = (d < 9) ? Fid[BB][aa] : df_make(0.0f, 0.0f);
      const df64 dtv = df_mul(kapd, trl);
      df64 M[3][3];
      for (int v = 0; v < 6; ++v) {
        int r, c;
        vo_idx(v, r, c);
        df64 val = df_mul(gd, dtau[d][v]);
        if (dphi) val = df_madd(val, gpd, taudd[v]);
        if (r == c) {
          if (tens) {
            val = df_madd(val, gd, dtv);
            if (dphi) val = df_madd(val, gpd, tvd);
          } else {
            val = df_add(val, dtv);
          }
        }
        M[r][c] = val; M[c][r] = val;
      }
      const df64 dpsip = tens ? df_madd(dpsi[d], kth, trl) : dpsi[d];
      if (d < 9)  // geometric term: - tau_degr ell^T, (tau ell^T)_{i aa} = (tau F^-T e_BB)_i
        for (int r = 0; r < 3; ++r) M[r][aa] = df_sub(M[r][aa], TF[r][BB]);
      df64 dP[3][3];
      for (int r = 0; r < 3; ++r)
        for (int A = 0; A < 3; ++A)
          dP[r][A] = df_madd(df_madd(df_mul(M[r][0], Fid[A][0]), M[r][1], Fid[A][1]), M[r][2], Fid[A][2]);
      df64 dL = active ? df_mul(gpd, dpsip) : df_make(0.0f, 0.0f);
      if (dphi) dL = df_add(dL, cLd);
      if (mapped) {
        if (d < 9) {
          for (int m = 0; m < 9; ++m) Dm[m][d] = df_join(dP[m / 3][m % 3]);
          Lv[d] = df_join(dL);
        } else {
          for (int m = 0; m < 9; ++m) Pv[m] = df_join(dP[m / 3][m % 3]);
          Lphi = df_join(dL);
        }
      } else if (d < 9) {
        const int n = 3 * aa + BB;
        for (int m = 0; m <= n; ++m) {
          const int r = m / 3, A = m % 3;
          lin[(long long)(kWA + sym9(m, n)) * stride] = df_join(df_mul(wsc2[A][BB], dP[r][A]));
        }
        lin[(long long)(kWC + n) * stride] = df_join(df_mul(df_mul(wsc[BB], sphi), dL));
      } else {
        for (int m = 0; m < 9; ++m) lin[(long long)(kWP + m) * stride] = df_join(df_mul(wsc[m % 3], dP[m / 3][m % 3]));
        lin[(long long)kWD * stride] = df_join(df_mul(df_mul(wd, sphi), dL));
      }
    }
    if (!mapped) {
      for (int A = 0; A < 3; ++A) lin[(long long)(kWK + A) * stride] = wdet * sg[A] * sg[A] * ph.kphi;
      for (int pr = 0; pr < 3; ++pr) lin[(long long)(kWKX + pr) * stride] = 0.0;
    } else {
      // parent frame: A_hat[(r, al), (c, be)] = w det J sum_{A,B} G[al][A] D[(r, A), (c, B)] G[be][B]
      double T[9][9];
      for (int m = 0; m < 9; ++m)
        for (int c = 0; c < 3; ++c)
          for (int be = 0; be < 3; ++be)
            T[m][3 * c + be] = Dm[m][3 * c] * Gx[be][0] + Dm[m][3 * c + 1] * Gx[be][1] + Dm[m][3 * c + 2] * Gx[be][2];
      for (int n = 0; n < 9; ++n)
        for (int m = 0; m <= n; ++m) {
          const int r = m / 3, al = m % 3;
          const double v = Gx[al][0] * T[3 * r][n] + Gx[al][1] * T[3 * r + 1][n] + Gx[al][2] * T[3 * r + 2][n];
          lin[(long long)(kWA + sym9(m, n)) * stride] = wdet * v;
        }
      for (int r = 0; r < 3; ++r)
        for (int al = 0; al < 3; ++al) {
          lin[(long long)(kWP + 3 * r + al) * stride] =
              wdet * (Gx[al][0] * Pv[3 * r] + Gx[al][1] * Pv[3 * r + 1] + Gx[al][2] * Pv[3 * r + 2]);
          lin[(long long)(kWC + 3 * r + al) * stride] =
              wdet * gl.s_phi * (Gx[al][0] * Lv[3 * r] + Gx[al][1] * Lv[3 * r + 1] + Gx[al][2] * Lv[3 * r + 2]);
        }
      lin[(long long)kWD * stride] = wdet * gl.s_phi * Lphi;
      double K[3][3];
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be)
          K[al][be] = wdet * ph.kphi * (Gx[al][0] * Gx[be][0] + Gx[al][1] * Gx[be][1] + Gx[al][2] * Gx[be][2]);
      for (int al = 0; al < 3; ++al) lin[(long long)(kWK + al) * stride] = K[al][al];
      lin[(long long)(kWKX + 0) * stride] = K[0][1];
      lin[(long long)(kWKX + 1) * stride] = K[0][2];
      lin[(long long)(kWKX + 2) * stride] = K[1][2];
    }
  }
  if (status) atomicOr(a.status, status);
}

cudaError_t launch_pointwise(const PointArgs& a, cudaStream_t st) {
  if (a.nq == 0) return cudaSuccess;
  long long nb = (a.nq + 127) / 128;
  k_pointwise<<<(unsigned)nb, 128, 0, st>>>(a); note_launch();
  return cudaGetLastError();
}

}  // namespace pff
