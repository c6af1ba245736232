"""Independent numpy restatement of the paper's closed-form linearisation.

Used only to pin the oracle's dual-number tangent.  It follows the principal
format of Appendix A for the update, Appendix B (Eq. hencky-stress-linearization
with the eigenvector variation for distinct eigenvalues, Box A1) for the branch
stresses and Appendix C (Eqs. linear-degraded-stress-linearization,
maxwell-dtau-dphi, prandtl-dtau-dphi, linearized-local-damage-residual,
history-field-linearization, energy-displacement-linearization,
maxwell-energy-dphi, prandtl-energy-dphi) for the coupled terms.  Valid at
points with distinct eigenvalues of every branch's trial b.
"""
import numpy as np
from scipy.optimize import brentq

VI = [0, 1, 2, 1, 0, 0]
VJ = [0, 1, 2, 2, 2, 1]


def _sym(v):
    A = np.empty((3, 3))
    for k in range(6):
        A[VI[k], VJ[k]] = A[VJ[k], VI[k]] = v[k]
    return A


def branches(phase_vec):
    """(kind, E, nu, extra, history offset) per branch of one phase."""
    out = [("hooke", phase_vec[2], phase_vec[3], None, None)]
    if phase_vec[4]:
        out.append(("maxwell", phase_vec[5], phase_vec[6], phase_vec[7], 0))
    if phase_vec[8]:
        law = tuple(phase_vec[11:15]) if len(phase_vec) == 15 else (phase_vec[11], 0.0, phase_vec[11], 0.0)
        out.append(("prandtl", phase_vec[9], phase_vec[10], law, 6))
    return out


def yield_stress(law, ep):
    """Linear + Voce hardening law (Eq. plasticity-strain-hardening-law) and its slope."""
    s0, Hl, sinf, beta = law
    return s0 + Hl * ep + (sinf - s0) * (1 - np.exp(-beta * ep)), Hl + (sinf - s0) * beta * np.exp(-beta * ep)


def point(inp, hist, phase_vec, glob):
    """Primal quantities at one point (principal format, Appendix A)."""
    G = inp[:9].reshape(3, 3)
    phi = inp[9]
    F = np.eye(3) + G
    J = np.linalg.det(F)
    theta = np.log(J)
    at, eta, zeta, dt, s_phi = glob
    g = (1 - phi) ** 2 + eta
    gp = -2 * (1 - phi)
    br = []
    kap_tot = 0.0
    for kind, E, nu, extra, off in branches(phase_vec):
        mu = E / (2 * (1 + nu))
        kap = E / (3 * (1 - 2 * nu))
        kap_tot += kap
        C = np.eye(3) if off is None else _sym(hist[off:off + 6])
        b = F @ C @ F.T
        bi, N = np.linalg.eigh(b)
        eps = 0.5 * np.log(bi)
        epsd = eps - eps.sum() / 3
        q = 2 * mu * np.sqrt(1.5 * np.sum(epsd ** 2))
        a, da_dphi, yield_, dgam, Hs = 1.0, 0.0, False, 0.0, 0.0
        if kind == "maxwell" and np.isfinite(extra):
            c = mu * dt / extra
            a = 1 / (1 + c * g)
            da_dphi = -a * a * c * gp
        elif kind == "prandtl" and g * q - yield_stress(extra, hist[12])[0] > 0:
            # Box 2, degraded: g q - 3 g mu dgam - sigma_y(eps_p,n + dgam) = 0, bracketed
            # root (f(0) > 0 >= f(dgam_max) for a non-decreasing sigma_y)
            f = lambda x: g * q - 3 * g * mu * x - yield_stress(extra, hist[12] + x)[0]
            hi = (g * q - yield_stress(extra, hist[12])[0]) / (3 * g * mu)
            dgam = brentq(f, 0.0, hi, xtol=1e-300, rtol=1e-15, maxiter=500) if f(hi) < 0 else hi
            Hs = yield_stress(extra, hist[12] + dgam)[1]
            a = 1 - 3 * mu * dgam / q
            # implicit derivative of dgam in phi (through g), Box A1 / App. C
            da_dphi = -3 * mu / q * (q - 3 * mu * dgam) * gp / (3 * g * mu + Hs)
            yield_ = True
        br.append(dict(kind=kind, mu=mu, kap=kap, bi=bi, N=N, epsd=epsd, a=a, da_dphi=da_dphi,
                       q=q, yield_=yield_, taui=2 * mu * a * epsd, dgam=dgam, H=Hs, g=g))
    taud = sum(b["N"] @ np.diag(b["taui"]) @ b["N"].T for b in br)
    psid = sum(b["mu"] * b["a"] ** 2 * np.sum(b["epsd"] ** 2) for b in br)
    tauv = kap_tot * theta * np.eye(3)
    psiv = 0.5 * kap_tot * theta ** 2
    tens = theta >= 0
    if tens:
        taudeg = g * (taud + tauv)
        psip = psid + psiv
    else:
        taudeg = g * taud + tauv
        psip = psid
    return dict(F=F, theta=theta, g=g, gp=gp, br=br, taud=taud, tauv=tauv, taudeg=taudeg,
                psip=psip, tens=tens, kap_tot=kap_tot)


def directional(inp, hist, phase_vec, glob, dF, dphi, dgphi):
    """Variation of (f0_phi, P, f1_phi) in direction (dF, dphi, dgphi)."""
    s = point(inp, hist, phase_vec, glob)
    at, eta, zeta, dt, s_phi = glob
    F, g, gp = s["F"], s["g"], s["gp"]
    Finv = np.linalg.inv(F)
    ell = dF @ Finv
    dtaud = np.zeros((3, 3))
    dpsid = 0.0
    for b in s["br"]:
        N, bi, mu, a = b["N"], b["bi"], b["mu"], b["a"]
        lh = N.T @ ell @ N
        dbh = lh * bi[None, :] + bi[:, None] * lh.T           # N^T db N, db = ell b + b ell^T
        deps = np.diag(dbh) / (2 * bi)                          # App. B principal strain variation
        depsd_tr = deps - deps.sum() / 3
        epsd = b["epsd"]
        da = b["da_dphi"] * dphi
        if b["kind"] == "prandtl" and b["yield_"]:
            taud_tr = 2 * mu * epsd
            dq = 1.5 * np.dot(taud_tr, 2 * mu * depsd_tr) / b["q"]   # Eq. plasticity-dq-trial-vonMises
            # Eq. plasticity-dtau-vonMises with the degraded consistency condition:
            # d dgam = g dq / (3 g mu + H) at fixed phi, a = 1 - 3 mu dgam / q
            ddgam = b["g"] * dq / (3 * b["g"] * mu + b["H"])
            da = da - 3 * mu * ddgam / b["q"] + 3 * mu * b["dgam"] * dq / b["q"] ** 2
        depsd = a * depsd_tr + da * epsd                        # Box A1 (degraded form)
        dtaui = 2 * mu * depsd
        tau_i = b["taui"]
        dth = np.diag(dtaui)
        for i in range(3):
            for j in range(3):
                if i != j:
                    dth[i, j] = (tau_i[i] - tau_i[j]) / (bi[i] - bi[j]) * dbh[i, j]
        dtaud += N @ dth @ N.T
        dpsid += 2 * mu * a * np.dot(epsd, depsd)               # tau_d : d eps_d^e
    dth_vol = np.trace(ell)
    dtauv = s["kap_tot"] * dth_vol * np.eye(3)
    dpsiv = s["kap_tot"] * s["theta"] * dth_vol
    if s["tens"]:
        dtaudeg = g * (dtaud + dtauv) + gp * dphi * (s["taud"] + s["tauv"])
        dpsip = dpsid + dpsiv
    else:
        dtaudeg = dtauv + g * dtaud + gp * dphi * s["taud"]
        dpsip = dpsid
    dP = (dtaudeg - s["taudeg"] @ ell.T) @ Finv.T
    Hn = hist[13]
    active = s["psip"] > Hn
    H = s["psip"] if active else Hn
    dH = dpsip if active else 0.0
    c0 = 8 / 3 if at == 1 else 2.0
    Gc, l0 = phase_vec[0], phase_vec[1]
    app = 0.0 if at == 1 else 2.0
    dL = (2 * H + Gc / (c0 * l0) * app + zeta / dt) * dphi + gp * dH
    kphi = s_phi * 2 * Gc * l0 / c0
    return s_phi * dL, dP, kphi * dgphi


def tangent16(inp, hist, phase_vec, glob):
    """16x16 pointwise tangent in the oracle's layout (rows f0[4], f1[4][3];
    cols values[4], gradients[4][3])."""
    D = np.zeros((16, 16))
    for col in range(16):
        if col < 3:
            continue  # u values do not enter
        dF = np.zeros((3, 3))
        dphi = 0.0
        dg = np.zeros(3)
        if col == 3:
            dphi = 1.0
        elif col < 13:
            k = col - 4
            dF[k // 3, k % 3] = 1.0
        else:
            dg[col - 13] = 1.0
        df0, dP, df1 = directional(inp, hist, phase_vec, glob, dF, dphi, dg)
        D[3, col] = df0
        D[4:13, col] = dP.ravel()
        D[13:16, col] = df1
    return D
