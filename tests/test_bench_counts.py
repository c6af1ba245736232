"""The roofline numerator of the bench: algorithmic flops of one element of the
Jacobian action, counted here by running an explicit loop version of one
element's action (sum-factorised basis work, collocated gradient, the
stored-word map at each point) that tallies its multiply-adds, against
bench.apply_counts.  The loop version also checks itself against a dense
evaluation of the same action, so the count belongs to a correct computation."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _counted_action(P, Q, rng):
    """One element, four fields: y = B^T D(words) B x with B = (values,
    gradients) at Q^3 points, done by 1D contractions; returns (y, MACs, y_dense)."""
    B = rng.uniform(-1, 1, (Q, P))      # 1D basis at the points
    Dc = rng.uniform(-1, 1, (Q, Q))     # collocated 1D derivative at the points
    x = rng.uniform(-1, 1, (4, P, P, P))
    macs = 0

    def c1(M, v, axis):                 # 1D contraction along one axis, counted
        nonlocal macs
        out = np.tensordot(M, v, axes=([1], [axis]))
        macs += M.shape[0] * M.shape[1] * (v.size // v.shape[axis])
        return np.moveaxis(out, 0, axis)

    # forward: values at the points, then three collocated derivatives
    val, grad = [], []
    for f in range(4):
        v = c1(B, c1(B, c1(B, x[f], 2), 1), 0)             # P^3 Q + P^2 Q^2 + P Q^3
        val.append(v)
        grad.append([c1(Dc, v, a) for a in range(3)])      # 3 Q^4
    # pointwise: symmetric 9x9 block on the displacement gradients, dP/dphi,
    # d(sL)/dF, d(sL)/dphi and the diagonal phase-gradient coefficients
    nq = Q ** 3
    A = rng.uniform(-1, 1, (nq, 9, 9)); A = A + A.transpose(0, 2, 1)
    Pw, Cw = rng.uniform(-1, 1, (nq, 9)), rng.uniform(-1, 1, (nq, 9))
    Dw, Kw = rng.uniform(-1, 1, nq), rng.uniform(-1, 1, (nq, 3))
    gu = np.stack([grad[f][a].ravel() for f in range(3) for a in range(3)], 1)     # [nq, 9]
    phi = val[3].ravel()
    gphi = np.stack([grad[3][a].ravel() for a in range(3)], 1)
    ou = np.zeros((nq, 9))
    for m in range(9):
        for n in range(m, 9):
            ou[:, m] += A[:, m, n] * gu[:, n]; macs += nq
            if n != m:
                ou[:, n] += A[:, m, n] * gu[:, m]; macs += nq
    ou += Pw * phi[:, None]; macs += 9 * nq
    o0 = (Cw * gu).sum(1) + Dw * phi; macs += 10 * nq
    og = Kw * gphi; macs += 3 * nq
    # backward: transposed derivatives and interpolation
    y = np.zeros_like(x)
    for f in range(4):
        comps = [ou[:, 3 * f + a] for a in range(3)] if f < 3 else [og[:, a] for a in range(3)]
        t = sum(c1(Dc.T, comps[a].reshape(Q, Q, Q), a) for a in range(3))        # 3 Q^4
        if f == 3:
            t = t + o0.reshape(Q, Q, Q)
        y[f] = c1(B.T, c1(B.T, c1(B.T, t, 0), 1), 2)      # P Q^3 + P^2 Q^2 + P^3 Q
    # dense check: the same operator through explicit 3D matrices
    B3 = np.einsum("ia,jb,kc->ijkabc", B, B, B).reshape(nq, P ** 3)
    G3 = [np.einsum("im,mjkabc->ijkabc", Dc, B3.reshape(Q, Q, Q, P, P, P)).reshape(nq, -1),
          np.einsum("jm,imkabc->ijkabc", Dc, B3.reshape(Q, Q, Q, P, P, P)).reshape(nq, -1),
          np.einsum("km,ijmabc->ijkabc", Dc, B3.reshape(Q, Q, Q, P, P, P)).reshape(nq, -1)]
    xs = x.reshape(4, -1)
    gud = np.stack([G3[a] @ xs[f] for f in range(3) for a in range(3)], 1)
    phd = B3 @ xs[3]
    gpd = np.stack([G3[a] @ xs[3] for a in range(3)], 1)
    oud = np.einsum("qmn,qn->qm", A * np.triu(np.ones((9, 9)))[None] + (A * np.triu(np.ones((9, 9)), 1)[None]).transpose(0, 2, 1), gud) + Pw * phd[:, None]
    o0d = (Cw * gud).sum(1) + Dw * phd
    yd = np.zeros_like(xs)
    for f in range(3):
        yd[f] = sum(G3[a].T @ oud[:, 3 * f + a] for a in range(3))
    yd[3] = sum(G3[a].T @ (Kw[:, a] * gpd[:, a]) for a in range(3)) + B3.T @ o0d
    return y.reshape(4, -1), macs, yd


@pytest.mark.parametrize("P,Q", [(5, 5), (3, 5), (2, 5), (3, 3), (4, 4)])
def test_apply_counts_matches_counted_loops(P, Q):
    import bench
    y, macs, yd = _counted_action(P, Q, np.random.default_rng(P * 10 + Q))
    assert np.linalg.norm(y - yd) <= 1e-12 * np.linalg.norm(yd)
    assert bench.apply_counts(P, Q) == 2 * macs
