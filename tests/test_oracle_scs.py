"""Pins for the oracle of the SCS iteration around the projection (no GPU).

App. D.1's iteration u~ = (I + Q)^{-1}(u + v), u = Pi_C(u~ - v),
v = v - u~ + u is checked against: a dense solve of (I + Q) for the affine
step (a library routine), the cone projection's own pins (it is the
oracle's proj), and convergence to the known optimum of a small SDP."""
import numpy as np

import oracle
from oracle import scs as S
from paper_2606_20519_gb300 import workloads as W


def _problem(rng, sides, k):
    offs = np.cumsum([0] + [n * (n + 1) // 2 for n in sides])
    m = int(offs[-1])
    A, _ = np.linalg.qr(rng.standard_normal((m, k)))
    return A, rng.standard_normal(m), rng.standard_normal(k), offs


def test_affine_step_equals_dense_solve():
    rng = W.rng_for(7900)
    A, b, c, offs = _problem(rng, [3, 4], 6)
    m, k = A.shape
    Q = np.zeros((k + m + 1, k + m + 1))
    Q[:k, k:k + m] = A.T
    Q[:k, -1] = c
    Q[k:k + m, :k] = -A
    Q[k:k + m, -1] = b
    Q[-1, :k] = -c
    Q[-1, k:k + m] = -b
    w = rng.standard_normal(k + m + 1)
    want = np.linalg.solve(np.eye(k + m + 1) + Q, w)
    px, py, hp = S.setup(A, b, c)
    zx, zy = S.m_inverse(A, w[:k], w[k:k + m])
    tau = (w[-1] + c @ zx + b @ zy) / (1 + hp)
    got = np.concatenate([zx - tau * px, zy - tau * py, [tau]])
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_one_iteration_by_hand():
    rng = W.rng_for(7910)
    A, b, c, offs = _problem(rng, [3], 2)
    m, k = A.shape
    u = np.concatenate([rng.standard_normal(k + m), [1.0]])
    v = np.concatenate([np.zeros(k), rng.standard_normal(m), [0.5]])
    un, vn = S.iterate(A, b, c, offs, u, v, 1)
    Q = np.block([[np.zeros((k, k)), A.T, c[:, None]], [-A, np.zeros((m, m)), b[:, None]],
                  [-c[None, :], -b[None, :], np.zeros((1, 1))]])
    ut = np.linalg.solve(np.eye(k + m + 1) + Q, u + v)
    t = ut - v
    want_u = np.concatenate([t[:k], oracle.proj(t[k:k + m]), [max(t[-1], 0.0)]])
    np.testing.assert_allclose(un, want_u, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(vn, v - ut + want_u, rtol=1e-12, atol=1e-12)


def test_converges_to_known_optimum():
    """min -<C, X> s.t. S = B - X is PSD, C PSD: the optimum is X = B with dual
    Y = C (A = I, orthonormal).  In SCS form x = svec(X), c = -svec(C),
    s = b - x, b = svec(B); the iterates give x/tau -> b, y/tau -> svec(C)."""
    rng = W.rng_for(7920)
    n = 3
    Cm = W.sym_gaussian(rng, n)
    Cm = Cm @ Cm.T + 0.5 * np.eye(n)
    Bm = W.sym_gaussian(rng, n)
    b, cs = W.to_svec(Bm), W.to_svec(Cm)
    m = b.size
    A = np.eye(m)
    offs = [0, m]
    u = np.concatenate([np.zeros(2 * m), [1.0]])
    v = np.concatenate([np.zeros(2 * m), [1.0]])
    u, v = S.iterate(A, b, -cs, offs, u, v, 3000)
    tau = u[-1]
    assert tau > 0
    np.testing.assert_allclose(u[:m] / tau, b, atol=1e-6)
    np.testing.assert_allclose(u[m:2 * m] / tau, cs, atol=1e-6)
