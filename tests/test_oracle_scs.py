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


# ---- the structured operator (App. D.2: A x and A^T y contracted over local bases)
def test_kron_columns_golden_two_qubits():
    """Hand-written Kronecker products of two-dimensional local matrices:
    diag(1, -1)/sqrt(2) (x) (E01 + E10)/sqrt(2), and the product of two
    antisymmetric factors (E01 - E10)/sqrt(2), which is symmetric."""
    B, anti = W.real_local_basis(2)
    assert list(anti) == [False, False, False, True]
    F1 = 0.5 * np.array([[0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 0, -1], [0, 0, -1, 0]], dtype=float)
    F2 = 0.5 * np.array([[0, 0, 0, 1], [0, 0, -1, 0], [0, -1, 0, 0], [1, 0, 0, 0]], dtype=float)
    cols = S.kron_columns([B, B], [1 * 4 + 2, 3 * 4 + 3])
    np.testing.assert_allclose(cols[:, 0], oracle.svec(F1), atol=1e-15)
    np.testing.assert_allclose(cols[:, 1], oracle.svec(F2), atol=1e-15)


def test_process_allowed_matches_the_paper_count_and_is_symmetric():
    """The allowed coefficients of App. B number 2 d^6 - 3 d^4 + 2 d^2; the
    real subset's Kronecker products are symmetric."""
    for d in (2, 3):
        assert W.process_allowed(d, real=False).size == 2 * d ** 6 - 3 * d ** 4 + 2 * d ** 2
    B, _ = W.real_local_basis(2)
    for flat in W.process_allowed(2):
        mu = np.unravel_index(int(flat), (4, 4, 4, 4))
        F = np.kron(np.kron(np.kron(B[mu[0]], B[mu[1]]), B[mu[2]]), B[mu[3]])
        assert np.array_equal(F, F.T)


def test_kron_contractions_match_the_explicit_columns():
    rng = W.rng_for(7950)
    B, _ = W.real_local_basis(2)
    bases, index = [B] * 4, W.process_allowed(2)
    A = S.kron_columns(bases, index)
    # orthonormal local bases and symmetric products: A^T A = I (App. D.3)
    np.testing.assert_allclose(A.T @ A, np.eye(index.size), atol=1e-14)
    x = rng.standard_normal(index.size)
    y = rng.standard_normal(A.shape[0])
    np.testing.assert_allclose(S.kron_apply(bases, index, x), A @ x, atol=1e-13)
    np.testing.assert_allclose(S.kron_apply_t(bases, index, y), A.T @ y, atol=1e-13)
    # mixed local dimensions: modes of sides 2 and 3
    B3, _ = W.real_local_basis(3)
    idx = np.array([0, 5, 9, 20, 35])  # symmetric products (35: two antisymmetric factors)
    A2 = S.kron_columns([B, B3], idx)
    x2 = rng.standard_normal(idx.size)
    y2 = rng.standard_normal(A2.shape[0])
    np.testing.assert_allclose(S.kron_apply([B, B3], idx, x2), A2 @ x2, atol=1e-13)
    np.testing.assert_allclose(S.kron_apply_t([B, B3], idx, y2), A2.T @ y2, atol=1e-13)


def test_kron_iteration_matches_the_dense_iteration():
    rng = W.rng_for(7960)
    B, _ = W.real_local_basis(2)
    bases, index = [B] * 4, W.process_allowed(2)
    A = S.kron_columns(bases, index)
    m, k = A.shape
    b, c = rng.standard_normal(m), rng.standard_normal(k)
    u = np.concatenate([rng.standard_normal(k + m), [1.0]])
    v = np.concatenate([np.zeros(k), rng.standard_normal(m), [0.3]])
    offs = [0, m]
    uk, vk = S.iterate_kron(bases, index, b, c, offs, u, v, 3)
    ud, vd = S.iterate(A, b, c, offs, u, v, 3)
    np.testing.assert_allclose(uk, ud, atol=1e-12)
    np.testing.assert_allclose(vk, vd, atol=1e-12)
