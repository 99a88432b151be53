"""Pins for the FP64 CPU oracle (no GPU).

The oracle is checked against what the definition of the projection fixes
(App. D.1 vec_R map and Moreau decomposition, App. D.2 projection by
eigendecomposition with negative eigenvalues set to zero) rather than
against itself: hand-worked fixtures, closed forms, exact constructions,
invariants, LAPACK as a third witness and brute force on tiny sizes.  The
last test plants known mistakes in the oracle and shows that a pin fails.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2606_20519_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def rand_sym(rng, n):
    return W.sym_gaussian(rng, n)


def proj_from_factors(Q, lam):
    """Closed-form projection of Q diag(lam) Q^T."""
    return (Q * np.maximum(lam, 0.0)[None, :]) @ Q.T


# ------------------------------------------------------------------ svec map

def test_svec_golden_fixture():
    g = json.load(open(os.path.join(GOLDEN, "svec_3x3.json")))
    A = np.array(g["matrix"])
    # the fixture holds the correctly rounded k*sqrt(2); computing it as
    # k * fl(sqrt(2)) may differ by one unit in the last place
    np.testing.assert_allclose(oracle.svec(A), np.array(g["svec"]), rtol=2.3e-16, atol=0)
    np.testing.assert_allclose(oracle.smat(np.array(g["svec"])), A, rtol=2.3e-16, atol=0)
    # the input generator's layout is an independent implementation
    np.testing.assert_allclose(W.to_svec(A), np.array(g["svec"]), rtol=2.3e-16, atol=0)


def test_svec_isometry_and_layout():
    rng = W.rng_for(1)
    for n in (1, 2, 5, 17):
        A, B = rand_sym(rng, n), rand_sym(rng, n)
        sa, sb = oracle.svec(A), oracle.svec(B)
        assert abs(sa @ sb - np.trace(A @ B)) <= 1e-12 * (1 + np.abs(A).sum() * np.abs(B).sum())
        np.testing.assert_allclose(sa, W.to_svec(A), rtol=0, atol=0)
        np.testing.assert_allclose(oracle.smat(sa), A, rtol=1e-15, atol=1e-15)


# -------------------------------------------------------------- closed forms

def test_golden_2x2_and_moreau():
    g = json.load(open(os.path.join(GOLDEN, "proj_2x2.json")))
    x = np.array(g["x_svec"])
    np.testing.assert_allclose(oracle.proj(x), g["proj_svec"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.proj(-x), g["proj_neg_svec"], rtol=0, atol=1e-15)


def test_golden_3x3():
    g = json.load(open(os.path.join(GOLDEN, "proj_3x3.json")))
    X = np.array(g["x_matrix_times_6"]) / 6.0
    P = np.array(g["proj_matrix_times_3"]) / 3.0
    y, lam = oracle.proj(oracle.svec(X), return_eigs=True)
    np.testing.assert_allclose(oracle.smat(y), P, rtol=0, atol=1e-14)
    np.testing.assert_allclose(np.sort(lam), g["eigenvalues"], rtol=0, atol=1e-14)
    # Euler: DPi(X)[X] = Pi(X)
    np.testing.assert_allclose(oracle.jvp(oracle.svec(X), oracle.svec(X)), oracle.svec(P), atol=1e-13)


def test_closed_form_2x2_random():
    rng = W.rng_for(2)
    for _ in range(200):
        a, b, c = rng.standard_normal(3) * 10.0 ** rng.uniform(-3, 3, 3)
        m, r = 0.5 * (a + c), np.hypot(0.5 * (a - c), b)
        lp, lm = m + r, m - r
        X = np.array([[a, b], [b, c]])
        if lm >= 0:
            P = X
        elif lp <= 0:
            P = np.zeros((2, 2))
        else:
            # eigenvector of lp: (b, lp - a) or (lp - c, b), the better conditioned one
            v = np.array([b, lp - a]) if abs(lp - a) >= abs(lp - c) else np.array([lp - c, b])
            v /= np.linalg.norm(v)
            P = lp * np.outer(v, v)
        y = oracle.smat(oracle.proj(oracle.svec(X)))
        assert np.abs(y - P).max() <= 1e-13 * max(abs(a), abs(b), abs(c))


def test_diagonal_is_exact():
    rng = W.rng_for(3)
    d = rng.standard_normal(33)
    y = oracle.smat(oracle.proj(oracle.svec(np.diag(d))))
    np.testing.assert_array_equal(y, np.diag(np.maximum(d, 0.0)))


def test_psd_and_nsd_inputs():
    rng = W.rng_for(4)
    for n in (3, 20, 41):
        G = rng.standard_normal((n, n))
        Xp = G @ G.T
        y = oracle.proj(oracle.svec(Xp))
        assert rel(y, oracle.svec(Xp)) <= 1e-13
        y = oracle.proj(oracle.svec(-Xp))
        assert np.linalg.norm(y) <= 1e-13 * np.linalg.norm(Xp)


def test_n1_and_n0_and_nonfinite():
    for v in (-2.5, 0.0, 3.25):
        assert oracle.proj(np.array([v]))[0] == max(v, 0.0)
    assert oracle.proj(np.zeros(0)).size == 0
    x = W.to_svec(np.eye(3))
    x[2] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.proj(x)


# -------------------------------------------------------------- constructions

@pytest.mark.parametrize("maker,n", [
    (W.spectrum_plain, 81), (W.spectrum_admm, 60), (W.spectrum_precision, 64),
    (W.spectrum_vjp, 50)])
def test_construction_pin(maker, n):
    rng = W.rng_for(5 + n)
    lam = maker(rng, n)
    X, Q, lam = W.from_spectrum(rng, lam)
    y = oracle.proj(W.to_svec(X))
    assert rel(y, W.to_svec(proj_from_factors(Q, lam))) <= 1e-12


def test_single_projection_workload_pin():
    x, Q, lam = W.single_projection()
    assert x.size == 3321 and (lam == 0).sum() == 1
    assert rel(oracle.proj(x), W.to_svec(proj_from_factors(Q, lam))) <= 1e-12


def test_lapack_witness():
    rng = W.rng_for(6)
    for n in (7, 48, 90):
        X = rand_sym(rng, n) + rng.uniform(-0.5, 0.5) * np.eye(n)
        w, V = np.linalg.eigh(X)
        P = (V * np.maximum(w, 0)) @ V.T
        assert rel(oracle.proj(W.to_svec(X)), W.to_svec(P)) <= 1e-12


# ------------------------------------------------------------------ invariants

def test_homogeneity_exact():
    rng = W.rng_for(7)
    x = W.to_svec(rand_sym(rng, 23))
    y = oracle.proj(x)
    for k in (-3, 5):
        np.testing.assert_array_equal(oracle.proj(x * 2.0 ** k), y * 2.0 ** k)


def test_permutation_equivariance():
    rng = W.rng_for(8)
    X = rand_sym(rng, 30)
    p = rng.permutation(30)
    Y = oracle.smat(oracle.proj(W.to_svec(X)))
    Yp = oracle.smat(oracle.proj(W.to_svec(X[np.ix_(p, p)])))
    assert np.abs(Yp - Y[np.ix_(p, p)]).max() <= 1e-13 * np.abs(X).max()


def test_moreau_idempotence_kkt():
    rng = W.rng_for(9)
    for n in (2, 13, 64):
        X = rand_sym(rng, n)
        x = W.to_svec(X)
        yp, yn = oracle.proj(x), oracle.proj(-x)
        s = np.linalg.norm(x)
        assert np.linalg.norm(yp - yn - x) <= 1e-13 * s            # X = Pi(X) - Pi(-X)
        assert abs(yp @ yn) <= 1e-13 * s * s                        # <Pi(X), Pi(-X)> = 0
        assert np.linalg.norm(oracle.proj_moreau(x) - yp) <= 1e-13 * s
        assert np.linalg.norm(oracle.proj(yp) - yp) <= 1e-13 * s    # idempotent
        Y = oracle.smat(yp)
        assert np.linalg.eigvalsh(Y).min() >= -1e-13 * s            # Y >= 0
        assert np.linalg.eigvalsh(Y - X).min() >= -1e-13 * s        # Y - X >= 0
        assert abs(np.trace(Y @ (Y - X))) <= 1e-13 * s * s          # complementarity


def test_brute_force_tiny():
    rng = W.rng_for(10)
    for n in (1, 2, 3):
        for _ in range(5):
            X = rand_sym(rng, n)
            Y = oracle.smat(oracle.proj(W.to_svec(X)))
            best = np.linalg.norm(Y - X)
            L = rng.standard_normal((20000, n, n))
            cand = L @ np.swapaxes(L, 1, 2)
            # also scaled candidates near the solution
            cand = np.concatenate([cand, Y[None] + 0.01 * cand[:5000]])
            d = np.linalg.norm(cand - X[None], axis=(1, 2))
            assert d.min() >= best - 1e-12


def test_thread_count_independence():
    rng = W.rng_for(11)
    x = W.to_svec(rand_sym(rng, 57))
    oracle.set_threads(1)
    try:
        y1 = oracle.proj(x)
        oracle.set_threads(4)
        y4 = oracle.proj(x)
    finally:
        oracle.set_threads(0)
    np.testing.assert_array_equal(y1, y4)


def test_batched_wrapper():
    b = W.uneven_batch(restarts=2, small_sides=(4, 9), copies=1, big_sides=(16,))
    y = oracle.proj_batched(b.x, b.offsets)
    for i in range(b.count):
        a, e = b.offsets[i], b.offsets[i + 1]
        np.testing.assert_array_equal(y[a:e], oracle.proj(b.x[a:e]))


# ------------------------------------------------------------- derivative pins

def _ip(a, b):
    return float(np.dot(a, b))


def test_jvp_euler_and_projections():
    rng = W.rng_for(12)
    X = rand_sym(rng, 24)
    x = W.to_svec(X)
    yp, yn = oracle.proj(x), oracle.proj(-x)
    s = np.linalg.norm(x)
    assert np.linalg.norm(oracle.jvp(x, x) - yp) <= 1e-12 * s        # J[X] = Pi(X)
    assert np.linalg.norm(oracle.jvp(x, yp) - yp) <= 1e-12 * s       # J[Pi(X)] = Pi(X)
    assert np.linalg.norm(oracle.jvp(x, yn)) <= 1e-12 * s            # J[Pi(-X)] = 0


def test_jvp_symmetry_and_bounds():
    rng = W.rng_for(13)
    x = W.to_svec(rand_sym(rng, 20))
    a, b = rng.standard_normal(x.size), rng.standard_normal(x.size)
    Ja, Jb = oracle.jvp(x, a), oracle.jvp(x, b)
    assert abs(_ip(a, Jb) - _ip(Ja, b)) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)
    for h in (a, b):
        q = _ip(h, oracle.jvp(x, h))
        assert -1e-12 <= q <= _ip(h, h) * (1 + 1e-12)


def test_jvp_definite_cases():
    rng = W.rng_for(14)
    G = rng.standard_normal((15, 15))
    Xp = G @ G.T + np.eye(15)
    h = rng.standard_normal(W.svec_len(15))
    assert rel(oracle.jvp(W.to_svec(Xp), h), h) <= 1e-12
    assert np.linalg.norm(oracle.jvp(W.to_svec(-Xp), h)) <= 1e-12 * np.linalg.norm(h)


def test_jvp_diagonal_divided_differences():
    rng = W.rng_for(15)
    d = np.array([1.5, -0.25, 0.75, -2.0, 3.0, -0.5])
    H = rand_sym(rng, d.size)
    out = oracle.smat(oracle.jvp(W.to_svec(np.diag(d)), W.to_svec(H)))
    relu = np.maximum(d, 0.0)
    for i in range(d.size):
        for j in range(d.size):
            if d[i] == d[j]:
                L = 1.0 if d[i] > 0 else 0.0
            else:
                L = (relu[i] - relu[j]) / (d[i] - d[j])
            assert abs(out[i, j] - L * H[i, j]) <= 1e-14 * (1 + abs(H[i, j]))


def test_jvp_vs_central_differences():
    # well separated spectrum: the +-1e-9 clusters of the stress case moved to +-1e-3
    rng = W.rng_for(16)
    lam = W.spectrum_vjp(rng, 40, cluster=1e-3)
    X, Q, lam = W.from_spectrum(rng, lam)
    x = W.to_svec(X)
    h = rng.standard_normal(x.size)
    fd = oracle.fd_jvp(x, h, 1e-6)
    assert rel(oracle.jvp(x, h), fd) <= 1e-6


# ---------------------------------------------------------------- planted bugs

def _pins_pass():
    """A compact set of pins; returns False as soon as one fails."""
    try:
        g = json.load(open(os.path.join(GOLDEN, "proj_2x2.json")))
        if np.abs(oracle.proj(np.array(g["x_svec"])) - g["proj_svec"]).max() > 1e-14:
            return False
        rng = W.rng_for(17)
        lam = W.spectrum_plain(rng, 21)
        X, Q, lam = W.from_spectrum(rng, lam)
        if rel(oracle.proj(W.to_svec(X)), W.to_svec(proj_from_factors(Q, lam))) > 1e-12:
            return False
        gs = json.load(open(os.path.join(GOLDEN, "svec_3x3.json")))
        if np.abs(oracle.svec(np.array(gs["matrix"])) - gs["svec"]).max() > 1e-15:
            return False
        return True
    except oracle.OracleError:
        return False


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(mutation):
    assert _pins_pass()
    oracle.set_mutation(mutation)
    try:
        assert not _pins_pass(), f"mutation {mutation} slipped through the pins"
    finally:
        oracle.set_mutation(0)
    assert _pins_pass()
