"""Pins for the oracle of the factorization-free approximate projection (no GPU).

Conclusions ("Approximate semidefinite-cone projections"): Pi is approximated
by a composite matrix polynomial of matrix products whose scalar map
reproduces eigenvalue thresholding.  The oracle's reading (scaled
Newton-Schulz for sign, Chen & Chow 2014) is pinned here against things
other than itself: a brute-force minimax search for the scaling, the
Jacobi eigendecomposition of the main oracle (a scalar function of a
symmetric matrix acts on its eigenvalues), diagonal inputs, the error bound
against the exact projection, and exact homogeneity.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import poly as P
from paper_2606_20519_gb300 import workloads as W


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def cubic(alpha, t):
    return 0.5 * alpha * t * (3.0 - alpha * alpha * t * t)


@pytest.mark.parametrize("l", [1e-6, 1e-3, 0.05, 0.3, 0.7, 0.99])
def test_scaling_is_the_capped_minimax_cubic(l):
    """alpha of each step minimises max |1 - g(t)| over [l, 1] among the odd
    cubics (alpha t / 2)(3 - alpha^2 t^2) whose value at t = 1 is at least
    1/2: a grid search over alpha finds the same alpha."""
    alphas, lows = P.poly_schedule(l, 1)
    alpha = alphas[0]
    t = np.concatenate([np.geomspace(l, 1.0, 4001), [1.0 / alpha]])
    t = t[(t >= l) & (t <= 1.0)]

    def worst(a):
        return float(np.max(np.abs(1.0 - cubic(a, t))))

    grid = np.linspace(1.0, math.sqrt(3.0), 20001)
    grid = grid[cubic(grid, 1.0) >= 0.5]
    best = grid[int(np.argmin([worst(a) for a in grid]))]
    assert abs(best - alpha) <= 2 * (grid[1] - grid[0]) + 1e-9
    # the maximum 1 sits at 1/alpha inside [l, 1], the next bound is g(l)
    assert abs(cubic(alpha, 1.0 / alpha) - 1.0) <= 1e-15
    assert lows[1] == pytest.approx(cubic(alpha, l), rel=1e-15)
    assert cubic(alpha, l) <= cubic(alpha, 1.0) + 1e-15
    if l >= 0.3:
        # uncapped: equioscillation g(l) = g(1) (Chen & Chow)
        assert abs(cubic(alpha, l) - cubic(alpha, 1.0)) <= 1e-15
    else:
        # capped: g(1) = 1/2 exactly
        assert abs(cubic(alpha, 1.0) - 0.5) <= 1e-15


def test_schedule_limits_and_steps():
    # l = 1 gives the plain Newton-Schulz step 3t/2 - t^3/2
    a, b, _ = P.poly_coeffs(1.0 - 1e-16, 1)
    assert a[0] == pytest.approx(1.5, abs=1e-15) and b[0] == pytest.approx(-0.5, abs=1e-15)
    for lo, k in ((1e-3, 13), (1e-7, 24), (1e-9, 29)):
        alphas, lows = P.poly_schedule(lo)
        assert len(alphas) == k
        assert 1.0 - lows[-1] <= P.AUTO_TOL and 1.0 - lows[-2] > P.AUTO_TOL
        assert all(lows[i + 1] > lows[i] for i in range(k - 1))
    assert len(P.poly_schedule(1e-7, 5)[0]) == 5
    for bad in (0.0, 1.0, -1e-3, 2.0):
        with pytest.raises(ValueError):
            P.poly_schedule(bad)


@pytest.mark.parametrize("lo", [1e-3, 1e-9])
def test_scalar_composite_bounds(lo):
    """|f(t) - sign t| <= 1 - l_K above lo, 0 <= f(t) sign(t) <= 1 everywhere."""
    _, _, lk = P.poly_coeffs(lo)
    t = np.concatenate([np.geomspace(1e-14, 1.0, 20001), np.linspace(0.0, 1.0, 2001)])
    f = P.poly_scalar(t, lo)
    fm = P.poly_scalar(-t, lo)
    np.testing.assert_array_equal(fm, -f)  # odd
    assert np.all(f >= 0.0) and np.all(f <= 1.0 + 1e-15)
    big = t >= lo
    assert np.max(np.abs(1.0 - f[big])) <= (1.0 - lk) + 4e-16


@pytest.mark.parametrize("n,lo", [(9, 1e-3), (24, 1e-7), (40, 1e-9)])
def test_matrix_form_equals_scalar_composite_on_eigenvalues(n, lo):
    """f(X/sigma) by matrix products = V f(lam/sigma) V^T with (lam, V) from
    the Jacobi oracle: the same composite, two independent evaluations."""
    rng = W.rng_for(7100 + n)
    lam = np.concatenate([rng.uniform(-1, 1, n - 4), [1e-9, -2e-8, 3e-4, 0.0]])
    X, Q, _ = W.from_spectrum(rng, lam)
    x = W.to_svec(X)
    got = P.proj_poly(x, lo)
    lj, V = oracle.eig(x)
    sigma = math.sqrt(float(np.sum(lj * lj)))
    f = P.poly_scalar(lj / sigma, lo)
    want = oracle.svec((V * (0.5 * lj * (1.0 + f))[None, :]) @ V.T)
    assert rel(got, want) <= 1e-12


def test_diagonal_input_acts_entrywise():
    rng = W.rng_for(7200)
    d = np.concatenate([rng.uniform(-2, 2, 20), [0.0, 1e-12, -1e-12]])
    X = np.diag(d)
    got = oracle.smat(P.proj_poly(W.to_svec(X), 1e-6))
    sigma = math.sqrt(float(np.sum(d * d)))
    want = 0.5 * d * (1.0 + P.poly_scalar(d / sigma, 1e-6))
    np.testing.assert_allclose(np.diag(got), want, rtol=1e-14, atol=1e-300)
    assert np.max(np.abs(got - np.diag(np.diag(got)))) == 0.0


@pytest.mark.parametrize("lo", [1e-3, 1e-7])
def test_error_bound_against_exact_projection(lo):
    """||proj_poly - Pi||_F stays within the per-eigenvalue bound, and the
    bound is met closely when the spectrum has eigenvalues below lo * sigma."""
    rng = W.rng_for(7300)
    n = 48
    lam = np.concatenate([rng.uniform(0.05, 1, 20), rng.uniform(-1, -0.05, 16),
                          rng.uniform(-1, 1, 12) * 1e-4 * lo])
    X, Q, _ = W.from_spectrum(rng, lam)
    x = W.to_svec(X)
    exact = W.to_svec((Q * np.maximum(lam, 0.0)[None, :]) @ Q.T)
    err = np.linalg.norm(P.proj_poly(x, lo) - exact)
    bound = P.poly_error_bound(lam, lo)
    assert err <= bound * (1 + 1e-6) + 1e-13 * np.linalg.norm(exact)
    # the tiny eigenvalues are not resolved: each costs about |lam| / 2
    tiny = np.abs(lam) < lo * np.linalg.norm(lam)
    assert err >= 0.4 * 0.5 * np.linalg.norm(lam[tiny])


def test_resolved_spectrum_matches_exact_projection():
    rng = W.rng_for(7400)
    lam = np.concatenate([rng.uniform(1e-3, 1, 30), rng.uniform(-1, -1e-3, 30)])
    X, Q, _ = W.from_spectrum(rng, lam)
    x = W.to_svec(X)
    exact = W.to_svec((Q * np.maximum(lam, 0.0)[None, :]) @ Q.T)
    assert rel(P.proj_poly(x, 1e-6), exact) <= 1e-13
    assert rel(P.proj_poly(x, 1e-6), oracle.proj(x)) <= 1e-13


def test_homogeneity_zero_and_batching():
    rng = W.rng_for(7500)
    x = W.to_svec(W.sym_gaussian(rng, 17))
    y = P.proj_poly(x, 1e-6)
    for k in (-3, 5):
        np.testing.assert_array_equal(P.proj_poly(x * 2.0 ** k, 1e-6), y * 2.0 ** k)
    np.testing.assert_array_equal(P.proj_poly(np.zeros(W.svec_len(6)), 1e-6), np.zeros(W.svec_len(6)))
    # side 1: x (1 + l_K) / 2 for x > 0 (f(1) = l_K), 0 for x <= 0
    _, _, lk = P.poly_coeffs(1e-6)
    assert P.proj_poly(np.array([3.0]), 1e-6)[0] == pytest.approx(3.0 * 0.5 * (1 + lk), rel=1e-15)
    assert P.proj_poly(np.array([-3.0]), 1e-6)[0] == 0.0
    xs = [W.to_svec(W.sym_gaussian(rng, n)) for n in (3, 1, 8)]
    offs = np.cumsum([0] + [len(v) for v in xs])
    got = P.proj_poly_batched(np.concatenate(xs), offs, 1e-6)
    np.testing.assert_array_equal(got, np.concatenate([P.proj_poly(v, 1e-6) for v in xs]))


def _pins_hold(x, lam, exact):
    alphas, _ = P.poly_schedule(0.5, 1)
    t = np.linspace(0.5, 1.0, 4001)
    grid = np.linspace(1.0, math.sqrt(3.0), 2001)
    best = grid[int(np.argmin([np.max(np.abs(1 - cubic(a, t))) for a in grid]))]
    minimax_ok = abs(best - alphas[0]) <= 2e-3
    y = P.proj_poly(x, 1e-6)
    bound_ok = np.linalg.norm(y - exact) <= P.poly_error_bound(lam, 1e-6) * (1 + 1e-6) + 1e-12 * np.linalg.norm(exact)
    lj, V = oracle.eig(x)
    f = P.poly_scalar(lj / np.linalg.norm(lj), 1e-6)
    spectral_ok = rel(y, oracle.svec((V * (0.5 * lj * (1 + f))[None, :]) @ V.T)) <= 1e-12
    return minimax_ok, bound_ok, spectral_ok


@pytest.mark.parametrize("mutation", [1, 2, 3])
def test_planted_mistakes_fail_a_pin(mutation):
    """Each planted mistake in the oracle breaks at least one of the pins above."""
    rng = W.rng_for(7600)
    # scaled away from ||X||_F = 1, with eigenvalues near the resolution lo
    lam = 7.0 * np.concatenate([rng.uniform(1e-3, 1, 10), rng.uniform(-1, -1e-3, 10), [3e-6, -8e-6, 2e-5]])
    X, Q, _ = W.from_spectrum(rng, lam)
    x = W.to_svec(X)
    exact = W.to_svec((Q * np.maximum(lam, 0.0)[None, :]) @ Q.T)
    assert all(_pins_hold(x, lam, exact))
    P.set_mutation(mutation)
    try:
        held = _pins_hold(x, lam, exact)
    finally:
        P.set_mutation(0)
    assert not all(held)


@pytest.mark.parametrize("n,lo", [(6, 1e-3), (20, 1e-9)])
def test_hermitian_composite_against_lapack_eigh(n, lo):
    """Complex Hermitian cones: the matrix form equals the scalar composite
    applied to the eigenvalues of LAPACK's complex eigh (an independent
    evaluation), and real input reduces to the real composite."""
    rng = W.rng_for(7700 + n)
    lam = np.concatenate([rng.uniform(-1, 1, n - 2), [4e-8, -1e-6]])
    X, U, _ = W.herm_from_spectrum(rng, lam)
    x = W.to_hsvec(X)
    got = P.herm_proj_poly(x, lo)
    w, V = np.linalg.eigh(X)
    sigma = np.linalg.norm(w)
    f = P.poly_scalar(w / sigma, lo)
    want = W.to_hsvec((V * (0.5 * w * (1.0 + f))[None, :]) @ V.conj().T)
    assert rel(got, want) <= 1e-12
    # error bound against the exact projection (complex Jacobi oracle)
    assert np.linalg.norm(got - oracle.herm_proj(x)) <= P.poly_error_bound(lam, lo) + 1e-12 * np.linalg.norm(got)
    # a real symmetric matrix gives the real composite (embedded in the Hermitian layout)
    R = W.sym_gaussian(rng, n)
    yr = oracle.smat(P.proj_poly(W.to_svec(R), lo))
    np.testing.assert_allclose(oracle.herm_smat(P.herm_proj_poly(W.to_hsvec(R.astype(complex)), lo)), yr,
                               rtol=0, atol=1e-13 * np.abs(yr).max())
