"""Pins of the complex Hermitian oracle (oracle.herm_proj): what the
definition Pi(X) = V diag(max(lambda, 0)) V^H and the mathematics fix,
independently of the oracle's own complex Jacobi arithmetic."""
import numpy as np
import pytest

import oracle
from paper_2606_20519_gb300 import workloads as W


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def real_svec_to_herm_svec(x):
    """The real symmetric svec of a cone rewritten as a Hermitian svec with zero imaginary parts."""
    n = oracle.side_of(x.size)
    A = oracle.smat(x)
    return W.to_hsvec(A.astype(np.complex128))


def test_hsvec_roundtrip_and_isometry():
    rng = W.rng_for(61)
    for n in (1, 2, 5, 9):
        A, B = W.herm_gaussian(rng, n), W.herm_gaussian(rng, n)
        a, b = oracle.herm_svec(A), oracle.herm_svec(B)
        assert np.array_equal(a, W.to_hsvec(A))
        assert np.allclose(oracle.herm_smat(a), A, atol=1e-15)
        # <svec A, svec B> = Re tr(A B) (the vec map is an isometry, App. D.1)
        assert abs(a @ b - np.trace(A @ B).real) <= 1e-12 * max(1.0, abs(a @ b))


def test_real_symmetric_special_case_matches_real_oracle():
    rng = W.rng_for(62)
    for n in (2, 7, 20):
        x = W.to_svec(W.sym_gaussian(rng, n))
        yr = oracle.proj(x)
        yh = oracle.herm_proj(real_svec_to_herm_svec(x))
        assert rel(yh, real_svec_to_herm_svec(yr)) <= 1e-13


def test_two_by_two_closed_form():
    rng = W.rng_for(63)
    for _ in range(100):
        a, d = rng.normal(size=2)
        b = complex(*rng.normal(size=2))
        H = np.array([[a, b], [np.conj(b), d]])
        r = np.sqrt(((a - d) / 2) ** 2 + abs(b) ** 2)
        l1, l2 = (a + d) / 2 + r, (a + d) / 2 - r
        # eigenvector of l1: (b, l1 - a) normalised (or e1 when b = 0 and a >= d)
        v = np.array([b, l1 - a]) if abs(b) > 0 else np.array([1.0, 0.0])
        v = v / np.linalg.norm(v)
        P1 = np.outer(v, v.conj())
        expect = max(l1, 0.0) * P1 + max(l2, 0.0) * (np.eye(2) - P1)
        y = oracle.herm_smat(oracle.herm_proj(W.to_hsvec(H)))
        assert np.allclose(y, expect, atol=1e-13)


def test_construction_with_haar_unitary():
    rng = W.rng_for(64)
    for n in (5, 16, 40):
        lam = np.concatenate([rng.uniform(0.1, 2, n // 2), rng.uniform(-2, -0.1, n - n // 2)])
        X, U, lam = W.herm_from_spectrum(rng, lam)
        exact = W.to_hsvec((U * np.maximum(lam, 0)) @ U.conj().T)
        assert rel(oracle.herm_proj(W.to_hsvec(X)), exact) <= 1e-12
        assert rel(oracle.herm_proj(W.to_hsvec(X), route=1), exact) <= 1e-12


def test_moreau_idempotence_psd_and_lapack_witness():
    rng = W.rng_for(65)
    n = 12
    X = W.herm_gaussian(rng, n)
    x = W.to_hsvec(X)
    p, m = oracle.herm_proj(x), oracle.herm_proj(-x)
    assert rel(p - m, x) <= 1e-13                 # X = Pi(X) - Pi(-X)
    assert abs(p @ m) <= 1e-12 * np.linalg.norm(p) * np.linalg.norm(m)  # <Pi(X), Pi(-X)> = 0
    assert rel(oracle.herm_proj(p), p) <= 1e-13    # idempotent
    assert np.linalg.eigvalsh(oracle.herm_smat(p)).min() >= -1e-12 * np.linalg.norm(p)
    w, V = np.linalg.eigh(X)                       # LAPACK as a third witness
    assert rel(p, W.to_hsvec((V * np.maximum(w, 0)) @ V.conj().T)) <= 1e-12


def test_unitary_equivariance_and_homogeneity():
    rng = W.rng_for(66)
    n = 10
    X = W.herm_gaussian(rng, n)
    D = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, n)))
    lhs = oracle.herm_smat(oracle.herm_proj(W.to_hsvec(D @ X @ D.conj().T)))
    rhs = D @ oracle.herm_smat(oracle.herm_proj(W.to_hsvec(X))) @ D.conj().T
    assert np.allclose(lhs, rhs, atol=1e-13)
    x = W.to_hsvec(X)
    assert np.array_equal(oracle.herm_proj(4.0 * x), 4.0 * oracle.herm_proj(x))


def test_brute_force_side_one_and_thread_independence():
    for v in (-1.5, 0.0, 2.25):
        assert oracle.herm_proj(np.array([v]))[0] == max(v, 0.0)
    rng = W.rng_for(67)
    x = W.to_hsvec(W.herm_gaussian(rng, 33))
    t0 = oracle.max_threads()
    oracle.set_threads(1)
    a = oracle.herm_proj(x)
    oracle.set_threads(t0)
    b = oracle.herm_proj(x)
    assert np.array_equal(a, b)
