"""Factorization-free approximate projection -- TEST INFRASTRUCTURE ONLY.

Only the test suite and the CPU legs of ``bench.py`` import this module; the
product path never does, and the two share no code.

Conclusions ("Approximate semidefinite-cone projections"): the exact
projection may be replaced by a composite matrix polynomial, built from
matrix-matrix products alone, whose scalar map reproduces the thresholding
t -> max(t, 0) of the eigenvalues.  The paper names the approach but prints
no polynomial.  Reading taken here:

* max(t, 0) = t (1 + sign t) / 2, so Pi(X) = (X + X sign(X)) / 2;
* sign is approximated on the spectrum of X / ||X||_F (inside [-1, 1]) by a
  scaled Newton-Schulz iteration.  On [l, 1] the odd cubic
  g(t) = (alpha t / 2)(3 - alpha^2 t^2), 1 <= alpha <= sqrt(3), rises to its
  maximum 1 at t = 1/alpha and falls to g(1) beyond it, so it maps [l, 1]
  into [min(g(l), g(1)), 1].  The minimax choice alpha^2 = 3 / (1 + l + l^2)
  (Chen & Chow 2014; g(l) = g(1)) sends the top of the interval down to the
  new lower bound, where the rounding of a low-precision product is
  amplified by about 1 / l; the scaling is therefore capped so that
  g(1) >= 1/2: alpha_k = min(sqrt(3 / (1 + l_k + l_k^2)), 2 cos(2 pi / 9)),
  2 cos(2 pi / 9) being the root of alpha (3 - alpha^2) / 2 = 1/2 in
  [1, sqrt(3)].  Either way g(l_k) <= g(1), so l_{k+1} = g_k(l_k).  Starting
  from l_0 = lo, the composite f = g_{K-1} o ... o g_0 satisfies
  |f(t) - sign t| <= 1 - l_K for lo <= |t| <= 1 and 0 <= f(t) sign(t) <= 1
  for all |t| <= 1;
* steps = 0 picks the smallest K with 1 - l_K <= 1e-15 (at most 200).

In matrix form one step is S <- a_k S + b_k S (S S) with a_k = 3 alpha_k / 2
and b_k = -alpha_k^3 / 2, from S_0 = X / ||X||_F (= X / ||x||_2 on svec,
svec being an isometry, App. D.1); X = 0 gives 0.  S is a symmetric matrix
function of X, and each step keeps it symmetric ((S + S^T) / 2 after the
product): a non-symmetric rounding residue is not a function of X, and the
iteration amplifies it.

Pins: ``tests/test_oracle_poly.py`` (the scaling against a brute-force
minimax search, the matrix form against the scalar composite applied to the
Jacobi eigendecomposition, diagonal inputs, the error bound against the exact
projection, exact homogeneity).
"""
from __future__ import annotations

import math

import numpy as np

from . import herm_smat, herm_svec, smat, svec

AUTO_TOL = 1e-15
MAX_STEPS = 200
ALPHA_CAP = 2.0 * math.cos(2.0 * math.pi / 9.0)  # alpha (3 - alpha^2) / 2 = 1/2

# A planted mistake (tests only): 1 drops the 1 + l^2 term of the scaling,
# 2 scales S_0 by ||X||_F^2, 3 flips the sign of X sign(X) in the output.
_mutation = 0


def set_mutation(m: int) -> None:
    """Plant a known mistake in this oracle (tests only); 0 restores it."""
    global _mutation
    _mutation = int(m)


def poly_schedule(lo: float, steps: int = 0):
    """Scalings alpha_k and lower bounds l_0 .. l_K of the composite (capped Chen & Chow 2014)."""
    if not (0.0 < lo < 1.0):
        raise ValueError("lo must lie in (0, 1)")
    if steps < 0 or steps > MAX_STEPS:
        raise ValueError("steps must lie in [0, 200]")
    alphas, lows = [], [float(lo)]
    l = float(lo)
    while True:
        if steps > 0 and len(alphas) == steps:
            break
        if steps == 0 and (1.0 - l <= AUTO_TOL or len(alphas) == MAX_STEPS):
            break
        alpha = min(math.sqrt(3.0 / (1.0 + l + (0.0 if _mutation == 1 else l * l))), ALPHA_CAP)
        l = 0.5 * alpha * l * (3.0 - alpha * alpha * l * l)
        alphas.append(alpha)
        lows.append(l)
    return alphas, lows


def poly_coeffs(lo: float, steps: int = 0):
    """(a_k, b_k) of S <- a_k S + b_k S^3 for every step, and the final lower bound l_K."""
    alphas, lows = poly_schedule(lo, steps)
    a = [1.5 * al for al in alphas]
    b = [-0.5 * al ** 3 for al in alphas]
    return a, b, lows[-1]


def poly_scalar(t, lo: float, steps: int = 0):
    """The composite f applied to numbers t in [-1, 1] (elementwise)."""
    a, b, _ = poly_coeffs(lo, steps)
    s = np.asarray(t, dtype=np.float64).copy()
    for ak, bk in zip(a, b):
        s = ak * s + bk * (s * (s * s))
    return s


def proj_poly_dense(X: np.ndarray, lo: float, steps: int = 0) -> np.ndarray:
    """(X + X f(X / ||X||_F)) / 2 of a dense symmetric matrix."""
    X = np.asarray(X, dtype=np.float64)
    sigma = math.sqrt(float(np.sum(X * X)))
    if sigma == 0.0:
        return np.zeros_like(X)
    a, b, _ = poly_coeffs(lo, steps)
    S = X / (sigma * sigma if _mutation == 2 else sigma)
    for ak, bk in zip(a, b):
        S = ak * S + bk * (S @ (S @ S))
        S = 0.5 * (S + S.T)
    return 0.5 * (X - X @ S) if _mutation == 3 else 0.5 * (X + X @ S)


def proj_poly(x, lo: float, steps: int = 0) -> np.ndarray:
    """The approximate projection on one svec cone."""
    x = np.asarray(x, dtype=np.float64)
    if x.size == 0:
        return x.copy()
    Y = proj_poly_dense(smat(x), lo, steps)
    return svec(0.5 * (Y + Y.T))


def proj_poly_batched(x, offsets, lo: float, steps: int = 0) -> np.ndarray:
    """proj_poly cone by cone on a packed buffer split by ``offsets``."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    for i in range(len(offsets) - 1):
        a, b = int(offsets[i]), int(offsets[i + 1])
        out[a:b] = proj_poly(x[a:b], lo, steps)
    return out


def herm_proj_poly(x, lo: float, steps: int = 0) -> np.ndarray:
    """The approximate projection of a complex Hermitian cone on its Hermitian
    svec: the same composite on X / ||X||_F (complex Frobenius norm), every
    iterate kept Hermitian, Y = (X + X S) / 2 (Conclusions: the construction
    acts on the spectrum only, so it carries over to Hermitian matrices)."""
    x = np.asarray(x, dtype=np.float64)
    if x.size == 0:
        return x.copy()
    X = herm_smat(x)
    sigma = math.sqrt(float(np.sum(np.abs(X) ** 2)))
    if sigma == 0.0:
        return np.zeros_like(x)
    a, b, _ = poly_coeffs(lo, steps)
    S = X / sigma
    for ak, bk in zip(a, b):
        S = ak * S + bk * (S @ (S @ S))
        S = 0.5 * (S + S.conj().T)
    Y = 0.5 * (X + X @ S)
    return herm_svec(0.5 * (Y + Y.conj().T))


def herm_proj_poly_batched(x, sides, lo: float, steps: int = 0) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    o = 0
    for n in sides:
        out[o:o + n * n] = herm_proj_poly(x[o:o + n * n], lo, steps)
        o += n * n
    return out


def poly_error_bound(lam, lo: float, steps: int = 0) -> float:
    """Frobenius bound on proj_poly - Pi for a matrix with eigenvalues lam.

    Per eigenvalue the error is |lam| |sign(lam) - f(lam / sigma)| / 2, at most
    |lam| / 2 below lo * sigma and |lam| (1 - l_K) / 2 above it."""
    lam = np.asarray(lam, dtype=np.float64)
    sigma = math.sqrt(float(np.sum(lam * lam)))
    if sigma == 0.0:
        return 0.0
    _, _, lk = poly_coeffs(lo, steps)
    small = np.abs(lam) < lo * sigma
    e2 = float(np.sum(lam[small] ** 2)) + (1.0 - lk) ** 2 * float(np.sum(lam[~small] ** 2))
    return 0.5 * math.sqrt(e2)
