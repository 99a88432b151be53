"""The SCS iteration around the PSD projection -- TEST INFRASTRUCTURE ONLY.

Only the test suite and the CPU legs of ``bench.py`` import this module; the
product path never does, and the two share no code.

App. D.1: SCS solves min c^T x s.t. A x + s = b, s in K (here K a product of
PSD cones in svec form) through the homogeneous self-dual embedding with
u = (x, y, tau), v = (r, s, kappa) and
    Q = [[0, A^T, c], [-A, 0, b], [-c^T, -b^T, 0]],
iterating (the paper's final iterates)
    u~ = (I + Q)^{-1} (u + v),
    u  = Pi_C(u~ - v),      C = R^k x K* x R_+  (K* = K, the PSD cone is self-dual),
    v  = v - u~ + u.
With M = [[I, A^T], [-A, I]] and h = (c, b), (I + Q)^{-1} w follows from
z = M^{-1} w_xy, p = M^{-1} h:  tau~ = (w_tau + h^T z) / (1 + h^T p),
(x~, y~) = z - tau~ p.  M^{-1}(a_x, a_y) solves (I + A^T A) z_x = a_x - A^T a_y,
z_y = a_y + A z_x; the paper's parametrization has A^T A = I (orthonormal
basis, App. D.3), so z_x = (a_x - A^T a_y) / 2 with one application of A
and one of A^T.

Reading taken: A is given as a dense matrix with orthonormal columns (the
paper applies it as Kronecker contractions of Gell-Mann bases, which are
out of scope here); no acceleration, over-relaxation or rescaling (the
paper's SCS adds them).  The PSD projection is the oracle's ``proj``.

Pins: ``tests/test_oracle_scs.py``.
"""
from __future__ import annotations

import numpy as np

from . import proj


def m_inverse(A, ax, ay):
    """M^{-1} (ax, ay) for A with orthonormal columns."""
    zx = 0.5 * (ax - A.T @ ay)
    zy = ay + A @ zx
    return zx, zy


def setup(A, b, c):
    """p = M^{-1} h and h^T p (computed once per problem)."""
    px, py = m_inverse(A, c, b)
    return px, py, float(c @ px + b @ py)


def project_cone(yv, offsets):
    """Pi onto the product of PSD cones (svec blocks split by offsets)."""
    out = np.empty_like(yv)
    for i in range(len(offsets) - 1):
        a, e = int(offsets[i]), int(offsets[i + 1])
        out[a:e] = proj(yv[a:e])
    return out


def iterate(A, b, c, offsets, u, v, iters: int):
    """``iters`` SCS iterations from (u, v); u, v = (x [k], y [m], tau [1])."""
    A = np.asarray(A, dtype=np.float64)
    m, k = A.shape
    u = np.asarray(u, dtype=np.float64).copy()
    v = np.asarray(v, dtype=np.float64).copy()
    px, py, hp = setup(A, b, c)
    for _ in range(iters):
        w = u + v
        zx, zy = m_inverse(A, w[:k], w[k:k + m])
        tau_t = (w[k + m] + c @ zx + b @ zy) / (1.0 + hp)
        ut = np.concatenate([zx - tau_t * px, zy - tau_t * py, [tau_t]])
        t = ut - v
        un = np.concatenate([t[:k], project_cone(t[k:k + m], offsets), [max(t[k + m], 0.0)]])
        v = v - ut + un
        u = un
    return u, v
