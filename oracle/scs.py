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

Reading taken: A has orthonormal columns and is given either as a dense
matrix or, as the paper applies it (App. D.2), as a structured operator whose
columns are svec of Kronecker products of local basis matrices
(``kron_apply``, ``kron_apply_t``); no acceleration, over-relaxation or
rescaling (the paper's SCS adds them).  The PSD projection is the oracle's
``proj``.

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


# ---- structured affine operator.  App. D.2 applies A x and A^T y as tensor
# contractions over local bases, never forming the Kronecker products
# F_mu = F1[mu_1] (x) ... (x) FS[mu_S].  Here column j of A is svec(F_mu) for
# the multi-index mu = unravel(index[j]) (C order over the local basis sizes),
# with np.kron's convention for the tensor product (mode 1 the slowest).  The
# checks form the columns explicitly (kron_columns) and contract them
# (kron_apply, kron_apply_t); the two are independent evaluations.
def kron_columns(bases, index):
    """Dense m x k matrix whose column j is svec(F_{mu_j})."""
    from . import svec
    shape = [len(B) for B in bases]
    cols = []
    for flat in np.asarray(index, dtype=np.int64):
        mu = np.unravel_index(int(flat), shape)
        F = np.ones((1, 1))
        for B, a in zip(bases, mu):
            F = np.kron(F, np.asarray(B[a], dtype=np.float64))
        cols.append(svec(F))
    return np.stack(cols, axis=1)


def _kron_subscripts(S):
    letters = "abcdefghijklmnopqrstuvwxyz"
    t, r, c = letters[:S], letters[S:2 * S], letters[2 * S:3 * S]
    return t, r, c


def kron_apply(bases, index, x):
    """svec(sum_j x_j F_{mu_j}) by contraction over the local bases."""
    from . import svec
    S = len(bases)
    shape = [len(B) for B in bases]
    N = int(np.prod([np.asarray(B).shape[1] for B in bases]))
    T = np.zeros(int(np.prod(shape)))
    T[np.asarray(index, dtype=np.int64)] = np.asarray(x, dtype=np.float64)
    t, r, c = _kron_subscripts(S)
    spec = t + "," + ",".join(t[s] + r[s] + c[s] for s in range(S)) + "->" + r + c
    W = np.einsum(spec, T.reshape(shape), *[np.asarray(B, dtype=np.float64) for B in bases], optimize="greedy")
    return svec(W.reshape(N, N))


def kron_apply_t(bases, index, y):
    """(<F_{mu_j}, smat(y)>)_j by contraction over the local bases."""
    from . import smat
    S = len(bases)
    dims = [np.asarray(B).shape[1] for B in bases]
    Y = smat(np.asarray(y, dtype=np.float64)).reshape(dims + dims)
    t, r, c = _kron_subscripts(S)
    spec = r + c + "," + ",".join(t[s] + r[s] + c[s] for s in range(S)) + "->" + t
    T = np.einsum(spec, Y, *[np.asarray(B, dtype=np.float64) for B in bases], optimize="greedy")
    return T.reshape(-1)[np.asarray(index, dtype=np.int64)]


def iterate_kron(bases, index, b, c, offsets, u, v, iters: int):
    """``iterate`` with A applied as the structured operator (orthonormal
    columns: orthonormal local bases and symmetric F_mu)."""
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    k, m = len(index), b.size
    u = np.asarray(u, dtype=np.float64).copy()
    v = np.asarray(v, dtype=np.float64).copy()

    def m_inv(ax, ay):
        zx = 0.5 * (ax - kron_apply_t(bases, index, ay))
        return zx, ay + kron_apply(bases, index, zx)

    px, py = m_inv(c, b)
    hp = float(c @ px + b @ py)
    for _ in range(iters):
        w = u + v
        zx, zy = m_inv(w[:k], w[k:k + m])
        tau_t = (w[k + m] + c @ zx + b @ zy) / (1.0 + hp)
        ut = np.concatenate([zx - tau_t * px, zy - tau_t * py, [tau_t]])
        t = ut - v
        un = np.concatenate([t[:k], project_cone(t[k:k + m], offsets), [max(t[k + m], 0.0)]])
        v = v - ut + un
        u = un
    return u, v
