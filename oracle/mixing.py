"""Positivity post-processing by mixing with a multiple of the identity --
TEST INFRASTRUCTURE ONLY.

Only the test suite and the CPU legs of ``bench.py`` import this module; the
product path never does, and the two share no code.

App. C (instrument step): the outcome blocks C_{a|x} of one input x are
mixed with the white-noise instrument N_{a|x} = (1/n_a) 1 (x) 1/d_Ao, whose
every eigenvalue is nu = 1/(n_a d_Ao):
    C~_{a|x} = p_x C_{a|x} + (1 - p_x) N_{a|x},
one p_x for all outcomes, so the trace-preserving constraint survives.  With
lambda_a = lambda_min(C_{a|x}): p_x = 1 if min_a lambda_a >= 0, otherwise
    p_x = min over the a with lambda_a < eps of (nu - eps) / (nu - lambda_a),
which makes lambda_min(C~_{a|x}) = p_x lambda_a + (1 - p_x) nu >= eps for all
a, with equality for the minimizing a.
App. D (process matrix): W' = (1 - l) W + l gamma 1 with the smallest l in
[0, 1] for which W' is PSD up to the tolerance -- the same rule with one
block, nu = gamma and p = 1 - l.

Reading taken: a group is the list of blocks that share one p (the outcomes
of one input, or a single process matrix), nu is given per group, and the
mixture adds (1 - p) nu to the diagonal; the paper's condition "min_a
lambda_a >= 0" decides p = 1 exactly as printed (blocks with 0 <= lambda_a <
eps are then left as they are).  lambda_min comes from the Jacobi oracle.

Pins: ``tests/test_oracle_mixing.py``.
"""
from __future__ import annotations

import numpy as np

from . import eig, smat, svec


def lambda_min(x) -> float:
    """Smallest eigenvalue of smat(x) (cyclic Jacobi)."""
    x = np.asarray(x, dtype=np.float64)
    if x.size == 1:
        return float(x[0])
    lam, _ = eig(x)
    return float(np.min(lam))


def lambda_min_batched(x, offsets) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return np.array([lambda_min(x[int(offsets[i]):int(offsets[i + 1])]) for i in range(len(offsets) - 1)])


def mixing_weight(lams, nu: float, eps: float) -> float:
    """p of one group from its blocks' smallest eigenvalues (App. C)."""
    lams = np.asarray(lams, dtype=np.float64)
    if np.min(lams) >= 0.0:
        return 1.0
    return float(min((nu - eps) / (nu - la) for la in lams if la < eps))


def mix_identity(x, offsets, groups, nu, eps: float):
    """(y, p): every block of group g becomes p_g C + (1 - p_g) nu_g 1 (svec)."""
    x = np.asarray(x, dtype=np.float64)
    y = x.copy()
    lam = lambda_min_batched(x, offsets)
    ps = []
    for g in range(len(groups) - 1):
        blocks = range(int(groups[g]), int(groups[g + 1]))
        p = mixing_weight([lam[i] for i in blocks], float(nu[g]), eps)
        ps.append(p)
        for i in blocks:
            a, b = int(offsets[i]), int(offsets[i + 1])
            C = smat(x[a:b])
            n = C.shape[0]
            y[a:b] = svec(p * C + (1.0 - p) * float(nu[g]) * np.eye(n))
    return y, np.array(ps)
