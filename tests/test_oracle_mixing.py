"""Pins for the oracle of the positivity post-processing (no GPU).

App. C mixes the outcome blocks of one instrument input with white noise
(App. D: a process matrix with the trivial process) using the largest weight
p that keeps every block PSD up to eps.  The oracle is checked against
LAPACK's eigenvalues, a brute-force search over p, the guarantee the paper
states (lambda_min of every mixed block >= eps, equality for one of them), and
the preserved partial-trace (trace-preserving) identity."""
import numpy as np
import pytest

import oracle
from oracle import mixing as M
from paper_2606_20519_gb300 import workloads as W


def test_lambda_min_against_lapack_and_constructions():
    rng = W.rng_for(7800)
    for n in (1, 2, 5, 30):
        A = W.sym_gaussian(rng, n)
        got = M.lambda_min(W.to_svec(A))
        assert abs(got - np.linalg.eigvalsh(A)[0]) <= 1e-13 * max(1.0, np.abs(A).max() * n)
    d = rng.uniform(-1, 1, 12)
    assert M.lambda_min(W.to_svec(np.diag(d))) == d.min()
    lam = np.concatenate([rng.uniform(-1, 1, 19), [-1.5]])
    X, _, _ = W.from_spectrum(rng, lam)
    assert abs(M.lambda_min(W.to_svec(X)) + 1.5) <= 1e-13


def _partial_trace_out(C, d_in, d_out):
    """tr over the output factor of a (d_in d_out) x (d_in d_out) matrix."""
    return np.einsum("iaja->ij", C.reshape(d_in, d_out, d_in, d_out))


def _instrument_group(rng, d, n_a, shift):
    """n_a random symmetric outcome blocks of side d^2 (d_Ai = d_Ao = d)."""
    blocks = []
    for _ in range(n_a):
        G = W.sym_gaussian(rng, d * d) * 0.1
        blocks.append(G + shift * np.eye(d * d))
    return blocks


@pytest.mark.parametrize("d,n_a", [(2, 2), (3, 3), (4, 2)])
def test_instrument_mixing_guarantee_and_trace(d, n_a):
    rng = W.rng_for(7810 + d)
    eps = 1e-12
    nu = 1.0 / (n_a * d)
    blocks = _instrument_group(rng, d, n_a, shift=0.05)
    x = np.concatenate([W.to_svec(B) for B in blocks])
    offs = np.cumsum([0] + [len(W.to_svec(B)) for B in blocks])
    y, p = M.mix_identity(x, offs, [0, n_a], [nu], eps)
    lams = [np.linalg.eigvalsh(B)[0] for B in blocks]
    assert min(lams) < 0  # the group needs mixing
    mixed = [oracle.smat(y[offs[i]:offs[i + 1]]) for i in range(n_a)]
    mins = [np.linalg.eigvalsh(Bm)[0] for Bm in mixed]
    assert min(mins) >= eps - 1e-13
    assert abs(min(mins) - eps) <= 1e-13  # equality for the worst outcome
    # brute force: the largest p on a fine grid that keeps every block >= eps
    grid = np.linspace(0, 1, 20001)
    ok = [q for q in grid if all(np.linalg.eigvalsh(q * B + (1 - q) * nu * np.eye(d * d))[0] >= eps for B in blocks)]
    assert abs(max(ok) - p[0]) <= 1e-4
    # the partial trace over the output is mixed the same way (trace preservation)
    s_in = sum(_partial_trace_out(B, d, d) for B in blocks)
    s_out = sum(_partial_trace_out(Bm, d, d) for Bm in mixed)
    np.testing.assert_allclose(s_out, p[0] * s_in + (1 - p[0]) * np.eye(d), atol=1e-13)


def test_psd_group_is_left_alone_and_process_case():
    rng = W.rng_for(7820)
    d = 3
    blocks = _instrument_group(rng, d, 2, shift=2.0)
    x = np.concatenate([W.to_svec(B) for B in blocks])
    offs = np.cumsum([0] + [len(W.to_svec(B)) for B in blocks])
    y, p = M.mix_identity(x, offs, [0, 2], [1.0 / 6.0], 1e-12)
    assert p[0] == 1.0
    np.testing.assert_array_equal(y, x)
    # process matrix: W' = (1 - l) W + l gamma 1, l = 1 - p, lambda_min(W') = eps
    n = 16
    lam = np.concatenate([rng.uniform(0, 0.2, n - 1), [-0.03]])
    Wm, _, _ = W.from_spectrum(rng, lam)
    gamma = 1.0 / n
    y, p = M.mix_identity(W.to_svec(Wm), [0, n * (n + 1) // 2], [0, 1], [gamma], 1e-12)
    assert abs(p[0] - (gamma - 1e-12) / (gamma + 0.03)) <= 1e-14
    assert abs(np.linalg.eigvalsh(oracle.smat(y))[0] - 1e-12) <= 1e-14
