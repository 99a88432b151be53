"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Tolerance: relative Frobenius error 1e-10 for the FP64 path (measured on
svec, which has the matrix's Frobenius norm because vec_R is an isometry).
Full-size cases the oracle cannot finish in seconds are checked against the
exact projection of their construction X = Q diag(lam) Q^T, whose value the
oracle is pinned to on smaller sizes, and against properties that hold at
any size (Moreau decomposition, positive semidefiniteness).
"""
import numpy as np
import pytest

import oracle
from paper_2606_20519_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2606_20519_gb300 import _lib, build
    build.build()
    _lib.load()
    torch.cuda.init()
    return _lib


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def gpu_proj_batched(lib, x, sides, **kw):
    xt = to_dev(x)
    y = lib.proj_batched(xt, sides, opts=lib.make_opts(**kw) if kw else None)
    st = lib.status(0)
    return y.cpu().numpy(), st


@pytest.mark.parametrize("n", [2, 3, 4, 5, 9, 16, 17, 18, 33, 40, 64, 81, 100, 130])
def test_random_symmetric_vs_oracle(lib, n):
    rng = W.rng_for(1000 + n)
    X = W.sym_gaussian(rng, n) + rng.uniform(-0.5, 0.5) * np.eye(n)
    x = W.to_svec(X)
    y, st = gpu_proj_batched(lib, x, [n])
    assert st == lib.OK
    assert rel(y, oracle.proj(x)) <= TOL


@pytest.mark.parametrize("band", [2, 4, 8, 16, 32])
def test_bandwidths(lib, band):
    rng = W.rng_for(2000 + band)
    n = 150
    X, Q, lam = W.from_spectrum(rng, W.spectrum_precision(rng, n))
    x = W.to_svec(X)
    y, st = gpu_proj_batched(lib, x, [n], band=band)
    assert st == lib.OK
    assert rel(y, oracle.proj(x)) <= TOL


def test_single_projection_workload(lib):
    x, Q, lam = W.single_projection()
    y, st = gpu_proj_batched(lib, x, [81])
    assert st == lib.OK
    assert rel(y, oracle.proj(x)) <= TOL


@pytest.mark.parametrize("maker", [W.spectrum_admm, W.spectrum_precision, W.spectrum_vjp, W.spectrum_plain])
def test_clustered_spectra(lib, maker):
    rng = W.rng_for(3000)
    n = 200
    X, Q, lam = W.from_spectrum(rng, maker(rng, n))
    x = W.to_svec(X)
    y, st = gpu_proj_batched(lib, x, [n])
    assert st == lib.OK
    assert rel(y, oracle.proj(x)) <= TOL


def test_uneven_batch_small(lib):
    b = W.uneven_batch(restarts=3, big_sides=(100, 130))
    y, st = gpu_proj_batched(lib, b.x, b.sides)
    assert st == lib.OK
    ref = oracle.proj_batched(b.x, b.offsets)
    for i in range(b.count):
        a, e = b.offsets[i], b.offsets[i + 1]
        assert rel(y[a:e], ref[a:e]) <= TOL, (i, b.sides[i])


def test_degenerate_cases(lib):
    import torch
    # sides 0 and 1 mixed with real cones; in place (y aliases x)
    sides = [1, 0, 3, 1, 2]
    rng = W.rng_for(4000)
    parts = []
    for n in sides:
        parts.append(W.to_svec(W.sym_gaussian(rng, n)) if n else np.zeros(0))
    x = np.concatenate(parts)
    x[0] = -1.5
    x[7] = 2.0
    ref = oracle.proj_batched(x, lib.shapes(sides)[0])
    xt = to_dev(x)
    lib.proj_batched(xt, sides, out=xt)
    assert lib.status(0) == lib.OK
    np.testing.assert_allclose(xt.cpu().numpy(), ref, rtol=0, atol=1e-13)
    # zero, PSD and NSD matrices
    n = 20
    G = rng.standard_normal((n, n))
    for X, want in ((np.zeros((n, n)), np.zeros((n, n))), (G @ G.T, G @ G.T), (-(G @ G.T), np.zeros((n, n)))):
        y, st = gpu_proj_batched(lib, W.to_svec(X), [n])
        assert st == lib.OK
        assert np.linalg.norm(y - W.to_svec(want)) <= 1e-12 * max(1.0, np.linalg.norm(X))


def test_nonfinite_input_reports_and_fills_nan(lib):
    rng = W.rng_for(5000)
    sides = [5, 6]
    x = np.concatenate([W.to_svec(W.sym_gaussian(rng, n)) for n in sides])
    x[3] = np.inf
    y, st = gpu_proj_batched(lib, x, sides)
    assert st == lib.ENONFINITE
    assert np.all(np.isnan(y[:15]))
    assert rel(y[15:], oracle.proj(x[15:])) <= TOL
    # the next clean call reports OK again
    y, st = gpu_proj_batched(lib, x[15:], [6])
    assert st == lib.OK


def test_explicit_sides_agree(lib):
    rng = W.rng_for(6000)
    n = 90
    x = W.to_svec(W.sym_gaussian(rng, n))
    ref = oracle.proj(x)
    for side in (1, 2):
        y, st = gpu_proj_batched(lib, x, [n], side=side)
        assert st == lib.OK
        assert rel(y, ref) <= TOL


def test_repeatable_bitwise(lib):
    rng = W.rng_for(7000)
    n = 120
    x = W.to_svec(W.sym_gaussian(rng, n))
    y1, _ = gpu_proj_batched(lib, x, [n])
    y2, _ = gpu_proj_batched(lib, x, [n])
    np.testing.assert_array_equal(y1, y2)


def test_single_entry_point(lib):
    import torch
    x, Q, lam = W.single_projection()
    xt = to_dev(x)
    y = lib.proj(xt, 81)
    assert lib.status(0) == lib.OK
    assert rel(y.cpu().numpy(), oracle.proj(x)) <= TOL
    assert lib.last_launch_count(0) > 0


def test_admm_sequence_625_first_steps(lib):
    seq, Q, lam = W.admm_sequence(steps=3)
    for x in seq:
        y, st = gpu_proj_batched(lib, x, [625])
        assert st == lib.OK
        assert rel(y, oracle.proj(x)) <= TOL


def test_precision_4096_construction(lib):
    # full size: checked against the construction's exact projection, and
    # by the Moreau decomposition with the projection of -X
    import torch
    b = W.precision_batch(batch=1)
    x = b.x
    Q, lam = b.extra["Q"][0], b.extra["lam"][0]
    y, st = gpu_proj_batched(lib, x, [4096])
    assert st == lib.OK
    P = (Q * np.maximum(lam, 0)) @ Q.T
    assert rel(y, W.to_svec(P)) <= TOL
    yn, st = gpu_proj_batched(lib, -x, [4096])
    assert np.linalg.norm(y - yn - x) <= TOL * np.linalg.norm(x)


@pytest.mark.parametrize("n", [256, 300, 401, 640, 660])
def test_medium_sides_vs_oracle(lib, n):
    """Lone cones between the one-CTA sizes and the ADMM side, on the
    ADMM-like spectrum (48 % clustered at zero): 401 leaves some CTAs of the
    group a column more than the others."""
    rng = W.rng_for(8100 + n)
    X, Q, lam = W.from_spectrum(rng, W.spectrum_admm(rng, n))
    x = W.to_svec(X)
    y, st = gpu_proj_batched(lib, x, [n])
    assert st == lib.OK
    assert rel(y, oracle.proj(x)) <= TOL


def test_few_large_cones_with_small_ones_in_place(lib):
    """Three large cones sharing the one-stage launch beside small cones on
    the one-CTA route, in place."""
    rng = W.rng_for(8200)
    sides = [300, 7, 520, 33, 640]
    x = np.concatenate([W.to_svec(W.sym_gaussian(rng, n) + rng.uniform(-0.5, 0.5) * np.eye(n)) for n in sides])
    ref = oracle.proj_batched(x, lib.shapes(sides)[0])
    xt = to_dev(x)
    lib.proj_batched(xt, sides, out=xt)
    assert lib.status(0) == lib.OK
    y = xt.cpu().numpy()
    offs = lib.shapes(sides)[0]
    for i, n in enumerate(sides):
        assert rel(y[offs[i]:offs[i + 1]], ref[offs[i]:offs[i + 1]]) <= TOL, n


def test_medium_side_nonfinite_then_repeatable(lib):
    """A NaN in a side-320 cone gives SCS_PSD_ENONFINITE and a NaN output;
    the next clean calls are correct and bit-for-bit equal."""
    rng = W.rng_for(8300)
    n = 320
    x = W.to_svec(W.sym_gaussian(rng, n))
    bad = x.copy()
    bad[1000] = np.nan
    y, st = gpu_proj_batched(lib, bad, [n])
    assert st == lib.ENONFINITE
    assert np.all(np.isnan(y))
    y1, st = gpu_proj_batched(lib, x, [n])
    assert st == lib.OK
    y2, _ = gpu_proj_batched(lib, x, [n])
    np.testing.assert_array_equal(y1, y2)
    assert rel(y1, oracle.proj(x)) <= TOL
