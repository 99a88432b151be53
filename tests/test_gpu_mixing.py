"""GPU parity of the positivity post-processing (App. C instrument mixing,
App. D process mixing): lambda_min per cone and the mixed blocks against the
oracle (Jacobi lambda_min, the paper's weight rule)."""
import numpy as np
import pytest

from oracle import mixing as M
from paper_2606_20519_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2606_20519_gb300 import _lib, build
    build.build()
    _lib.load()
    torch.cuda.init()
    return _lib


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def batch(seed, sides, shift=0.0):
    rng = W.rng_for(seed)
    return W.pack([W.to_svec(W.sym_gaussian(rng, n) + shift * np.eye(n)) for n in sides], sides)


@pytest.mark.parametrize("band", [0, 16])
def test_lambda_min_mixed_sides(lib, band):
    """One-stage (automatic) and two-stage (band 16) reductions; sides span
    the trivial case, small blocks, several tiles and a ragged tail."""
    sides = [1, 2, 5, 33, 64, 200, 625]
    b = batch(9800 + band, sides)
    opts = lib.make_opts(band=band) if band else None
    lam = lib.lambda_min(dev(b.x), b.sides, opts=opts).cpu().numpy()
    assert lib.status(0) == lib.OK
    want = M.lambda_min_batched(b.x, b.offsets)
    for i, n in enumerate(sides):
        Xn = np.abs(b.x[b.offsets[i]:b.offsets[i + 1]]).max() * n
        assert abs(lam[i] - want[i]) <= 1e-13 * max(1.0, Xn), (n, lam[i], want[i])


def test_lambda_min_constructions(lib):
    rng = W.rng_for(9810)
    lam0 = np.concatenate([rng.uniform(-1, 1, 99), [-1.25]])
    X, _, _ = W.from_spectrum(rng, lam0)
    d = rng.uniform(-2, 2, 40)
    b = W.pack([W.to_svec(X), W.to_svec(np.diag(d)), W.to_svec(np.zeros((7, 7)))], [100, 40, 7])
    lam = lib.lambda_min(dev(b.x), b.sides).cpu().numpy()
    assert abs(lam[0] + 1.25) <= 1e-13
    assert abs(lam[1] - d.min()) <= 1e-14
    assert abs(lam[2]) <= 1e-300


def test_mix_identity_instruments_and_process(lib):
    """Instrument groups (two outcomes, blocks of side d^2, nu = 1/(2d)) and a
    process matrix (one block, nu = gamma = 1/n), some of them PSD already."""
    rng = W.rng_for(9820)
    sides, svecs, groups, nu = [], [], [0], []
    for d, shift in ((2, 0.02), (3, 1.5), (4, 0.0), (8, 0.05)):
        for _ in range(2):
            n = d * d
            svecs.append(W.to_svec(0.1 * W.sym_gaussian(rng, n) + shift * np.eye(n)))
            sides.append(n)
        groups.append(len(sides))
        nu.append(1.0 / (2 * d))
    n = 625
    lamp = np.concatenate([rng.uniform(0, 0.01, n - 1), [-2e-4]])
    Wm, _, _ = W.from_spectrum(rng, lamp)
    svecs.append(W.to_svec(Wm))
    sides.append(n)
    groups.append(len(sides))
    nu.append(1.0 / n)
    b = W.pack(svecs, sides)
    eps = 1e-12
    y, p = lib.mix_identity(dev(b.x), b.sides, groups, nu, eps)
    assert lib.status(0) == lib.OK
    y, p = y.cpu().numpy(), p.cpu().numpy()
    wy, wp = M.mix_identity(b.x, b.offsets, groups, nu, eps)
    np.testing.assert_allclose(p, wp, rtol=1e-11, atol=1e-14)
    assert wp[1] == 1.0 and p[1] == 1.0  # the PSD group is left alone
    np.testing.assert_allclose(y, wy, rtol=0, atol=1e-13)
    # in place
    xt = dev(b.x)
    lib.mix_identity(xt, b.sides, groups, nu, eps, out=xt)
    np.testing.assert_allclose(xt.cpu().numpy(), wy, rtol=0, atol=1e-13)


def test_errors_and_nonfinite(lib):
    import torch
    b = batch(9830, [4, 6])
    x = b.x.copy()
    x[2] = np.nan
    y, p = lib.mix_identity(dev(x), b.sides, [0, 1, 2], [0.25, 0.25], 1e-12)
    assert lib.status(0) == lib.ENONFINITE
    p = p.cpu().numpy()
    assert np.isnan(p[0]) and not np.isnan(p[1])
    assert np.all(np.isnan(y.cpu().numpy()[:b.offsets[1]]))
    xt = dev(b.x)
    for groups in ([0, 1], [1, 2], [0, 2, 1, 2]):
        with pytest.raises(lib.ScsPsdError):
            lib.mix_identity(xt, b.sides, groups, [0.25] * (len(groups) - 1), 1e-12)
    with pytest.raises(lib.ScsPsdError):
        lib.lambda_min(torch.zeros(1, dtype=torch.float64, device="cuda"), [0, 1])
