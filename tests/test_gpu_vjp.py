"""GPU parity of the Daleckii-Krein VJP (scs_psd_proj_vjp) against the FP64
oracle's derivative, central differences and identities that hold at any
size (positive homogeneity gives J[X] = Pi(X); J is symmetric in svec
coordinates; J[Pi(X)] = Pi(X)).

Tolerances: 1e-10 relative on spectra whose opposite-sign eigenvalues are
well separated.  When eigenvalues +-delta straddle zero, the cross block of
the Loewner matrix is fixed by any backward-stable eigensolver only to about
eps * ||X||_2 / (2 delta), so the stress case uses a tolerance derived from
that conditioning bound."""
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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def vjp(lib, x, g, sides, want_y=False):
    import torch
    xt, gt = dev(x), dev(g)
    y = torch.empty_like(xt) if want_y else None
    xb = lib.proj_vjp(xt, gt, sides, y=y)
    st = lib.status(0)
    return xb.cpu().numpy(), (y.cpu().numpy() if want_y else None), st


@pytest.mark.parametrize("n", [2, 7, 40, 64, 100])
def test_vjp_vs_oracle_separated(lib, n):
    rng = W.rng_for(8000 + n)
    X, Q, lam = W.from_spectrum(rng, W.spectrum_vjp(rng, n, cluster=1e-3))
    x = W.to_svec(X)
    g = rng.standard_normal(x.size)
    xb, y, st = vjp(lib, x, g, [n], want_y=True)
    assert st == lib.OK
    assert rel(xb, oracle.jvp(x, g)) <= TOL
    assert rel(y, oracle.proj(x)) <= TOL


def test_vjp_batched_uneven(lib):
    b = W.uneven_batch(restarts=2, small_sides=(4, 9, 16), copies=1, big_sides=(50,))
    rng = W.rng_for(8100)
    g = rng.standard_normal(b.x.size)
    xb, _, st = vjp(lib, b.x, g, b.sides)
    assert st == lib.OK
    ref = oracle.jvp_batched(b.x, g, b.offsets)
    for i in range(b.count):
        s, e = b.offsets[i], b.offsets[i + 1]
        assert rel(xb[s:e], ref[s:e]) <= TOL


def test_vjp_matches_central_differences_of_gpu_projection(lib):
    rng = W.rng_for(8200)
    n = 60
    X, Q, lam = W.from_spectrum(rng, W.spectrum_vjp(rng, n, cluster=1e-3))
    x = W.to_svec(X)
    g = rng.standard_normal(x.size)
    h = 1e-6
    yp = lib.proj_batched(dev(x + h * g), [n]).cpu().numpy()
    ym = lib.proj_batched(dev(x - h * g), [n]).cpu().numpy()
    fd = (yp - ym) / (2 * h)
    xb, _, st = vjp(lib, x, g, [n])
    assert st == lib.OK
    assert rel(xb, fd) <= 1e-6


def test_vjp_stress_clusters_conditioning_tolerance(lib):
    rng = W.rng_for(8300)
    n = 130
    X, Q, lam = W.from_spectrum(rng, W.spectrum_vjp(rng, n, cluster=1e-9))
    x = W.to_svec(X)
    g = rng.standard_normal(x.size)
    xb, _, st = vjp(lib, x, g, [n])
    assert st == lib.OK
    ref = oracle.jvp(x, g)
    delta = 2e-9                      # smallest gap between opposite-sign eigenvalues
    bound = 10 * n * np.finfo(float).eps * np.abs(lam).max() / delta
    assert rel(xb, ref) <= bound


def test_full_size_identities(lib):
    # n = 1296 (d = 6), batch 8, the +-1e-9 stress spectrum: identities only
    b = W.vjp_batch(batch=8)
    x = b.x
    xb_euler, y, st = vjp(lib, x, x, b.sides, want_y=True)
    assert st == lib.OK
    for i in range(b.count):
        s, e = b.offsets[i], b.offsets[i + 1]
        Q, lam = b.extra["Q"][i], b.extra["lam"][i]
        P = W.to_svec((Q * np.maximum(lam, 0)) @ Q.T)
        assert rel(y[s:e], P) <= TOL                      # forward value
        assert rel(xb_euler[s:e], y[s:e]) <= TOL          # J[X] = Pi(X)
    rng = W.rng_for(8400)
    a, c = rng.standard_normal(x.size), rng.standard_normal(x.size)
    Ja, _, _ = vjp(lib, x, a, b.sides)
    Jc, _, _ = vjp(lib, x, c, b.sides)
    for i in range(b.count):
        s, e = b.offsets[i], b.offsets[i + 1]
        lhs, rhs = a[s:e] @ Jc[s:e], Ja[s:e] @ c[s:e]
        assert abs(lhs - rhs) <= 1e-10 * np.linalg.norm(a[s:e]) * np.linalg.norm(c[s:e])
        q = a[s:e] @ Ja[s:e]
        assert -1e-10 * (a[s:e] @ a[s:e]) <= q <= (a[s:e] @ a[s:e]) * (1 + 1e-10)


def test_autograd_wrapper(lib):
    import torch
    from paper_2606_20519_gb300.autograd import psd_project
    rng = W.rng_for(8500)
    sides = [5, 12]
    x = np.concatenate([W.to_svec(W.sym_gaussian(rng, n)) for n in sides])
    xt = dev(x).requires_grad_(True)
    y = psd_project(xt, sides)
    g = rng.standard_normal(x.size)
    (y * dev(g)).sum().backward()
    offs = lib.shapes(sides)[0]
    np.testing.assert_allclose(y.detach().cpu().numpy(), oracle.proj_batched(x, offs), rtol=0, atol=1e-12)
    ref = oracle.jvp_batched(x, g, offs)
    assert rel(xt.grad.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("side", [1, 2])
def test_vjp_both_routes(lib, side):
    """The block-structured derivative takes the positive pairs (route 0) or
    the non-positive ones (route 1) as its small side; both give DPi."""
    import torch
    n = 90
    rng = W.rng_for(8900 + side)
    # more positive than negative eigenvalues, so the automatic route would be 1;
    # none near zero, where Pi is not differentiable
    lam = np.concatenate([rng.uniform(0.01, 1, 60), rng.uniform(-1, -0.01, 30)])
    X, Q, lam = W.from_spectrum(rng, lam)
    x = W.to_svec(X)
    g = rng.standard_normal(x.size)
    y = torch.empty(x.size, dtype=torch.float64, device="cuda")
    xb = lib.proj_vjp(dev(x), dev(g), [n], y=y, opts=lib.make_opts(side=side))
    assert lib.status(0) == lib.OK
    assert rel(xb.cpu().numpy(), oracle.jvp(x, g)) <= TOL
    assert rel(y.cpu().numpy(), oracle.proj(x)) <= TOL
