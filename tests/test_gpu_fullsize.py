"""GPU parity at the workloads' full sizes, element by element against the
FP64 oracle, for the paths the measured configurations run:

* the derivative of a side-1296 cone (the differentiation workload's size,
  its +-1e-9 clusters moved to +-1e-3 so that the Loewner matrix is well
  conditioned, as the reading of App. E's derivative requires for 1e-10
  parity), in FP64 at 1e-10 and in the split precision at the split bound;
  at this size every product of the split derivative runs on the
  long-contraction kernel (K >= 256);
* the split derivative at n = 300, the smallest side whose products all
  take the long-contraction kernel;
* the full batch of uneven cones (64 restarts: 896 instrument blocks of
  sides 4..64 and 64 process blocks of sides 625 / 1296 in one call), every
  small cone and three process blocks against the oracle, the remaining
  process blocks by the optimality conditions of the projection;
* the two-stage route (dense -> band -> tridiagonal, band 16) at n = 1100,
  where the panel factorisation runs on a multi-CTA cluster and the band
  reduction on several sweeps at once;
* the one-stage reduction in double-float with the columns in global memory
  (sides 1700 and 1300), against the constructions.

The oracle (cyclic Jacobi) takes seconds to tens of seconds per cone at
these sizes on the host cores; each reference is computed once per module."""
import numpy as np
import pytest

import oracle
from paper_2606_20519_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10
TOL_SPLIT = 2e-7


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


@pytest.fixture(scope="module")
def vjp1296():
    """One side-1296 cone of the differentiation workload with separated
    clusters, a Gaussian cotangent and the oracle's derivative."""
    b = W.vjp_batch(batch=1, cluster=1e-3)
    x, g = b.x, b.extra["g"]
    Q, lam = b.extra["Q"][0], b.extra["lam"][0]
    return x, g, W.to_svec((Q * np.maximum(lam, 0)) @ Q.T), oracle.jvp(x, g)


def test_vjp_fp64_1296_vs_oracle(lib, vjp1296):
    import torch
    x, g, P, ref = vjp1296
    y = torch.empty(x.size, dtype=torch.float64, device="cuda")
    xb = lib.proj_vjp(dev(x), dev(g), [1296], y=y)
    assert lib.status(0) == lib.OK
    assert rel(xb.cpu().numpy(), ref) <= TOL
    assert rel(y.cpu().numpy(), P) <= TOL


def test_vjp_split_1296_vs_oracle(lib, vjp1296):
    import torch
    x, g, P, ref = vjp1296
    y = torch.empty(x.size, dtype=torch.float64, device="cuda")
    xb = lib.proj_vjp(dev(x), dev(g), [1296], y=y, opts=lib.make_opts(precision=lib.SPLIT_TF32))
    assert lib.status(0) == lib.OK
    assert rel(xb.cpu().numpy(), ref) <= TOL_SPLIT
    assert rel(y.cpu().numpy(), P) <= TOL_SPLIT


@pytest.mark.parametrize("n", [300, 301])
def test_vjp_split_long_contractions_vs_oracle(lib, n):
    rng = W.rng_for(8810 + n)
    X, Q, lam = W.from_spectrum(rng, W.spectrum_vjp(rng, n, cluster=1e-3))
    x = W.to_svec(X)
    g = rng.standard_normal(x.size)
    xb = lib.proj_vjp(dev(x), dev(g), [n], opts=lib.make_opts(precision=lib.SPLIT_TF32))
    assert lib.status(0) == lib.OK
    assert rel(xb.cpu().numpy(), oracle.jvp(x, g)) <= TOL_SPLIT


def kkt_residuals(y, x, n):
    """Optimality conditions of Y = Pi(X) on the GPU's eigenvalue solver
    (a checker only): lambda_min(Y), lambda_min(Y - X) and <Y, Y - X>,
    relative to ||X||_F."""
    import torch
    Y, X = W_smat(y, n), W_smat(x, n)
    nx = float(np.linalg.norm(x))
    t = torch.from_numpy(np.stack([Y, Y - X])).cuda()
    ev = torch.linalg.eigvalsh(t).cpu().numpy()
    comp = float(y @ (y - x))
    return ev[0].min() / nx, ev[1].min() / nx, comp / nx ** 2


def W_smat(s, n):
    r, c = np.triu_indices(n)
    A = np.zeros((n, n))
    v = s * np.where(r == c, 1.0, 1.0 / np.sqrt(2.0))
    A[r, c] = v
    A[c, r] = v
    return A


def test_uneven_batch_full_size(lib):
    """The 960-cone batch in one call, as the bench times it."""
    b = W.uneven_batch()
    y = lib.proj_batched(dev(b.x), b.sides).cpu().numpy()
    assert lib.status(0) == lib.OK
    big = [i for i in range(b.count) if b.sides[i] >= 625]
    small = [i for i in range(b.count) if b.sides[i] < 625]
    assert len(small) == 896 and len(big) == 64
    for i in small:
        s, e = b.offsets[i], b.offsets[i + 1]
        assert rel(y[s:e], oracle.proj(b.x[s:e])) <= TOL, (i, b.sides[i])
    # three process blocks against the oracle: the first 625, the first 1296 and the last 625
    first625 = next(i for i in big if b.sides[i] == 625)
    first1296 = next(i for i in big if b.sides[i] == 1296)
    last625 = [i for i in big if b.sides[i] == 625][-1]
    for i in (first625, first1296, last625):
        s, e = b.offsets[i], b.offsets[i + 1]
        assert rel(y[s:e], oracle.proj(b.x[s:e])) <= TOL, (i, b.sides[i])
    # every process block: Y >= 0, Y - X >= 0 and <Y, Y - X> = 0 to FP64 rounding
    for i in big:
        s, e = b.offsets[i], b.offsets[i + 1]
        ly, lz, comp = kkt_residuals(y[s:e], b.x[s:e], int(b.sides[i]))
        assert ly >= -1e-12 and lz >= -1e-12 and abs(comp) <= 1e-13, (i, ly, lz, comp)


def test_two_stage_multi_panel_1100(lib):
    """The two-stage route at a side where each panel is factored by a
    cluster of several CTAs (n = 1100 is not a multiple of the band)."""
    rng = W.rng_for(2100)
    n = 1100
    X, Q, lam = W.from_spectrum(rng, W.spectrum_precision(rng, n))
    x = W.to_svec(X)
    y = lib.proj_batched(dev(x), [n], opts=lib.make_opts(band=16)).cpu().numpy()
    assert lib.status(0) == lib.OK
    assert rel(y, oracle.proj(x)) <= TOL
    assert rel(y, W.to_svec((Q * np.maximum(lam, 0)) @ Q.T)) <= TOL
    assert lib.last_tuning(0)["band"] == 16


@pytest.mark.parametrize("sides", [[1700], [1700, 1300]])
def test_double_float_columns_in_l2(lib, sides):
    """Sides whose columns no longer fit in shared memory (one cone of 1700,
    and two cones sharing the SMs) run the one-stage reduction in
    double-float arithmetic with the columns kept in global memory; against
    the exact projection of the constructions, at 1e-10."""
    rng = W.rng_for(2200 + len(sides))
    xs, refs = [], []
    for n in sides:
        X, Q, lam = W.from_spectrum(rng, W.spectrum_admm(rng, n))
        xs.append(W.to_svec(X))
        refs.append(W.to_svec((Q * np.maximum(lam, 0)) @ Q.T))
    y = lib.proj_batched(dev(np.concatenate(xs)), sides).cpu().numpy()
    assert lib.status(0) == lib.OK
    o = 0
    for x, ref in zip(xs, refs):
        assert rel(y[o:o + x.size], ref) <= TOL
        o += x.size
