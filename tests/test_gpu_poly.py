"""GPU parity of the factorization-free approximate projection (scs_psd_proj_poly).

Conclusions ("Approximate semidefinite-cone projections"): the projection is
approximated by a composite matrix polynomial of matrix products.  The CUDA
path (grouped FP64 or split-TF32 GEMMs) is compared element by element with
the oracle's plain FP64 evaluation of the same composite: 1e-10 in FP64,
1e-6 (the split path's promise) with split-TF32 products.  At the benchmark's
full sizes the result is checked against the exact projection of the
construction within the composite's error bound, a property that holds at
any size."""
import numpy as np
import pytest

from oracle import poly as P
from paper_2606_20519_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-10
TOL_SPLIT = 1e-6


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


def run(lib, x, sides, lo, steps=0, precision=None, graphs=True, out=None):
    import torch
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    opts = lib.make_opts(precision=lib.FP64 if precision is None else precision, graphs=graphs)
    y = lib.proj_poly(xt, sides, lo, steps, opts=opts, out=out)
    return y.cpu().numpy(), lib.status(0)


def mixed_batch(seed, sides):
    rng = W.rng_for(seed)
    svecs = []
    for n in sides:
        lam = np.concatenate([rng.uniform(-1, 1, max(n - 2, 0)), [3e-7, -2e-6]])[:n]
        X, _, _ = W.from_spectrum(rng, lam)
        svecs.append(W.to_svec(X))
    return W.pack(svecs, sides)


SIDES = [1, 2, 7, 33, 64, 65, 130, 200]


@pytest.mark.parametrize("lo,steps", [(1e-6, 0), (1e-3, 3)])
def test_fp64_vs_oracle_mixed_sides(lib, lo, steps):
    b = mixed_batch(9500 + steps, SIDES)
    y, st = run(lib, b.x, b.sides, lo, steps)
    assert st == lib.OK
    want = P.proj_poly_batched(b.x, b.offsets, lo, steps)
    for i in range(b.count):
        s, e = b.offsets[i], b.offsets[i + 1]
        assert rel(y[s:e], want[s:e]) <= TOL_FP64, (int(b.sides[i]), rel(y[s:e], want[s:e]))


def test_split_vs_oracle_mixed_sides(lib):
    b = mixed_batch(9510, SIDES + [300])
    y, st = run(lib, b.x, b.sides, 1e-7, precision=lib.SPLIT_TF32)
    assert st == lib.OK
    want = P.proj_poly_batched(b.x, b.offsets, 1e-7)
    errs = [rel(y[b.offsets[i]:b.offsets[i + 1]], want[b.offsets[i]:b.offsets[i + 1]]) for i in range(b.count)]
    assert max(errs) <= TOL_SPLIT, errs


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_admm_first_iterate_n625(lib, precision):
    """The n = 625 ADMM iterate: element by element against the oracle's
    composite, and against the exact projection of the construction within
    the composite's error bound."""
    xs, Q, lam = W.admm_sequence(steps=1)
    x = xs[0]
    prec = lib.FP64 if precision == "fp64" else lib.SPLIT_TF32
    y, st = run(lib, x, [625], 1e-9, precision=prec)
    assert st == lib.OK
    assert rel(y, P.proj_poly(x, 1e-9)) <= (TOL_FP64 if precision == "fp64" else TOL_SPLIT)
    exact = W.to_svec((Q * np.maximum(lam, 0.0)[None, :]) @ Q.T)
    err = np.linalg.norm(y - exact)
    assert err <= P.poly_error_bound(lam, 1e-9) + (1e-12 if precision == "fp64" else 1e-6) * np.linalg.norm(exact)


def test_precision_batch_n4096_split_within_bound(lib):
    """Four n = 4096 cones of the precision spectrum on the split path: the
    error against the exact projection stays within the composite's bound
    plus the split promise (oracle at this size: the construction)."""
    b = W.precision_batch(batch=4)
    y, st = run(lib, b.x, b.sides, 1e-9, precision=lib.SPLIT_TF32)
    assert st == lib.OK
    for i in range(b.count):
        Q, lam = b.extra["Q"][i], b.extra["lam"][i]
        exact = W.to_svec((Q * np.maximum(lam, 0.0)[None, :]) @ Q.T)
        s, e = b.offsets[i], b.offsets[i + 1]
        err = np.linalg.norm(y[s:e] - exact)
        assert err <= P.poly_error_bound(lam, 1e-9) + TOL_SPLIT * np.linalg.norm(exact)


def test_graph_replay_is_bitwise_and_in_place(lib):
    import torch
    b = mixed_batch(9520, [5, 70, 129])
    xt = torch.from_numpy(b.x).cuda()
    opts = lib.make_opts(precision=lib.SPLIT_TF32)
    y1 = lib.proj_poly(xt, b.sides, 1e-6, opts=opts).cpu().numpy()
    assert not lib.last_replayed(0)
    y2 = lib.proj_poly(xt, b.sides, 1e-6, opts=opts).cpu().numpy()
    assert lib.last_replayed(0)
    np.testing.assert_array_equal(y1, y2)
    xi = xt.clone()
    lib.proj_poly(xi, b.sides, 1e-6, opts=opts, out=xi)
    np.testing.assert_array_equal(xi.cpu().numpy(), y1)
    assert lib.status(0) == lib.OK


def test_edge_cases(lib):
    import torch
    # zero cone, side-1 cones, empty cone
    sides = [4, 1, 1, 0, 3]
    rng = W.rng_for(9530)
    svecs = [np.zeros(10), np.array([2.5]), np.array([-1.0]), np.zeros(0), W.to_svec(W.sym_gaussian(rng, 3))]
    b = W.pack(svecs, sides)
    y, st = run(lib, b.x, b.sides, 1e-6)
    assert st == lib.OK
    np.testing.assert_allclose(y, P.proj_poly_batched(b.x, b.offsets, 1e-6), rtol=1e-12, atol=1e-300)
    assert np.all(y[:10] == 0.0)
    # non-finite input: that cone is NaN and the status says so; the others are unaffected
    b2 = mixed_batch(9540, [6, 9])
    x2 = b2.x.copy()
    x2[3] = np.inf
    y2, st2 = run(lib, x2, b2.sides, 1e-6)
    assert st2 == lib.ENONFINITE
    assert np.all(np.isnan(y2[:b2.offsets[1]]))
    want = P.proj_poly(b2.x[b2.offsets[1]:], 1e-6)
    assert rel(y2[b2.offsets[1]:], want) <= TOL_FP64
    # argument errors on the host
    xt = torch.zeros(6, dtype=torch.float64, device="cuda")
    for lo, steps in ((0.0, 0), (1.0, 0), (1e-3, 201), (1e-3, -2)):
        with pytest.raises(lib.ScsPsdError):
            lib.proj_poly(xt, [3], lo, steps)
    with pytest.raises(lib.ScsPsdError):
        lib.proj_poly(xt, [3], 1e-3, 0, offsets=[0, 5], )


@pytest.mark.parametrize("n", [64, 130, 300, 700])
def test_split_products_single_step(lib, n):
    """One composite step isolates the split-TF32 products from the
    iteration's amplification: S_0 = X/||X||_F, S_1 = a S_0 + b S_0^3,
    Y = (X + S_1 X)/2 against the oracle's FP64 evaluation.  A product
    carries 2^-31 of max|a| max|b| per term (the grid of a row's 256-wide K
    group); for Gaussian entries max/rms is about 4, so a product is good to
    about 16 x 2^-31 = 7.5e-9 relative, and three chained products to 5e-8."""
    rng = W.rng_for(9600 + n)
    x = W.to_svec(W.sym_gaussian(rng, n))
    y, st = run(lib, x, [n], 0.3, steps=1, precision=lib.SPLIT_TF32)
    assert st == lib.OK
    assert rel(y, P.proj_poly(x, 0.3, 1)) <= 5e-8


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_hermitian_cones(lib, precision):
    """Complex Hermitian cones through the real embedding (norm halved), against
    the oracle's complex evaluation of the composite."""
    import torch
    rng = W.rng_for(9700)
    sides = [3, 40, 90]
    xs = []
    for n in sides:
        lam = np.concatenate([rng.uniform(-1, 1, n - 1), [2e-7]])
        X, _, _ = W.herm_from_spectrum(rng, lam)
        xs.append(W.to_hsvec(X))
    x = np.concatenate(xs)
    xt = torch.from_numpy(x).cuda()
    prec = lib.FP64 if precision == "fp64" else lib.SPLIT_TF32
    y = lib.proj_poly_hermitian(xt, sides, 1e-7, opts=lib.make_opts(precision=prec)).cpu().numpy()
    assert lib.status(0) == lib.OK
    want = P.herm_proj_poly_batched(x, sides, 1e-7)
    assert rel(y, want) <= (TOL_FP64 if precision == "fp64" else TOL_SPLIT)
