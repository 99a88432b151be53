"""GPU parity of complex Hermitian cones (scs_psd_proj_hermitian) against
the complex Jacobi oracle, 1e-10 relative (FP64 path), and against the exact
projection of Haar-unitary constructions at a larger side."""
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


def run(lib, x, sides, **kw):
    import torch
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = lib.proj_hermitian(xt, sides, **kw)
    return y.cpu().numpy(), lib.status(0)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 130])
def test_single_cone_vs_oracle(lib, n):
    rng = W.rng_for(9700 + n)
    x = W.to_hsvec(W.herm_gaussian(rng, n))
    y, st = run(lib, x, [n])
    assert st == lib.OK
    assert rel(y, oracle.herm_proj(x)) <= TOL


def test_uneven_batch_and_in_place(lib):
    import torch
    sides = [0, 1, 4, 9, 2, 25, 16, 36]
    rng = W.rng_for(9750)
    x = np.concatenate([W.to_hsvec(W.herm_gaussian(rng, n)) for n in sides if n > 0])
    ref = oracle.herm_proj_batched(x, [n for n in sides])
    y, st = run(lib, x, sides)
    assert st == lib.OK
    assert rel(y, ref) <= TOL
    xt = torch.from_numpy(x.copy()).cuda()
    lib.proj_hermitian(xt, sides, out=xt)
    assert rel(xt.cpu().numpy(), ref) <= TOL


def test_construction_and_moreau_side(lib):
    rng = W.rng_for(9760)
    n = 300
    lam = np.concatenate([rng.uniform(0.01, 1, 120), rng.normal(0, 1e-6, 100), rng.uniform(-1, -0.01, 80)])
    X, U, lam = W.herm_from_spectrum(rng, lam)
    x = W.to_hsvec(X)
    exact = W.to_hsvec((U * np.maximum(lam, 0)) @ U.conj().T)
    for side in (0, 1, 2):
        y, st = run(lib, x, [n], opts=lib.make_opts(side=side))
        assert st == lib.OK
        assert rel(y, exact) <= TOL


@pytest.mark.parametrize("n", [40, 300])
def test_native_and_embedding_routes_agree_with_oracle(lib, n):
    """The native complex reduction (the automatic route for sides up to
    1100) and the real embedding of side 2n (taken when opts.band is set)
    both against the complex oracle."""
    rng = W.rng_for(9780 + n)
    x = W.to_hsvec(W.herm_gaussian(rng, n))
    ref = oracle.herm_proj(x)
    y_native, st = run(lib, x, [n])
    assert st == lib.OK
    assert rel(y_native, ref) <= TOL
    y_embed, st = run(lib, x, [n], opts=lib.make_opts(band=1))
    assert st == lib.OK
    assert rel(y_embed, ref) <= TOL
