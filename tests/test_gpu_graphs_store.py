"""Graph replay and the stored-eigendecomposition derivative, through the C-ABI.

* Replay: from the second call with the same shapes the launch sequence is a
  recorded CUDA graph; its results must be bit-identical to kernel-by-kernel
  launches (the same deterministic kernels run) for new inputs and new
  output buffers, for the projection and for the VJP.
* Store vs recompute (App. E back-propagates through the eigendecomposition):
  scs_psd_proj_store + scs_psd_vjp_stored must give the bits of
  scs_psd_proj_vjp; the stored pairs reconstruct X and are orthonormal; the
  oracle pins the result (1e-10) on spectra with separated signs.
* Side-1 cones in a derivative batch: DPi(x)[g] = g for x > 0, else 0."""
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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def mixed_batch(seed, sides):
    rng = W.rng_for(seed)
    parts = []
    for n in sides:
        X, _, _ = W.from_spectrum(rng, W.spectrum_vjp(rng, n, cluster=1e-3)) if n > 1 else (
            np.array([[rng.uniform(-1, 1)]]), None, None)
        parts.append(W.to_svec(X))
    return np.concatenate(parts), rng


SIDES = [1, 5, 1, 12, 30, 1, 64, 7]


def test_graph_replay_bitwise_projection(lib):
    eager = lib.make_opts(graphs=False)
    for rep in range(4):
        x, _ = mixed_batch(9100 + rep, SIDES)
        xt = dev(x)
        y_eager = lib.proj_batched(xt, SIDES, opts=eager)
        assert not lib.last_replayed(0)
        y_graph = lib.proj_batched(xt, SIDES)
        if rep >= 1:  # the first graph-enabled call of a plan runs eagerly
            assert lib.last_replayed(0)
        assert lib.status(0) == lib.OK
        assert np.array_equal(y_eager.cpu().numpy(), y_graph.cpu().numpy())
        assert rel(y_graph.cpu().numpy(), oracle.proj_batched(x, lib.shapes(SIDES)[0])) <= TOL


def test_graph_replay_bitwise_vjp_and_in_place(lib):
    eager = lib.make_opts(graphs=False)
    for rep in range(3):
        x, rng = mixed_batch(9200 + rep, SIDES)
        g = rng.standard_normal(x.size)
        xt, gt = dev(x), dev(g)
        xb_e = lib.proj_vjp(xt, gt, SIDES, opts=eager).cpu().numpy()
        xb_g = lib.proj_vjp(xt, gt, SIDES).cpu().numpy()
        assert np.array_equal(xb_e, xb_g)
        assert rel(xb_g, oracle.jvp_batched(x, g, lib.shapes(SIDES)[0])) <= TOL
    # in place through a replayed graph
    x, _ = mixed_batch(9300, SIDES)
    ref = lib.proj_batched(dev(x), SIDES, opts=eager).cpu().numpy()
    xt = dev(x)
    lib.proj_batched(xt, SIDES, out=xt)
    assert lib.last_replayed(0)
    assert np.array_equal(xt.cpu().numpy(), ref)


def test_store_then_vjp_matches_recompute_bitwise(lib):
    import torch
    x, rng = mixed_batch(9400, SIDES)
    g = rng.standard_normal(x.size)
    xt, gt = dev(x), dev(g)
    y, V, lam = lib.proj_store(xt, SIDES)
    xb_s = lib.vjp_stored(V, lam, gt, SIDES)
    y_r = torch.empty_like(xt)
    xb_r = lib.proj_vjp(xt, gt, SIDES, y=y_r)
    assert lib.status(0) == lib.OK
    assert np.array_equal(xb_s.cpu().numpy(), xb_r.cpu().numpy())
    assert np.array_equal(y.cpu().numpy(), y_r.cpu().numpy())
    assert rel(xb_s.cpu().numpy(), oracle.jvp_batched(x, g, lib.shapes(SIDES)[0])) <= TOL
    # the stored pairs are an eigendecomposition of each cone
    Vh, lh = V.cpu().numpy(), lam.cpu().numpy()
    vo = lo = so = 0
    for n in SIDES:
        Vi = Vh[vo:vo + n * n].reshape(n, n, order="F")
        li = lh[lo:lo + n]
        Xi = oracle.smat(x[so:so + n * (n + 1) // 2])
        assert np.linalg.norm(Vi.T @ Vi - np.eye(n)) <= 1e-12 * n
        assert np.linalg.norm(Vi @ np.diag(li) @ Vi.T - Xi) <= 1e-12 * max(1.0, np.linalg.norm(Xi))
        vo, lo, so = vo + n * n, lo + n, so + n * (n + 1) // 2


def test_side_one_cones_in_vjp(lib):
    sides = [1, 1, 1, 3]
    x, rng = mixed_batch(9500, sides)
    x[0], x[1], x[2] = 0.7, -0.2, 0.0
    g = rng.standard_normal(x.size)
    xb = lib.proj_vjp(dev(x), dev(g), sides).cpu().numpy()
    assert lib.status(0) == lib.OK
    assert xb[0] == g[0] and xb[1] == 0.0 and xb[2] == 0.0
    assert rel(xb, oracle.jvp_batched(x, g, lib.shapes(sides)[0])) <= TOL


def test_autograd_store_and_recompute_identical(lib):
    import torch
    from paper_2606_20519_gb300.autograd import psd_project, stores_eigenpairs
    x, rng = mixed_batch(9600, SIDES)
    g = rng.standard_normal(x.size)
    grads = []
    for recompute in (1, 2):
        opts = lib.make_opts(recompute=recompute)
        assert stores_eigenpairs(SIDES, opts) == (recompute == 2)
        xt = dev(x).requires_grad_(True)
        y = psd_project(xt, SIDES, opts)
        (y * dev(g)).sum().backward()
        grads.append(xt.grad.detach().cpu().numpy())
    assert np.array_equal(grads[0], grads[1])
    # a budget below the kept bytes forces recomputation
    assert not stores_eigenpairs(SIDES, lib.make_opts(mem_budget_bytes=64))


def test_reserve_builds_the_plan_ahead(lib):
    """After scs_psd_reserve, the first call with those shapes allocates no device memory."""
    import torch
    n, count = 210, 3
    lib.reserve(n, count)
    rng = W.rng_for(9800)
    x = np.concatenate([W.to_svec(W.sym_gaussian(rng, n)) for _ in range(count)])
    xt = dev(x)
    y = torch.empty_like(xt)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lib.proj_batched(xt, [n] * count, out=y)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 - (1 << 20)  # no workspace allocated by the call
    assert lib.status(0) == lib.OK
    assert rel(y.cpu().numpy(), oracle.proj_batched(x, lib.shapes([n] * count)[0])) <= TOL
