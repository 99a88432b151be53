"""GPU parity of the SCS iteration around the projection (App. D.1 final
iterates, closed-form affine step for orthonormal A) against the oracle."""
import numpy as np
import pytest

from oracle import scs as S
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("sides,k,iters", [([3, 5, 9], 20, 5), ([81], 300, 3), ([2, 40], 0, 4)])
def test_iterations_vs_oracle(lib, sides, k, iters):
    rng = W.rng_for(9900 + k)
    offs = np.cumsum([0] + [n * (n + 1) // 2 for n in sides])
    m = int(offs[-1])
    A = np.linalg.qr(rng.standard_normal((m, k)))[0] if k else np.zeros((m, 0))
    b, c = rng.standard_normal(m), rng.standard_normal(k)
    u = np.concatenate([rng.standard_normal(k + m), [1.0]])
    v = np.concatenate([np.zeros(k), rng.standard_normal(m), [0.3]])
    ug, vg = dev(u), dev(v)
    lib.scs_iterate(dev(A), dev(b), dev(c), sides, ug, vg, iters)
    assert lib.status(0) == lib.OK
    uw, vw = S.iterate(A, b, c, offs, u, v, iters)
    assert rel(ug.cpu().numpy(), uw) <= 1e-11
    assert rel(vg.cpu().numpy(), vw) <= 1e-11


def test_converges_to_known_optimum(lib):
    """min -<C, X> s.t. B - X PSD (A = I): x/tau -> svec(B), y/tau -> svec(C)."""
    rng = W.rng_for(7920)
    n = 3
    Cm = W.sym_gaussian(rng, n)
    Cm = Cm @ Cm.T + 0.5 * np.eye(n)
    Bm = W.sym_gaussian(rng, n)
    b, cs = W.to_svec(Bm), W.to_svec(Cm)
    m = b.size
    u = dev(np.concatenate([np.zeros(2 * m), [1.0]]))
    v = dev(np.concatenate([np.zeros(2 * m), [1.0]]))
    lib.scs_iterate(dev(np.eye(m)), dev(b), dev(-cs), [n], u, v, 3000)
    u = u.cpu().numpy()
    tau = u[-1]
    assert tau > 0
    np.testing.assert_allclose(u[:m] / tau, b, atol=1e-6)
    np.testing.assert_allclose(u[m:2 * m] / tau, cs, atol=1e-6)


def test_argument_errors(lib):
    import torch
    z = torch.zeros(10, dtype=torch.float64, device="cuda")
    A = torch.zeros((6, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.ScsPsdError):  # cones do not cover m
        lib.scs_iterate(A, z[:6], z[:2], [2], z[:9], z[:9], 1)
    with pytest.raises(lib.ScsPsdError):  # negative iteration count
        lib.scs_iterate(A, z[:6], z[:2], [3], z[:9], z[:9], -1)


# ---- the structured operator (App. D.2: A and A^T as contractions over local bases)
def _kron_case(rng, bases, index):
    m = svec_len(int(np.prod([B.shape[1] for B in bases])))
    k = len(index)
    b, c = rng.standard_normal(m), rng.standard_normal(k)
    u = np.concatenate([rng.standard_normal(k + m), [1.0]])
    v = np.concatenate([np.zeros(k), rng.standard_normal(m), [0.3]])
    return b, c, u, v


def svec_len(n):
    return n * (n + 1) // 2


def _run_kron(lib, bases, index, b, c, u, v, iters):
    import torch
    ug, vg = dev(u), dev(v)
    lib.scs_iterate_kron([dev(B) for B in bases], torch.from_numpy(np.asarray(index, dtype=np.int64)).cuda(),
                         dev(b), dev(c), ug, vg, iters)
    return ug.cpu().numpy(), vg.cpu().numpy()


@pytest.mark.parametrize("d,modes", [(2, 4), (3, 2)])
def test_kron_iterations_vs_oracle(lib, d, modes):
    rng = W.rng_for(9950 + 10 * d + modes)
    B, anti = W.real_local_basis(d)
    bases = [B] * modes
    if modes == 4:
        index = W.process_allowed(d)
    else:  # every symmetric product of two local elements
        kb = B.shape[0]
        index = np.array([f for f in range(kb * kb) if anti[f // kb] == anti[f % kb]])
    b, c, u, v = _kron_case(rng, bases, index)
    iters = 4
    ug, vg = _run_kron(lib, bases, index, b, c, u, v, iters)
    assert lib.status(0) == lib.OK
    m = b.size
    uw, vw = S.iterate_kron(bases, index, b, c, [0, m], u, v, iters)
    assert rel(ug, uw) <= 1e-11
    assert rel(vg, vw) <= 1e-11


def test_kron_matches_the_dense_operator_n81(lib):
    """d = 3, four subsystems (n = 81, 633 coefficients of the real process
    subspace): the structured products against the dense path with the
    same A formed column by column."""
    rng = W.rng_for(9960)
    B, _ = W.real_local_basis(3)
    bases, index = [B] * 4, W.process_allowed(3)
    A = S.kron_columns(bases, index)
    b, c, u, v = _kron_case(rng, bases, index)
    ug, vg = _run_kron(lib, bases, index, b, c, u, v, 3)
    assert lib.status(0) == lib.OK
    ud, vd = dev(u), dev(v)
    lib.scs_iterate(dev(A), dev(b), dev(c), [81], ud, vd, 3)
    assert lib.status(0) == lib.OK
    assert rel(ug, ud.cpu().numpy()) <= 1e-12
    assert rel(vg, vd.cpu().numpy()) <= 1e-12


def test_kron_bad_index_is_reported(lib):
    import torch
    B, _ = W.real_local_basis(2)
    bases = [B, B]
    index = np.array([0, 5, 16])  # 16 is past the 4 x 4 coefficient tensor
    rng = W.rng_for(9970)
    b, c, u, v = _kron_case(rng, bases, index)
    _run_kron(lib, bases, index, b, c, u, v, 1)
    assert lib.status(0) == lib.EINVAL
    with pytest.raises(lib.ScsPsdError):  # a local side beyond the maximum of 8
        big = torch.zeros((1, 9, 9), dtype=torch.float64, device="cuda")
        lib.scs_iterate_kron([big], torch.zeros(1, dtype=torch.int64, device="cuda"), dev(np.zeros(45)),
                             dev(np.zeros(1)), dev(np.zeros(47)), dev(np.zeros(47)), 1)
