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
