"""The autotuner (scs_psd_autotune) through the C-ABI: it returns a valid
launch-shape choice, later calls with these shapes use it, an explicit band
overrides it, and the tuned path stays at FP64 parity with the oracle."""
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


def test_autotune_choice_is_used_and_exact(lib):
    import torch
    sides = [1, 5, 12, 40, 130, 300]
    rng = W.rng_for(9900)
    x = np.concatenate([W.to_svec(W.sym_gaussian(rng, n)) for n in sides])
    xt = torch.from_numpy(x).cuda()
    x_before = xt.clone()
    ch = lib.autotune(xt, sides)
    assert ch["band"] in (0, 1, 8, 16, 32)
    assert ch["gemm_ctas"] in (1, 2, 4)
    assert ch["bt1_cols"] in (1, 2, 4, 8)
    assert ch["sy_share"] in (1, 2, 4)
    assert ch["ms"] > 0.0
    assert torch.equal(xt, x_before)  # the input is not modified
    y = lib.proj_batched(xt, sides)
    assert lib.status(0) == lib.OK
    used = lib.last_tuning(0)
    assert used == {k: ch[k] for k in lib.TUNING_FIELDS}
    ref = oracle.proj_batched(x, lib.shapes(sides)[0])
    assert rel(y.cpu().numpy(), ref) <= TOL
    # an explicit band wins over the tuned choice
    y16 = lib.proj_batched(xt, sides, opts=lib.make_opts(band=16))
    assert lib.last_tuning(0)["band"] == 16
    assert rel(y16.cpu().numpy(), ref) <= TOL
