"""The allocation-free entry point scs_psd_proj_static, called through the
C-ABI, against the FP64 oracle and against the regular entry point
scs_psd_proj.

scs_psd_proj_static serves callers that cannot allocate device memory (a
process whose GPU memory belongs to a pool or a framework's allocator, code
that may not allocate once it runs): its workspace is a fixed file-scope
device array shared by every call.  Checked here:
* two calls in a row of one side, then other sides (each re-lays out the
  shared array): the maximum side 256, the trivial sides 1 and 2, and an
  in-place call (y aliases x), each within the FP64-path tolerance of the
  oracle and of scs_psd_proj;
* a call of a side the static path has not planned before leaves the
  device's free memory unchanged (it plans inside the array, with no
  cudaMalloc);
* such a planning call is refused while the stream is being captured, and
  sides beyond the maximum are refused on the host.
This file is collected last so that a failure here does not hide the other
tests' results; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2606_20519_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def static_fn():
    import torch
    from paper_2606_20519_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    torch.cuda.init()
    fn = lib.scs_psd_proj_static
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def call(fn, x, y, n, stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return fn(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), n, ctypes.c_void_p(s.cuda_stream))


def cone(n, seed):
    rng = W.rng_for(7000 + seed)
    if n == 1:
        return np.array([rng.uniform(-1, 1)])
    X, Q, lam = W.from_spectrum(rng, W.spectrum_plain(rng, n))
    return W.to_svec(X)


def test_static_scratch_entry_point_matches_oracle_and_proj(static_fn):
    import torch
    from paper_2606_20519_gb300 import _lib
    for n, seed in [(81, 1), (81, 2), (200, 3), (256, 4), (1, 5), (2, 6), (1, 7)]:
        xh = cone(n, seed)
        x = torch.from_numpy(xh).cuda()
        y = torch.empty_like(x)
        rc = call(static_fn, x, y, n)
        assert rc == 0, _lib.strerror(rc)
        y_ref = _lib.proj(x, n)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert rel(a, oracle.proj(xh)) <= TOL, (n, seed)
        assert rel(a, b) <= TOL, (n, seed)
    # in place: y aliases x
    xh = cone(81, 8)
    x = torch.from_numpy(xh).cuda()
    assert call(static_fn, x, x, 81) == 0
    torch.cuda.synchronize()
    assert rel(x.cpu().numpy(), oracle.proj(xh)) <= TOL


def test_static_scratch_plans_without_allocating(static_fn):
    import torch
    from paper_2606_20519_gb300 import _lib
    n = 150  # a side the static path has not planned in this process
    xh = cone(n, 9)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty_like(x)
    # the array's set-up (first call on the device) and every kernel of this
    # side's launch sequence loaded before the measurement
    x0 = torch.from_numpy(cone(2, 12)).cuda()
    assert call(static_fn, x0, torch.empty_like(x0), 2) == 0
    _lib.proj(x, n)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc = call(static_fn, x, y, n)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert rc == 0, _lib.strerror(rc)
    assert free1 >= free0 - (1 << 20), (free0, free1)
    assert rel(y.cpu().numpy(), oracle.proj(xh)) <= TOL


def test_static_scratch_refuses_planning_inside_capture_and_large_sides(static_fn):
    import torch
    from paper_2606_20519_gb300 import _lib
    x = torch.from_numpy(cone(40, 10)).cuda()
    y = torch.empty_like(x)
    assert call(static_fn, x, y, 40) == 0
    torch.cuda.synchronize()
    # a call of another side would re-plan: refused while the stream is captured
    x2 = torch.from_numpy(cone(41, 11)).cuda()
    y2 = torch.empty_like(x2)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    rcs = []
    with torch.cuda.graph(g, stream=s):
        rcs.append(call(static_fn, x2, y2, 41, stream=s))
    assert rcs == [_lib.EINVAL]
    # sides beyond the static maximum are rejected on the host
    big = torch.zeros(300 * 301 // 2, dtype=torch.float64, device="cuda")
    assert call(static_fn, big, big, 300) == _lib.EINVAL
