"""The allocation-free entry point scs_psd_proj_static, called through the
C-ABI, against the regular entry point scs_psd_proj.

scs_psd_proj_static serves callers that cannot allocate device memory: its
workspace is a fixed file-scope device array shared by every call.  Two
calls in a row (and a third of another side, which re-lays out the shared
array) must each agree with scs_psd_proj within the FP64-path tolerance.
This file is collected last so that a failure here does not hide the other
tests' results; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2606_20519_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


def test_static_scratch_entry_point_matches_proj():
    import torch
    from paper_2606_20519_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    fn = lib.scs_psd_proj_static
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    stream = torch.cuda.current_stream()
    cases = [(81, 1), (81, 2), (200, 3)]
    for n, seed in cases:
        rng = W.rng_for(7000 + seed)
        X, Q, lam = W.from_spectrum(rng, W.spectrum_plain(rng, n))
        x = torch.from_numpy(W.to_svec(X)).cuda()
        y = torch.empty_like(x)
        rc = fn(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), n,
                ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, _lib.strerror(rc)
        y_ref = _lib.proj(x, n)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b), (n, seed)
    # sides beyond the static maximum are rejected on the host
    big = torch.zeros(300 * 301 // 2, dtype=torch.float64, device="cuda")
    assert fn(ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()), 300,
              ctypes.c_void_p(stream.cuda_stream)) == _lib.EINVAL
