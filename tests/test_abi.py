"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point that include/scs_psd.h declares, and host-side argument errors
are reported without touching a device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scs_psd.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int32_t|int64_t|const char\*)\s+(scs_psd_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_20519_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("scs_psd_proj", "scs_psd_proj_batched", "scs_psd_proj_vjp", "scs_psd_create",
                     "scs_psd_destroy", "scs_psd_status", "scs_psd_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2606_20519_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(scs_psd_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_strerror_and_null_handle(lib):
    from paper_2606_20519_gb300 import _lib
    assert _lib.strerror(0) == "ok"
    assert "invalid" in _lib.strerror(1)
    # a null handle is rejected on the host
    assert lib.scs_psd_proj(None, None, None, 3, None, None) == _lib.EINVAL
    v = ctypes.c_int32(0)
    assert lib.scs_psd_status(None, ctypes.byref(v)) == _lib.EINVAL
    assert lib.scs_psd_last_launch_count(None) == -1


def test_shapes_helper():
    from paper_2606_20519_gb300 import _lib
    offs, sides = _lib.shapes([1, 3, 0, 4])
    assert list(offs) == [0, 1, 7, 7, 17]
    assert sides.dtype.name == "int32"


def test_poly_schedule_matches_the_oracle(lib):
    """The library's composite coefficients (host function, no GPU) against
    the oracle's schedule for the factorization-free projection."""
    from oracle import poly as P
    from paper_2606_20519_gb300 import _lib as L
    for lo, steps in ((1e-3, 0), (1e-7, 0), (1e-9, 0), (0.25, 3)):
        a, b, lk = L.poly_schedule(lo, steps)
        oa, ob, olk = P.poly_coeffs(lo, steps)
        assert len(a) == len(oa)
        np.testing.assert_allclose(a, oa, rtol=4e-16, atol=0)
        np.testing.assert_allclose(b, ob, rtol=8e-16, atol=0)
        assert abs(lk - olk) <= 4e-16
    for lo, steps in ((0.0, 0), (1.0, 0), (1e-3, -1), (1e-3, 201)):
        with pytest.raises(L.ScsPsdError):
            L.poly_schedule(lo, steps)


def test_stats_record_layout_and_null_handle(lib):
    """The binding's records match the header's layout (four int32 and four
    doubles; the options struct keeps its size with the stats field), and
    statistics are refused without a handle."""
    from paper_2606_20519_gb300 import _lib
    assert ctypes.sizeof(_lib.ConeStats) == 48
    assert ctypes.sizeof(_lib.Opts) == 40
    out = (_lib.ConeStats * 1)()
    assert lib.scs_psd_last_stats(None, out, 1) == _lib.EINVAL
