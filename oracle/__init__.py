"""FP64 CPU oracle for the PSD-cone projection -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product path (the CUDA library and its
Python binding) never imports it, and the two share no code.

The arithmetic lives in ``psd_oracle.c`` (plain C, FP64, cyclic Jacobi, no
BLAS/LAPACK, compiled without FP contraction); this module compiles it with
gcc and wraps it with ctypes.  Functions follow App. D of the paper:

* ``smat`` / ``svec``  -- the vec_R map of App. D.1 (real symmetric case,
  lower triangle column by column, off-diagonals times sqrt(2));
* ``proj``             -- Pi(X) = V diag(max(lambda,0)) V^T (App. D.2);
* ``proj_moreau``      -- the same through X - Pi_-(X) (Moreau, App. D.1);
* ``jvp``              -- Daleckii-Krein derivative (App. E differentiates
  through the eigendecomposition), symmetric in svec coordinates, so it is
  also the VJP;
* ``fd_jvp``           -- central finite difference of ``proj``.

Every function is pinned by ``tests/test_oracle.py`` against closed forms,
invariants, constructions and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psd_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

OK, EINVAL, ENOMEM, ENOCONV, ENONFINITE = 0, 1, 2, 5, 6

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile psd_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.orc_smat.argtypes = [i64, dp, dp]
        lib.orc_svec.argtypes = [i64, dp, dp]
        lib.orc_eig_svec.argtypes = [i64, dp, dp, dp, ctypes.POINTER(ctypes.c_int)]
        lib.orc_eig_svec.restype = ctypes.c_int
        lib.orc_psd_proj_route.argtypes = [i64, dp, dp, dp, ctypes.c_int]
        lib.orc_psd_proj_route.restype = ctypes.c_int
        lib.orc_psd_jvp.argtypes = [i64, dp, dp, dp]
        lib.orc_psd_jvp.restype = ctypes.c_int
        lib.orc_hsmat.argtypes = [i64, dp, dp, dp]
        lib.orc_hsvec.argtypes = [i64, dp, dp, dp]
        lib.orc_herm_proj_route.argtypes = [i64, dp, dp, dp, ctypes.c_int]
        lib.orc_herm_proj_route.restype = ctypes.c_int
        lib.orc_set_mutation.argtypes = [ctypes.c_int]
        lib.orc_get_mutation.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def svec_len(n: int) -> int:
    return n * (n + 1) // 2


def side_of(length: int) -> int:
    n = int((np.sqrt(8 * length + 1) - 1) // 2)
    while svec_len(n) < length:
        n += 1
    if svec_len(n) != length:
        raise ValueError(f"{length} is not a triangular number")
    return n


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != OK:
        raise OracleError(f"{what}: oracle status {st}")


def set_threads(t: int) -> None:
    """OpenMP threads the oracle uses (0 = OpenMP default)."""
    _load().orc_set_threads(int(t))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def set_mutation(m: int) -> None:
    """Plant a known mistake in the oracle (tests only); 0 restores it."""
    _load().orc_set_mutation(int(m))


def smat(x) -> np.ndarray:
    x = _f64(x)
    n = side_of(x.size)
    A = np.empty((n, n))
    _load().orc_smat(n, _dp(x), _dp(A))
    return A


def svec(A) -> np.ndarray:
    A = _f64(A)
    n = A.shape[0]
    s = np.empty(svec_len(n))
    _load().orc_svec(n, _dp(A), _dp(s))
    return s


def eig(x):
    """(lam, V) of smat(x) by cyclic Jacobi; eigenvalues unsorted."""
    x = _f64(x)
    n = side_of(x.size)
    lam = np.empty(n)
    V = np.empty((n, n))
    sw = ctypes.c_int(0)
    _check(_load().orc_eig_svec(n, _dp(x), _dp(lam), _dp(V), ctypes.byref(sw)), "eig")
    return lam, V


def proj(x, return_eigs: bool = False):
    """Pi(X) on an svec buffer: svec(V diag(max(lam,0)) V^T)."""
    x = _f64(x)
    n = side_of(x.size)
    y = np.empty_like(x)
    lam = np.empty(max(n, 1))
    _check(_load().orc_psd_proj_route(n, _dp(x), _dp(y), _dp(lam), 0), "proj")
    return (y, lam[:n]) if return_eigs else y


def proj_moreau(x) -> np.ndarray:
    """Pi(X) computed as X - sum_{lam<0} lam v v^T (Moreau decomposition)."""
    x = _f64(x)
    n = side_of(x.size)
    y = np.empty_like(x)
    _check(_load().orc_psd_proj_route(n, _dp(x), _dp(y), None, 1), "proj_moreau")
    return y


def jvp(x, h) -> np.ndarray:
    """Daleckii-Krein derivative DPi(X)[H] on svec buffers (= VJP)."""
    x = _f64(x)
    h = _f64(h)
    n = side_of(x.size)
    if h.size != x.size:
        raise ValueError("x and h differ in length")
    out = np.empty_like(x)
    _check(_load().orc_psd_jvp(n, _dp(x), _dp(h), _dp(out)), "jvp")
    return out


def fd_jvp(x, h, step: float = 1e-6) -> np.ndarray:
    """Central difference (Pi(X + step H) - Pi(X - step H)) / (2 step)."""
    x = _f64(x)
    h = _f64(h)
    return (proj(x + step * h) - proj(x - step * h)) / (2.0 * step)


def proj_batched(x, offsets) -> np.ndarray:
    """Pi applied cone by cone to a packed buffer split by ``offsets``."""
    x = _f64(x)
    offsets = np.asarray(offsets, dtype=np.int64)
    y = np.empty_like(x)
    for i in range(len(offsets) - 1):
        a, b = int(offsets[i]), int(offsets[i + 1])
        y[a:b] = proj(x[a:b])
    return y


def jvp_batched(x, g, offsets) -> np.ndarray:
    x = _f64(x)
    g = _f64(g)
    offsets = np.asarray(offsets, dtype=np.int64)
    y = np.empty_like(x)
    for i in range(len(offsets) - 1):
        a, b = int(offsets[i]), int(offsets[i + 1])
        y[a:b] = jvp(x[a:b], g[a:b])
    return y


# ---- complex Hermitian cones (svec: per column the diagonal entry, then for
# every row below it sqrt(2) Re, sqrt(2) Im; n^2 reals)
def hside_of(length: int) -> int:
    n = int(round(np.sqrt(length)))
    if n * n != length:
        raise ValueError(f"{length} is not n^2")
    return n


def herm_smat(x) -> np.ndarray:
    """Complex Hermitian matrix of a Hermitian svec."""
    x = _f64(x)
    n = hside_of(x.size)
    Ar = np.empty((n, n)); Ai = np.empty((n, n))
    _load().orc_hsmat(n, _dp(x), _dp(Ar), _dp(Ai))
    return Ar + 1j * Ai


def herm_svec(A) -> np.ndarray:
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    Ar = np.ascontiguousarray(A.real); Ai = np.ascontiguousarray(A.imag)
    s = np.empty(n * n)
    _load().orc_hsvec(n, _dp(Ar), _dp(Ai), _dp(s))
    return s


def herm_proj(x, route: int = 0) -> np.ndarray:
    """Pi(X) of a complex Hermitian cone on its svec (complex Jacobi, FP64)."""
    x = _f64(x)
    n = hside_of(x.size)
    y = np.empty_like(x)
    _check(_load().orc_herm_proj_route(n, _dp(x), _dp(y), None, route), "orc_herm_proj_route")
    return y


def herm_proj_batched(x, sides) -> np.ndarray:
    x = _f64(x)
    y = np.empty_like(x)
    o = 0
    for n in sides:
        y[o:o + n * n] = herm_proj(x[o:o + n * n])
        o += n * n
    return y
