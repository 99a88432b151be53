"""ctypes binding of the scs_psd C-ABI (include/scs_psd.h).

Argument marshalling only: every arithmetic step of the projection runs in
the CUDA kernels of ``_build/libscs_psd.so``.  There is no CPU fallback; if
the library has not been built, loading fails with an error that says so.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libscs_psd.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOCONV, ENONFINITE = range(7)
FP64, SPLIT_TF32 = 0, 1


class ScsPsdError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (code {code})")


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("side", ctypes.c_int32), ("recompute", ctypes.c_int32),
                ("band", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_int64),
                ("wait_limit_cycles", ctypes.c_int64), ("graphs", ctypes.c_int32), ("stats", ctypes.c_int32)]


class KronOp(ctypes.Structure):
    _fields_ = [("nmodes", ctypes.c_int32), ("dims", ctypes.c_int32 * 6), ("nbasis", ctypes.c_int32 * 6),
                ("basis", ctypes.c_void_p * 6), ("nparams", ctypes.c_int64), ("index", ctypes.c_void_p)]


class ConeStats(ctypes.Structure):
    _fields_ = [("k_pos", ctypes.c_int32), ("k_neg", ctypes.c_int32), ("route", ctypes.c_int32),
                ("status", ctypes.c_int32), ("complementarity", ctypes.c_double), ("norm_y", ctypes.c_double),
                ("norm_x", ctypes.c_double), ("reserved", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_handles = {}

EXPORTS = ("scs_psd_create", "scs_psd_destroy", "scs_psd_proj", "scs_psd_proj_batched", "scs_psd_proj_vjp",
           "scs_psd_proj_store", "scs_psd_vjp_stored", "scs_psd_proj_static", "scs_psd_reserve", "scs_psd_status", "scs_psd_last_launch_count",
           "scs_psd_last_replayed", "scs_psd_strerror", "scs_psd_trace", "scs_psd_trace_read",
           "scs_psd_autotune", "scs_psd_last_tuning", "scs_psd_proj_hermitian", "scs_psd_proj_poly",
           "scs_psd_poly_schedule", "scs_psd_proj_poly_hermitian", "scs_psd_lambda_min", "scs_psd_mix_identity",
           "scs_psd_scs_iterate", "scs_psd_last_stats", "scs_psd_scs_iterate_kron")
NPHASES = 8
PHASES = ("unpack", "dense_to_band", "band_to_tridiag", "tridiag_dc", "backtransform_2", "backtransform_1",
          "reconstruct", "derivative")


def load(path: str | None = None):
    """Load the compiled library (raises if it has not been built)."""
    global _lib, LIB_PATH
    with _lock:
        if _lib is not None:
            return _lib
        if path is not None:
            LIB_PATH = path
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"scs_psd CUDA library not built ({LIB_PATH} missing); "
                               "run paper_2606_20519_gb300.build.build() first -- there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        op = ctypes.POINTER(Opts)
        lib.scs_psd_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
        lib.scs_psd_destroy.argtypes = [vp]
        lib.scs_psd_proj.argtypes = [vp, vp, vp, i64, op, vp]
        lib.scs_psd_proj_batched.argtypes = [vp, vp, vp, vp, vp, i32, op, vp]
        lib.scs_psd_proj_vjp.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, op, vp]
        lib.scs_psd_proj_store.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, op, vp]
        lib.scs_psd_vjp_stored.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, op, vp]
        lib.scs_psd_reserve.argtypes = [vp, i64, i32, op]
        lib.scs_psd_status.argtypes = [vp, ctypes.POINTER(i32)]
        lib.scs_psd_last_launch_count.argtypes = [vp]
        lib.scs_psd_last_launch_count.restype = i64
        lib.scs_psd_proj_hermitian.argtypes = [vp, vp, vp, vp, vp, i32, op, vp]
        lib.scs_psd_proj_poly.argtypes = [vp, vp, vp, vp, vp, i32, ctypes.c_double, i32, op, vp]
        lib.scs_psd_poly_schedule.argtypes = [ctypes.c_double, i32, vp, vp, ctypes.POINTER(ctypes.c_double)]
        lib.scs_psd_poly_schedule.restype = i32
        lib.scs_psd_proj_poly_hermitian.argtypes = [vp, vp, vp, vp, vp, i32, ctypes.c_double, i32, op, vp]
        lib.scs_psd_lambda_min.argtypes = [vp, vp, vp, vp, vp, i32, op, vp]
        lib.scs_psd_scs_iterate.argtypes = [vp, vp, vp, vp, i64, i64, vp, vp, i32, vp, vp, i32, op, vp]
        lib.scs_psd_mix_identity.argtypes = [vp, vp, vp, vp, vp, i32, vp, i32, vp, ctypes.c_double, vp, op, vp]
        lib.scs_psd_autotune.argtypes = [vp, vp, vp, vp, i32, op, vp, ctypes.POINTER(i32),
                                         ctypes.POINTER(ctypes.c_double)]
        lib.scs_psd_last_tuning.argtypes = [vp, ctypes.POINTER(i32)]
        lib.scs_psd_last_stats.argtypes = [vp, ctypes.POINTER(ConeStats), i32]
        lib.scs_psd_scs_iterate_kron.argtypes = [vp, ctypes.POINTER(KronOp), vp, vp, vp, vp, i32, op, vp]
        lib.scs_psd_last_replayed.argtypes = [vp]
        lib.scs_psd_last_replayed.restype = ctypes.c_int
        lib.scs_psd_trace.argtypes = [vp, ctypes.c_int]
        lib.scs_psd_trace_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        lib.scs_psd_strerror.argtypes = [ctypes.c_int]
        lib.scs_psd_strerror.restype = ctypes.c_char_p
        for name in EXPORTS:
            getattr(lib, name)
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().scs_psd_strerror(int(code)).decode()
    except Exception:  # pragma: no cover - used while formatting errors
        return "error"


def _check(rc: int, what: str):
    if rc != OK:
        raise ScsPsdError(rc, what)


def handle(device: int):
    with _lock:
        h = _handles.get(device)
    if h is not None:
        return h
    lib = load()
    hv = ctypes.c_void_p()
    _check(lib.scs_psd_create(ctypes.byref(hv), int(device)), "scs_psd_create")
    with _lock:
        _handles[device] = hv
    return hv


def make_opts(precision: int = FP64, side: int = 0, band: int = 0, wait_limit_cycles: int = 0,
              recompute: int = 0, mem_budget_bytes: int = 0, graphs: bool = True, stats: bool = False) -> Opts:
    return Opts(precision, side, recompute, band, mem_budget_bytes, wait_limit_cycles, 0 if graphs else 1,
                1 if stats else 0)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream_ptr(t):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _check_tensor(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")


def shapes(sides):
    """(offsets int64[count+1], sides int32[count]) host arrays for a side list."""
    sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    lens = sides.astype(np.int64) * (sides.astype(np.int64) + 1) // 2
    offsets = np.zeros(sides.size + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    return offsets, sides


def proj(x, n: int, out=None, opts: Opts | None = None):
    """y = svec(Pi(smat(x))) for one side-n cone (C-ABI scs_psd_proj)."""
    import torch
    _check_tensor(x, "x")
    if out is None:
        out = torch.empty_like(x)
    _check_tensor(out, "out")
    lib = load()
    rc = lib.scs_psd_proj(handle(x.device.index), _ptr(x), _ptr(out), int(n),
                          ctypes.byref(opts) if opts is not None else None, _stream_ptr(x))
    _check(rc, "scs_psd_proj")
    return out


def proj_batched(x, sides, out=None, opts: Opts | None = None, offsets=None):
    """Projection of many uneven cones packed in one svec buffer."""
    import torch
    _check_tensor(x, "x")
    if offsets is None:
        offsets, sides = shapes(sides)
    else:
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    if out is None:
        out = torch.empty_like(x)
    _check_tensor(out, "out")
    lib = load()
    rc = lib.scs_psd_proj_batched(handle(x.device.index), _ptr(x), _ptr(out),
                                  offsets.ctypes.data_as(ctypes.c_void_p), sides.ctypes.data_as(ctypes.c_void_p),
                                  int(sides.size), ctypes.byref(opts) if opts is not None else None, _stream_ptr(x))
    _check(rc, "scs_psd_proj_batched")
    return out


def proj_vjp(x, g, sides, xbar=None, y=None, opts: Opts | None = None, offsets=None):
    """xbar = DPi(X)^T g (Daleckii-Krein), optionally y = Pi(x) as well."""
    import torch
    _check_tensor(x, "x")
    _check_tensor(g, "g")
    if offsets is None:
        offsets, sides = shapes(sides)
    else:
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    if xbar is None:
        xbar = torch.empty_like(x)
    lib = load()
    rc = lib.scs_psd_proj_vjp(handle(x.device.index), _ptr(x), _ptr(g), _ptr(xbar), _ptr(y),
                              offsets.ctypes.data_as(ctypes.c_void_p), sides.ctypes.data_as(ctypes.c_void_p),
                              int(sides.size), ctypes.byref(opts) if opts is not None else None, _stream_ptr(x))
    _check(rc, "scs_psd_proj_vjp")
    return xbar


def _shape_arrays(sides, offsets):
    if offsets is None:
        return shapes(sides)
    return (np.ascontiguousarray(np.asarray(offsets, dtype=np.int64)),
            np.ascontiguousarray(np.asarray(sides, dtype=np.int32)))


def eig_sizes(sides) -> tuple[int, int]:
    """Doubles of a stored eigendecomposition: (sum n^2 for V, sum n for lam)."""
    s = np.asarray(sides, dtype=np.int64)
    return int((s * s).sum()), int(s.sum())


def proj_store(x, sides, y=None, V=None, lam=None, opts: Opts | None = None, offsets=None, want_y=True):
    """y = Pi(x) and every eigenpair (V, lam) of every cone (C-ABI scs_psd_proj_store).
    Returns (y or None, V, lam)."""
    import torch
    _check_tensor(x, "x")
    offsets, sides = _shape_arrays(sides, offsets)
    nv, nl = eig_sizes(sides)
    if want_y and y is None:
        y = torch.empty_like(x)
    if V is None:
        V = torch.empty(nv, dtype=torch.float64, device=x.device)
    if lam is None:
        lam = torch.empty(nl, dtype=torch.float64, device=x.device)
    _check_tensor(V, "V")
    _check_tensor(lam, "lam")
    if V.numel() < nv or lam.numel() < nl:
        raise ValueError("V or lam too small for the shapes")
    rc = load().scs_psd_proj_store(handle(x.device.index), _ptr(x), _ptr(y), _ptr(V), _ptr(lam),
                                   offsets.ctypes.data_as(ctypes.c_void_p), sides.ctypes.data_as(ctypes.c_void_p),
                                   int(sides.size), ctypes.byref(opts) if opts is not None else None,
                                   _stream_ptr(x))
    _check(rc, "scs_psd_proj_store")
    return y, V, lam


def vjp_stored(V, lam, g, sides, xbar=None, opts: Opts | None = None, offsets=None):
    """xbar = DPi(X)^T g from an eigendecomposition kept by proj_store (C-ABI scs_psd_vjp_stored)."""
    import torch
    _check_tensor(V, "V")
    _check_tensor(lam, "lam")
    _check_tensor(g, "g")
    offsets, sides = _shape_arrays(sides, offsets)
    nv, nl = eig_sizes(sides)
    if V.numel() < nv or lam.numel() < nl:
        raise ValueError("V or lam too small for the shapes")
    if xbar is None:
        xbar = torch.empty_like(g)
    rc = load().scs_psd_vjp_stored(handle(g.device.index), _ptr(V), _ptr(lam), _ptr(g), _ptr(xbar),
                                   offsets.ctypes.data_as(ctypes.c_void_p), sides.ctypes.data_as(ctypes.c_void_p),
                                   int(sides.size), ctypes.byref(opts) if opts is not None else None,
                                   _stream_ptr(g))
    _check(rc, "scs_psd_vjp_stored")
    return xbar


def hshapes(sides):
    """(offsets int64[count+1], sides int32[count]) of Hermitian cones (n^2 reals each)."""
    sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    offsets = np.zeros(sides.size + 1, dtype=np.int64)
    np.cumsum(sides.astype(np.int64) ** 2, out=offsets[1:])
    return offsets, sides


def proj_hermitian(x, sides, out=None, opts: Opts | None = None, offsets=None):
    """Projection of complex Hermitian cones on their Hermitian svec (C-ABI scs_psd_proj_hermitian)."""
    import torch
    _check_tensor(x, "x")
    if offsets is None:
        offsets, sides = hshapes(sides)
    else:
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    if out is None:
        out = torch.empty_like(x)
    _check_tensor(out, "out")
    rc = load().scs_psd_proj_hermitian(handle(x.device.index), _ptr(x), _ptr(out),
                                       offsets.ctypes.data_as(ctypes.c_void_p),
                                       sides.ctypes.data_as(ctypes.c_void_p), int(sides.size),
                                       ctypes.byref(opts) if opts is not None else None, _stream_ptr(x))
    _check(rc, "scs_psd_proj_hermitian")
    return out


def poly_schedule(lo: float, steps: int = 0):
    """(a, b, l_final) of the composite scs_psd_proj_poly applies (C-ABI scs_psd_poly_schedule)."""
    lib = load()
    k = lib.scs_psd_poly_schedule(float(lo), int(steps), None, None, None)
    if k < 0:
        _check(-k, "scs_psd_poly_schedule")
    a = np.zeros(k, dtype=np.float64)
    b = np.zeros(k, dtype=np.float64)
    lk = ctypes.c_double(0.0)
    lib.scs_psd_poly_schedule(float(lo), int(steps), a.ctypes.data_as(ctypes.c_void_p),
                              b.ctypes.data_as(ctypes.c_void_p), ctypes.byref(lk))
    return a, b, lk.value


def proj_poly(x, sides, lo: float, steps: int = 0, out=None, opts: Opts | None = None, offsets=None):
    """Factorization-free approximate projection of packed svec cones (C-ABI scs_psd_proj_poly)."""
    import torch
    _check_tensor(x, "x")
    if offsets is None:
        offsets, sides = shapes(sides)
    else:
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    if out is None:
        out = torch.empty_like(x)
    _check_tensor(out, "out")
    rc = load().scs_psd_proj_poly(handle(x.device.index), _ptr(x), _ptr(out), offsets.ctypes.data_as(ctypes.c_void_p),
                                  sides.ctypes.data_as(ctypes.c_void_p), int(sides.size), float(lo), int(steps),
                                  ctypes.byref(opts) if opts is not None else None, _stream_ptr(x))
    _check(rc, "scs_psd_proj_poly")
    return out


def proj_poly_hermitian(x, sides, lo: float, steps: int = 0, out=None, opts: Opts | None = None, offsets=None):
    """Factorization-free approximate projection of complex Hermitian cones (C-ABI scs_psd_proj_poly_hermitian)."""
    import torch
    _check_tensor(x, "x")
    if offsets is None:
        offsets, sides = hshapes(sides)
    else:
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    if out is None:
        out = torch.empty_like(x)
    _check_tensor(out, "out")
    rc = load().scs_psd_proj_poly_hermitian(handle(x.device.index), _ptr(x), _ptr(out),
                                            offsets.ctypes.data_as(ctypes.c_void_p),
                                            sides.ctypes.data_as(ctypes.c_void_p), int(sides.size), float(lo),
                                            int(steps), ctypes.byref(opts) if opts is not None else None,
                                            _stream_ptr(x))
    _check(rc, "scs_psd_proj_poly_hermitian")
    return out


def lambda_min(x, sides, out=None, opts: Opts | None = None, offsets=None):
    """Smallest eigenvalue of every cone (C-ABI scs_psd_lambda_min): a float64 CUDA tensor of count values."""
    import torch
    _check_tensor(x, "x")
    if offsets is None:
        offsets, sides = shapes(sides)
    else:
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    if out is None:
        out = torch.empty(int(sides.size), dtype=torch.float64, device=x.device)
    _check_tensor(out, "out")
    rc = load().scs_psd_lambda_min(handle(x.device.index), _ptr(x), _ptr(out), offsets.ctypes.data_as(ctypes.c_void_p),
                                   sides.ctypes.data_as(ctypes.c_void_p), int(sides.size),
                                   ctypes.byref(opts) if opts is not None else None, _stream_ptr(x))
    _check(rc, "scs_psd_lambda_min")
    return out


def mix_identity(x, sides, groups, nu, eps: float, out=None, p_out=None, opts: Opts | None = None, offsets=None):
    """Positivity post-processing by mixing with nu * identity per group (C-ABI scs_psd_mix_identity).
    Returns (y, p)."""
    import torch
    _check_tensor(x, "x")
    if offsets is None:
        offsets, sides = shapes(sides)
    else:
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    groups = np.ascontiguousarray(np.asarray(groups, dtype=np.int32))
    nu = np.ascontiguousarray(np.asarray(nu, dtype=np.float64))
    if out is None:
        out = torch.empty_like(x)
    _check_tensor(out, "out")
    ng = int(groups.size) - 1
    if p_out is None:
        p_out = torch.empty(max(ng, 1), dtype=torch.float64, device=x.device)
    rc = load().scs_psd_mix_identity(handle(x.device.index), _ptr(x), _ptr(out),
                                     offsets.ctypes.data_as(ctypes.c_void_p), sides.ctypes.data_as(ctypes.c_void_p),
                                     int(sides.size), groups.ctypes.data_as(ctypes.c_void_p), ng,
                                     nu.ctypes.data_as(ctypes.c_void_p), float(eps), _ptr(p_out),
                                     ctypes.byref(opts) if opts is not None else None, _stream_ptr(x))
    _check(rc, "scs_psd_mix_identity")
    return out, p_out[:ng]


def scs_iterate(A, b, c, sides, u, v, iters: int, opts: Opts | None = None, offsets=None):
    """SCS iterations around the projection (C-ABI scs_psd_scs_iterate); A is an m x k float64 CUDA
    tensor with orthonormal columns (column-major, i.e. A.T contiguous); u, v updated in place."""
    for t, nm in ((b, "b"), (u, "u"), (v, "v")):
        _check_tensor(t, nm)
    m, k = int(A.shape[0]), int(A.shape[1])
    Acm = A.t().contiguous() if not A.t().is_contiguous() else A.t()
    if offsets is None:
        offsets, sides = shapes(sides)
    else:
        offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        sides = np.ascontiguousarray(np.asarray(sides, dtype=np.int32))
    rc = load().scs_psd_scs_iterate(handle(u.device.index), _ptr(Acm), _ptr(b), _ptr(c) if k else None, m, k,
                                    offsets.ctypes.data_as(ctypes.c_void_p), sides.ctypes.data_as(ctypes.c_void_p),
                                    int(sides.size), _ptr(u), _ptr(v), int(iters),
                                    ctypes.byref(opts) if opts is not None else None, _stream_ptr(u))
    _check(rc, "scs_psd_scs_iterate")
    return u, v


def kron_operator(bases, index):
    """The C-ABI description of a structured operator: bases is a list of
    float64 CUDA tensors of shape (k_s, d_s, d_s) holding B_s[b][i, j] (made
    column-major per matrix here), index an int64 CUDA tensor of flat indices.
    Returns (KronOp, tensors to keep alive while the operator is in use)."""
    import torch
    if len(bases) < 1 or len(bases) > 6:
        raise ValueError("1 to 6 modes")
    _check_index = index
    if not isinstance(_check_index, torch.Tensor) or not index.is_cuda or index.dtype != torch.int64:
        raise TypeError("index must be an int64 CUDA tensor")
    keep = [index.contiguous()]
    op = KronOp()
    op.nmodes = len(bases)
    for s_, B in enumerate(bases):
        if not isinstance(B, torch.Tensor) or not B.is_cuda or B.dtype != torch.float64 or B.dim() != 3:
            raise TypeError("each local basis must be a float64 CUDA tensor of shape (k, d, d)")
        Bc = B.transpose(1, 2).contiguous()
        keep.append(Bc)
        op.dims[s_] = int(B.shape[1])
        op.nbasis[s_] = int(B.shape[0])
        op.basis[s_] = Bc.data_ptr()
    op.nparams = int(keep[0].numel())
    op.index = keep[0].data_ptr() if op.nparams else None
    return op, keep


def scs_iterate_kron(bases, index, b, c, u, v, iters: int, opts: Opts | None = None):
    """SCS iterations around the projection of one cone of side prod d_s with
    the structured operator (C-ABI scs_psd_scs_iterate_kron); u, v updated in place."""
    for t, nm in ((b, "b"), (c, "c"), (u, "u"), (v, "v")):
        _check_tensor(t, nm)
    op, keep = kron_operator(bases, index)
    rc = load().scs_psd_scs_iterate_kron(handle(u.device.index), ctypes.byref(op), _ptr(b), _ptr(c), _ptr(u),
                                         _ptr(v), int(iters), ctypes.byref(opts) if opts is not None else None,
                                         _stream_ptr(u))
    del keep
    _check(rc, "scs_psd_scs_iterate_kron")
    return u, v


TUNING_FIELDS = ("band", "gemm_ctas", "bt1_cols", "sy_share")


def autotune(x, sides, opts: Opts | None = None, offsets=None) -> dict:
    """Time launch-shape candidates on x and keep the fastest for these shapes
    (C-ABI scs_psd_autotune); returns the choice and its time per call."""
    _check_tensor(x, "x")
    offsets, sides = _shape_arrays(sides, offsets)
    out = (ctypes.c_int32 * 4)()
    ms = ctypes.c_double(0.0)
    rc = load().scs_psd_autotune(handle(x.device.index), _ptr(x), offsets.ctypes.data_as(ctypes.c_void_p),
                                 sides.ctypes.data_as(ctypes.c_void_p), int(sides.size),
                                 ctypes.byref(opts) if opts is not None else None, _stream_ptr(x), out,
                                 ctypes.byref(ms))
    _check(rc, "scs_psd_autotune")
    d = dict(zip(TUNING_FIELDS, [int(v) for v in out]))
    d["ms"] = float(ms.value)
    return d


def last_tuning(device: int = 0) -> dict:
    """Launch shapes of the last call on the device."""
    out = (ctypes.c_int32 * 4)()
    _check(load().scs_psd_last_tuning(handle(device), out), "scs_psd_last_tuning")
    return dict(zip(TUNING_FIELDS, [int(v) for v in out]))


def reserve(max_n: int, max_count: int = 1, opts: Opts | None = None, device: int = 0) -> None:
    """Build the plan of max_count cones of side max_n ahead of the first call (C-ABI scs_psd_reserve)."""
    _check(load().scs_psd_reserve(handle(device), int(max_n), int(max_count),
                                  ctypes.byref(opts) if opts is not None else None), "scs_psd_reserve")


def status(device: int = 0) -> int:
    """Synchronise and return the device status of the work since the last query."""
    v = ctypes.c_int32(0)
    _check(load().scs_psd_status(handle(device), ctypes.byref(v)), "scs_psd_status")
    return int(v.value)


STATS_FIELDS = ("k_pos", "k_neg", "route", "status", "complementarity", "norm_y", "norm_x")


def last_stats(count: int, device: int = 0) -> list[dict]:
    """Per-cone statistics of the last call made with make_opts(stats=True) (C-ABI scs_psd_last_stats)."""
    out = (ConeStats * max(1, int(count)))()
    _check(load().scs_psd_last_stats(handle(device), out, int(count)), "scs_psd_last_stats")
    return [{f: getattr(out[i], f) for f in STATS_FIELDS} for i in range(int(count))]


def last_launch_count(device: int = 0) -> int:
    return int(load().scs_psd_last_launch_count(handle(device)))


def last_replayed(device: int = 0) -> bool:
    """True if the last call on the device replayed a recorded CUDA graph."""
    return load().scs_psd_last_replayed(handle(device)) == 1


def trace(enable: bool, device: int = 0) -> None:
    """Turn per-phase CUDA-event timing on or off."""
    _check(load().scs_psd_trace(handle(device), int(bool(enable))), "scs_psd_trace")


def trace_read(device: int = 0):
    """{phase: (ms, intervals)} summed since the last read (synchronises)."""
    ms = (ctypes.c_double * NPHASES)()
    cnt = (ctypes.c_int64 * NPHASES)()
    _check(load().scs_psd_trace_read(handle(device), ms, cnt), "scs_psd_trace_read")
    return {PHASES[i]: (float(ms[i]), int(cnt[i])) for i in range(NPHASES)}
