"""Python binding of the h2rs C-ABI (``include/h2rs.h``) through ctypes.

Argument marshalling only: every step of the factorisation and solve runs in the
library's CUDA kernels.  Functions keep the C names.  Vectors are float64 torch
tensors in cluster-tree order, either 1-D (one right-hand side) or 2-D of shape
(n, nrhs) in column-major layout (``stride(0) == 1``; see :func:`colmajor`), on the
GPU (used in place) or on the host (copied by the library).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libh2rs.so")

H2_PREC_FP64 = 0
H2_PREC_FP32 = 1
H2_PREC_TF32X3 = 2

ERRORS = {0: "H2_OK", -1: "H2_ERR_ARG", -2: "H2_ERR_OOM", -3: "H2_ERR_SINGULAR",
          -4: "H2_ERR_RANK_CAP", -5: "H2_ERR_NONFINITE", -6: "H2_ERR_NO_CONVERGENCE",
          -7: "H2_ERR_TIMEOUT", -8: "H2_ERR_CUDA", -9: "H2_ERR_STATE"}

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_dp = ctypes.POINTER(ctypes.c_double)


class h2_matrix_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("depth", ctypes.c_int32), ("values_on_device", ctypes.c_int32),
                ("node_start", _i64p), ("node_size", _i64p), ("rank", _i64p),
                ("U_off", _i64p), ("U", _dp), ("E_off", _i64p), ("E", _dp),
                ("adm_ptr", _i64p), ("adm_col", _i64p), ("S_off", _i64p), ("S", _dp),
                ("inad_ptr", _i64p), ("inad_col", _i64p), ("D_off", _i64p), ("D", _dp),
                ("stream", ctypes.c_void_p)]


class h2_factor_opts(ctypes.Structure):
    _fields_ = [("eps_lu", ctypes.c_double), ("norm_a", ctypes.c_double), ("precision", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p), ("sys_norm_a", _dp),
                ("force_ranks", ctypes.POINTER(ctypes.c_int32)), ("k_cap", ctypes.c_int32)]


class h2_factor_stats(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int32), ("top_level", ctypes.c_int32), ("top_size", ctypes.c_int64),
                ("factor_bytes", ctypes.c_int64), ("peak_bytes", ctypes.c_int64),
                ("error_level", ctypes.c_int32), ("error_box", ctypes.c_int32),
                ("factor_ms", ctypes.c_double), ("phase_ms", ctypes.c_double * 8),
                ("phase_flops", ctypes.c_double * 8), ("phase_bytes", ctypes.c_double * 8),
                ("kernel_ms", ctypes.c_double * 16), ("kernel_launches", ctypes.c_int64 * 16),
                ("host_ms", ctypes.c_double * 4), ("schur_reread_bytes", ctypes.c_double)]


PHASES = ["augment", "project", "lu_trsm", "schur", "close", "top", "leaf_load", "other"]
KERNELS = ["gather", "basis", "proj", "zero", "lu", "trsm", "schur", "close", "top", "load", "pack"]
H2_FLAG_TIME_KERNELS = 1
H2_FLAG_DEBUG_SHORT_WAIT = 2
H2_FLAG_W_TRIANGULAR = 4
H2_FLAG_W_INVERSE = 8

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("h2_matrix_create", ctypes.c_int, [ctypes.POINTER(h2_matrix_desc), ctypes.POINTER(ctypes.c_void_p)]),
    ("h2_matrix_destroy", None, [ctypes.c_void_p]),
    ("h2_matrix_create_batch", ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(h2_matrix_desc),
                                              ctypes.POINTER(ctypes.c_void_p)]),
    ("h2_matrix_batch_info", ctypes.c_int, [ctypes.c_void_p, _i32p, _i64p]),
    ("h2_matvec", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]),
    ("h2_matvec_static", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_int64]),
    ("h2_factor_create", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(h2_factor_opts),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    ("h2_factor_destroy", None, [ctypes.c_void_p]),
    ("h2_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_int32]),
    ("h2_refine_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_int32, ctypes.c_int32, _i32p, _dp]),
    ("h2_factor_stats_get", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(h2_factor_stats)]),
    ("h2_layout_counts", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _i64p, _i64p]),
    ("h2_layout_get", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _i64p, _i64p, _i32p, _i64p, _i64p,
                                     _i32p, _i64p]),
    ("h2_plan_query", ctypes.c_int, [ctypes.POINTER(h2_matrix_desc), ctypes.c_int32, _i64p, _i64p, _i32p,
                                     _i64p, _i64p, _i32p]),
    ("h2_plan_query_batch", ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(h2_matrix_desc), ctypes.c_int32,
                                           _i64p, _i64p, _i32p, _i64p, _i64p, _i32p, _i32p, _i32p]),
    ("h2_kernel_launch_count", ctypes.c_int64, []),
    ("h2_last_error", ctypes.c_char_p, []),
    ("h2_version", ctypes.c_char_p, []),
]

EXPORTED = [s[0] for s in _SIGS]

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2509_11152_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class H2Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(rc: int) -> None:
    if rc != 0:
        raise H2Error(rc, lib().h2_last_error().decode())


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _vals(t: torch.Tensor):
    t = t.contiguous()
    return t, ctypes.cast(ctypes.c_void_p(t.data_ptr()), _dp)


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """A column-major (n, nrhs) copy of ``t`` (1-D tensors become (n, 1))."""
    if t.dim() == 1:
        t = t.reshape(-1, 1)
    return t.t().contiguous().t()


def _vec(t: torch.Tensor):
    """(pointer, nrhs, ld, on_device) of a float64 vector / column-major matrix."""
    if t.dtype != torch.float64:
        raise TypeError("vectors must be float64")
    if t.dim() == 1:
        if not t.is_contiguous():
            raise ValueError("1-D vector must be contiguous")
        return t.data_ptr(), 1, t.shape[0], int(t.is_cuda)
    if t.dim() != 2 or t.stride(0) != 1:
        raise ValueError("2-D vectors must be column-major (stride(0) == 1); use colmajor()")
    ld = t.stride(1) if t.shape[1] > 1 else t.shape[0]
    return t.data_ptr(), t.shape[1], ld, int(t.is_cuda)


def make_desc(A, stream=None):
    """Descriptor of an ``h2gen.H2Matrix`` plus the arrays that must stay alive."""
    keep = {}
    d = h2_matrix_desc()
    d.n = int(A.n)
    d.depth = int(A.depth)
    on_dev = A.U.is_cuda
    d.values_on_device = int(on_dev)
    for name in ("node_start", "node_size", "rank", "U_off", "E_off", "adm_ptr", "adm_col", "S_off",
                 "inad_ptr", "inad_col", "D_off"):
        arr = np.ascontiguousarray(np.asarray(getattr(A, name), dtype=np.int64))
        keep[name] = arr
        setattr(d, name, _ptr(arr, ctypes.c_int64))
    for name in ("U", "E", "S", "D"):
        t = getattr(A, name)
        if not torch.is_tensor(t):
            t = torch.from_numpy(np.ascontiguousarray(t))
        t = t.to(torch.float64)
        t, p = _vals(t)
        keep[name] = t
        setattr(d, name, p)
    d.stream = ctypes.c_void_p(stream) if stream else None
    return d, keep


class Matrix:
    """Owning handle of an ``h2_matrix``."""

    def __init__(self, handle, n):
        self.handle = handle
        self.n = n

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.h2_matrix_destroy(self.handle)
            self.handle = None


class Factor:
    """Owning handle of an ``h2_factor`` (keeps its matrix alive)."""

    def __init__(self, handle, matrix, precision):
        self.handle = handle
        self.matrix = matrix
        self.precision = precision

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.h2_factor_destroy(self.handle)
            self.handle = None


def h2_matrix_create(A, stream=None) -> Matrix:
    d, keep = make_desc(A, stream)
    h = ctypes.c_void_p()
    _check(lib().h2_matrix_create(ctypes.byref(d), ctypes.byref(h)))
    del keep
    return Matrix(h, int(A.n))


def h2_matrix_create_batch(As, stream=None) -> Matrix:
    """One block-diagonal matrix of the independent H^2 matrices ``As`` (vectors are
    the systems' vectors stacked in this order)."""
    descs, keeps = zip(*[make_desc(A, stream) for A in As])
    arr = (h2_matrix_desc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _check(lib().h2_matrix_create_batch(len(descs), arr, ctypes.byref(h)))
    del keeps
    return Matrix(h, int(sum(int(A.n) for A in As)))


def h2_matrix_batch_info(M: Matrix) -> np.ndarray:
    """Row offsets of the systems of ``M`` (nsys + 1 entries)."""
    ns = ctypes.c_int32()
    _check(lib().h2_matrix_batch_info(M.handle, ctypes.byref(ns), None))
    off = np.zeros(ns.value + 1, np.int64)
    _check(lib().h2_matrix_batch_info(M.handle, None, _ptr(off, ctypes.c_int64)))
    return off


def h2_factor_create(M: Matrix, eps_lu: float, norm_a, precision: int = H2_PREC_FP64,
                     stream=None, flags: int = 0, force_ranks=None, k_cap: int = 0) -> Factor:
    """``norm_a``: ||A||_2, or for a batch one norm per system (a sequence).
    ``force_ranks``: debug, the augmented ranks of every level (a sequence of arrays,
    leaves first) that the factorisation must use instead of truncating."""
    o = h2_factor_opts()
    o.eps_lu = float(eps_lu)
    keep = None
    if np.ndim(norm_a) == 0:
        o.norm_a = float(norm_a)
    else:
        keep = np.ascontiguousarray(np.asarray(norm_a, dtype=np.float64))
        o.norm_a = float(keep.max())
        o.sys_norm_a = _ptr(keep, ctypes.c_double)
    o.precision = int(precision)
    o.flags = int(flags)
    o.k_cap = int(k_cap)
    if force_ranks is not None:
        fr = np.ascontiguousarray(np.concatenate([np.asarray(r, dtype=np.int32).ravel() for r in force_ranks])
                                  if len(force_ranks) else np.zeros(0, np.int32))
        o.force_ranks = fr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        keep = (keep, fr)
    o.stream = ctypes.c_void_p(stream) if stream else None
    h = ctypes.c_void_p()
    _check(lib().h2_factor_create(M.handle, ctypes.byref(o), ctypes.byref(h)))
    return Factor(h, M, precision)


def h2_solve(Z: Factor, b: torch.Tensor) -> torch.Tensor:
    """In place: ``b`` is overwritten with ``A^-1 b``; returns ``b``."""
    p, nrhs, ld, dev = _vec(b)
    _check(lib().h2_solve(Z.handle, nrhs, ctypes.c_void_p(p), ld, dev))
    return b


def h2_matvec(M: Matrix, x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    px, nrhs, ldx, dev = _vec(x)
    py, nrhs_y, ldy, dev_y = _vec(y)
    if nrhs != nrhs_y or dev != dev_y:
        raise ValueError("x and y must match in shape and device")
    _check(lib().h2_matvec(M.handle, nrhs, ctypes.c_void_p(px), ldx, ctypes.c_void_p(py), ldy, dev))
    return y


def h2_matvec_static(M: Matrix, x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """``h2_matvec`` without device allocation (x, y on the GPU; see the header)."""
    px, nrhs, ldx, dev = _vec(x)
    py, nrhs_y, ldy, dev_y = _vec(y)
    if nrhs != nrhs_y or not dev or not dev_y:
        raise ValueError("x and y must be GPU tensors of the same shape")
    _check(lib().h2_matvec_static(M.handle, nrhs, ctypes.c_void_p(px), ldx, ctypes.c_void_p(py), ldy))
    return y


def h2_refine_solve(Z: Factor, M: Matrix, b: torch.Tensor, x: torch.Tensor, tol: float = 1e-10,
                    maxit: int = 20):
    """Returns (iterations, backward error, converged)."""
    pb, nrhs, ldb, dev = _vec(b)
    px, nrhs_x, ldx, dev_x = _vec(x)
    if nrhs != nrhs_x or dev != dev_x:
        raise ValueError("b and x must match in shape and device")
    it = ctypes.c_int32()
    be = ctypes.c_double()
    rc = lib().h2_refine_solve(Z.handle, M.handle, nrhs, ctypes.c_void_p(pb), ldb, ctypes.c_void_p(px), ldx,
                               float(tol), int(maxit), dev, ctypes.byref(it), ctypes.byref(be))
    if rc not in (0, -6):
        _check(rc)
    return it.value, be.value, rc == 0


def h2_factor_stats_get(Z: Factor) -> dict:
    s = h2_factor_stats()
    _check(lib().h2_factor_stats_get(Z.handle, ctypes.byref(s)))
    return dict(nlevels=s.nlevels, top_level=s.top_level, top_size=s.top_size, factor_bytes=s.factor_bytes,
                peak_bytes=s.peak_bytes, error_level=s.error_level, error_box=s.error_box,
                factor_ms=s.factor_ms, phase_ms=dict(zip(PHASES, list(s.phase_ms))),
                phase_flops=dict(zip(PHASES, list(s.phase_flops))),
                phase_bytes=dict(zip(PHASES, list(s.phase_bytes))),
                kernel_ms=dict(zip(KERNELS, list(s.kernel_ms))),
                kernel_launches=dict(zip(KERNELS, list(s.kernel_launches))),
                host_ms=dict(zip(["work_lists", "uploads", "level_setup_close", "rank_readback"],
                                 list(s.host_ms))),
                schur_reread_bytes=s.schur_reread_bytes)


def h2_layout_get(Z: Factor, level: int) -> dict:
    nbox = ctypes.c_int64()
    nblk = ctypes.c_int64()
    _check(lib().h2_layout_counts(Z.handle, level, ctypes.byref(nbox), ctypes.byref(nblk)))
    nb, nk = nbox.value, nblk.value
    out = dict(sizes=np.zeros(nb, np.int64), ranks=np.zeros(nb, np.int64), colour=np.zeros(nb, np.int32),
               row_ptr=np.zeros(nb + 1, np.int64), col=np.zeros(nk, np.int64), kind=np.zeros(nk, np.int32),
               offset=np.zeros(nk + 1, np.int64))
    _check(lib().h2_layout_get(Z.handle, level, _ptr(out["sizes"], ctypes.c_int64),
                               _ptr(out["ranks"], ctypes.c_int64), _ptr(out["colour"], ctypes.c_int32),
                               _ptr(out["row_ptr"], ctypes.c_int64), _ptr(out["col"], ctypes.c_int64),
                               _ptr(out["kind"], ctypes.c_int32), _ptr(out["offset"], ctypes.c_int64)))
    return out


def h2_plan_query(A, level: int) -> dict:
    """Host-only: structure of skeletonised level ``level`` (0 = leaves) as planned by
    the library (no GPU needed; only the index arrays of ``A`` are read)."""
    d, keep = make_desc(A)
    nbox = ctypes.c_int64()
    nblk = ctypes.c_int64()
    _check(lib().h2_plan_query(ctypes.byref(d), level, ctypes.byref(nbox), ctypes.byref(nblk),
                               None, None, None, None))
    nb, nk = nbox.value, nblk.value
    out = dict(colour=np.zeros(nb, np.int32), row_ptr=np.zeros(nb + 1, np.int64), col=np.zeros(nk, np.int64),
               kind=np.zeros(nk, np.int32))
    _check(lib().h2_plan_query(ctypes.byref(d), level, None, None, _ptr(out["colour"], ctypes.c_int32),
                               _ptr(out["row_ptr"], ctypes.c_int64), _ptr(out["col"], ctypes.c_int64),
                               _ptr(out["kind"], ctypes.c_int32)))
    del keep
    return out


def h2_plan_query_batch(As, level: int) -> dict:
    """Host-only: forest level ``level`` (0 = leaves) of the batch ``As`` as planned by
    the library, with each box's state and system."""
    descs, keeps = zip(*[make_desc(A) for A in As])
    arr = (h2_matrix_desc * len(descs))(*descs)
    nbox = ctypes.c_int64()
    nblk = ctypes.c_int64()
    _check(lib().h2_plan_query_batch(len(descs), arr, level, ctypes.byref(nbox), ctypes.byref(nblk),
                                     None, None, None, None, None, None))
    nb, nk = nbox.value, nblk.value
    out = dict(colour=np.zeros(nb, np.int32), row_ptr=np.zeros(nb + 1, np.int64), col=np.zeros(nk, np.int64),
               kind=np.zeros(nk, np.int32), state=np.zeros(nb, np.int32), system=np.zeros(nb, np.int32))
    _check(lib().h2_plan_query_batch(len(descs), arr, level, None, None, _ptr(out["colour"], ctypes.c_int32),
                                     _ptr(out["row_ptr"], ctypes.c_int64), _ptr(out["col"], ctypes.c_int64),
                                     _ptr(out["kind"], ctypes.c_int32), _ptr(out["state"], ctypes.c_int32),
                                     _ptr(out["system"], ctypes.c_int32)))
    del keeps
    return out


def h2_version() -> str:
    return lib().h2_version().decode()
