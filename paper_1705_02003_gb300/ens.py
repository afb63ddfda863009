"""ctypes binding of libens (include/ens.h): the same entry points, taking torch
tensors for device arrays and numpy arrays for host arrays.

Argument marshalling only -- every step runs in the CUDA kernels of the
library.  There is no CPU fallback: if the library cannot be built or loaded,
``load()`` raises.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np
import torch

from . import build as _build

FD5_LOGKL, Q1_ROT, FD7_AXIS, Q1_3D_KL, Q1_3D_DISC = 1, 2, 3, 4, 5
KINDS = {"fd5": FD5_LOGKL, "q1": Q1_ROT, "fd7": FD7_AXIS, "q1_3d_kl": Q1_3D_KL, "q1_3d_disc": Q1_3D_DISC}

OK, EINVAL, ECUDA, ENOMEM, ETIMEOUT, ENOTSUP = 0, -1, -2, -3, -4, -5
LANE_CONVERGED, LANE_MAXIT, LANE_BREAKDOWN, LANE_BADINPUT, LANE_INACTIVE = 0, 1, 2, 3, 4

EXPORTS = ("ens_create", "ens_destroy", "ens_last_error", "ens_problem_size", "ens_pattern",
           "ens_assemble", "ens_pcg_workspace_size", "ens_pcg_solve", "ens_group", "ens_sort_chunk",
           "ens_sg_refine", "ens_sg_initial", "ens_sg_eval", "ens_qoi", "ens_spmv",
           "ens_pcg_solve_static", "ens_pcg_ir_workspace_size", "ens_pcg_solve_ir",
           "ens_adjoint_workspace_size", "ens_adjoint_grad", "ens_param_indicator",
           "ens_stream_workspace_size", "ens_solve_stream", "ens_pcg_branches", "ens_check_pattern",
           "ens_mg_workspace_size", "ens_mg_setup", "ens_mg_level", "ens_mg_apply", "ens_mgpcg_solve",
           "ens_sg_points", "ens_fp64_peak", "ens_fp64_peak_flops", "ens_adjoint_solve_workspace_size",
           "ens_adjoint_solve_grad", "ens_pcg_cluster_size")

_lib = None
_lock = threading.Lock()


class EnsError(RuntimeError):
    pass


class Problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("nparam", ctypes.c_int),
                ("aniso", ctypes.c_double)]


def problem(kind, n: int, nparam: int, aniso: float) -> Problem:
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    return Problem(k, int(n), int(nparam), float(aniso))


def load(path: str | None = None):
    """Build (if stale) and load libens.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            so = path or _build.build()
            L = ctypes.CDLL(so)
            _declare(L)
            _lib = L
        return _lib


def _declare(L):
    c = ctypes
    vp = c.c_void_p
    L.ens_create.argtypes = [c.POINTER(vp), c.c_int]
    L.ens_destroy.argtypes = [vp]
    L.ens_last_error.argtypes = [vp]
    L.ens_last_error.restype = c.c_char_p
    L.ens_problem_size.argtypes = [c.POINTER(Problem), c.POINTER(c.c_int), c.POINTER(c.c_int64)]
    L.ens_pattern.argtypes = [vp, c.POINTER(Problem), vp, vp, vp]
    L.ens_assemble.argtypes = [vp, c.POINTER(Problem), c.c_int, c.c_int, vp, vp, vp, vp, c.c_int, vp,
                               vp, vp]
    L.ens_check_pattern.argtypes = [vp, c.c_int, c.c_int64, vp, vp, vp]
    L.ens_pcg_branches.argtypes = [vp, c.c_int]
    L.ens_pcg_branches.restype = c.c_int
    L.ens_pcg_cluster_size.argtypes = [vp, c.c_int, c.c_int64, c.c_int, c.c_int]
    L.ens_pcg_cluster_size.restype = c.c_int
    L.ens_pcg_workspace_size.argtypes = [c.c_int, c.c_int64, c.c_int, c.c_int]
    L.ens_pcg_workspace_size.restype = c.c_size_t
    L.ens_pcg_solve.argtypes = [vp, c.c_int, c.c_int64, c.c_int, c.c_int, vp, vp, vp, vp, vp, vp, vp,
                                c.c_double, c.c_int, vp, vp, vp, vp, c.c_size_t, vp]
    L.ens_group.argtypes = [vp, c.c_int, c.c_int, vp, vp, vp, c.c_int, vp, c.c_int, vp, vp,
                            c.POINTER(c.c_int), vp]
    L.ens_sort_chunk.argtypes = [vp, c.c_int, vp, c.c_int, vp, c.POINTER(c.c_int), vp]
    L.ens_sg_eval.argtypes = [vp, c.c_int, c.c_int, vp, vp, vp, c.c_int, vp, vp, vp, vp]
    L.ens_qoi.argtypes = [vp, c.c_int, c.c_int, c.c_int, vp, vp, vp, vp]
    L.ens_spmv.argtypes = [vp, c.c_int, c.c_int64, c.c_int, c.c_int, vp, vp, vp, vp, vp, vp, vp, c.c_size_t, vp]
    L.ens_stream_workspace_size.argtypes = [c.POINTER(Problem), c.c_int, c.c_int]
    L.ens_stream_workspace_size.restype = c.c_size_t
    L.ens_solve_stream.argtypes = [vp, c.POINTER(Problem), c.c_int, c.c_int, c.c_int, vp, vp, vp, c.c_double,
                                   c.c_int, c.c_int, vp, vp, vp, vp, vp, c.c_size_t, vp]
    L.ens_param_indicator.argtypes = [vp, c.POINTER(Problem), c.c_int, vp, vp, vp]
    L.ens_mg_workspace_size.argtypes = [c.POINTER(Problem), c.c_int, c.c_int, c.c_int]
    L.ens_mg_workspace_size.restype = c.c_size_t
    L.ens_mg_setup.argtypes = [vp, c.POINTER(Problem), c.c_int, c.c_int, c.c_int, vp, vp, vp, vp, c.c_size_t, vp]
    L.ens_mg_level.argtypes = [vp, c.POINTER(Problem), c.c_int, c.c_int, c.c_int, c.c_int, vp, vp, vp, c.c_size_t,
                               vp]
    L.ens_mg_apply.argtypes = [vp, c.POINTER(Problem), c.c_int, c.c_int, c.c_int, vp, vp, vp, vp, vp, vp, c.c_size_t,
                               vp]
    L.ens_mgpcg_solve.argtypes = [vp, c.POINTER(Problem), c.c_int, c.c_int, c.c_int, vp, vp, vp, vp, vp, vp,
                                  c.c_double, c.c_int, vp, vp, vp, vp, c.c_size_t, vp]
    L.ens_adjoint_workspace_size.argtypes = [c.POINTER(Problem), c.c_int, c.c_int]
    L.ens_adjoint_workspace_size.restype = c.c_size_t
    L.ens_adjoint_grad.argtypes = [vp, c.POINTER(Problem), c.c_int, c.c_int, vp, vp, vp, vp, vp, c.c_size_t, vp]
    L.ens_adjoint_solve_workspace_size.argtypes = [c.POINTER(Problem), c.c_int, c.c_int]
    L.ens_adjoint_solve_workspace_size.restype = c.c_size_t
    L.ens_adjoint_solve_grad.argtypes = [vp, c.POINTER(Problem), c.c_int, c.c_int, vp, vp, vp, vp, vp, vp, c.c_double,
                                         c.c_int, vp, vp, vp, vp, vp, vp, vp, c.c_size_t, vp]
    L.ens_pcg_ir_workspace_size.argtypes = [c.c_int, c.c_int64, c.c_int, c.c_int]
    L.ens_pcg_ir_workspace_size.restype = c.c_size_t
    L.ens_pcg_solve_ir.argtypes = [vp, c.c_int, c.c_int64, c.c_int, c.c_int, vp, vp, vp, vp, vp, vp, vp, vp,
                                   c.c_double, c.c_double, c.c_int, c.c_int, vp, vp, vp, vp, vp, c.c_size_t, vp]
    L.ens_pcg_solve_static.argtypes = [vp, c.c_int, c.c_int64, c.c_int, c.c_int, vp, vp, vp, vp, vp, vp, vp,
                                       c.c_double, c.c_int, vp, vp, vp, vp]
    i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    L.ens_sg_refine.argtypes = [c.c_int, c.c_int, i8p, i32p, c.c_int, f64p, c.c_double, c.c_int,
                                c.c_int, i8p, i32p]
    L.ens_sg_initial.argtypes = [c.c_int, c.c_int, c.c_int, i8p, i32p]
    L.ens_sg_points.argtypes = [c.c_int, c.c_int, i8p, i32p, f64p]
    L.ens_fp64_peak.argtypes = [vp, c.c_int, c.c_int, vp, vp]
    L.ens_fp64_peak_flops.argtypes = [c.c_int, c.c_int]
    L.ens_fp64_peak_flops.restype = c.c_double


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("device array expected (CUDA tensor)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check_dtype(t, dt, name):
    if t is not None and t.dtype != dt:
        raise TypeError(f"{name} must be {dt}, got {t.dtype}")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Handle:
    """Owns an ens_handle (graph cache, capture stream) for one device."""

    def __init__(self, device: int | None = None):
        L = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = ctypes.c_void_p()
        rc = L.ens_create(ctypes.byref(h), self.device)
        if rc != OK:
            raise EnsError(f"ens_create failed ({rc})")
        self._h = h

    @property
    def ptr(self):
        return self._h

    def check(self, rc, what):
        if rc != OK:
            msg = load().ens_last_error(self._h).decode()
            raise EnsError(f"{what} failed ({rc}): {msg}")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ens_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def ens_problem_size(prob: Problem):
    J = ctypes.c_int()
    nnz = ctypes.c_int64()
    rc = load().ens_problem_size(ctypes.byref(prob), ctypes.byref(J), ctypes.byref(nnz))
    if rc != OK:
        raise EnsError(f"ens_problem_size failed ({rc})")
    return J.value, nnz.value


def ens_pattern(h: Handle, prob: Problem, rowptr, colidx, stream=None):
    _check_dtype(rowptr, torch.int32, "rowptr")
    _check_dtype(colidx, torch.int32, "colidx")
    J, nnz = ens_problem_size(prob)
    if rowptr.numel() != J + 1 or colidx.numel() != nnz:
        raise ValueError("rowptr/colidx sizes do not match the problem")
    h.check(load().ens_pattern(h.ptr, ctypes.byref(prob), _ptr(rowptr), _ptr(colidx), _stream(stream)),
            "ens_pattern")


def ens_assemble(h: Handle, prob: Problem, S: int, E: int, xi, rowptr, colidx, vals, dinv=None, b=None,
                 stream=None):
    J, nnz = ens_problem_size(prob)
    _check_dtype(xi, torch.float64, "xi")
    if vals.dtype not in (torch.float64, torch.float32):
        raise TypeError("vals must be float64 or float32")
    if xi.numel() != E * S * prob.nparam or vals.numel() != E * nnz * S:
        raise ValueError("xi / vals sizes do not match E, S, nparam, nnz")
    for t, nm in ((dinv, "dinv"), (b, "b")):
        if t is not None:
            _check_dtype(t, torch.float64, nm)
            if t.numel() != E * J * S:
                raise ValueError(f"{nm} size does not match E * J * S")
    rc = load().ens_assemble(h.ptr, ctypes.byref(prob), int(S), int(E), _ptr(xi), _ptr(rowptr),
                             _ptr(colidx), _ptr(vals), int(vals.dtype == torch.float32), _ptr(dinv),
                             _ptr(b), _stream(stream))
    h.check(rc, "ens_assemble")


def ens_check_pattern(h: Handle, J: int, nnz: int, rowptr, colidx, stream=None):
    """Validate a CSR graph; raises EnsError naming the failed checks."""
    _check_dtype(rowptr, torch.int32, "rowptr")
    _check_dtype(colidx, torch.int32, "colidx")
    if rowptr.numel() != J + 1 or colidx.numel() != nnz:
        raise ValueError("rowptr must hold J + 1 and colidx nnz entries")
    h.check(load().ens_check_pattern(h.ptr, int(J), int(nnz), _ptr(rowptr), _ptr(colidx), _stream(stream)),
            "ens_check_pattern")


def ens_pcg_branches(h: Handle, E: int) -> int:
    """Independent while-loop branches ens_pcg_solve runs for E ensembles."""
    return int(load().ens_pcg_branches(h.ptr, int(E)))


def ens_pcg_cluster_size(h: Handle, J: int, nnz: int, S: int, E: int) -> int:
    """CTAs per ensemble of the one-launch cluster schedule ens_pcg_solve uses
    for this problem, or 0 where it runs the graph loop."""
    return int(load().ens_pcg_cluster_size(h.ptr, int(J), int(nnz), int(S), int(E)))


def ens_pcg_workspace_size(J: int, nnz: int, S: int, E: int) -> int:
    return int(load().ens_pcg_workspace_size(int(J), int(nnz), int(S), int(E)))


def ens_pcg_solve(h: Handle, J: int, nnz: int, S: int, E: int, rowptr, colidx, vals, dinv, b, x, active,
                  rtol: float, maxit: int, iters, relres, status, work, stream=None):
    for t, nm, dt in ((vals, "vals", torch.float64), (dinv, "dinv", torch.float64), (b, "b", torch.float64),
                      (x, "x", torch.float64), (iters, "iters", torch.int32), (relres, "relres", torch.float64),
                      (status, "status", torch.int32), (rowptr, "rowptr", torch.int32),
                      (colidx, "colidx", torch.int32)):
        _check_dtype(t, dt, nm)
    if active is not None:
        _check_dtype(active, torch.uint8, "active")
    if vals.numel() != E * nnz * S or x.numel() != E * J * S or iters.numel() != E * S:
        raise ValueError("array sizes do not match E, J, nnz, S")
    if work.dtype != torch.uint8:
        raise TypeError("work must be a uint8 tensor")
    rc = load().ens_pcg_solve(h.ptr, int(J), int(nnz), int(S), int(E), _ptr(rowptr), _ptr(colidx),
                              _ptr(vals), _ptr(dinv), _ptr(b), _ptr(x), _ptr(active), float(rtol),
                              int(maxit), _ptr(iters), _ptr(relres), _ptr(status), _ptr(work),
                              work.numel(), _stream(stream))
    h.check(rc, "ens_pcg_solve")


def ens_spmv(h: Handle, J: int, nnz: int, S: int, E: int, rowptr, colidx, vals, p, q, pq, work, stream=None):
    """q = A p per lane (and pq = p^T q per lane): the PCG loop's SpMV kernel alone."""
    for t, nm in ((vals, "vals"), (p, "p"), (q, "q")):
        _check_dtype(t, torch.float64, nm)
    if pq is not None:
        _check_dtype(pq, torch.float64, "pq")
    if vals.numel() != E * nnz * S or p.numel() != E * J * S or q.numel() != E * J * S:
        raise ValueError("array sizes do not match E, J, nnz, S")
    rc = load().ens_spmv(h.ptr, int(J), int(nnz), int(S), int(E), _ptr(rowptr), _ptr(colidx), _ptr(vals),
                         _ptr(p), _ptr(q), _ptr(pq), _ptr(work), work.numel(), _stream(stream))
    h.check(rc, "ens_spmv")


def ens_mg_workspace_size(prob: Problem, S: int, E: int, mixed: bool = False) -> int:
    """Bytes of workspace of the multigrid calls (0 when the problem has no hierarchy);
    mixed: the V-cycle runs in float."""
    return int(load().ens_mg_workspace_size(ctypes.byref(prob), int(S), int(E), int(bool(mixed))))


def _mg_sizes(prob, S, E, vals, work):
    J, nnz = ens_problem_size(prob)
    _check_dtype(vals, torch.float64, "vals")
    if vals.numel() != E * nnz * S:
        raise ValueError("vals size does not match E, nnz, S")
    if work.dtype != torch.uint8:
        raise TypeError("work must be a uint8 tensor")
    return J, nnz


def ens_mg_setup(h: Handle, prob: Problem, S: int, E: int, rowptr, colidx, vals, work, stream=None, mixed=False):
    """Build the per-sample multigrid hierarchy of the fine values into work."""
    _mg_sizes(prob, S, E, vals, work)
    rc = load().ens_mg_setup(h.ptr, ctypes.byref(prob), int(S), int(E), int(bool(mixed)), _ptr(rowptr),
                             _ptr(colidx), _ptr(vals), _ptr(work), work.numel(), _stream(stream))
    h.check(rc, "ens_mg_setup")


def ens_mg_level(h: Handle, prob: Problem, S: int, E: int, level: int, vals_out, lmax_out, work, stream=None,
                 mixed=False):
    """Copy a level's Galerkin values [E][nnz_l][S] and Gershgorin bounds [E][S] out of work."""
    for t, nm in ((vals_out, "vals_out"), (lmax_out, "lmax_out")):
        if t is not None:
            _check_dtype(t, torch.float64, nm)
    rc = load().ens_mg_level(h.ptr, ctypes.byref(prob), int(S), int(E), int(bool(mixed)), int(level),
                             _ptr(vals_out), _ptr(lmax_out), _ptr(work), work.numel(), _stream(stream))
    h.check(rc, "ens_mg_level")


def ens_mg_apply(h: Handle, prob: Problem, S: int, E: int, rowptr, colidx, vals, r, z, work, stream=None,
                 mixed=False):
    """z = one V-cycle applied to r (hierarchy of the last ens_mg_setup on work)."""
    J, _ = _mg_sizes(prob, S, E, vals, work)
    for t, nm in ((r, "r"), (z, "z")):
        _check_dtype(t, torch.float64, nm)
        if t.numel() != E * J * S:
            raise ValueError(f"{nm} size does not match E, J, S")
    rc = load().ens_mg_apply(h.ptr, ctypes.byref(prob), int(S), int(E), int(bool(mixed)), _ptr(rowptr), _ptr(colidx),
                             _ptr(vals), _ptr(r), _ptr(z), _ptr(work), work.numel(), _stream(stream))
    h.check(rc, "ens_mg_apply")


def ens_mgpcg_solve(h: Handle, prob: Problem, S: int, E: int, rowptr, colidx, vals, b, x, active, rtol: float,
                    maxit: int, iters, relres, status, work, stream=None, mixed=False):
    """Multigrid-preconditioned ensemble CG (after ens_mg_setup on work)."""
    J, _ = _mg_sizes(prob, S, E, vals, work)
    for t, nm, dt in ((b, "b", torch.float64), (x, "x", torch.float64), (iters, "iters", torch.int32),
                      (relres, "relres", torch.float64), (status, "status", torch.int32)):
        _check_dtype(t, dt, nm)
    if active is not None:
        _check_dtype(active, torch.uint8, "active")
    if b.numel() != E * J * S or x.numel() != E * J * S or iters.numel() != E * S:
        raise ValueError("array sizes do not match E, J, S")
    rc = load().ens_mgpcg_solve(h.ptr, ctypes.byref(prob), int(S), int(E), int(bool(mixed)), _ptr(rowptr),
                                _ptr(colidx), _ptr(vals), _ptr(b), _ptr(x), _ptr(active), float(rtol), int(maxit),
                                _ptr(iters), _ptr(relres), _ptr(status), _ptr(work), work.numel(), _stream(stream))
    h.check(rc, "ens_mgpcg_solve")


def ens_pcg_ir_workspace_size(J: int, nnz: int, S: int, E: int) -> int:
    return int(load().ens_pcg_ir_workspace_size(int(J), int(nnz), int(S), int(E)))


def ens_pcg_solve_ir(h: Handle, J: int, nnz: int, S: int, E: int, rowptr, colidx, vals, vals32, dinv, b, x,
                     active, rtol: float, rtol_inner: float, maxit_inner: int, maxit_outer: int, iters,
                     outer_its, relres, status, work, stream=None):
    """FP32 inner Jacobi-PCG inside FP64 iterative refinement (see include/ens.h)."""
    for t, nm, dt in ((vals, "vals", torch.float64), (vals32, "vals32", torch.float32),
                      (dinv, "dinv", torch.float64), (b, "b", torch.float64), (x, "x", torch.float64),
                      (iters, "iters", torch.int32), (outer_its, "outer_its", torch.int32),
                      (relres, "relres", torch.float64), (status, "status", torch.int32)):
        _check_dtype(t, dt, nm)
    if vals.numel() != E * nnz * S or vals32.numel() != E * nnz * S or x.numel() != E * J * S:
        raise ValueError("array sizes do not match E, J, nnz, S")
    rc = load().ens_pcg_solve_ir(h.ptr, int(J), int(nnz), int(S), int(E), _ptr(rowptr), _ptr(colidx), _ptr(vals),
                                 _ptr(vals32), _ptr(dinv), _ptr(b), _ptr(x), _ptr(active), float(rtol),
                                 float(rtol_inner), int(maxit_inner), int(maxit_outer), _ptr(iters),
                                 _ptr(outer_its), _ptr(relres), _ptr(status), _ptr(work), work.numel(),
                                 _stream(stream))
    h.check(rc, "ens_pcg_solve_ir")


def ens_stream_workspace_size(prob: Problem, S: int, E: int) -> int:
    return int(load().ens_stream_workspace_size(ctypes.byref(prob), int(S), int(E)))


def ens_solve_stream(h: Handle, prob: Problem, S: int, E: int, xi, order, rtol: float, maxit: int, chunk: int,
                     iters, status, relres, qoi=None, w=None, work=None, stream=None):
    """Continuous ensemble batching of the samples xi[M][N] (see include/ens.h)."""
    M = iters.numel()
    _check_dtype(xi, torch.float64, "xi")
    for t, nm, dt in ((iters, "iters", torch.int32), (status, "status", torch.int32),
                      (relres, "relres", torch.float64)):
        _check_dtype(t, dt, nm)
    if order is not None:
        _check_dtype(order, torch.int32, "order")
    if qoi is not None:
        _check_dtype(qoi, torch.float64, "qoi")
    if w is not None:
        _check_dtype(w, torch.float64, "w")
    if xi.numel() != M * prob.nparam:
        raise ValueError("xi must be [M][nparam]")
    if work is None:
        work = torch.empty(ens_stream_workspace_size(prob, S, E), dtype=torch.uint8, device=xi.device)
    rc = load().ens_solve_stream(h.ptr, ctypes.byref(prob), int(S), int(E), int(M), _ptr(xi), _ptr(order), _ptr(w),
                                 float(rtol), int(maxit), int(chunk), _ptr(iters), _ptr(status), _ptr(relres),
                                 _ptr(qoi), _ptr(work), work.numel(), _stream(stream))
    h.check(rc, "ens_solve_stream")


def ens_param_indicator(h: Handle, prob: Problem, xi, H, stream=None):
    """H[m] = max_x lambda_max / lambda_min of A(x, xi_m) (the "par" grouping key)."""
    _check_dtype(xi, torch.float64, "xi")
    _check_dtype(H, torch.float64, "H")
    M = H.numel()
    if xi.numel() != M * prob.nparam:
        raise ValueError("xi must be [M][nparam]")
    rc = load().ens_param_indicator(h.ptr, ctypes.byref(prob), int(M), _ptr(xi), _ptr(H), _stream(stream))
    h.check(rc, "ens_param_indicator")


def ens_adjoint_workspace_size(prob: Problem, S: int, E: int) -> int:
    return int(load().ens_adjoint_workspace_size(ctypes.byref(prob), int(S), int(E)))


def ens_adjoint_grad(h: Handle, prob: Problem, S: int, E: int, xi, u, lam, grad, work, stream=None):
    """grad[E][S][N] = -lam^T (dA/dxi) u per lane."""
    J, _ = ens_problem_size(prob)
    for t, nm in ((xi, "xi"), (u, "u"), (lam, "lam"), (grad, "grad")):
        _check_dtype(t, torch.float64, nm)
    if u.numel() != E * J * S or lam.numel() != E * J * S or grad.numel() != E * S * prob.nparam:
        raise ValueError("u / lam / grad sizes do not match E, J, S, nparam")
    rc = load().ens_adjoint_grad(h.ptr, ctypes.byref(prob), int(S), int(E), _ptr(xi), _ptr(u), _ptr(lam),
                                 _ptr(grad), _ptr(work), work.numel(), _stream(stream))
    h.check(rc, "ens_adjoint_grad")


def ens_adjoint_solve_workspace_size(prob: Problem, S: int, E: int) -> int:
    return int(load().ens_adjoint_solve_workspace_size(ctypes.byref(prob), int(S), int(E)))


def ens_adjoint_solve_grad(h: Handle, prob: Problem, S: int, E: int, xi, rowptr, colidx, u, w, active,
                           rtol: float, maxit: int, Q, grad, lam, iters, relres, status, work, stream=None):
    """Adjoint solve A lam = w, Q = w^T u and dQ/dxi = -lam^T (dA/dxi) u per lane."""
    J, _ = ens_problem_size(prob)
    for t, nm, dt in ((xi, "xi", torch.float64), (u, "u", torch.float64), (w, "w", torch.float64),
                      (Q, "Q", torch.float64), (grad, "grad", torch.float64), (lam, "lam", torch.float64),
                      (iters, "iters", torch.int32), (relres, "relres", torch.float64),
                      (status, "status", torch.int32)):
        _check_dtype(t, dt, nm)
    if (u.numel() != E * J * S or lam.numel() != E * J * S or w.numel() != J or grad.numel() != E * S * prob.nparam
            or Q.numel() != E * S or iters.numel() != E * S):
        raise ValueError("array sizes do not match E, J, S, nparam")
    rc = load().ens_adjoint_solve_grad(h.ptr, ctypes.byref(prob), int(S), int(E), _ptr(xi), _ptr(rowptr),
                                       _ptr(colidx), _ptr(u), _ptr(w), _ptr(active), float(rtol), int(maxit),
                                       _ptr(Q), _ptr(grad), _ptr(lam), _ptr(iters), _ptr(relres), _ptr(status),
                                       _ptr(work), work.numel(), _stream(stream))
    h.check(rc, "ens_adjoint_solve_grad")


STATIC_SCRATCH_BYTES = 8 << 20


def ens_pcg_solve_static(h, J: int, nnz: int, S: int, E: int, rowptr, colidx, vals, dinv, b, x, active,
                         rtol: float, maxit: int, iters, relres, status, stream=None):
    """ens_pcg_solve without a caller workspace: for callers that may not
    allocate device memory; scratch is the library's fixed 8 MiB device array.
    h may be None."""
    for t, nm, dt in ((vals, "vals", torch.float64), (dinv, "dinv", torch.float64), (b, "b", torch.float64),
                      (x, "x", torch.float64), (iters, "iters", torch.int32), (relres, "relres", torch.float64),
                      (status, "status", torch.int32)):
        _check_dtype(t, dt, nm)
    if vals.numel() != E * nnz * S or x.numel() != E * J * S or iters.numel() != E * S:
        raise ValueError("array sizes do not match E, J, nnz, S")
    rc = load().ens_pcg_solve_static(h.ptr if h is not None else None, int(J), int(nnz), int(S), int(E),
                                     _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(dinv), _ptr(b), _ptr(x),
                                     _ptr(active), float(rtol), int(maxit), _ptr(iters), _ptr(relres),
                                     _ptr(status), _stream(stream))
    if h is not None:
        h.check(rc, "ens_pcg_solve_static")
    elif rc != OK:
        raise EnsError(f"ens_pcg_solve_static failed ({rc})")


def ens_group(h: Handle, lvl, idx, surplus, yq, S: int, pred, perm, stream=None) -> int:
    M, N = (0, yq.shape[1]) if lvl is None else tuple(lvl.shape)
    Mq = yq.shape[0]
    _check_dtype(yq, torch.float64, "yq")
    _check_dtype(pred, torch.float64, "pred")
    _check_dtype(perm, torch.int32, "perm")
    if M:
        _check_dtype(lvl, torch.int8, "lvl")
        _check_dtype(idx, torch.int32, "idx")
        _check_dtype(surplus, torch.float64, "surplus")
    n_ens = ctypes.c_int()
    rc = load().ens_group(h.ptr, int(N), int(M), _ptr(lvl) if M else None, _ptr(idx) if M else None,
                          _ptr(surplus) if M else None, int(Mq), _ptr(yq), int(S), _ptr(pred), _ptr(perm),
                          ctypes.byref(n_ens), _stream(stream))
    h.check(rc, "ens_group")
    return n_ens.value


def ens_sg_eval(h: Handle, lvl, idx, surplus, yq, out, values=None, stream=None):
    """out = surrogate(yq), or values - surrogate(yq) (the surpluses) if values is given."""
    M, N = (0, yq.shape[1]) if lvl is None else tuple(lvl.shape)
    _check_dtype(yq, torch.float64, "yq")
    _check_dtype(out, torch.float64, "out")
    if values is not None:
        _check_dtype(values, torch.float64, "values")
    if M:
        _check_dtype(lvl, torch.int8, "lvl")
        _check_dtype(idx, torch.int32, "idx")
        _check_dtype(surplus, torch.float64, "surplus")
    rc = load().ens_sg_eval(h.ptr, int(N), int(M), _ptr(lvl) if M else None, _ptr(idx) if M else None,
                            _ptr(surplus) if M else None, int(yq.shape[0]), _ptr(yq), _ptr(values),
                            _ptr(out), _stream(stream))
    h.check(rc, "ens_sg_eval")


def ens_qoi(h: Handle, J: int, S: int, E: int, x, out, w=None, stream=None):
    """out[e][s] = sum_j x^2 (w None) or sum_j w_j x (w a [J] tensor)."""
    _check_dtype(x, torch.float64, "x")
    _check_dtype(out, torch.float64, "out")
    if w is not None:
        _check_dtype(w, torch.float64, "w")
        if w.numel() != J:
            raise ValueError("w must have J entries")
    if x.numel() != E * J * S or out.numel() != E * S:
        raise ValueError("x / out sizes do not match E, J, S")
    rc = load().ens_qoi(h.ptr, int(J), int(S), int(E), _ptr(x), _ptr(w), _ptr(out), _stream(stream))
    h.check(rc, "ens_qoi")


def ens_sort_chunk(h: Handle, keys, S: int, perm, stream=None) -> int:
    _check_dtype(keys, torch.float64, "keys")
    _check_dtype(perm, torch.int32, "perm")
    n_ens = ctypes.c_int()
    rc = load().ens_sort_chunk(h.ptr, int(keys.numel()), _ptr(keys), int(S), _ptr(perm),
                               ctypes.byref(n_ens), _stream(stream))
    h.check(rc, "ens_sort_chunk")
    return n_ens.value


def ens_sg_refine(lvl, idx, first: int, surplus, tau: float, max_level: int, max_out: int = 1 << 16):
    """(host) children of the points first..M-1 with |surplus| >= tau."""
    lvl = np.ascontiguousarray(lvl, np.int8)
    idx = np.ascontiguousarray(idx, np.int32)
    M, N = lvl.shape
    ol = np.zeros((max_out, N), np.int8)
    oi = np.zeros((max_out, N), np.int32)
    cnt = load().ens_sg_refine(int(N), int(M), lvl, idx, int(first),
                               np.ascontiguousarray(surplus, np.float64), float(tau), int(max_level),
                               int(max_out), ol, oi)
    if cnt < 0:
        raise EnsError(f"ens_sg_refine failed ({cnt})")
    return ol[:cnt].copy(), oi[:cnt].copy()


def ens_sg_initial(N: int, level: int, max_out: int = 1 << 16):
    """(host) the full sparse grid of levels 0..level."""
    lvl = np.zeros((max_out, N), np.int8)
    idx = np.zeros((max_out, N), np.int32)
    M = load().ens_sg_initial(int(N), int(level), int(max_out), lvl, idx)
    if M < 0:
        raise EnsError(f"ens_sg_initial failed ({M})")
    return lvl[:M].copy(), idx[:M].copy()


def ens_sg_points(lvl, idx) -> np.ndarray:
    """(host) y[m][n] = idx 2^(1 - lvl) - 1 of the grid points (exact)."""
    lvl = np.ascontiguousarray(lvl, np.int8)
    idx = np.ascontiguousarray(idx, np.int32)
    M, N = lvl.shape
    y = np.zeros((M, N), np.float64)
    rc = load().ens_sg_points(int(N), int(M), lvl, idx, y)
    if rc != OK:
        raise EnsError(f"ens_sg_points failed ({rc})")
    return y


def ens_fp64_peak(h: "Handle", blocks: int, iters: int, sink: torch.Tensor, stream=None) -> float:
    """Launch the FP64 fused multiply-add throughput kernel; returns its
    floating-point operation count (time it with events on the stream)."""
    _check_dtype(sink, torch.float64, "sink")
    h.check(load().ens_fp64_peak(h.ptr, int(blocks), int(iters), _ptr(sink), _stream(stream)), "ens_fp64_peak")
    return float(load().ens_fp64_peak_flops(int(blocks), int(iters)))
