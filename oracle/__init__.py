"""CPU FP64 oracle for the ensemble-PCG / surrogate-grouping method of
D'Elia, Phipps, Rushdi, Ebeida (arXiv 1705.02003).

TEST INFRASTRUCTURE ONLY.  The product package never imports this module; only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference arm do.  It shares no code with the CUDA path: the arithmetic lives
in plain C (``problem.c``, ``pcg.c``, ``sgrid.c``, built with
``-O2 -ffp-contract=off``), and this file only marshals numpy arrays.

Parity status of each function is pinned by ``tests/test_oracle_*.py``
(closed forms, manufactured solutions, brute force and the paper's printed
conventions); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_SRC = ["problem.c", "pcg.c", "sgrid.c", "mg.c"]

FD5_LOGKL = 1
Q1_ROT = 2
FD7_AXIS = 3
Q1_3D_KL = 4      # Section 4, Test 1 (3-D trilinear FEM, exponential-covariance KL field)
Q1_3D_DISC = 5    # Section 4, Test 2 (the same with the discontinuous ahat(xi))

CONVERGED, MAXIT, BREAKDOWN, BADINPUT = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``oracle/_build/liboracle.so``."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_SO):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_SO) >= newest:
            return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp] + srcs + ["-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
        return _lib


_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def _declare(L):
    c = ctypes
    L.or_problem_size.argtypes = [c.c_int, c.c_int, c.POINTER(c.c_int), c.POINTER(c.c_int64)]
    L.or_pattern.argtypes = [c.c_int, c.c_int, _i64p, _i32p]
    L.or_assemble.argtypes = [c.c_int, c.c_int, c.c_int, c.c_double, _f64p, _i64p, _i32p, _f64p, _f64p]
    L.or_tensor.argtypes = [c.c_int, c.c_int, c.c_double, _f64p, _f64p, _f64p]
    L.or_param_indicator.argtypes = [c.c_int, c.c_int, c.c_int, c.c_double, _f64p]
    L.or_param_indicator.restype = c.c_double
    L.or_kl_1d.argtypes = [c.c_int, c.POINTER(c.c_double), c.POINTER(c.c_double)]
    L.or_kl_lambda.argtypes = [c.c_int]
    L.or_kl_lambda.restype = c.c_double
    L.or_kl_mode.argtypes = [c.c_int, _f64p]
    L.or_kl_mode.restype = c.c_double
    L.or_spmv.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p, _f64p]
    L.or_spmv.restype = None
    L.or_jacobi.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p]
    L.or_pcg.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p, c.c_double, c.c_int, _f64p,
                         c.POINTER(c.c_int), c.POINTER(c.c_double)]
    L.or_pcg_history.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p, c.c_double, c.c_int, _f64p,
                                 c.POINTER(c.c_int), c.POINTER(c.c_double), _f64p]
    L.or_mg_levels.argtypes = [c.c_int, _i32p]
    L.or_mg_galerkin.argtypes = [c.c_int, _i64p, _i32p, _f64p, c.c_int, _i64p, _i32p, _f64p]
    L.or_mg_prolong.argtypes = [c.c_int, c.c_int, _f64p, _f64p]
    L.or_mg_prolong.restype = None
    L.or_mg_restrict.argtypes = [c.c_int, c.c_int, _f64p, _f64p]
    L.or_mg_restrict.restype = None
    L.or_gershgorin.argtypes = [c.c_int, _i64p, _i32p, _f64p]
    L.or_gershgorin.restype = c.c_double
    L.or_cheb.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p, c.c_double, _f64p, _f64p]
    L.or_cheb.restype = None
    L.or_mg_coarse.argtypes = [c.c_int, _i64p, _i32p, _f64p, c.c_int, _f64p, c.POINTER(c.c_double)]
    L.or_mg_apply.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p, _f64p]
    L.or_mgpcg.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p, c.c_double, c.c_int, _f64p,
                           c.POINTER(c.c_int), c.POINTER(c.c_double)]
    L.or_mg_apply32.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p, _f64p]
    L.or_mgpcg32.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p, c.c_double, c.c_int, _f64p,
                             c.POINTER(c.c_int), c.POINTER(c.c_double)]
    L.or_solve_batch.argtypes = [c.c_int, c.c_int, c.c_int, c.c_double, c.c_int, _f64p, c.c_double,
                                 c.c_int, c.c_int, _i32p, _i32p, _f64p, _f64p, c.c_void_p]
    L.or_pcg_ir.argtypes = [c.c_int, _i64p, _i32p, _f64p, _f64p, c.c_double, c.c_double, c.c_int,
                            c.c_int, _f64p, c.POINTER(c.c_int), c.POINTER(c.c_int),
                            c.POINTER(c.c_double)]
    L.or_adjoint_grad.argtypes = [c.c_int, c.c_int, c.c_int, c.c_double, _f64p, _f64p, c.c_double,
                                  c.c_int, c.POINTER(c.c_double), _f64p, c.POINTER(c.c_int),
                                  c.POINTER(c.c_int)]
    L.or_sg_coord.argtypes = [c.c_int, c.c_int64]
    L.or_sg_coord.restype = c.c_double
    L.or_hat.argtypes = [c.c_int, c.c_int64, c.c_double]
    L.or_hat.restype = c.c_double
    L.or_sg_points.argtypes = [c.c_int, c.c_int, _i8p, _i32p, _f64p]
    L.or_sg_points.restype = None
    L.or_sg_eval.argtypes = [c.c_int, c.c_int, _i8p, _i32p, _f64p, c.c_int, _f64p, _f64p]
    L.or_sg_eval.restype = None
    L.or_sg_initial.argtypes = [c.c_int, c.c_int, c.c_int, _i8p, _i32p]
    L.or_sg_refine.argtypes = [c.c_int, c.c_int, _i8p, _i32p, c.c_int, _f64p, c.c_double, c.c_int,
                               c.c_int, _i8p, _i32p]
    L.or_sort_perm.argtypes = [c.c_int, _f64p, _i32p]
    L.or_sort_perm.restype = None
    L.or_work_ratio.argtypes = [c.c_int, c.c_int, _i32p, _f64p]
    L.or_work_ratio.restype = c.c_double


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# problem
# ---------------------------------------------------------------------------
def problem_size(kind: int, n: int):
    J = ctypes.c_int()
    nnz = ctypes.c_int64()
    if lib().or_problem_size(kind, n, ctypes.byref(J), ctypes.byref(nnz)):
        raise ValueError("bad problem kind/size")
    return J.value, nnz.value


def pattern(kind: int, n: int):
    J, nnz = problem_size(kind, n)
    rowptr = np.zeros(J + 1, np.int64)
    colidx = np.zeros(nnz, np.int32)
    if lib().or_pattern(kind, n, rowptr, colidx):
        raise ValueError("pattern failed")
    return rowptr, colidx


def assemble(kind: int, n: int, nparam: int, aniso: float, xi, rowptr=None, colidx=None):
    """One sample's CSR values (pattern order) and load vector."""
    if rowptr is None:
        rowptr, colidx = pattern(kind, n)
    J = len(rowptr) - 1
    vals = np.zeros(int(rowptr[-1]), np.float64)
    b = np.zeros(J, np.float64)
    rc = lib().or_assemble(kind, n, nparam, float(aniso), _f64(xi), rowptr, colidx, vals, b)
    if rc:
        raise ValueError(f"assemble failed ({rc})")
    return vals, b


def tensor(kind: int, nparam: int, aniso: float, xi, x):
    d = 3 if kind in (FD7_AXIS, Q1_3D_KL, Q1_3D_DISC) else 2
    K = np.zeros(d * d, np.float64)
    if lib().or_tensor(kind, nparam, float(aniso), _f64(xi), _f64(x), K):
        raise ValueError("tensor failed")
    return K.reshape(d, d)


def kl_1d(which: int):
    """(w, lambda) of the first even (0) or odd (1) 1-D exponential-kernel mode."""
    w = ctypes.c_double()
    lam = ctypes.c_double()
    if lib().or_kl_1d(int(which), ctypes.byref(w), ctypes.byref(lam)):
        raise ValueError("which must be 0 or 1")
    return w.value, lam.value


def kl_lambda(k: int) -> float:
    """3-D covariance eigenvalue of parameter k = 1..4 (sigma0 included)."""
    return lib().or_kl_lambda(int(k))


def kl_mode(k: int, x) -> float:
    """3-D KL mode b_k(x) of parameter k = 1..4 at x in [0, 1]^3."""
    return lib().or_kl_mode(int(k), _f64(x))


def param_indicator(kind: int, n: int, nparam: int, aniso: float, xi) -> float:
    """H(xi) = max over the evaluation points of lambda_max / lambda_min of A."""
    return lib().or_param_indicator(kind, n, nparam, float(aniso), _f64(xi))


# ---------------------------------------------------------------------------
# solver
# ---------------------------------------------------------------------------
def spmv(rowptr, colidx, vals, x):
    J = len(rowptr) - 1
    y = np.zeros(J, np.float64)
    lib().or_spmv(J, rowptr, colidx, _f64(vals), _f64(x), y)
    return y


def jacobi(rowptr, colidx, vals):
    J = len(rowptr) - 1
    d = np.zeros(J, np.float64)
    if lib().or_jacobi(J, rowptr, colidx, _f64(vals), d):
        raise ValueError("missing diagonal")
    return d


def pcg(rowptr, colidx, vals, b, rtol: float, maxit: int):
    """Per-sample Jacobi-PCG. Returns (x, iters, status, relres)."""
    J = len(rowptr) - 1
    x = np.zeros(J, np.float64)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().or_pcg(J, rowptr, colidx, _f64(vals), _f64(b), float(rtol), int(maxit), x,
                      ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, st, rr.value


def pcg_history(rowptr, colidx, vals, b, rtol: float, maxit: int):
    """pcg() that also returns ||r_k|| / ||b|| after every update k = 1..iters
    (Section 4's per-sample convergence record at every iteration).  With
    rtol = 0 it runs exactly maxit iterations (barring breakdown).
    Returns (x, iters, status, relres, history[iters])."""
    J = len(rowptr) - 1
    x = np.zeros(J, np.float64)
    hist = np.zeros(max(1, int(maxit)), np.float64)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().or_pcg_history(J, rowptr, colidx, _f64(vals), _f64(b), float(rtol), int(maxit), x,
                              ctypes.byref(it), ctypes.byref(rr), hist)
    return x, it.value, st, rr.value, hist[: it.value].copy()


# ---- multigrid V-cycle preconditioner of the trilinear problems (mg.c) ----

def mg_levels(n: int):
    """Interior nodes per axis of each level: [n, (n-1)/2, ..., 3]."""
    ns = np.zeros(8, np.int32)
    L = lib().or_mg_levels(int(n), ns)
    if L < 1:
        raise ValueError(f"no multigrid hierarchy for n = {n} (n = 2^k - 1, k >= 2)")
    return [int(v) for v in ns[:L]]


def mg_galerkin(nf: int, rpf, cif, vf, nc: int):
    """P^T A P of a fine 27-point matrix, in the coarse level's pattern."""
    rpc, cic = pattern(Q1_3D_KL, nc)
    vc = np.zeros(len(cic), np.float64)
    if lib().or_mg_galerkin(int(nf), rpf, cif, _f64(vf), int(nc), rpc, cic, vc):
        raise ValueError("bad levels or pattern")
    return vc


def mg_prolong(nf: int, nc: int, ec):
    ef = np.zeros(nf ** 3, np.float64)
    lib().or_mg_prolong(int(nf), int(nc), _f64(ec), ef)
    return ef


def mg_restrict(nf: int, nc: int, rf):
    rc = np.zeros(nc ** 3, np.float64)
    lib().or_mg_restrict(int(nf), int(nc), _f64(rf), rc)
    return rc


def gershgorin(rowptr, colidx, vals) -> float:
    return lib().or_gershgorin(len(rowptr) - 1, rowptr, colidx, _f64(vals))


def cheb(rowptr, colidx, vals, dinv, lmax: float, b, x):
    """Degree-2 Chebyshev smoothing of A x = b from x (returns the new x)."""
    x = _f64(x).copy()
    lib().or_cheb(len(rowptr) - 1, rowptr, colidx, _f64(vals), _f64(dinv), float(lmax), _f64(b), x)
    return x


def mg_coarse(n: int, rowptr, colidx, vals, level: int):
    """(values, Gershgorin bound) of level `level` of the hierarchy."""
    nl = mg_levels(n)[level]
    _, nnz = problem_size(Q1_3D_KL, nl)
    vc = np.zeros(nnz, np.float64)
    lm = ctypes.c_double()
    if lib().or_mg_coarse(int(n), rowptr, colidx, _f64(vals), int(level), vc, ctypes.byref(lm)):
        raise ValueError("hierarchy setup failed")
    return vc, lm.value


def mg_apply(n: int, rowptr, colidx, vals, r):
    """z = one V-cycle applied to r."""
    z = np.zeros(n ** 3, np.float64)
    if lib().or_mg_apply(int(n), rowptr, colidx, _f64(vals), _f64(r), z):
        raise ValueError("hierarchy setup failed")
    return z


def mgpcg(n: int, rowptr, colidx, vals, b, rtol: float, maxit: int):
    """CG preconditioned by one V-cycle per iteration. Returns (x, iters, status, relres)."""
    x = np.zeros(n ** 3, np.float64)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().or_mgpcg(int(n), rowptr, colidx, _f64(vals), _f64(b), float(rtol), int(maxit), x,
                        ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, st, rr.value


def mg_apply32(n: int, rowptr, colidx, vals, r):
    """z = one V-cycle in float (hierarchy rounded to float) applied to r."""
    z = np.zeros(n ** 3, np.float64)
    if lib().or_mg_apply32(int(n), rowptr, colidx, _f64(vals), _f64(r), z):
        raise ValueError("hierarchy setup failed")
    return z


def mgpcg32(n: int, rowptr, colidx, vals, b, rtol: float, maxit: int):
    """CG (FP64) preconditioned by the float V-cycle. Returns (x, iters, status, relres)."""
    x = np.zeros(n ** 3, np.float64)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().or_mgpcg32(int(n), rowptr, colidx, _f64(vals), _f64(b), float(rtol), int(maxit), x,
                          ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, st, rr.value


def solve_batch_mg(kind: int, n: int, nparam: int, aniso: float, xi, rtol: float, maxit: int,
                   nthreads: int = 1, want_x: bool = False):
    """solve_batch with the multigrid preconditioner (one sample per task)."""
    from concurrent.futures import ThreadPoolExecutor

    xi = _f64(xi)
    M = xi.shape[0]
    rp, ci = pattern(kind, n)

    def one(m):
        vals, b = assemble(kind, n, nparam, aniso, xi[m], rp, ci)
        x, it, st, rr = mgpcg(n, rp, ci, vals, b, rtol, maxit)
        return x, it, st, rr, float(np.dot(x, x))

    if nthreads > 1:
        with ThreadPoolExecutor(nthreads) as ex:
            res = list(ex.map(one, range(M)))
    else:
        res = [one(m) for m in range(M)]
    out = dict(iters=np.array([r[1] for r in res], np.int32), status=np.array([r[2] for r in res], np.int32),
               relres=np.array([r[3] for r in res]), G=np.array([r[4] for r in res]))
    if want_x:
        out["x"] = np.array([r[0] for r in res])
    return out


def solve_batch(kind: int, n: int, nparam: int, aniso: float, xi, rtol: float, maxit: int,
                nthreads: int = 1, want_x: bool = False):
    """Assemble + solve each row of ``xi`` [M][N] independently.

    Returns dict(iters, status, relres, G, x?) where G = ||u||_2^2."""
    xi = _f64(xi)
    M = xi.shape[0]
    J, _ = problem_size(kind, n)
    iters = np.zeros(M, np.int32)
    status = np.zeros(M, np.int32)
    relres = np.zeros(M, np.float64)
    G = np.zeros(M, np.float64)
    xout = np.zeros((M, J), np.float64) if want_x else None
    ptr = xout.ctypes.data if want_x else None
    rc = lib().or_solve_batch(kind, n, nparam, float(aniso), M, xi, float(rtol), int(maxit),
                              int(nthreads), iters, status, relres, G, ptr)
    if rc:
        raise ValueError(f"solve_batch failed ({rc})")
    out = dict(iters=iters, status=status, relres=relres, G=G)
    if want_x:
        out["x"] = xout
    return out


def pcg_ir(rowptr, colidx, vals, b, rtol_outer=1e-10, rtol_inner=1e-6, maxit_inner=20000,
           maxit_outer=50):
    J = len(rowptr) - 1
    x = np.zeros(J, np.float64)
    oi = ctypes.c_int()
    ii = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().or_pcg_ir(J, rowptr, colidx, _f64(vals), _f64(b), float(rtol_outer),
                         float(rtol_inner), int(maxit_inner), int(maxit_outer), x,
                         ctypes.byref(oi), ctypes.byref(ii), ctypes.byref(rr))
    return x, oi.value, ii.value, st, rr.value


def region_weights(n: int, dim: int):
    """Weights of the quantity of interest Q = mean of u over [0.4, 0.6]^dim
    (the differentiation workload): w_p = 1/|R| on the interior nodes p whose
    coordinates x = i/(n+1) all lie in [0.4, 0.6], else 0; node order x fastest.
    The test 0.4 <= i/(n+1) <= 0.6 is taken exactly, as 5i >= 2(n+1) and
    5i <= 3(n+1)."""
    inside = [i for i in range(1, n + 1) if 5 * i >= 2 * (n + 1) and 5 * i <= 3 * (n + 1)]
    J = n ** dim
    w = np.zeros(J, np.float64)
    count = len(inside) ** dim
    for j in range(J):
        coords = [(j // n ** d) % n + 1 for d in range(dim)]
        if all(c in inside for c in coords):
            w[j] = 1.0 / count
    return w


def adjoint_grad(kind: int, n: int, nparam: int, aniso: float, xi, w, rtol: float, maxit: int):
    """Q = w^T u and dQ/dxi = -lambda^T (dA/dxi) u for one sample."""
    grad = np.zeros(nparam, np.float64)
    Q = ctypes.c_double()
    itf = ctypes.c_int()
    ita = ctypes.c_int()
    st = lib().or_adjoint_grad(kind, n, nparam, float(aniso), _f64(xi), _f64(w), float(rtol),
                               int(maxit), ctypes.byref(Q), grad, ctypes.byref(itf),
                               ctypes.byref(ita))
    if st < 0:
        raise ValueError("adjoint_grad failed")
    return Q.value, grad, itf.value, ita.value, st


# ---------------------------------------------------------------------------
# sparse grid + grouping
# ---------------------------------------------------------------------------
def sg_coord(l: int, i: int) -> float:
    return lib().or_sg_coord(int(l), int(i))


def hat(l: int, i: int, y: float) -> float:
    return lib().or_hat(int(l), int(i), float(y))


def sg_points(lvl, idx):
    lvl = np.ascontiguousarray(lvl, np.int8)
    idx = np.ascontiguousarray(idx, np.int32)
    M, N = lvl.shape
    y = np.zeros((M, N), np.float64)
    lib().or_sg_points(N, M, lvl, idx, y)
    return y


def sg_eval(lvl, idx, surplus, yq):
    lvl = np.ascontiguousarray(lvl, np.int8)
    idx = np.ascontiguousarray(idx, np.int32)
    yq = _f64(yq)
    M, N = lvl.shape
    Q = yq.shape[0]
    out = np.zeros(Q, np.float64)
    if Q:
        lib().or_sg_eval(N, M, lvl, idx, _f64(surplus), Q, yq, out)
    return out


def sg_initial(N: int, level: int, max_out: int = 1 << 16):
    lvl = np.zeros((max_out, N), np.int8)
    idx = np.zeros((max_out, N), np.int32)
    M = lib().or_sg_initial(N, level, max_out, lvl, idx)
    if M < 0:
        raise ValueError("sg_initial overflow")
    return lvl[:M].copy(), idx[:M].copy()


def sg_refine(lvl, idx, first: int, surplus, tau: float, max_level: int, max_out: int = 1 << 16):
    lvl = np.ascontiguousarray(lvl, np.int8)
    idx = np.ascontiguousarray(idx, np.int32)
    M, N = lvl.shape
    ol = np.zeros((max_out, N), np.int8)
    oi = np.zeros((max_out, N), np.int32)
    cnt = lib().or_sg_refine(N, M, lvl, idx, int(first), _f64(surplus), float(tau), int(max_level),
                             max_out, ol, oi)
    if cnt < 0:
        raise ValueError("sg_refine overflow")
    return ol[:cnt].copy(), oi[:cnt].copy()


def sort_perm(keys):
    keys = _f64(keys)
    perm = np.zeros(len(keys), np.int32)
    lib().or_sort_perm(len(keys), keys, perm)
    return perm


def work_ratio(S: int, perm, iters) -> float:
    perm = np.ascontiguousarray(perm, np.int32)
    return lib().or_work_ratio(int(S), len(perm), perm, _f64(iters))
