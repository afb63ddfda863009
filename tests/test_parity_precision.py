"""GPU parity of the precision layer: FP32 matrix values and inner Jacobi-PCG
inside FP64 iterative refinement (ens_pcg_solve_ir) against the FP64 oracle.

Bars: every returned x within 1e-8 relative of the oracle's FP64 solution
(solved to 1e-13), and its FP64 residual ||b - A x|| <= 1e-10 ||b|| with the
oracle's matrix."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import OKIND, Case, elem_err
from paper_1705_02003_gb300 import ens, inputs

pytestmark = pytest.mark.gpu

NTH = os.cpu_count() or 4


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


def solve_ir(c, rtol=1e-10, rtol_inner=1e-6, maxit_inner=20000, maxit_outer=30, active=None):
    E, S, J, nnz = c.E, c.S, c.J, c.nnz
    v32 = torch.empty(E * nnz * S, dtype=torch.float32, device="cuda")
    ens.ens_assemble(c.h, c.prob, S, E, c.xi, c.rowptr, c.colidx, v32)
    x = torch.full((E * J * S,), float("nan"), dtype=torch.float64, device="cuda")
    it = torch.zeros(E * S, dtype=torch.int32, device="cuda")
    oit = torch.zeros(E * S, dtype=torch.int32, device="cuda")
    st = torch.zeros(E * S, dtype=torch.int32, device="cuda")
    rr = torch.zeros(E * S, dtype=torch.float64, device="cuda")
    work = torch.empty(ens.ens_pcg_ir_workspace_size(J, nnz, S, E), dtype=torch.uint8, device="cuda")
    ens.ens_pcg_solve_ir(c.h, J, nnz, S, E, c.rowptr, c.colidx, c.vals, v32, c.dinv, c.b, x,
                         c.active if active is None else active, rtol, rtol_inner, maxit_inner, maxit_outer,
                         it, oit, rr, st, work)
    torch.cuda.synchronize()
    xs = x.view(E, J, S).permute(0, 2, 1).reshape(E * S, J).cpu().numpy()
    return dict(x=xs, iters=it.cpu().numpy(), outer=oit.cpu().numpy(), status=st.cpu().numpy(),
                relres=rr.cpu().numpy())


def dense_residual(kind, n, N, aniso, xi, x):
    """||b - A x|| / ||b|| with the oracle's matrix (scipy CSR product)."""
    import scipy.sparse as sp

    rp, ci = O.pattern(OKIND[kind], n)
    vals, b = O.assemble(OKIND[kind], n, N, aniso, xi, rp, ci)
    A = sp.csr_matrix((vals, ci, rp), shape=(len(b), len(b)))
    return np.linalg.norm(b - A @ x) / np.linalg.norm(b)


@pytest.mark.parametrize("kind,n,N,aniso,S,M", [("fd7", 12, 6, 2.0, 32, 40), ("fd5", 40, 8, 3.0, 8, 13),
                                                ("q1", 32, 4, 4.0, 16, 16), ("fd7", 10, 6, 3.0, 1, 3)])
def test_ir_matches_fp64_oracle(h, kind, n, N, aniso, S, M):
    xi = inputs.draws(M, N, seed=40 + n)
    c = Case(h, kind, n, N, aniso, S, xi)
    got = solve_ir(c)
    ref = O.solve_batch(OKIND[kind], n, N, aniso, xi, 1e-13, 100000, nthreads=NTH, want_x=True)
    for s in range(M):
        assert got["status"][s] == ens.LANE_CONVERGED, (s, got["status"][s])
        assert got["relres"][s] <= 1e-10
        assert got["outer"][s] >= 1 and got["iters"][s] >= got["outer"][s]
        err = elem_err(got["x"][s], ref["x"][s])
        assert err <= 1e-8, (s, err)
        assert dense_residual(kind, n, N, aniso, xi[s], got["x"][s]) <= 1e-10
    for L in range(M, c.E * S):
        assert got["status"][L] == ens.LANE_INACTIVE and np.all(got["x"][L] == 0)


def test_ir_full_size_sampled_lane(h):
    """The 128^3 workload's problem, one ensemble of 32 in the bench's launch
    shape; lane 7 against the oracle."""
    wl = inputs.WORKLOADS["fd7_128_mixed"]
    xi = inputs.draws(wl.S, wl.nparam, seed=wl.seed)
    c = Case(h, wl.kind, wl.n, wl.nparam, wl.aniso, wl.S, xi)
    got = solve_ir(c, rtol=wl.rtol)
    assert np.all(got["status"] == ens.LANE_CONVERGED)
    assert np.all(got["relres"] <= wl.rtol)
    ref = O.solve_batch(O.FD7_AXIS, wl.n, wl.nparam, wl.aniso, xi[7:8], 1e-12, 100000, want_x=True)
    err = elem_err(got["x"][7], ref["x"][0])
    assert err <= 1e-8, err


def test_ir_degenerate_cases(h):
    xi = inputs.draws(8, 2, seed=41)
    c = Case(h, "fd5", 16, 2, 3.0, 8, xi)
    z = solve_ir(c, maxit_outer=0)
    assert np.all(z["status"] == ens.LANE_MAXIT) and np.all(z["x"] == 0) and np.all(z["outer"] == 0)
    assert np.allclose(z["relres"], 1.0)
    act = torch.tensor([1, 0, 1, 0, 0, 0, 0, 1], dtype=torch.uint8, device="cuda")
    got = solve_ir(c, active=act)
    full = solve_ir(c)
    for L in range(8):
        if act[L]:
            assert got["status"][L] == ens.LANE_CONVERGED
            assert np.array_equal(got["x"][L], full["x"][L])
        else:
            assert got["status"][L] == ens.LANE_INACTIVE and np.all(got["x"][L] == 0)
    bad = xi.copy()
    bad[2, 0] = np.nan
    cb = Case(h, "fd5", 16, 2, 3.0, 8, bad)
    gb = solve_ir(cb)
    assert gb["status"][2] in (ens.LANE_BADINPUT, ens.LANE_BREAKDOWN)
    keep = [L for L in range(8) if L != 2]
    assert np.array_equal(gb["x"][keep], full["x"][keep])
