"""ens_pcg_solve_static: the ensemble PCG for callers that may not allocate
device memory (code under an allocator that owns all device memory, plug-ins
that may not create allocations), whose scratch is the library's fixed
device array instead of a caller workspace.  Its results must match
ens_pcg_solve's on consecutive calls, and a problem too large for the fixed
array must be refused with a clear error.  Collected last on purpose."""
import numpy as np
import pytest
import torch

from gpu_util import Case, elem_err
from paper_1705_02003_gb300 import ens, inputs

pytestmark = pytest.mark.gpu


def solve_static(c, rtol, maxit, h=None):
    E, S, J = c.E, c.S, c.J
    x = torch.full((E * J * S,), float("nan"), dtype=torch.float64, device="cuda")
    iters = torch.full((E * S,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((E * S,), -7, dtype=torch.int32, device="cuda")
    relres = torch.empty(E * S, dtype=torch.float64, device="cuda")
    ens.ens_pcg_solve_static(h, J, c.nnz, S, E, c.rowptr, c.colidx, c.vals, c.dinv, c.b, x, c.active, rtol,
                             maxit, iters, relres, status)
    torch.cuda.synchronize()
    xs = x.view(E, J, S).permute(0, 2, 1).reshape(E * S, J).cpu().numpy()
    return dict(x=xs, iters=iters.cpu().numpy(), status=status.cpu().numpy(), relres=relres.cpu().numpy())


def same_as_workspace_solve(c, got, ref):
    assert np.array_equal(got["status"], ref["status"])
    assert np.array_equal(got["iters"], ref["iters"])
    for L in range(c.E * c.S):
        if not np.any(ref["x"][L]):
            assert np.all(got["x"][L] == 0)  # a padding lane
        else:
            assert elem_err(got["x"][L], ref["x"][L]) <= 1e-10, L


def test_static_scratch_solve_matches_workspace_solve(ens_lib):
    h = ens.Handle(0)
    # 20 samples in ensembles of 8: the last ensemble has 4 padding lanes
    c = Case(h, "fd5", 32, 2, 3.0, 8, inputs.draws(20, 2, seed=31))
    ref = c.solve(1e-8, 20000)
    for _ in range(2):  # two calls in a row through the same fixed array
        same_as_workspace_solve(c, solve_static(c, 1e-8, 20000), ref)
    # another problem and lane count through the array the last call left behind
    c2 = Case(h, "q1", 24, 4, 4.0, 16, inputs.draws(16, 4, seed=32))
    ref2 = c2.solve(1e-8, 20000)
    for _ in range(2):
        same_as_workspace_solve(c2, solve_static(c2, 1e-8, 20000, h=h), ref2)
    h.close()


def test_static_scratch_refuses_oversize_problems(ens_lib):
    h = ens.Handle(0)
    p = ens.problem("q1", 256, 4, 4.0)
    J, nnz = ens.ens_problem_size(p)
    S, E = 16, 2
    assert ens.ens_pcg_workspace_size(J, nnz, S, E) > ens.STATIC_SCRATCH_BYTES
    f64 = dict(dtype=torch.float64, device="cuda")
    rowptr = torch.zeros(J + 1, dtype=torch.int32, device="cuda")
    colidx = torch.zeros(nnz, dtype=torch.int32, device="cuda")
    vals = torch.zeros(E * nnz * S, **f64)
    vec = torch.zeros(E * J * S, **f64)
    it = torch.zeros(E * S, dtype=torch.int32, device="cuda")
    rr = torch.zeros(E * S, **f64)
    with pytest.raises(ens.EnsError, match="static scratch"):
        ens.ens_pcg_solve_static(h, J, nnz, S, E, rowptr, colidx, vals, vec, vec, vec, None, 1e-8, 10, it, rr,
                                 it.clone())
    h.close()
