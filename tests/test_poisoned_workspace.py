"""Reads of unwritten scratch memory (compute-sanitizer is not available on
this pool): every solve runs once on a workspace filled with 0xFF bytes (a NaN
in every FP64 and FP32 slot, -1 in every integer) and once on a zeroed one; the
results must be identical bit for bit, so no kernel depends on scratch it did
not write first.  Covers the FP64 solve (several branches), the FP32-in-FP64
refinement and the streamed solve with refills and re-packing."""
import numpy as np
import pytest
import torch

from gpu_util import Case
from paper_1705_02003_gb300 import batching, ens, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


def _solve(c, work, rtol=1e-8, maxit=5000):
    E, S, J = c.E, c.S, c.J
    x = torch.empty(E * J * S, dtype=torch.float64, device="cuda")
    it = torch.empty(E * S, dtype=torch.int32, device="cuda")
    st = torch.empty_like(it)
    rr = torch.empty(E * S, dtype=torch.float64, device="cuda")
    ens.ens_pcg_solve(c.h, J, c.nnz, S, E, c.rowptr, c.colidx, c.vals, c.dinv, c.b, x, c.active, rtol, maxit, it,
                      rr, st, work)
    torch.cuda.synchronize()
    return x.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy(), rr.cpu().numpy()


@pytest.mark.parametrize("kind,n,N,aniso,S,M", [("q1", 20, 4, 4.0, 16, 45), ("fd5", 24, 2, 3.0, 8, 30)])
def test_pcg_solve_ignores_workspace_contents(h, kind, n, N, aniso, S, M):
    c = Case(h, kind, n, N, aniso, S, inputs.draws(M, N, seed=60 + n))
    size = ens.ens_pcg_workspace_size(c.J, c.nnz, S, c.E)
    work = torch.empty(size, dtype=torch.uint8, device="cuda")
    work.fill_(255)
    a = _solve(c, work)
    work.zero_()
    b = _solve(c, work)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    assert np.all(np.isfinite(a[0]))


def test_refinement_ignores_workspace_contents(h):
    c = Case(h, "fd7", 10, 6, 2.0, 8, inputs.draws(16, 6, seed=61))
    E, S, J, nnz = c.E, c.S, c.J, c.nnz
    v32 = torch.empty(E * nnz * S, dtype=torch.float32, device="cuda")
    ens.ens_assemble(h, c.prob, S, E, c.xi, c.rowptr, c.colidx, v32)
    work = torch.empty(ens.ens_pcg_ir_workspace_size(J, nnz, S, E), dtype=torch.uint8, device="cuda")
    out = []
    for fill in (255, 0):
        work.fill_(fill)
        x = torch.empty(E * J * S, dtype=torch.float64, device="cuda")
        it = torch.empty(E * S, dtype=torch.int32, device="cuda")
        oit, st = torch.empty_like(it), torch.empty_like(it)
        rr = torch.empty(E * S, dtype=torch.float64, device="cuda")
        ens.ens_pcg_solve_ir(h, J, nnz, S, E, c.rowptr, c.colidx, c.vals, v32, c.dinv, c.b, x, c.active, 1e-10,
                             1e-4, 5000, 50, it, oit, rr, st, work)
        torch.cuda.synchronize()
        out.append([t.cpu().numpy() for t in (x, it, oit, st, rr)])
    for u, v in zip(*out):
        assert np.array_equal(u, v)


def test_stream_ignores_workspace_contents(h):
    prob = ens.problem("fd5", 20, 8, 3.0)
    xi = torch.from_numpy(inputs.draws(37, 8, seed=62)).cuda()
    S, E = 4, 3
    work = torch.empty(ens.ens_stream_workspace_size(prob, S, E), dtype=torch.uint8, device="cuda")
    out = []
    for fill in (255, 0):
        work.fill_(fill)
        r = batching.solve_stream(h, prob, xi, S, E, 1e-8, 5000, chunk=5, work=work)
        torch.cuda.synchronize()
        out.append([r[k].cpu().numpy() for k in ("iters", "status", "relres", "qoi")])
    for u, v in zip(*out):
        assert np.array_equal(u, v)
