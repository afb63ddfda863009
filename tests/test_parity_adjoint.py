"""GPU parity of the differentiation layer: Q = w^T u and dQ/dxi from the
adjoint ensemble solve (ens_adjoint_grad behind torch.autograd.Function),
against the oracle's adjoint gradient and against central finite differences
of the GPU forward map (h = 1e-6, forward solves to rtol 1e-13)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1705_02003_gb300 import adjoint, ens, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


CASES = [("fd5", 31, 8, 3.0, 8, 10), ("fd7", 9, 6, 3.0, 4, 6), ("fd5", 24, 2, 3.0, 1, 3)]


@pytest.mark.parametrize("kind,n,N,aniso,S,M", CASES)
def test_adjoint_gradient_matches_oracle(h, kind, n, N, aniso, S, M):
    dim = 3 if kind == "fd7" else 2
    w = inputs.region_weights(n, dim)
    xi = inputs.draws(M, N, seed=50 + n) * 0.9
    sol = adjoint.AdjointSolver(h, ens.problem(kind, n, N, aniso), S, M, torch.from_numpy(w), 1e-13, 100000)
    x = torch.from_numpy(xi).cuda()
    q = sol.forward(x).cpu().numpy()
    g = sol.gradient(x, recompute_forward=False).cpu().numpy()
    okind = {"fd5": O.FD5_LOGKL, "fd7": O.FD7_AXIS}[kind]
    for s in range(M):
        Qo, go, _, _, st = O.adjoint_grad(okind, n, N, aniso, xi[s], O.region_weights(n, dim), 1e-13, 100000)
        assert st == O.CONVERGED
        assert q[s] == pytest.approx(Qo, rel=1e-10)
        assert np.all(np.abs(g[s] - go) <= 1e-9 * np.maximum(1e-3, np.abs(go))), (s, g[s], go)


def test_adjoint_gradient_matches_central_differences(h):
    n, N, aniso, S, M = 31, 8, 3.0, 8, 4
    w = inputs.region_weights(n, 2)
    xi = inputs.draws(M, N, seed=60) * 0.9
    sol = adjoint.AdjointSolver(h, ens.problem("fd5", n, N, aniso), S, 2 * N * M, torch.from_numpy(w), 1e-13,
                                100000)
    x = torch.from_numpy(xi).cuda()
    g = sol.gradient(x, recompute_forward=True).cpu().numpy()
    hh = 1e-6
    pts = []
    for s in range(M):
        for k in range(N):
            for sg in (1, -1):
                e = xi[s].copy()
                e[k] += sg * hh
                pts.append(e)
    qs = sol.forward(torch.from_numpy(np.array(pts)).cuda()).cpu().numpy().reshape(M, N, 2)
    gfd = (qs[:, :, 0] - qs[:, :, 1]) / (2 * hh)
    assert np.all(np.abs(g - gfd) <= 1e-6 * np.maximum(1.0, np.abs(gfd))), np.abs(g - gfd).max()


def test_autograd_function_and_recompute(h):
    n, N, aniso, S, M = 24, 8, 3.0, 8, 9
    w = inputs.region_weights(n, 2)
    xi = torch.from_numpy(inputs.draws(M, N, seed=61)).cuda().requires_grad_(True)
    sol = adjoint.AdjointSolver(h, ens.problem("fd5", n, N, aniso), S, M, torch.from_numpy(w), 1e-12, 100000)
    coef = torch.linspace(0.5, 2.0, M, dtype=torch.float64, device="cuda")
    loss = (coef * adjoint.qoi(xi, sol, recompute=True)).sum()
    loss.backward()
    g1 = xi.grad.clone()
    direct = sol.gradient(xi.detach(), recompute_forward=True)
    assert torch.equal(g1, coef[:, None] * direct)
    xi.grad = None
    loss = (coef * adjoint.qoi(xi, sol, recompute=False)).sum()
    loss.backward()
    assert torch.equal(xi.grad, g1)  # stored and recomputed forward solutions agree bit for bit


def test_adjoint_full_size_sampled_lane(h):
    """The 512 x 512 workload's problem in its launch shape (one ensemble of 32);
    lane 5 against the oracle's adjoint."""
    wl = inputs.WORKLOADS["fd5_512_adjoint"]
    w = inputs.region_weights(wl.n, 2)
    xi = inputs.draws(wl.S, wl.nparam, seed=wl.seed)
    sol = adjoint.AdjointSolver(h, ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso), wl.S, wl.S,
                                torch.from_numpy(w), 1e-10, wl.maxit)
    x = torch.from_numpy(xi).cuda()
    q = sol.forward(x).cpu().numpy()
    g = sol.gradient(x, recompute_forward=False).cpu().numpy()
    assert torch.all(sol.last["forward_status"] == ens.LANE_CONVERGED)
    assert torch.all(sol.last["adjoint_status"] == ens.LANE_CONVERGED)
    Qo, go, _, _, st = O.adjoint_grad(O.FD5_LOGKL, wl.n, wl.nparam, wl.aniso, xi[5], O.region_weights(wl.n, 2), 1e-10,
                                      wl.maxit)
    assert q[5] == pytest.approx(Qo, rel=1e-7)
    assert np.all(np.abs(g[5] - go) <= 1e-6 * np.maximum(1e-3, np.abs(go))), (g[5], go)


@pytest.mark.parametrize("kind,aniso", [("q1", 4.0), ("q1_3d_kl", 0.0), ("q1_3d_disc", 0.0)])
def test_fem_problems_have_no_adjoint(h, kind, aniso):
    p = ens.problem(kind, 8, 4, aniso)
    J, _ = ens.ens_problem_size(p)
    z = torch.zeros(J * 2, dtype=torch.float64, device="cuda")
    work = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ens.EnsError, match="only the FD problems"):
        ens.ens_adjoint_grad(h, p, 2, 1, torch.zeros(8, dtype=torch.float64, device="cuda"), z, z,
                             torch.zeros(8, dtype=torch.float64, device="cuda"), work)


def test_adjoint_solve_grad_equals_the_split_calls(h):
    """ens_adjoint_solve_grad (assembly, adjoint solve, Q and gradient in one
    call) gives bit for bit what the separate entry points give: ens_assemble,
    ens_pcg_solve with right-hand side w, ens_qoi and ens_adjoint_grad."""
    n, N, aniso, S, M = 20, 8, 3.0, 8, 11
    prob = ens.problem("fd5", n, N, aniso)
    w = torch.from_numpy(inputs.region_weights(n, 2)).cuda()
    x = torch.from_numpy(inputs.draws(M, N, seed=62)).cuda()
    sol = adjoint.AdjointSolver(h, prob, S, M, w.cpu(), 1e-11, 100000)
    q = sol.forward(x)
    g = sol.gradient(x, recompute_forward=False)
    lam = sol.lam.clone()
    E, J = sol.Emax, sol.J
    L = E * S
    vals = torch.empty(E * sol.nnz * S, dtype=torch.float64, device="cuda")
    dinv = torch.empty(E * J * S, dtype=torch.float64, device="cuda")
    ens.ens_assemble(h, prob, S, E, sol.xi[: L * N], sol.rowptr, sol.colidx, vals, dinv)
    b = w.view(1, J, 1).expand(E, J, S).contiguous().view(-1)
    lam2 = torch.empty(E * J * S, dtype=torch.float64, device="cuda")
    it2 = torch.empty(L, dtype=torch.int32, device="cuda")
    st2, rr2 = torch.empty_like(it2), torch.empty(L, dtype=torch.float64, device="cuda")
    work = torch.empty(ens.ens_pcg_workspace_size(J, sol.nnz, S, E), dtype=torch.uint8, device="cuda")
    ens.ens_pcg_solve(h, J, sol.nnz, S, E, sol.rowptr, sol.colidx, vals, dinv, b, lam2, sol.active[:L], 1e-11,
                      100000, it2, rr2, st2, work)
    g2 = torch.empty(L * N, dtype=torch.float64, device="cuda")
    gw = torch.empty(ens.ens_adjoint_workspace_size(prob, S, E), dtype=torch.uint8, device="cuda")
    ens.ens_adjoint_grad(h, prob, S, E, sol.xi[: L * N], sol.u, lam2, g2, gw)
    q2 = torch.empty(L, dtype=torch.float64, device="cuda")
    ens.ens_qoi(h, J, S, E, sol.u, q2, w=w)
    torch.cuda.synchronize()
    per_lane = lambda t: t[: E * J * S].view(E, J, S).permute(0, 2, 1).reshape(L, J)[:M]
    assert torch.equal(per_lane(lam), per_lane(lam2))
    assert torch.equal(g, g2.view(L, N)[:M])
    assert torch.equal(sol.last["adjoint_iters"], it2[:M])
    assert torch.equal(q, q2[:M])
    assert torch.equal(sol.q[:M], q2[:M])


def test_adjoint_solve_grad_refuses_fem_problems(h):
    for kind, aniso in (("q1", 4.0), ("q1_3d_kl", 0.0)):
        p = ens.problem(kind, 8, 4, aniso)
        assert ens.ens_adjoint_solve_workspace_size(p, 2, 1) == 0
