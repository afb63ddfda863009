"""Differentiation layer: Q(xi) = w^T u(xi) for a batch of samples as a
torch.autograd.Function, with the gradient from one adjoint ensemble solve.

forward:  assemble A(xi_s) for all samples (K1), solve A u = b in ensembles
          (K2-K4), Q_s = w^T u_s (ens_qoi).
backward: one call of ens_adjoint_solve_grad: solve A lambda = w with the same
          kernels (A is symmetric), then dQ/dxi = -lambda^T (dA/dxi) u (K8),
          times dL/dQ.

With recompute=True the forward solutions are not kept between forward and
backward: backward solves for u again (the memory of one set of solution
fields instead of two, for the largest problems).
"""
from __future__ import annotations

import math

import torch

from . import ens


class AdjointSolver:
    """Device buffers for up to max_samples samples of one FD problem."""

    def __init__(self, handle: ens.Handle, prob: ens.Problem, S: int, max_samples: int, weights: torch.Tensor,
                 rtol: float, maxit: int):
        self.h, self.prob, self.S = handle, prob, int(S)
        self.N = prob.nparam
        self.rtol, self.maxit = float(rtol), int(maxit)
        self.J, self.nnz = ens.ens_problem_size(prob)
        dev = torch.device("cuda", handle.device)
        self.dev = dev
        self.w = weights.to(dev, torch.float64).contiguous()
        if self.w.numel() != self.J:
            raise ValueError("weights must have J entries")
        self.rowptr = torch.empty(self.J + 1, dtype=torch.int32, device=dev)
        self.colidx = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        ens.ens_pattern(handle, prob, self.rowptr, self.colidx)
        self.Emax = max(1, math.ceil(max_samples / self.S))
        L = self.Emax * self.S
        f64 = dict(dtype=torch.float64, device=dev)
        self.xi = torch.empty(L * self.N, **f64)
        self.vals = torch.empty(self.Emax * self.nnz * self.S, **f64)
        self.dinv = torch.empty(self.Emax * self.J * self.S, **f64)
        self.b = torch.empty(self.Emax * self.J * self.S, **f64)
        self.u = torch.empty(self.Emax * self.J * self.S, **f64)
        self.lam = torch.empty(self.Emax * self.J * self.S, **f64)
        self.active = torch.empty(L, dtype=torch.uint8, device=dev)
        self.iters = torch.empty(L, dtype=torch.int32, device=dev)
        self.status = torch.empty(L, dtype=torch.int32, device=dev)
        self.relres = torch.empty(L, **f64)
        self.q = torch.empty(L, **f64)
        self.grad = torch.empty(L * self.N, **f64)
        self.work = torch.empty(ens.ens_pcg_workspace_size(self.J, self.nnz, self.S, self.Emax), dtype=torch.uint8,
                                device=dev)
        self.gwork = torch.empty(ens.ens_adjoint_solve_workspace_size(prob, self.S, self.Emax), dtype=torch.uint8,
                                 device=dev)
        self.last = {}

    def _load(self, xi: torch.Tensor):
        M = xi.shape[0]
        E = math.ceil(M / self.S)
        if E > self.Emax:
            raise ValueError("too many samples for this solver")
        L = E * self.S
        xv = self.xi[: L * self.N].view(L, self.N)
        xv[:M].copy_(xi)
        if L > M:
            xv[M:].copy_(xi[M - 1:M].expand(L - M, self.N))
        self.active[:L].fill_(1)
        if L > M:
            self.active[M:L].fill_(0)
        return M, E, L

    def _solve(self, E, L, out):
        J, S, nnz = self.J, self.S, self.nnz
        vals, dinv, b = self.vals[: E * nnz * S], self.dinv[: E * J * S], self.b[: E * J * S]
        ens.ens_assemble(self.h, self.prob, S, E, self.xi[: L * self.N], self.rowptr, self.colidx, vals, dinv, b)
        ens.ens_pcg_solve(self.h, J, nnz, S, E, self.rowptr, self.colidx, vals, dinv, b, out[: E * J * S],
                          self.active[:L], self.rtol, self.maxit, self.iters[:L], self.relres[:L], self.status[:L],
                          self.work)

    def forward(self, xi: torch.Tensor) -> torch.Tensor:
        """Q[M] for the samples xi[M][N] (device f64)."""
        M, E, L = self._load(xi)
        self._solve(E, L, self.u)
        ens.ens_qoi(self.h, self.J, self.S, E, self.u[: E * self.J * self.S], self.q[:L], w=self.w)
        self.last = dict(forward_iters=self.iters[:M].clone(), forward_status=self.status[:M].clone())
        return self.q[:M].clone()

    def gradient(self, xi: torch.Tensor, recompute_forward: bool) -> torch.Tensor:
        """dQ/dxi [M][N]; solves for u again first when recompute_forward."""
        M, E, L = self._load(xi)
        if recompute_forward:
            self._solve(E, L, self.u)
        n = E * self.J * self.S
        ens.ens_adjoint_solve_grad(self.h, self.prob, self.S, E, self.xi[: L * self.N], self.rowptr, self.colidx,
                                   self.u[:n], self.w, self.active[:L], self.rtol, self.maxit, self.q[:L],
                                   self.grad[: L * self.N], self.lam[:n], self.iters[:L], self.relres[:L],
                                   self.status[:L], self.gwork)
        self.last["adjoint_iters"] = self.iters[:M].clone()
        self.last["adjoint_status"] = self.status[:M].clone()
        return self.grad[: M * self.N].view(M, self.N).clone()


class EnsembleQoI(torch.autograd.Function):
    """Q = QoI(xi) with dQ/dxi from the adjoint ensemble solve."""

    @staticmethod
    def forward(ctx, xi: torch.Tensor, solver: AdjointSolver, recompute: bool = True):
        q = solver.forward(xi.detach())
        ctx.solver = solver
        ctx.recompute = bool(recompute)
        ctx.save_for_backward(xi.detach())
        return q

    @staticmethod
    def backward(ctx, gq: torch.Tensor):
        (xi,) = ctx.saved_tensors
        g = ctx.solver.gradient(xi, recompute_forward=ctx.recompute)
        return gq.to(g.dtype)[:, None] * g, None, None


def qoi(xi: torch.Tensor, solver: AdjointSolver, recompute: bool = True) -> torch.Tensor:
    return EnsembleQoI.apply(xi, solver, recompute)
