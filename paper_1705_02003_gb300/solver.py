"""Batched ensemble solves on one GPU: device buffers for up to E_max ensembles
of S samples of one problem, and the assemble -> PCG -> QoI pipeline through
the C ABI.  PyTorch only provides the device memory and the stream.

Samples arrive already in ensemble order (consecutive runs of S form the
ensembles, Section 3.1); a short last run is padded with copies of its last
sample whose lanes are masked inactive, so they cost no updates and report
status ENS_LANE_INACTIVE.
"""
from __future__ import annotations

import math

import torch

from . import ens


class EnsembleSolver:
    """precond = "jacobi" (ens_pcg_solve), "mg" (ens_mg_setup + ens_mgpcg_solve:
    the multigrid V-cycle of the trilinear problems) or "mg32" (the same with
    the V-cycle in float, CG in double)."""

    def __init__(self, handle: ens.Handle, prob: ens.Problem, S: int, max_samples: int, rtol: float,
                 maxit: int, device=None, precond: str = "jacobi"):
        if precond not in ("jacobi", "mg", "mg32"):
            raise ValueError(f"unknown preconditioner {precond}")
        self.h = handle
        self.prob = prob
        self.precond = precond
        self.S = int(S)
        self.N = prob.nparam
        self.rtol = float(rtol)
        self.maxit = int(maxit)
        dev = torch.device("cuda", handle.device) if device is None else torch.device(device)
        self.dev = dev
        self.J, self.nnz = ens.ens_problem_size(prob)
        self.rowptr = torch.empty(self.J + 1, dtype=torch.int32, device=dev)
        self.colidx = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        ens.ens_pattern(handle, prob, self.rowptr, self.colidx)
        self.Emax = max(1, math.ceil(max_samples / self.S))
        lanes = self.Emax * self.S
        f64 = dict(dtype=torch.float64, device=dev)
        self.xi = torch.empty(lanes * self.N, **f64)
        self.vals = torch.empty(self.Emax * self.nnz * self.S, **f64)
        self.dinv = torch.empty(self.Emax * self.J * self.S, **f64)
        self.b = torch.empty(self.Emax * self.J * self.S, **f64)
        self.x = torch.empty(self.Emax * self.J * self.S, **f64)
        self.active = torch.empty(lanes, dtype=torch.uint8, device=dev)
        self.iters = torch.empty(lanes, dtype=torch.int32, device=dev)
        self.status = torch.empty(lanes, dtype=torch.int32, device=dev)
        self.relres = torch.empty(lanes, **f64)
        self.qoi = torch.empty(lanes, **f64)
        self.mixed = precond == "mg32"
        if precond != "jacobi":
            need = ens.ens_mg_workspace_size(prob, self.S, self.Emax, self.mixed)
            if need == 0:
                raise ValueError("this problem has no multigrid hierarchy (trilinear problems, n = 2^k - 1)")
        else:
            need = ens.ens_pcg_workspace_size(self.J, self.nnz, self.S, self.Emax)
        self.work = torch.empty(need, dtype=torch.uint8, device=dev)

    def bytes_per_iteration(self, E: int) -> int:
        """Algorithmic bytes of one PCG iteration of E ensembles: values, graph,
        and the nine vector streams (x r/w, r r/w, p r/w, q w/r, D^-1 r)."""
        return E * (8 * self.nnz * self.S + 4 * self.nnz + 4 * (self.J + 1) + 72 * self.J * self.S)

    def solve(self, xi: torch.Tensor, weights: torch.Tensor | None = None):
        """Solve the samples xi[M][N] (device f64, ensemble order).

        Returns views (iters, status, relres, qoi), each [M], valid until the
        next call.  qoi = ||u||_2^2, or w^T u when weights[J] is given."""
        M = xi.shape[0]
        S = self.S
        E = math.ceil(M / S)
        if E > self.Emax:
            raise ValueError(f"{M} samples exceed the solver's capacity {self.Emax * S}")
        if M == 0:
            z = torch.empty(0, dtype=torch.int32, device=self.dev)
            return z, z, torch.empty(0, dtype=torch.float64, device=self.dev), torch.empty(0, dtype=torch.float64, device=self.dev)
        L = E * S
        xv = self.xi[: L * self.N].view(L, self.N)
        xv[:M].copy_(xi)
        if L > M:
            xv[M:].copy_(xi[M - 1:M].expand(L - M, self.N))
        act = self.active[:L]
        act.fill_(1)
        if L > M:
            act[M:].fill_(0)
        J, nnz = self.J, self.nnz
        vals = self.vals[: E * nnz * S]
        dinv = self.dinv[: E * J * S]
        b = self.b[: E * J * S]
        x = self.x[: E * J * S]
        ens.ens_assemble(self.h, self.prob, S, E, self.xi[: L * self.N], self.rowptr, self.colidx, vals, dinv, b)
        if self.precond != "jacobi":
            ens.ens_mg_setup(self.h, self.prob, S, E, self.rowptr, self.colidx, vals, self.work, mixed=self.mixed)
            ens.ens_mgpcg_solve(self.h, self.prob, S, E, self.rowptr, self.colidx, vals, b, x, act, self.rtol,
                                self.maxit, self.iters[:L], self.relres[:L], self.status[:L], self.work,
                                mixed=self.mixed)
        else:
            ens.ens_pcg_solve(self.h, J, nnz, S, E, self.rowptr, self.colidx, vals, dinv, b, x, act, self.rtol,
                              self.maxit, self.iters[:L], self.relres[:L], self.status[:L], self.work)
        ens.ens_qoi(self.h, J, S, E, x, self.qoi[:L], w=weights)
        return self.iters[:M], self.status[:M], self.relres[:M], self.qoi[:M]

    def solution(self, M: int) -> torch.Tensor:
        """x of the last solve as [E][J][S] (device view)."""
        E = math.ceil(M / self.S)
        return self.x[: E * self.J * self.S].view(E, self.J, self.S)

    @staticmethod
    def trips(iters: torch.Tensor, status: torch.Tensor) -> int:
        """Trips of the device while loop for one solve (K2-K4 launched per trip):
        one per iteration of the slowest lane, plus the trip in which a lane
        broke down, and at least one."""
        if iters.numel() == 0:
            return 1
        t = iters.to(torch.int64) + (status == ens.LANE_BREAKDOWN).to(torch.int64)
        return max(1, int(t.max().item()))
