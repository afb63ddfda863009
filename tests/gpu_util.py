"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
on seeded inputs and lay the results out per sample."""
import math

import numpy as np
import torch

import oracle as O
from paper_1705_02003_gb300 import ens

OKIND = {"fd5": O.FD5_LOGKL, "q1": O.Q1_ROT, "fd7": O.FD7_AXIS, "q1_3d_kl": O.Q1_3D_KL,
         "q1_3d_disc": O.Q1_3D_DISC}


class Case:
    """Device buffers for E ensembles of S lanes of one problem."""

    def __init__(self, h, kind, n, N, aniso, S, xi, active=None):
        self.h, self.kind, self.n, self.N, self.aniso, self.S = h, kind, n, N, aniso, S
        self.prob = ens.problem(kind, n, N, aniso)
        self.J, self.nnz = ens.ens_problem_size(self.prob)
        xi = np.asarray(xi, np.float64)
        M = xi.shape[0]
        self.E = E = math.ceil(M / S)
        pad = E * S - M
        if pad:
            xi = np.concatenate([xi, np.repeat(xi[-1:], pad, axis=0)])
        self.M = M
        self.xi_h = xi
        dev = "cuda"
        self.xi = torch.from_numpy(xi).to(dev).contiguous()
        self.rowptr = torch.empty(self.J + 1, dtype=torch.int32, device=dev)
        self.colidx = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        ens.ens_pattern(h, self.prob, self.rowptr, self.colidx)
        self.vals = torch.empty(E * self.nnz * S, dtype=torch.float64, device=dev)
        self.dinv = torch.empty(E * self.J * S, dtype=torch.float64, device=dev)
        self.b = torch.empty(E * self.J * S, dtype=torch.float64, device=dev)
        ens.ens_assemble(h, self.prob, S, E, self.xi, self.rowptr, self.colidx, self.vals, self.dinv, self.b)
        if active is None:
            active = np.ones(E * S, np.uint8)
            active[M:] = 0
        self.active = torch.from_numpy(np.asarray(active, np.uint8)).to(dev)

    def solve(self, rtol, maxit, vals=None, active=None):
        E, S, J = self.E, self.S, self.J
        dev = "cuda"
        x = torch.full((E * J * S,), float("nan"), dtype=torch.float64, device=dev)
        iters = torch.full((E * S,), -7, dtype=torch.int32, device=dev)
        status = torch.full((E * S,), -7, dtype=torch.int32, device=dev)
        relres = torch.empty(E * S, dtype=torch.float64, device=dev)
        work = torch.empty(ens.ens_pcg_workspace_size(J, self.nnz, S, E), dtype=torch.uint8, device=dev)
        ens.ens_pcg_solve(self.h, J, self.nnz, S, E, self.rowptr, self.colidx,
                          self.vals if vals is None else vals, self.dinv, self.b, x,
                          self.active if active is None else active, rtol, maxit, iters, relres, status, work)
        torch.cuda.synchronize()
        xs = x.view(E, J, S).permute(0, 2, 1).reshape(E * S, J).cpu().numpy()
        return dict(x=xs, iters=iters.cpu().numpy(), status=status.cpu().numpy(), relres=relres.cpu().numpy())

    def lane_vals(self):
        """vals as [E*S][nnz] (per sample)."""
        E, S = self.E, self.S
        return self.vals.view(E, self.nnz, S).permute(0, 2, 1).reshape(E * S, self.nnz).cpu().numpy()

    def lane_vec(self, t):
        E, S = self.E, self.S
        return t.view(E, self.J, S).permute(0, 2, 1).reshape(E * S, self.J).cpu().numpy()

    def mg_work(self, mixed=False):
        return torch.empty(ens.ens_mg_workspace_size(self.prob, self.S, self.E, mixed), dtype=torch.uint8,
                           device="cuda")

    def solve_mg(self, rtol, maxit, vals=None, b=None, active=None, work=None, mixed=False):
        """Multigrid setup + MG-PCG through the C ABI; results per lane as solve()."""
        E, S, J = self.E, self.S, self.J
        dev = "cuda"
        vals = self.vals if vals is None else vals
        work = self.mg_work(mixed) if work is None else work
        x = torch.full((E * J * S,), float("nan"), dtype=torch.float64, device=dev)
        iters = torch.full((E * S,), -7, dtype=torch.int32, device=dev)
        status = torch.full((E * S,), -7, dtype=torch.int32, device=dev)
        relres = torch.empty(E * S, dtype=torch.float64, device=dev)
        ens.ens_mg_setup(self.h, self.prob, S, E, self.rowptr, self.colidx, vals, work, mixed=mixed)
        ens.ens_mgpcg_solve(self.h, self.prob, S, E, self.rowptr, self.colidx, vals, self.b if b is None else b, x,
                            self.active if active is None else active, rtol, maxit, iters, relres, status, work,
                            mixed=mixed)
        torch.cuda.synchronize()
        xs = x.view(E, J, S).permute(0, 2, 1).reshape(E * S, J).cpu().numpy()
        return dict(x=xs, iters=iters.cpu().numpy(), status=status.cpu().numpy(), relres=relres.cpu().numpy())

    def upload_lanes(self, per_lane, J):
        """[E*S][J] host array -> device [E][J][S]."""
        E, S = self.E, self.S
        a = np.asarray(per_lane, np.float64).reshape(E, S, J).transpose(0, 2, 1).copy()
        return torch.from_numpy(a.ravel()).to("cuda")


def elem_err(x, x0):
    """max_j |x_j - x0_j| / max_j |x0_j|: an element-wise bound relative to the
    largest entry (a relative 2-norm could hide large errors in small entries)."""
    x, x0 = np.asarray(x), np.asarray(x0)
    return float(np.max(np.abs(x - x0)) / np.max(np.abs(x0)))


def grouping_on_oracle_counts(h, r):
    """Feed the oracle run's grid and iteration surpluses to ens_group level by
    level; predictions and permutations must equal the oracle's bit for bit."""
    S = r["S"]
    for (a, b), pred_o, perm_o in zip(r["levels"][1:], r["pred"][1:], r["perms"]["sur"][1:]):
        yq = O.sg_points(r["lvl"][a:b], r["idx"][a:b])
        pred = torch.empty(b - a, dtype=torch.float64, device="cuda")
        perm = torch.empty(b - a, dtype=torch.int32, device="cuda")
        dev = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
        ens.ens_group(h, dev(r["lvl"][:a]), dev(r["idx"][:a]), dev(r["cI"][:a]), dev(yq), S, pred, perm)
        assert np.array_equal(pred.cpu().numpy(), pred_o)
        assert np.array_equal(perm.cpu().numpy(), perm_o)
