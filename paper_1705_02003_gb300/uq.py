"""The grid-generation and grouping loop of Section 3.1 ("The algorithm",
steps 1-4 of the flowchart) on the GPU path.

    Y_0 = initial sparse grid (levels 0..init_level), grouped in generation order
    loop:
      1. solve the newest points in ensembles -> G(y) = ||u||_2^2, I(y) = iterations
      2. surpluses of G and I at the new points (ens_sg_eval with values)
      3. refine the new points whose |surplus of G| >= tau (ens_sg_refine, host);
         stop when nothing is refined or |Y| + |Y_new| > n_max
      4. group the new points by the iteration surrogate (ens_group) and go to 1.

Groupings: "sur" (the surrogate, Section 3.1), "par" (the anisotropy indicator
of Section 3.2), "nat" (generation order), "rand" (a seeded permutation), all
with S-sample ensembles; "its" (sorted by the actual counts, known only
afterwards) is reported through R only.

The grid table (levels, indices, surpluses) stays on the device in generation
order; per level the host reads back only the G surpluses it refines on.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import ens, inputs
from .solver import EnsembleSolver


def coords(lvl: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Grid-point coordinates y_{l,i} = i 2^(1-l) - 1 per dimension (ens_sg_points)."""
    return ens.ens_sg_points(lvl, idx)


def work_ratio(S: int, perm: np.ndarray, iters: np.ndarray) -> float:
    """Eq. (R): S sum_k max_{i in k} I_i / sum_i I_i over the real samples."""
    it = np.asarray(iters, np.float64)[perm]
    num = sum(float(it[k:k + S].max()) for k in range(0, len(it), S))
    return S * num / float(it.sum())


def level_surpluses(h: ens.Handle, lvl: np.ndarray, lvl_d: torch.Tensor, idx_d: torch.Tensor,
                    y_d: torch.Tensor, values: torch.Tensor) -> torch.Tensor:
    """Surpluses c = v - (surrogate of the lower levels)(y) of a grid listed in
    non-decreasing level order, one level at a time (Eq. hierSGint)."""
    c = torch.empty(len(lvl), dtype=torch.float64, device=values.device)
    lev = lvl.sum(axis=1)
    for L in range(int(lev.max()) + 1):
        a, b = int(np.searchsorted(lev, L, "left")), int(np.searchsorted(lev, L, "right"))
        if b > a:
            ens.ens_sg_eval(h, lvl_d[:a] if a else None, idx_d[:a], c[:a], y_d[a:b], c[a:b], values=values[a:b])
    return c


class PilotGrouping:
    """Surrogate grouping of a sample set that is not generated adaptively
    (Section 5: pre-select samples, evaluate them, and build the iteration
    surrogate from the results).  The pre-selected samples are the full sparse
    grid of levels 0..level; they are solved in ensembles of the solver's S in
    generation order, their iteration counts are hierarchized level by level,
    and a set of draws is then grouped by the surrogate's prediction (sort and
    chunk, ens_group)."""

    def __init__(self, handle: ens.Handle, solver: EnsembleSolver, level: int):
        self.h = handle
        self.solver = solver
        self.level = level
        self.lvl, self.idx = ens.ens_sg_initial(solver.N, level)
        dev = solver.dev
        self.lvl_d = torch.from_numpy(self.lvl).to(dev)
        self.idx_d = torch.from_numpy(self.idx).to(dev)
        self.y_d = torch.from_numpy(coords(self.lvl, self.idx)).to(dev)
        self.I = None
        self.cI = None

    def build(self):
        """Solve the pilot points and form the iteration surpluses."""
        sol = self.solver
        M = len(self.lvl)
        cap = sol.Emax * sol.S
        I = torch.empty(M, dtype=torch.float64, device=sol.dev)
        for a in range(0, M, cap):
            b = min(M, a + cap)
            it, st, rr, q = sol.solve(self.y_d[a:b])
            I[a:b] = it.to(torch.float64)
        self.I = I
        self.cI = level_surpluses(self.h, self.lvl, self.lvl_d, self.idx_d, self.y_d, I)
        return self

    def group(self, xi: torch.Tensor, S: int, pred: torch.Tensor | None = None):
        """(pred, perm, n_ens) for the draws xi[M][N] (device f64, inside
        [-1, 1]^N): predicted iterations, the ensemble order, the ensemble count."""
        M = xi.shape[0]
        pred = torch.empty(M, dtype=torch.float64, device=xi.device) if pred is None else pred
        perm = torch.empty(M, dtype=torch.int32, device=xi.device)
        n_ens = ens.ens_group(self.h, self.lvl_d, self.idx_d, self.cI, xi.contiguous(), S, pred, perm)
        return pred, perm, n_ens


class Adaptive:
    """Runs the loop for one workload with one grouping."""

    def __init__(self, handle: ens.Handle, wl: inputs.Workload, S: int | None = None,
                 solver: EnsembleSolver | None = None, per_sample: bool = False, repack: bool = False,
                 chunk: int = 64, precond: str = "jacobi"):
        self.h = handle
        self.wl = wl
        self.S = wl.S if S is None else S
        self.per_sample = per_sample
        self.prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
        cap = min(wl.n_max, 16384)
        if solver is None:
            solver = EnsembleSolver(handle, self.prob, 1 if per_sample else self.S,
                                    1 if per_sample else cap, wl.rtol, wl.maxit, precond=precond)
        if repack and solver.precond != "jacobi":
            raise ValueError("lane re-packing runs the Jacobi solver")
        self.solver = solver
        self.dev = solver.dev
        self.launches = 0
        self.solve_sets = []
        # repack: solve each level through the batching layer (ens_solve_stream),
        # which gathers the live lanes of partly converged ensembles into fewer
        # ensembles every `chunk` trips; the groups are still the grouping's.
        self.repack = repack
        self.chunk = chunk
        self.stream_work = None
        self.sink = None  # optional callable(solver, M) run after every solve call
        self.time_calls = False  # record CUDA events around every ensemble solve call
        self.call_events = []

    def _solve(self, y_dev: torch.Tensor, order: torch.Tensor, offset: int):
        """Solve the points y_dev[order] and return (G, I) in point order.
        Records which global points each solve call held (for launch counts)."""
        M = y_dev.shape[0]
        G = torch.empty(M, dtype=torch.float64, device=self.dev)
        I = torch.empty(M, dtype=torch.float64, device=self.dev)
        xi = y_dev.index_select(0, order)
        if self.per_sample:
            order_h = order.cpu().numpy()
            for j in range(M):
                it, st, rr, q = self._call(xi[j:j + 1])
                if self.sink:
                    self.sink(self.solver, 1)
                G[order[j:j + 1]] = q
                I[order[j:j + 1]] = it.to(torch.float64)
                self.solve_sets.append(np.array([offset + order_h[j]]))
        elif self.repack:
            from . import batching

            E = -(-M // self.solver.S)
            need = ens.ens_stream_workspace_size(self.prob, self.solver.S, E)
            if self.stream_work is None or self.stream_work.numel() < need:
                self.stream_work = torch.empty(need, dtype=torch.uint8, device=self.dev)
            out = batching.solve_stream(self.h, self.prob, xi, self.solver.S, E, self.wl.rtol, self.wl.maxit,
                                        chunk=self.chunk, work=self.stream_work)
            G[order] = out["qoi"]
            I[order] = out["iters"].to(torch.float64)
            self.solve_sets.append(offset + order.cpu().numpy())
        else:
            # a level larger than the solver's capacity is solved in calls of
            # whole ensembles (capacity is a multiple of S), which leaves every
            # ensemble -- and so every sample's result -- as in one call
            cap = self.solver.Emax * self.solver.S
            order_h = order.cpu().numpy()
            for a0 in range(0, M, cap):
                a1 = min(M, a0 + cap)
                it, st, rr, q = self._call(xi[a0:a1])
                if self.sink:
                    self.sink(self.solver, a1 - a0)
                G[order[a0:a1]] = q
                I[order[a0:a1]] = it.to(torch.float64)
                self.solve_sets.append(offset + order_h[a0:a1])
        return G, I

    def _call(self, xs: torch.Tensor):
        """One solve call, bracketed by CUDA events when time_calls is set."""
        if not self.time_calls:
            return self.solver.solve(xs)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record()
        out = self.solver.solve(xs)
        ev[1].record()
        self.call_events.append((xs.shape[0], ev))
        return out

    def call_times(self):
        """(M, milliseconds) of every ensemble solve call of the last run made
        with time_calls set (synchronises the device)."""
        torch.cuda.synchronize()
        return [(M, ev[0].elapsed_time(ev[1])) for M, ev in self.call_events]

    def kernel_launches(self, I: np.ndarray) -> int:
        """Kernels of libens launched by the last run: per solve call assembly,
        PCG init, finish and QoI, and three kernels per trip of each loop
        branch (a branch runs until the slowest sample of its ensembles stops);
        plus the grouping and surplus kernels counted in run()."""
        n = self.launches
        S = self.solver.S
        for pts in self.solve_sets:
            it = I[pts]
            E = -(-len(it) // S)
            nb = ens.ens_pcg_branches(self.h, E)
            n += 4
            for b in range(nb):
                e0, e1 = b * E // nb, (b + 1) * E // nb
                n += 3 * max(1, int(it[e0 * S:e1 * S].max()))
        return n

    def run(self, grouping: str = "sur", seed: int = 0, record_trips: bool = False,
            stop_after: int | None = None, resume: dict | None = None):
        """Run the loop.  stop_after = k returns after k refined levels with
        done = False; resume = such a result (or load_run of a saved one)
        continues from there exactly as an uninterrupted run would."""
        wl, S, dev = self.wl, self.S, self.dev
        N = wl.nparam
        self.launches = 0
        self.solve_sets = []
        self.call_events = []
        if resume is None:
            lvl, idx = ens.ens_sg_initial(N, wl.init_level)
            y = coords(lvl, idx)
            lvl_d = torch.from_numpy(lvl).to(dev)
            idx_d = torch.from_numpy(idx).to(dev)
            y_d = torch.from_numpy(y).to(dev)
            M0 = len(lvl)
            order = torch.arange(M0, device=dev)
            G, I = self._solve(y_d, order, 0)
            # surpluses of the initial grid, one level at a time (Eq. hierSGint)
            cG = level_surpluses(self.h, lvl, lvl_d, idx_d, y_d, G)
            cI = level_surpluses(self.h, lvl, lvl_d, idx_d, y_d, I)
            self.launches += 2 * len(np.unique(lvl.sum(axis=1)))
            levels = [(0, M0)]
            perms = [np.arange(M0, dtype=np.int32)]
            preds = [np.zeros(M0)]
            rng_seed = seed
            first = 0
        else:
            if resume["done"] or resume["grouping"] != grouping or resume["S"] != S:
                raise ValueError("resume needs an unfinished run of the same grouping and S")
            lvl, idx = resume["lvl"], resume["idx"]
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
            lvl_d, idx_d, y_d = t(lvl), t(idx), t(resume["y"])
            G, I, cG, cI = t(resume["G"]), t(resume["I"]), t(resume["cG"]), t(resume["cI"])
            levels = [tuple(l) for l in resume["levels"]]
            perms = list(resume["perms"])
            preds = list(resume["preds"])
            rng_seed = resume["rng_seed"]
            first = levels[-1][0]
        refined = 0
        done = True
        while True:
            if stop_after is not None and refined >= stop_after:
                done = False
                break
            cG_host = cG[first:].cpu().numpy()
            cG_all = np.concatenate([np.zeros(first), cG_host])
            nl, ni = ens.ens_sg_refine(lvl, idx, first, cG_all, wl.tau, wl.max_level)
            if len(nl) == 0 or len(lvl) + len(nl) > wl.n_max:
                break
            Mn = len(nl)
            yn = torch.from_numpy(coords(nl, ni)).to(dev)
            pred = torch.empty(Mn, dtype=torch.float64, device=dev)
            if grouping == "sur":
                perm = torch.empty(Mn, dtype=torch.int32, device=dev)
                ens.ens_group(self.h, lvl_d, idx_d, cI, yn, S, pred, perm)
                self.launches += 2
            elif grouping == "par":
                # parameter-based grouping (Section 3.2): sort by the anisotropy indicator H
                perm = torch.empty(Mn, dtype=torch.int32, device=dev)
                ens.ens_param_indicator(self.h, self.prob, yn, pred)
                ens.ens_sort_chunk(self.h, pred, S, perm)
                self.launches += 2
            elif grouping == "nat":
                perm = torch.arange(Mn, dtype=torch.int32, device=dev)
            elif grouping == "rand":
                perm = torch.from_numpy(inputs.rand_perm(Mn, rng_seed)).to(dev)
                rng_seed += 1
            else:
                raise ValueError(f"unknown grouping {grouping}")
            Gn, In = self._solve(yn, perm.to(torch.int64), len(lvl))
            cGn = torch.empty(Mn, dtype=torch.float64, device=dev)
            cIn = torch.empty(Mn, dtype=torch.float64, device=dev)
            ens.ens_sg_eval(self.h, lvl_d, idx_d, cG, yn, cGn, values=Gn)
            ens.ens_sg_eval(self.h, lvl_d, idx_d, cI, yn, cIn, values=In)
            self.launches += 2
            first = len(lvl)
            levels.append((first, first + Mn))
            perms.append(perm.cpu().numpy())
            preds.append(pred.cpu().numpy() if grouping in ("sur", "par") else np.zeros(Mn))
            lvl = np.concatenate([lvl, nl])
            idx = np.concatenate([idx, ni])
            lvl_d = torch.cat([lvl_d, torch.from_numpy(nl).to(dev)])
            idx_d = torch.cat([idx_d, torch.from_numpy(ni).to(dev)])
            y_d = torch.cat([y_d, yn])
            G = torch.cat([G, Gn])
            I = torch.cat([I, In])
            cG = torch.cat([cG, cGn])
            cI = torch.cat([cI, cIn])
            refined += 1
        return dict(lvl=lvl, idx=idx, y=y_d.cpu().numpy(), G=G.cpu().numpy(), I=I.cpu().numpy(),
                    cG=cG.cpu().numpy(), cI=cI.cpu().numpy(), levels=levels, perms=perms, preds=preds,
                    S=S, grouping=grouping, rng_seed=rng_seed, done=done)


def save_run(run: dict, path: str) -> None:
    """Write a run of Adaptive.run (finished or not) to an .npz checkpoint."""
    arrays = {k: run[k] for k in ("lvl", "idx", "y", "G", "I", "cG", "cI")}
    for j, (p, q) in enumerate(zip(run["perms"], run["preds"])):
        arrays[f"perm{j}"] = p
        arrays[f"pred{j}"] = q
    meta = {"levels": [list(map(int, l)) for l in run["levels"]], "S": int(run["S"]),
            "grouping": run["grouping"], "rng_seed": int(run["rng_seed"]), "done": bool(run["done"])}
    np.savez(path, meta=np.array(json.dumps(meta)), **arrays)


def load_run(path: str) -> dict:
    """Read a checkpoint written by save_run."""
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(str(z["meta"]))
        run = {k: z[k] for k in ("lvl", "idx", "y", "G", "I", "cG", "cI")}
        n = len(meta["levels"])
        run["perms"] = [z[f"perm{j}"] for j in range(n)]
        run["preds"] = [z[f"pred{j}"] for j in range(n)]
    run.update(levels=[tuple(l) for l in meta["levels"]], S=meta["S"], grouping=meta["grouping"],
               rng_seed=meta["rng_seed"], done=meta["done"])
    return run


def ratios(run: dict, S: int | None = None):
    """R_l per level and R overall (Eqs. Rl, R) for the run's grouping and for
    the iteration-sorted ("its") grouping of the same levels."""
    S = run["S"] if S is None else S
    out = {}
    for name in ("run", "its"):
        Rl, num, den = [], 0.0, 0.0
        for (a, b), perm in zip(run["levels"], run["perms"]):
            it = run["I"][a:b]
            p = np.argsort(it, kind="stable") if name == "its" else perm
            r = work_ratio(S, p, it)
            Rl.append(r)
            num += r * it.sum() / S
            den += it.sum()
        out[name] = (Rl, S * num / den)
    return out
