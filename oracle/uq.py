"""Oracle: the grid-generation and grouping loop of the paper's flowchart
(Section 3.1, "The algorithm", steps 1-4), composed from the C routines in
``sgrid.c`` and a per-sample solver.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

    Y_0 = initial sparse grid, grouped in generation order
    loop:
      1. solve every point of the newest level -> G(y) = ||u||^2, I(y) = iterations
      2. surpluses of G and I at the new points: c = v - (surrogate of older points)(y)
      3. refine the new points with |c_G| >= tau (children not already present;
         children above ``max_level`` are not made)
         stop if nothing is refined, or if |Y| + |Y_new| > n_max (not admitted)
      4. group the new points: sort by the iteration surrogate I^ (stable), chunk by S
"""
from __future__ import annotations

import numpy as np

from . import sg_eval, sg_initial, sg_points, sg_refine, sort_perm, work_ratio


def hierarchize(lvl, idx, values):
    """Surpluses of a grid listed in non-decreasing level order:
    c_m = v_m - sum_{m' < m} c_{m'} psi_{m'}(y_m)."""
    y = sg_points(lvl, idx)
    c = np.zeros(len(values), np.float64)
    for m in range(len(values)):
        pred = sg_eval(lvl[:m], idx[:m], c[:m], y[m:m + 1])[0] if m else 0.0
        c[m] = values[m] - pred
    return c


def adaptive(solve, N: int, S: int, tau: float, init_level: int, max_level: int, n_max: int,
             rng_seed: int = 0):
    """Run the loop.  ``solve(points[M][N]) -> (G[M], iters[M])``.

    Returns a dict with the grid (lvl, idx, y), per-point G, I, surpluses, the
    level boundaries, the surrogate predictions and the surrogate / natural /
    random / iteration-sorted permutations of each level."""
    lvl, idx = sg_initial(N, init_level)
    y = sg_points(lvl, idx)
    G, I = solve(y)
    G = np.asarray(G, np.float64)
    I = np.asarray(I, np.float64)
    cG = hierarchize(lvl, idx, G)
    cI = hierarchize(lvl, idx, I)
    M0 = len(lvl)
    levels = [(0, M0)]
    pred = [np.zeros(M0)]
    perms = {"sur": [np.arange(M0, dtype=np.int32)], "nat": [np.arange(M0, dtype=np.int32)]}
    rng = np.random.default_rng(rng_seed)
    perms["rand"] = [np.arange(M0, dtype=np.int32)]
    perms["its"] = [sort_perm(I)]
    first = 0
    while True:
        nl, ni = sg_refine(lvl, idx, first, cG, tau, max_level)
        if len(nl) == 0 or len(lvl) + len(nl) > n_max:
            break
        yn = sg_points(nl, ni)
        p = sg_eval(lvl, idx, cI, yn)
        predG = sg_eval(lvl, idx, cG, yn)
        Gn, In = solve(yn)
        Gn = np.asarray(Gn, np.float64)
        In = np.asarray(In, np.float64)
        first = len(lvl)
        levels.append((first, first + len(nl)))
        pred.append(p)
        perms["sur"].append(sort_perm(p))
        perms["nat"].append(np.arange(len(nl), dtype=np.int32))
        perms["rand"].append(rng.permutation(len(nl)).astype(np.int32))
        perms["its"].append(sort_perm(In))
        lvl = np.concatenate([lvl, nl])
        idx = np.concatenate([idx, ni])
        y = np.concatenate([y, yn])
        G = np.concatenate([G, Gn])
        I = np.concatenate([I, In])
        cG = np.concatenate([cG, Gn - predG])
        cI = np.concatenate([cI, In - p])
    return dict(lvl=lvl, idx=idx, y=y, G=G, I=I, cG=cG, cI=cI, levels=levels, pred=pred,
                perms=perms, S=S)


def ratios(run, S: int | None = None):
    """R_l per level and R overall (Eqs. Rl, R) for each grouping."""
    S = run["S"] if S is None else S
    out = {}
    for name, plist in run["perms"].items():
        Rl = []
        num = 0.0
        den = 0.0
        for (a, b), perm in zip(run["levels"], plist):
            it = run["I"][a:b]
            Rl.append(work_ratio(S, perm, it))
            den += float(np.sum(it))
            num += Rl[-1] * float(np.sum(it)) / S
        out[name] = (Rl, S * num / den)
    return out
