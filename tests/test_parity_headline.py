"""The headline workload end to end against the oracle: the grid-generation and
grouping loop of Section 3.1 on the Q1 256 x 256 problem (4 parameters,
rotated anisotropy up to 10^4, 265 adaptive points in 3 levels, S = 16), every
sample solved by the GPU path and by the oracle.

Checked for the ensemble path (S = 16, surrogate grouping) and for one sample
per call (S = 1):
  - the same grid and levels (the grid follows from G alone);
  - G = ||u||^2 of every sample within 1e-10 relative;
  - every sample's iteration count within one of the oracle's, or every
    stopping decision consistent with the oracle's residual history to within
    the oracle's own rounding drift (tests/stopping.py): the samples whose
    residual hovers at the threshold;
  - predictions and groupings of every refined level bit-exact when the GPU
    surrogate is fed the oracle's iteration counts.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle as O
from oracle import uq as ouq
from paper_1705_02003_gb300 import ens, inputs, uq
from stopping import oracle_check

pytestmark = pytest.mark.gpu

WL = inputs.WORKLOADS["q1_256_adaptive"]


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


@pytest.fixture(scope="module")
def oracle_run():
    threads = os.cpu_count() or 1

    def solve(y):
        out = O.solve_batch(O.Q1_ROT, WL.n, WL.nparam, WL.aniso, y, WL.rtol, WL.maxit, nthreads=threads)
        assert np.all(out["status"] == O.CONVERGED)
        return out["G"], out["iters"]

    return ouq.adaptive(solve, WL.nparam, WL.S, WL.tau, WL.init_level, WL.max_level, WL.n_max)


def stop_checks(y, counts, counts_oracle):
    """oracle_check of each point y[m] (tests/stopping.py), in parallel."""
    rp, ci = O.pattern(O.Q1_ROT, WL.n)

    def one(args):
        ym, k, ko = args
        vals, b = O.assemble(O.Q1_ROT, WL.n, WL.nparam, WL.aniso, ym, rp, ci)
        return oracle_check(O, rp, ci, vals, b, WL.rtol, int(k), int(ko))[0]

    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        return list(ex.map(one, zip(y, counts, counts_oracle)))


def check_run(run, r):
    """Same grid, G within 1e-10, and every count within one of the oracle's or
    its stops consistent with the oracle's residual history."""
    assert np.array_equal(run["lvl"], r["lvl"]) and np.array_equal(run["idx"], r["idx"])
    assert run["levels"] == r["levels"]
    assert len(run["I"]) == 265
    np.testing.assert_allclose(run["G"], r["G"], rtol=1e-10, atol=0)
    Ig, Io = run["I"].astype(int), r["I"].astype(int)
    off = np.nonzero(Ig != Io)[0]
    ok = stop_checks(r["y"][off], Ig[off], Io[off])
    bad = [(int(m), int(Io[m]), int(Ig[m])) for m, c in zip(off, ok) if not c and abs(Ig[m] - Io[m]) > 1]
    assert not bad, f"stops inconsistent with the oracle's residual history (sample, oracle, gpu): {bad}"
    print(f"\n{len(off)} of {len(Ig)} counts differ from the oracle's (max {np.abs(Ig - Io).max()}); "
          f"{sum(ok)} of them consistent with its residual history")


def test_headline_loop_ensembles_match_oracle(h, oracle_run):
    run = uq.Adaptive(h, WL).run("sur")
    check_run(run, oracle_run)


def test_headline_loop_one_sample_per_call_matches_oracle(h, oracle_run):
    run = uq.Adaptive(h, WL, per_sample=True).run("sur")
    check_run(run, oracle_run)


def test_headline_grouping_bit_exact_on_oracle_counts(h, oracle_run):
    r = oracle_run

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    for (a, b), pred_o, perm_o in zip(r["levels"][1:], r["pred"][1:], r["perms"]["sur"][1:]):
        yq = O.sg_points(r["lvl"][a:b], r["idx"][a:b])
        pred = torch.empty(b - a, dtype=torch.float64, device="cuda")
        perm = torch.empty(b - a, dtype=torch.int32, device="cuda")
        ens.ens_group(h, dev(r["lvl"][:a]), dev(r["idx"][:a]), dev(r["cI"][:a]), dev(yq), WL.S, pred, perm)
        assert np.array_equal(pred.cpu().numpy(), pred_o)
        assert np.array_equal(perm.cpu().numpy(), perm_o)
