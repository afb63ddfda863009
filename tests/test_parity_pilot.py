"""GPU parity of surrogate grouping for a sample set that is not generated
adaptively (Section 5: pre-select samples, evaluate them, build the iteration
surrogate from the results): the full sparse grid of levels 0..1 in six
dimensions (256 points) is solved, its iteration counts hierarchized, and 256
uniform draws grouped by the surrogate.  The surpluses, predictions and the
grouping equal the oracle's bit for bit whenever the pilot iteration counts
agree, and the grouping beats generation order on the draws' own counts."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from oracle import uq as ouq
from paper_1705_02003_gb300 import ens, inputs, uq
from paper_1705_02003_gb300.solver import EnsembleSolver

pytestmark = pytest.mark.gpu

KIND, N_GRID, N, ANISO, S, RTOL, MAXIT = "fd7", 12, 6, 3.0, 8, 1e-8, 20000


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


def test_pilot_grouping_matches_oracle_and_groups_well(h):
    prob = ens.problem(KIND, N_GRID, N, ANISO)
    sol = EnsembleSolver(h, prob, S, 256, RTOL, MAXIT)
    pg = uq.PilotGrouping(h, sol, level=1).build()
    assert len(pg.lvl) == 2 ** N + N * 2 ** (N - 1)  # corners, then one coordinate at the centre
    threads = os.cpu_count() or 4
    y = O.sg_points(pg.lvl, pg.idx)
    o = O.solve_batch(O.FD7_AXIS, N_GRID, N, ANISO, y, RTOL, MAXIT, nthreads=threads)
    I_gpu = pg.I.cpu().numpy()
    assert np.max(np.abs(I_gpu - o["iters"])) <= 1
    cI_o = ouq.hierarchize(pg.lvl, pg.idx, o["iters"].astype(np.float64))

    draws = inputs.draws(256, N, seed=31)
    pred, perm, n_ens = pg.group(torch.from_numpy(draws).cuda(), S)
    pred_g, perm_g = pred.cpu().numpy(), perm.cpu().numpy()
    assert n_ens == 256 // S
    assert sorted(perm_g.tolist()) == list(range(256))
    assert perm_g.tolist() == sorted(range(256), key=lambda i: pred_g[i])  # stable ascending sort
    # fed the oracle's pilot counts, the GPU surrogate and grouping are the oracle's bit for bit
    pred_o = O.sg_eval(pg.lvl, pg.idx, cI_o, draws)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pred2 = torch.empty(256, dtype=torch.float64, device="cuda")
    perm2 = torch.empty(256, dtype=torch.int32, device="cuda")
    ens.ens_group(h, dev(pg.lvl), dev(pg.idx), dev(cI_o), dev(draws), S, pred2, perm2)
    assert np.array_equal(pred2.cpu().numpy(), pred_o)
    assert np.array_equal(perm2.cpu().numpy(), O.sort_perm(pred_o))
    if np.array_equal(I_gpu, o["iters"]):
        assert np.array_equal(pg.cI.cpu().numpy(), cI_o)
        assert np.array_equal(pred_g, pred_o)
        assert np.array_equal(perm_g, O.sort_perm(pred_o))

    # the draws' own iteration counts (the oracle's): surrogate order against generation order
    od = O.solve_batch(O.FD7_AXIS, N_GRID, N, ANISO, draws, RTOL, MAXIT, nthreads=threads)
    it = od["iters"].astype(np.float64)
    R_sur = uq.work_ratio(S, perm_g, it)
    R_nat = uq.work_ratio(S, np.arange(256), it)
    R_its = uq.work_ratio(S, np.argsort(it, kind="stable"), it)
    assert R_its <= R_sur + 1e-12
    assert R_sur < R_nat
