"""GPU parity of the grouping step (K6 surrogate, K7 sort-and-chunk) and of the
whole adaptive loop against the oracle.  Predictions and permutations are
compared bit for bit when both sides are fed the same grid and iteration
counts."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import grouping_on_oracle_counts
from oracle import uq as ouq
from paper_1705_02003_gb300 import ens, inputs, uq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


def dev(a, dt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dt is None else t.to(dt)).cuda()


@pytest.fixture(scope="module")
def small_run():
    """The oracle's adaptive loop on the 32 x 32 5-point workload."""
    wl = inputs.WORKLOADS["fd5_32_adaptive"]

    def solve(y):
        out = O.solve_batch(O.FD5_LOGKL, wl.n, wl.nparam, wl.aniso, y, wl.rtol, wl.maxit, nthreads=8)
        return out["G"], out["iters"]

    return ouq.adaptive(solve, N=2, S=wl.S, tau=wl.tau, init_level=wl.init_level, max_level=wl.max_level,
                        n_max=wl.n_max)


def synthetic_grid(N, levels, seed):
    """A larger refined grid from an analytic function (no PDE solves)."""
    rng = np.random.default_rng(seed)
    lvl, idx = O.sg_initial(N, 1)
    y = O.sg_points(lvl, idx)
    f = lambda Y: np.exp(-np.sum((Y - 0.3) ** 2, axis=1) * 3.0) + 0.1 * Y[:, 0]
    c = ouq.hierarchize(lvl, idx, f(y))
    first = 0
    for _ in range(levels):
        nl, ni = O.sg_refine(lvl, idx, first, c, 1e-3, 64)
        if not len(nl):
            break
        yn = O.sg_points(nl, ni)
        cn = f(yn) - O.sg_eval(lvl, idx, c, yn)
        first = len(lvl)
        lvl, idx, c = np.concatenate([lvl, nl]), np.concatenate([idx, ni]), np.concatenate([c, cn])
    # iteration-like surpluses: integers with structure
    cI = np.round(rng.standard_normal(len(lvl)) * 20.0)
    return lvl, idx, cI


def test_surrogate_and_grouping_bit_exact_on_the_oracle_run(h, small_run):
    r = small_run
    for (a, b), pred_o, perm_o in zip(r["levels"][1:], r["pred"][1:], r["perms"]["sur"][1:]):
        yq = O.sg_points(r["lvl"][a:b], r["idx"][a:b])
        pred = torch.empty(b - a, dtype=torch.float64, device="cuda")
        perm = torch.empty(b - a, dtype=torch.int32, device="cuda")
        n_ens = ens.ens_group(h, dev(r["lvl"][:a]), dev(r["idx"][:a]), dev(r["cI"][:a]), dev(yq), r["S"], pred,
                              perm)
        assert n_ens == -(-(b - a) // r["S"])
        assert np.array_equal(pred.cpu().numpy(), pred_o)
        assert np.array_equal(perm.cpu().numpy(), perm_o)
        # surpluses of the new points through the values form
        cI = torch.empty(b - a, dtype=torch.float64, device="cuda")
        ens.ens_sg_eval(h, dev(r["lvl"][:a]), dev(r["idx"][:a]), dev(r["cI"][:a]), dev(yq), cI,
                        values=dev(r["I"][a:b]))
        assert np.array_equal(cI.cpu().numpy(), r["cI"][a:b])


@pytest.mark.parametrize("N,levels,Mq", [(4, 4, 500), (2, 7, 2000), (6, 3, 4096), (8, 2, 333), (4, 4, 40000)])
def test_surrogate_bit_exact_on_larger_grids(h, N, levels, Mq):
    lvl, idx, cI = synthetic_grid(N, levels, seed=N)
    rng = np.random.default_rng(N + 1)
    yq = rng.uniform(-1, 1, (Mq, N))
    yq[: Mq // 4] = np.round(yq[: Mq // 4] * 64) / 64  # dyadic points hit basis kinks exactly
    want = O.sg_eval(lvl, idx, cI, yq)
    pred = torch.empty(Mq, dtype=torch.float64, device="cuda")
    perm = torch.empty(Mq, dtype=torch.int32, device="cuda")
    ens.ens_group(h, dev(lvl), dev(idx), dev(cI), dev(yq), 16, pred, perm)
    assert np.array_equal(pred.cpu().numpy(), want)
    assert np.array_equal(perm.cpu().numpy(), O.sort_perm(want) if Mq <= 16384 else np.argsort(want, kind="stable"))


@pytest.mark.parametrize("Mq", [1, 2, 3, 31, 1000, 4097, 16384, 16385, 50000, 300000])
def test_sort_chunk_matches_stable_sort(h, Mq):
    """One-block sort up to 16384 keys, device-wide beyond: both equal a stable
    ascending sort (the oracle's insertion sort; numpy's stable argsort for the
    sizes an insertion sort cannot reach)."""
    rng = np.random.default_rng(Mq)
    keys = rng.integers(0, 40, Mq).astype(np.float64)  # many ties
    keys[rng.random(Mq) < 0.1] = -0.0
    perm = torch.empty(Mq, dtype=torch.int32, device="cuda")
    n_ens = ens.ens_sort_chunk(h, dev(keys), 8, perm)
    assert n_ens == -(-Mq // 8)
    want = O.sort_perm(keys) if Mq <= 16384 else np.argsort(keys, kind="stable")
    assert np.array_equal(perm.cpu().numpy(), want)
    # NaN keys go last, in index order (the oracle's insertion sort has no rule for NaN)
    keys[rng.random(Mq) < 0.01] = np.nan
    ens.ens_sort_chunk(h, dev(keys), 8, perm)
    assert np.array_equal(perm.cpu().numpy(), np.argsort(keys, kind="stable"))


def test_sort_puts_nan_last_and_rejects_oversize(h):
    keys = np.array([3.0, np.nan, 1.0, np.inf, -np.inf, np.nan, 1.0])
    perm = torch.empty(7, dtype=torch.int32, device="cuda")
    ens.ens_sort_chunk(h, dev(keys), 2, perm)
    assert perm.cpu().numpy().tolist() == [4, 2, 6, 0, 3, 1, 5]
    # more than 2^26 keys is refused before any buffer is touched
    import ctypes

    n_ens = ctypes.c_int()
    kd = dev(keys)
    rc = ens.load().ens_sort_chunk(h.ptr, (1 << 26) + 1, kd.data_ptr(), 2, perm.data_ptr(), ctypes.byref(n_ens),
                                   None)
    assert rc == ens.EINVAL


def test_qoi_matches_definition(h):
    rng = np.random.default_rng(3)
    E, J, S = 3, 1000, 8
    x = rng.standard_normal((E, J, S))
    w = rng.random(J)
    out = torch.empty(E * S, dtype=torch.float64, device="cuda")
    ens.ens_qoi(h, J, S, E, dev(x.ravel()), out)
    np.testing.assert_allclose(out.cpu().numpy(), (x**2).sum(axis=1).ravel(), rtol=1e-13)
    ens.ens_qoi(h, J, S, E, dev(x.ravel()), out, w=dev(w))
    np.testing.assert_allclose(out.cpu().numpy(), np.einsum("j,ejs->es", w, x).ravel(), rtol=1e-12)


def test_adaptive_loop_matches_oracle(h, small_run):
    """The whole flowchart loop on the GPU path: same grid, iteration counts
    within one, G within 1e-10, and R of each level from the run's groups."""
    wl = inputs.WORKLOADS["fd5_32_adaptive"]
    ad = uq.Adaptive(h, wl)
    run = ad.run("sur")
    r = small_run
    assert np.array_equal(run["lvl"], r["lvl"]) and np.array_equal(run["idx"], r["idx"])
    assert run["levels"] == r["levels"]
    assert np.max(np.abs(run["I"] - r["I"])) <= 1
    np.testing.assert_allclose(run["G"], r["G"], rtol=1e-10)
    grouping_on_oracle_counts(h, r)
    if np.array_equal(run["I"], r["I"]):
        for p, po in zip(run["perms"][1:], r["perms"]["sur"][1:]):
            assert np.array_equal(p, po)
    R = uq.ratios(run)
    Ro = ouq.ratios(r)
    if np.array_equal(run["I"], r["I"]):
        np.testing.assert_allclose(R["run"][0], Ro["sur"][0], rtol=1e-12)
    for lev, (a, b) in enumerate(run["levels"]):
        assert R["run"][0][lev] >= 1.0


@pytest.mark.parametrize("kind,n,N,aniso", [("fd5", 32, 2, 3.0), ("q1", 64, 4, 4.0), ("fd7", 12, 6, 2.0),
                                            ("fd5", 40, 8, 3.0)])
def test_param_indicator_matches_oracle(h, kind, n, N, aniso):
    from gpu_util import OKIND

    M = 37
    xi = inputs.draws(M, N, seed=70 + n)
    xi[:8] = np.round(xi[:8] * 4) / 4  # dyadic points, as on a sparse grid: many equal indicators
    H = torch.empty(M, dtype=torch.float64, device="cuda")
    ens.ens_param_indicator(h, ens.problem(kind, n, N, aniso), dev(xi), H)
    Hg = H.cpu().numpy()
    Ho = np.array([O.param_indicator(OKIND[kind], n, N, aniso, xi[m]) for m in range(M)])
    np.testing.assert_allclose(Hg, Ho, rtol=1e-12)
    perm = torch.empty(M, dtype=torch.int32, device="cuda")
    ens.ens_sort_chunk(h, H, 8, perm)
    # a stable ascending sort of the GPU keys (Python's sort is stable)
    assert perm.cpu().numpy().tolist() == sorted(range(M), key=lambda i: Hg[i])


def test_parameter_grouping_in_the_loop(h):
    """The loop with "par" grouping visits the same grid (grouping never
    changes the grid) and its R is at least the iteration-sorted R on full
    levels."""
    wl = inputs.WORKLOADS["fd5_32_adaptive"]
    ad = uq.Adaptive(h, wl)
    sur = ad.run("sur")
    par = ad.run("par")
    assert np.array_equal(sur["lvl"], par["lvl"]) and np.array_equal(sur["I"], par["I"])
    R = uq.ratios(par)
    for lev, (a, b) in enumerate(par["levels"]):
        if (b - a) % wl.S == 0:
            assert R["its"][0][lev] <= R["run"][0][lev] + 1e-12


@pytest.mark.parametrize("grouping", ["sur", "rand"])
def test_checkpoint_resume_equals_uninterrupted(h, tmp_path, grouping):
    """A run stopped after one refined level, written to disk, read back and
    resumed ends bit for bit where the uninterrupted run ends (the random
    grouping also carries its seed over)."""
    wl = inputs.WORKLOADS["fd5_32_adaptive"]
    ad = uq.Adaptive(h, wl)
    full = ad.run(grouping, seed=3)
    part = ad.run(grouping, seed=3, stop_after=1)
    assert full["done"] and not part["done"] and len(part["levels"]) == 2 < len(full["levels"])
    path = str(tmp_path / "run.npz")
    uq.save_run(part, path)
    rest = ad.run(grouping, resume=uq.load_run(path))
    assert rest["done"] and rest["levels"] == full["levels"]
    for k in ("lvl", "idx", "y", "G", "I", "cG", "cI"):
        assert np.array_equal(rest[k], full[k]), k
    for a, b in zip(rest["perms"], full["perms"]):
        assert np.array_equal(a, b)
    with pytest.raises(ValueError):
        ad.run("nat" if grouping != "nat" else "sur", resume=uq.load_run(path))


def test_empty_inputs_are_no_ops(h):
    """Empty inputs at every step of the path: no points to group or sort, no
    ensembles to solve, no samples to stream -- each returns without work."""
    from paper_1705_02003_gb300 import batching
    from paper_1705_02003_gb300.solver import EnsembleSolver

    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    perm = torch.empty(0, dtype=torch.int32, device="cuda")
    assert ens.ens_sort_chunk(h, empty, 8, perm) == 0
    lvl, idx = ens.ens_sg_initial(2, 1)
    cI = torch.zeros(len(lvl), dtype=torch.float64, device="cuda")
    assert ens.ens_group(h, dev(lvl), dev(idx), cI, torch.empty(0, 2, dtype=torch.float64, device="cuda"), 8,
                         empty, perm) == 0
    prob = ens.problem("fd5", 8, 2, 3.0)
    sol = EnsembleSolver(h, prob, 8, 8, 1e-8, 100)
    it, st, rr, q = sol.solve(torch.empty(0, 2, dtype=torch.float64, device="cuda"))
    assert it.numel() == st.numel() == rr.numel() == q.numel() == 0
    J, nnz = sol.J, sol.nnz
    ens.ens_pcg_solve(h, J, nnz, 8, 0, sol.rowptr, sol.colidx, sol.vals[:0], sol.dinv[:0], sol.b[:0], sol.x[:0],
                      None, 1e-8, 100, sol.iters[:0], sol.relres[:0], sol.status[:0], sol.work)
    out = batching.solve_stream(h, prob, torch.empty(0, 2, dtype=torch.float64, device="cuda"), 8, 1, 1e-8, 100)
    assert out["iters"].numel() == 0


def test_levels_larger_than_the_solver_are_solved_in_whole_ensembles(h):
    """A solver that holds one ensemble at a time runs every level in calls of
    whole ensembles; the loop's results equal the one-call run bit for bit."""
    from paper_1705_02003_gb300.solver import EnsembleSolver

    wl = inputs.WORKLOADS["fd5_32_adaptive"]
    full = uq.Adaptive(h, wl).run("sur")
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    small = uq.Adaptive(h, wl, solver=EnsembleSolver(h, prob, wl.S, wl.S, wl.rtol, wl.maxit))
    part = small.run("sur")
    assert max(b - a for a, b in full["levels"]) > wl.S  # some level really needed several calls
    assert len(small.solve_sets) > len(full["levels"])
    for k in ("lvl", "idx", "G", "I", "cG", "cI"):
        assert np.array_equal(part[k], full[k]), k
    for a, b in zip(part["perms"], full["perms"]):
        assert np.array_equal(a, b)
