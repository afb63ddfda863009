"""The one-launch cluster schedule of ens_pcg_solve (problems of at most 1024
unknowns) against the graph loop: the same outcome, bit for bit, for every
lane, including lanes that are padding, start converged, break down, carry a
NaN parameter or stop at maxit.  The two schedules perform the same operations
in the same order (Section 2.3's per-sample recurrences), so nothing may
differ.  The oracle parity of the solve at these sizes is covered by the other
tests, which run on the default handle and therefore on this schedule."""
import numpy as np
import pytest

from gpu_util import Case
from paper_1705_02003_gb300 import ens, inputs

pytestmark = pytest.mark.gpu


def handle_with(var, value):
    mp = pytest.MonkeyPatch()
    mp.setenv(var, value)
    try:
        return ens.Handle(0)
    finally:
        mp.undo()


@pytest.fixture(scope="module")
def handles(ens_lib):
    """The one-launch schedule wherever it fits (past the work bound too, so
    that every kernel variant runs), and the graph loop only."""
    return handle_with("ENS_PCG_FUSED", "2"), handle_with("ENS_PCG_FUSED", "0")


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint64 if a.dtype == np.float64 else np.uint32)


def same(got, ref):
    for k in ("x", "iters", "status", "relres"):
        assert np.array_equal(bits(got[k]), bits(ref[k])), k


def run_both(handles, kind, n, N, aniso, S, M, rtol, maxit, seed, perturb=None):
    hf, hl = handles
    xi = inputs.draws(M, N, seed=seed)
    out = []
    for h in (hf, hl):
        c = Case(h, kind, n, N, aniso, S, xi)
        if perturb:
            perturb(c)
        out.append(c.solve(rtol, maxit))
    assert ens.ens_pcg_cluster_size(hf, c.J, c.nnz, S, c.E) > 0, "the one-launch schedule did not run"
    assert ens.ens_pcg_cluster_size(hl, c.J, c.nnz, S, c.E) == 0
    return out[0], out[1], c


# (kind, n, N, aniso): 5-, 9-, 7- and 27-point rows; 1 to 16 row tiles of 64
# rows (4 and 25 unknowns: a cluster of one CTA), with ragged last tiles (961
# unknowns: a last tile of one row).  On the
# 7-point 10^3 problem the +-100-row neighbours do not fit the 256-row windows,
# so p goes through global memory there.
PROBLEMS = [("fd5", 2, 2, 3.0), ("fd5", 5, 2, 3.0), ("fd5", 15, 2, 3.0), ("fd5", 32, 2, 3.0),
            ("q1", 16, 4, 4.0), ("q1", 31, 4, 4.0), ("fd7", 10, 6, 3.0), ("q1_3d_kl", 7, 4, 0.0)]


@pytest.mark.parametrize("prob", PROBLEMS, ids=lambda p: f"{p[0]}_{p[1]}")
@pytest.mark.parametrize("S", [1, 8, 16, 32])
def test_cluster_schedule_equals_graph_loop(handles, prob, S):
    kind, n, N, aniso = prob
    got, ref, c = run_both(handles, kind, n, N, aniso, S, 3 * S - (1 if S > 1 else 0), 1e-8, 5000, seed=S)
    same(got, ref)
    assert np.all(got["status"][: c.M] == ens.LANE_CONVERGED)


@pytest.mark.parametrize("S", [1, 2, 4, 8, 16, 32])
def test_every_lane_count(handles, S):
    got, ref, _ = run_both(handles, "fd5", 32, 2, 3.0, S, 2 * S, 1e-8, 5000, seed=100 + S)
    same(got, ref)


def test_lane_outcomes(handles):
    """A zero load (converged at 0 trips), zero values (p^T A p = 0: breakdown
    in the first trip), a NaN parameter (bad input), padding lanes, and lanes
    stopped by maxit, side by side in one ensemble."""
    S = 16

    def perturb(c):
        b = c.b.view(c.E, c.J, S)
        b[0, :, 2] = 0.0
        v = c.vals.view(c.E, c.nnz, S)
        v[1, :, 5] = 0.0

    hf, hl = handles
    xi = inputs.draws(2 * S - 3, 2, seed=9)
    xi[S + 4, 0] = np.nan
    outs = []
    for h in (hf, hl):
        c = Case(h, "fd5", 32, 2, 3.0, S, xi)
        perturb(c)
        outs.append(c.solve(1e-8, 5000))
        outs.append(c.solve(1e-12, 40))  # most lanes stop at maxit
    assert ens.ens_pcg_cluster_size(hf, c.J, c.nnz, S, c.E) > 0
    for got, ref in ((outs[0], outs[2]), (outs[1], outs[3])):
        same(got, ref)
    st = outs[0]["status"]
    assert st[2] == ens.LANE_CONVERGED and outs[0]["iters"][2] == 0
    assert st[S + 5] == ens.LANE_BREAKDOWN
    assert st[S + 4] == ens.LANE_BADINPUT
    assert np.all(st[2 * S - 3:] == ens.LANE_INACTIVE)
    assert np.sum(outs[1]["status"] == ens.LANE_MAXIT) >= S


@pytest.mark.parametrize("maxit", [0, 1, 2])
def test_tiny_maxit(handles, maxit):
    got, ref, _ = run_both(handles, "q1", 16, 4, 4.0, 8, 13, 1e-8, maxit, seed=4)
    same(got, ref)
    assert np.all(got["iters"][:13] == maxit)


def test_many_ensembles(handles):
    """The largest ensemble count (of 2 to 64) whose clusters are all resident."""
    hf, _ = handles
    J, nnz = ens.ens_problem_size(ens.problem("fd5", 32, 2, 3.0))
    E = max(e for e in (2, 4, 8, 16, 32, 64) if ens.ens_pcg_cluster_size(hf, J, nnz, 8, e) > 0)
    got, ref, c = run_both(handles, "fd5", 32, 2, 3.0, 8, 8 * E, 1e-8, 5000, seed=21)
    assert c.E == E
    same(got, ref)


def test_where_the_graph_loop_runs(handles):
    """Past 16 tiles, at S = 64, or with more ensembles than resident clusters."""
    hf, _ = handles
    J, nnz = ens.ens_problem_size(ens.problem("fd5", 33, 2, 3.0))
    assert J > 1024 and ens.ens_pcg_cluster_size(hf, J, nnz, 16, 4) == 0
    J, nnz = ens.ens_problem_size(ens.problem("fd5", 32, 2, 3.0))
    assert ens.ens_pcg_cluster_size(hf, J, nnz, 16, 2) == 16
    assert ens.ens_pcg_cluster_size(hf, J, nnz, 64, 1) == 0
    assert ens.ens_pcg_cluster_size(hf, J, nnz, 16, 20000) == 0


def test_host_loop_handle_keeps_the_kernels(ens_lib):
    h = handle_with("ENS_PCG_HOST_LOOP", "1")
    J, nnz = ens.ens_problem_size(ens.problem("fd5", 32, 2, 3.0))
    assert ens.ens_pcg_cluster_size(h, J, nnz, 8, 3) == 0


def test_default_handle_applies_the_work_bound(ens_lib):
    """64 S (nnz/J + 7) <= 26000 multiply-adds per CTA and trip."""
    h = ens.Handle(0)
    J, nnz = ens.ens_problem_size(ens.problem("fd5", 32, 2, 3.0))
    assert ens.ens_pcg_cluster_size(h, J, nnz, 8, 3) == 16
    assert ens.ens_pcg_cluster_size(h, J, nnz, 32, 1) == 16
    J, nnz = ens.ens_problem_size(ens.problem("q1", 31, 4, 4.0))
    assert ens.ens_pcg_cluster_size(h, J, nnz, 16, 1) == 16
    assert ens.ens_pcg_cluster_size(h, J, nnz, 32, 1) == 0
    J, nnz = ens.ens_problem_size(ens.problem("q1_3d_kl", 7, 4, 0.0))
    assert ens.ens_pcg_cluster_size(h, J, nnz, 8, 1) == 6
    assert ens.ens_pcg_cluster_size(h, J, nnz, 16, 1) == 0


def test_null_active_mask(handles):
    """active = NULL (every lane active) on both schedules."""
    import torch

    S, E = 8, 2
    outs = []
    for h in handles:
        c = Case(h, "fd5", 32, 2, 3.0, S, inputs.draws(S * E, 2, seed=31))
        J, nnz = c.J, c.nnz
        x = torch.empty(E * J * S, dtype=torch.float64, device="cuda")
        it = torch.empty(E * S, dtype=torch.int32, device="cuda")
        st = torch.empty_like(it)
        rr = torch.empty(E * S, dtype=torch.float64, device="cuda")
        work = torch.empty(ens.ens_pcg_workspace_size(J, nnz, S, E), dtype=torch.uint8, device="cuda")
        ens.ens_pcg_solve(h, J, nnz, S, E, c.rowptr, c.colidx, c.vals, c.dinv, c.b, x, None, 1e-8, 5000, it, rr, st,
                          work)
        torch.cuda.synchronize()
        outs.append(dict(x=x.cpu().numpy(), iters=it.cpu().numpy(), status=st.cpu().numpy(),
                         relres=rr.cpu().numpy()))
    assert ens.ens_pcg_cluster_size(handles[0], J, nnz, S, E) > 0
    same(outs[0], outs[1])
    assert np.all(outs[0]["status"] == ens.LANE_CONVERGED)
