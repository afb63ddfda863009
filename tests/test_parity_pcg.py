"""GPU parity of the graph, the ensemble assembly (K1) and the ensemble
Jacobi-PCG (K2-K4) against the CPU oracle, through the C ABI.

Bars (FP64): matrix values within 1e-13 relative (the two sides differ only in
the last bits of exp/sin/pow); iteration counts within +-1; solutions within
1e-10 relative wherever the counts agree, and both within the tolerance where
they differ by one; padding, masking, lane order and batch size change nothing,
bit for bit.
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import OKIND, Case, elem_err, grouping_on_oracle_counts
from paper_1705_02003_gb300 import ens, inputs

pytestmark = pytest.mark.gpu

NTH = os.cpu_count() or 4


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


def oracle_solve(case, rtol, maxit, rows=None):
    xi = case.xi_h[: case.M] if rows is None else case.xi_h[rows]
    return O.solve_batch(OKIND[case.kind], case.n, case.N, case.aniso, xi, rtol, maxit, nthreads=NTH,
                         want_x=True)


def check_against_oracle(case, got, ref, rtol, lanes):
    for j, L in enumerate(lanes):
        assert got["status"][L] == ref["status"][j] == O.CONVERGED, (L, got["status"][L], ref["status"][j])
        di = int(got["iters"][L]) - int(ref["iters"][j])
        assert abs(di) <= 1, (L, got["iters"][L], ref["iters"][j])
        xo = ref["x"][j]
        err = elem_err(got["x"][L], xo)
        if di == 0:
            assert err <= 1e-10, (L, err)
        else:
            assert got["relres"][L] <= rtol and ref["relres"][j] <= rtol
            assert err <= 1e-6, (L, err)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("wl", list(inputs.WORKLOADS.values()), ids=lambda w: w.name)
def test_pattern_bit_exact(h, wl):
    p = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    J, nnz = ens.ens_problem_size(p)
    rp = torch.empty(J + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(nnz, dtype=torch.int32, device="cuda")
    ens.ens_pattern(h, p, rp, ci)
    orp, oci = O.pattern(OKIND[wl.kind], wl.n)
    assert np.array_equal(rp.cpu().numpy().astype(np.int64), orp)
    assert np.array_equal(ci.cpu().numpy(), oci)


ASM_CASES = [
    ("fd5", 32, 2, 3.0, 8, 19),
    ("fd5", 20, 8, 3.0, 32, 40),
    ("q1", 24, 4, 4.0, 16, 21),
    ("fd7", 10, 6, 3.0, 32, 33),
    ("fd7", 9, 6, 2.0, 4, 7),
]


@pytest.mark.parametrize("kind,n,N,aniso,S,M", ASM_CASES)
def test_assembly_matches_oracle(h, kind, n, N, aniso, S, M):
    xi = inputs.draws(M, N, seed=n)
    c = Case(h, kind, n, N, aniso, S, xi)
    V = c.lane_vals()
    D = c.lane_vec(c.dinv)
    B = c.lane_vec(c.b)
    rp, ci = O.pattern(OKIND[kind], n)
    for s in range(M):
        vals, b = O.assemble(OKIND[kind], n, N, aniso, xi[s], rp, ci)
        np.testing.assert_allclose(V[s], vals, rtol=1e-13, atol=0)
        np.testing.assert_array_equal(B[s], b)
        np.testing.assert_allclose(D[s], O.jacobi(rp, ci, vals), rtol=1e-13, atol=0)


def test_assembly_f32_is_rounded_f64(h):
    xi = inputs.draws(8, 6, seed=3)
    c = Case(h, "fd7", 8, 6, 2.0, 8, xi)
    v32 = torch.empty(c.E * c.nnz * c.S, dtype=torch.float32, device="cuda")
    ens.ens_assemble(h, c.prob, c.S, c.E, c.xi, c.rowptr, c.colidx, v32)
    assert torch.equal(v32, c.vals.to(torch.float32))


SOLVE_CASES = [
    # kind, n, N, aniso, S, M  (M not a multiple of S: a padded last ensemble)
    ("fd5", 32, 2, 3.0, 8, 37),     # the 32 x 32 adaptive workload's problem
    ("q1", 40, 4, 4.0, 16, 21),
    ("fd7", 12, 6, 3.0, 32, 40),
    ("fd5", 24, 8, 3.0, 4, 11),
    ("fd5", 16, 2, 3.0, 1, 5),
    ("fd5", 16, 2, 3.0, 2, 5),
    ("fd5", 16, 3, 3.0, 64, 70),
    ("fd5", 40, 8, 3.0, 32, 45),    # 5-point rows at S = 16, 32: the two-lane SpMV variant
    ("fd5", 50, 4, 3.0, 16, 20),    # (J = 1600, 2500: ragged last tile)
    ("fd5", 2, 2, 3.0, 8, 5),       # the smallest grids (n = 2): 4 and 8 unknowns, one row tile
    ("q1", 2, 4, 4.0, 16, 3),
    ("fd7", 2, 6, 3.0, 32, 33),
]


@pytest.mark.parametrize("kind,n,N,aniso,S,M", SOLVE_CASES)
def test_pcg_matches_oracle(h, kind, n, N, aniso, S, M):
    rtol, maxit = 1e-8, 20000
    xi = inputs.draws(M, N, seed=100 + n)
    c = Case(h, kind, n, N, aniso, S, xi)
    got = c.solve(rtol, maxit)
    ref = oracle_solve(c, rtol, maxit)
    check_against_oracle(c, got, ref, rtol, range(M))
    # padded lanes are inactive, zero and cost nothing
    for L in range(M, c.E * S):
        assert got["status"][L] == ens.LANE_INACTIVE and got["iters"][L] == 0
        assert np.all(got["x"][L] == 0)


@pytest.mark.parametrize("name,lanes", [("q1_256_adaptive", [0, 17, 31]), ("fd7_64_batch", [5, 30]),
                                        ("fd5_512_adjoint", [3])])
def test_pcg_full_size_sampled_lanes(h, name, lanes):
    """The full-size problems in the launch shape the bench uses (S lanes, E
    ensembles in one call); a few sampled lanes against the oracle."""
    wl = inputs.WORKLOADS[name]
    E = 2 if wl.S <= 16 else 1
    xi = inputs.draws(E * wl.S, wl.nparam, seed=wl.seed)
    c = Case(h, wl.kind, wl.n, wl.nparam, wl.aniso, wl.S, xi)
    got = c.solve(1e-8, wl.maxit)
    assert np.all(got["status"] == ens.LANE_CONVERGED)
    ref = oracle_solve(c, 1e-8, wl.maxit, rows=lanes)
    check_against_oracle(c, got, ref, 1e-8, lanes)


@pytest.mark.parametrize("name,M", [("q1_256_adaptive", 3), ("q1_256_adaptive", 32), ("fd7_64_batch", 3),
                                    ("fd7_64_batch", 8)])
def test_one_lane_ensembles_full_size(h, name, M):
    """S = 1 on the full-size problems, M one-lane ensembles in one call: a few
    (256-row tiles; 512 on 64^3) and a batch that fills the GPU (4096-row tiles;
    on the 7-point 64^3 rows in dealt 256-row chunks).  Sampled lanes against
    the oracle."""
    wl = inputs.WORKLOADS[name]
    xi = inputs.draws(M, wl.nparam, seed=wl.seed + 1)
    c = Case(h, wl.kind, wl.n, wl.nparam, wl.aniso, 1, xi)
    got = c.solve(1e-8, wl.maxit)
    assert np.all(got["status"] == ens.LANE_CONVERGED)
    lanes = [0, M - 1]
    ref = oracle_solve(c, 1e-8, wl.maxit, rows=lanes)
    check_against_oracle(c, got, ref, 1e-8, lanes)


@pytest.mark.parametrize("S", [2, 4, 8])
def test_small_ensembles_full_size(h, S):
    """S = 2, 4, 8 on Q1 256^2 (tiles of 4096 / S rows, whatever E): a sample
    gives the same bits alone and in a batch of three ensembles, and sampled
    lanes agree with the oracle."""
    wl = inputs.WORKLOADS["q1_256_adaptive"]
    xi = inputs.draws(3 * S, wl.nparam, seed=wl.seed + 2)
    c = Case(h, wl.kind, wl.n, wl.nparam, wl.aniso, S, xi)
    batch = c.solve(1e-8, wl.maxit)
    alone = Case(h, wl.kind, wl.n, wl.nparam, wl.aniso, S, xi[S:2 * S]).solve(1e-8, wl.maxit)
    assert np.array_equal(batch["x"][S:2 * S], alone["x"])
    assert np.array_equal(batch["iters"][S:2 * S], alone["iters"])
    assert np.all(batch["status"] == ens.LANE_CONVERGED)
    lanes = [0, 2 * S - 1]
    check_against_oracle(c, batch, oracle_solve(c, 1e-8, wl.maxit, rows=lanes), 1e-8, lanes)


# ---------------------------------------------------------------------------
# invariants (bit-exact on the GPU)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n", [("q1", 24), ("fd5", 40)])  # one and two lanes per SpMV thread
def test_masked_lane_equals_full_ensemble_and_order_free(h, kind, n):
    xi = inputs.draws(16, 4, seed=5)
    c = Case(h, kind, n, 4, 4.0 if kind == "q1" else 3.0, 16, xi)
    full = c.solve(1e-8, 5000)
    again = c.solve(1e-8, 5000)
    for k in ("x", "iters", "status", "relres"):
        assert np.array_equal(full[k], again[k])  # deterministic
    for s in (0, 7, 15):
        act = torch.zeros(16, dtype=torch.uint8, device="cuda")
        act[s] = 1
        one = c.solve(1e-8, 5000, active=act)
        assert np.array_equal(one["x"][s], full["x"][s])
        assert one["iters"][s] == full["iters"][s]
        others = [L for L in range(16) if L != s]
        assert np.all(one["status"][others] == ens.LANE_INACTIVE)
    perm = np.random.default_rng(1).permutation(16)
    cp = Case(h, kind, n, 4, 4.0 if kind == "q1" else 3.0, 16, xi[perm])
    pp = cp.solve(1e-8, 5000)
    assert np.array_equal(pp["x"], full["x"][perm])
    assert np.array_equal(pp["iters"], full["iters"][perm])


def test_batch_size_does_not_change_results(h):
    xi = inputs.draws(24, 2, seed=6)
    alone = Case(h, "fd5", 32, 2, 3.0, 8, xi[8:16]).solve(1e-8, 5000)
    batch = Case(h, "fd5", 32, 2, 3.0, 8, xi).solve(1e-8, 5000)
    assert np.array_equal(batch["x"][8:16], alone["x"])
    assert np.array_equal(batch["iters"][8:16], alone["iters"])


def test_dealt_row_chunks_keep_results_independent_of_batch_and_lane(h):
    """7-point rows on 56^3 (J = 175,616: row tiles of 512 rows, so K2 deals its
    256-row chunks across the blocks): a sample gives the same bits alone, in a
    batch of three ensembles, at another lane, and with the loop launched from
    the host; and the solve agrees with the oracle."""
    n, N, aniso, S = 56, 6, 3.0, 8
    xi = inputs.draws(24, N, seed=9) * 0.7
    batch = Case(h, "fd7", n, N, aniso, S, xi).solve(1e-8, 5000)
    alone = Case(h, "fd7", n, N, aniso, S, xi[8:16]).solve(1e-8, 5000)
    assert np.array_equal(batch["x"][8:16], alone["x"]) and np.array_equal(batch["iters"][8:16], alone["iters"])
    rev = Case(h, "fd7", n, N, aniso, S, xi[8:16][::-1].copy()).solve(1e-8, 5000)
    assert np.array_equal(rev["x"][::-1], alone["x"]) and np.array_equal(rev["iters"][::-1], alone["iters"])
    hh = _handle_with({"ENS_PCG_HOST_LOOP": "1"})
    host = Case(hh, "fd7", n, N, aniso, S, xi[8:16]).solve(1e-8, 5000)
    assert np.array_equal(host["x"], alone["x"]) and np.array_equal(host["iters"], alone["iters"])
    hh.close()
    c = Case(h, "fd7", n, N, aniso, S, xi[8:10])
    ref = oracle_solve(c, 1e-8, 5000)
    check_against_oracle(c, c.solve(1e-8, 5000), ref, 1e-8, [0, 1])


def _handle_with(env: dict):
    """A handle created while the environment holds `env` (read at ens_create)."""
    import os

    saved = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return ens.Handle(0)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def test_loop_branches_do_not_change_results(h):
    """Five ensembles with different iteration counts: one graph branch per
    ensemble (the default), two branches, one branch and the host loop give
    the same solutions, counts and residuals bit for bit, and each branch
    stops on its own (the maxit cap still applies per lane)."""
    xi = inputs.draws(40, 4, seed=12)
    xi[:8, 0] = 0.95  # a strongly anisotropic ensemble: many more iterations
    ref = Case(h, "q1", 20, 4, 4.0, 8, xi).solve(1e-8, 5000)
    assert ens.ens_pcg_branches(h, 5) == 5 and ens.ens_pcg_branches(h, 40) == 16
    for env in ({"ENS_PCG_BRANCHES": "2"}, {"ENS_PCG_BRANCHES": "1"}, {"ENS_PCG_HOST_LOOP": "1"}):
        h2 = _handle_with(env)
        nb = ens.ens_pcg_branches(h2, 5)
        assert nb == (1 if "ENS_PCG_HOST_LOOP" in env else int(env["ENS_PCG_BRANCHES"]))
        got = Case(h2, "q1", 20, 4, 4.0, 8, xi).solve(1e-8, 5000)
        for k in ("x", "iters", "status", "relres"):
            assert np.array_equal(got[k], ref[k]), (env, k)
        capped = Case(h2, "q1", 20, 4, 4.0, 8, xi).solve(1e-8, 7)
        assert np.all(capped["iters"] == 7) and np.all(capped["status"] == ens.LANE_MAXIT)
        h2.close()
    it = ref["iters"].reshape(5, 8).max(axis=1)
    assert it.max() > it.min()  # the branches really ran different trip counts


# ---------------------------------------------------------------------------
# degenerate cases and status codes
# ---------------------------------------------------------------------------
def test_maxit_zero_and_one(h):
    xi = inputs.draws(8, 2, seed=7)
    c = Case(h, "fd5", 16, 2, 3.0, 8, xi)
    z = c.solve(1e-8, 0)
    assert np.all(z["status"] == ens.LANE_MAXIT) and np.all(z["iters"] == 0) and np.all(z["x"] == 0)
    one = c.solve(1e-8, 1)
    assert np.all(one["status"] == ens.LANE_MAXIT) and np.all(one["iters"] == 1)
    rp, ci = O.pattern(O.FD5_LOGKL, 16)
    for s in range(8):
        vals, b = O.assemble(O.FD5_LOGKL, 16, 2, 3.0, xi[s], rp, ci)
        x, it, st, _ = O.pcg(rp, ci, vals, b, 1e-8, 1)
        assert st == O.MAXIT and it == 1
        np.testing.assert_allclose(one["x"][s], x, rtol=1e-13, atol=0)


def test_nan_parameter_flags_only_its_lane(h):
    xi = inputs.draws(8, 2, seed=8)
    base = Case(h, "fd5", 16, 2, 3.0, 8, xi).solve(1e-8, 5000)
    bad = xi.copy()
    bad[3, 1] = np.nan
    got = Case(h, "fd5", 16, 2, 3.0, 8, bad).solve(1e-8, 5000)
    assert got["status"][3] == ens.LANE_BADINPUT and got["iters"][3] == 0
    keep = [L for L in range(8) if L != 3]
    assert np.array_equal(got["x"][keep], base["x"][keep])
    assert np.array_equal(got["iters"][keep], base["iters"][keep])


def test_breakdown_guard_freezes_one_lane(h):
    xi = inputs.draws(8, 2, seed=9)
    c = Case(h, "fd5", 16, 2, 3.0, 8, xi)
    base = c.solve(1e-8, 5000)
    v = c.vals.view(c.nnz, 8).clone()
    v[:, 5] = -v[:, 5]  # lane 5 now has p^T A p < 0
    got = c.solve(1e-8, 5000, vals=v.view(-1))
    assert got["status"][5] == ens.LANE_BREAKDOWN and got["iters"][5] == 0 and np.all(got["x"][5] == 0)
    keep = [L for L in range(8) if L != 5]
    assert np.array_equal(got["x"][keep], base["x"][keep])


def test_all_lanes_inactive(h):
    xi = inputs.draws(4, 2, seed=10)
    c = Case(h, "fd5", 16, 2, 3.0, 4, xi, active=np.zeros(4, np.uint8))
    got = c.solve(1e-8, 100)
    assert np.all(got["status"] == ens.LANE_INACTIVE) and np.all(got["x"] == 0)


def test_argument_errors(h):
    xi = inputs.draws(8, 2, seed=11)
    c = Case(h, "fd5", 16, 2, 3.0, 8, xi)
    J, nnz, E = c.J, c.nnz, c.E
    x = torch.empty(E * J * 8, dtype=torch.float64, device="cuda")
    it = torch.empty(8, dtype=torch.int32, device="cuda")
    st = torch.empty(8, dtype=torch.int32, device="cuda")
    rr = torch.empty(8, dtype=torch.float64, device="cuda")
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(ens.EnsError, match="workspace"):
        ens.ens_pcg_solve(h, J, nnz, 8, E, c.rowptr, c.colidx, c.vals, c.dinv, c.b, x, None, 1e-8, 10, it, rr, st,
                          small)
    with pytest.raises(ens.EnsError):
        ens.ens_pcg_solve(h, J, nnz, 8, E, c.rowptr, c.colidx, c.vals, c.dinv, c.b, x, None, -1.0, 10, it, rr,
                          st, small)
    with pytest.raises(ens.EnsError):
        ens.ens_assemble(h, ens.problem("fd5", 16, 2, 3.0), 3, 1, c.xi[:3], c.rowptr, c.colidx,
                         torch.empty(3 * nnz, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("kind,n,N,aniso,S,M", [("q1", 30, 4, 4.0, 16, 20), ("fd7", 9, 6, 3.0, 8, 9),
                                                ("fd5", 20, 8, 3.0, 1, 3), ("fd5", 12, 2, 3.0, 64, 64),
                                                ("fd5", 50, 4, 3.0, 16, 20), ("fd5", 40, 8, 3.0, 32, 33),
                                                ("q1", 30, 4, 4.0, 1, 3), ("fd7", 60, 6, 3.0, 1, 2)])
def test_spmv_matches_oracle_and_lane_dots(h, kind, n, N, aniso, S, M):
    """K2 alone: each row sum is taken in the oracle's column order, with one
    rounding per fused multiply-add instead of two, so every row agrees with
    the oracle within the summation bound 2 k eps sum_k |a_k p_k|.  Matrix
    values and p come from the oracle side and are uploaded."""
    xi = inputs.draws(M, N, seed=21)
    c = Case(h, kind, n, N, aniso, S, xi)
    rng = np.random.default_rng(22)
    rp, ci = O.pattern(OKIND[kind], n)
    V = np.stack([O.assemble(OKIND[kind], n, N, aniso, c.xi_h[L], rp, ci)[0] for L in range(c.E * S)])
    vals = torch.from_numpy(V.reshape(c.E, S, c.nnz).transpose(0, 2, 1).copy()).cuda().reshape(-1)
    P = rng.standard_normal((c.E * S, c.J))
    p = torch.from_numpy(P.reshape(c.E, S, c.J).transpose(0, 2, 1).copy()).cuda().reshape(-1)
    q = torch.empty_like(p)
    pq = torch.empty(c.E * S, dtype=torch.float64, device="cuda")
    work = torch.empty(ens.ens_pcg_workspace_size(c.J, c.nnz, S, c.E), dtype=torch.uint8, device="cuda")
    ens.ens_spmv(h, c.J, c.nnz, S, c.E, c.rowptr, c.colidx, vals, p, q, pq, work)
    Q = c.lane_vec(q)
    eps = np.finfo(np.float64).eps
    for L in range(c.E * S):
        ref = O.spmv(rp, ci, V[L], P[L])
        mag = O.spmv(rp, ci, np.abs(V[L]), np.abs(P[L]))
        assert np.all(np.abs(Q[L] - ref) <= 2 * 9 * eps * mag)
        assert pq[L].item() == pytest.approx(float(P[L] @ ref), rel=1e-12)
