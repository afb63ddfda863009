"""GPU parity of the multigrid preconditioner and MG-PCG (csrc/mg.cu) against
the oracle (oracle/mg.c): the hierarchy's Galerkin operators and Gershgorin
bounds bit for bit, one V-cycle (FP64 and float), the solve on the oracle's
matrices (FP64 and mixed precision) and at the full 32^3-cell size, status
codes, lane independence, and the adaptive loop of Section 3.1 run with the
multigrid solver."""
import dataclasses
import os

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import OKIND, Case, elem_err, grouping_on_oracle_counts
from oracle import uq as ouq
from paper_1705_02003_gb300 import ens, inputs, uq

pytestmark = pytest.mark.gpu
KINDS = ["q1_3d_kl", "q1_3d_disc"]


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


def draws(M, seed):
    """Uniform draws plus the points on Test 2's jumps and the mean."""
    xi = inputs.draws(M, 4, seed=seed)
    xi[0] = [0.25, 0.25, 0.25, 0.0]   # r = sqrt(3)/4
    xi[1] = [0.5, -0.5, 0.0, 0.5]     # r = sqrt(3)/2
    xi[2] = [0.0, 0.0, 0.0, 0.0]
    return xi


def oracle_system(c, kind):
    """The oracle's assembled values and loads of every lane, and the same
    uploaded in the ensemble layout."""
    rp, ci = O.pattern(OKIND[kind], c.n)
    V, B = [], []
    for L in range(c.E * c.S):
        v, b = O.assemble(OKIND[kind], c.n, 4, 0.0, c.xi_h[L], rp, ci)
        V.append(v)
        B.append(b)
    return rp, ci, V, B, c.upload_lanes(V, c.nnz), c.upload_lanes(B, c.J)


@pytest.mark.parametrize("kind", KINDS)
def test_hierarchy_matches_oracle_bit_for_bit(h, kind):
    n, S, M = 15, 8, 11
    c = Case(h, kind, n, 4, 0.0, S, draws(M, 11))
    rp, ci, V, _, vals, _ = oracle_system(c, kind)
    work = c.mg_work()
    ens.ens_mg_setup(h, c.prob, S, c.E, c.rowptr, c.colidx, vals, work)
    ns = O.mg_levels(n)
    for level, nl in enumerate(ns):
        _, nnz_l = O.problem_size(OKIND[kind], nl)
        lm = torch.empty(c.E * S, dtype=torch.float64, device="cuda")
        vo = torch.empty(c.E * nnz_l * S, dtype=torch.float64, device="cuda") if level else None
        ens.ens_mg_level(h, c.prob, S, c.E, level, vo, lm, work)
        torch.cuda.synchronize()
        lm = lm.cpu().numpy()
        vg = vo.view(c.E, nnz_l, S).permute(0, 2, 1).reshape(c.E * S, nnz_l).cpu().numpy() if level else None
        for L in range(M):
            vc, lmax = O.mg_coarse(n, rp, ci, V[L], level)
            assert lm[L] == lmax, (level, L)
            if level:
                np.testing.assert_array_equal(vg[L], vc)


@pytest.mark.parametrize("kind", KINDS)
def test_vcycle_matches_oracle(h, kind):
    """One V-cycle on the same hierarchy: fused multiply-adds against separate
    roundings through the smoothers and the coarsest solve (~1e-14 measured
    scale; bar 1e-11 of the result's largest entry, element by element)."""
    n, S, M = 15, 8, 11
    c = Case(h, kind, n, 4, 0.0, S, draws(M, 12))
    rp, ci, V, _, vals, _ = oracle_system(c, kind)
    rng = np.random.default_rng(5)
    R = rng.standard_normal((c.E * S, c.J))
    r = c.upload_lanes(R, c.J)
    z = torch.empty_like(r)
    work = c.mg_work()
    ens.ens_mg_setup(h, c.prob, S, c.E, c.rowptr, c.colidx, vals, work)
    ens.ens_mg_apply(h, c.prob, S, c.E, c.rowptr, c.colidx, vals, r, z, work)
    torch.cuda.synchronize()
    Z = c.lane_vec(z)
    for L in range(M):
        zo = O.mg_apply(n, rp, ci, V[L], R[L])
        assert elem_err(Z[L], zo) <= 1e-11, L


@pytest.mark.parametrize("kind", KINDS)
def test_float_vcycle_matches_oracle(h, kind):
    """The mixed-precision V-cycle (float copy of the hierarchy, float
    arithmetic): against the oracle's float V-cycle and its FP64 one, 1e-5 of
    the result's largest entry, element by element (float rounding ~2e-7 on
    each side; fused multiply-adds and the coarsest inverse against separate
    roundings and triangular solves)."""
    n, S, M = 15, 8, 11
    c = Case(h, kind, n, 4, 0.0, S, draws(M, 16))
    rp, ci, V, _, vals, _ = oracle_system(c, kind)
    rng = np.random.default_rng(6)
    R = rng.standard_normal((c.E * S, c.J))
    r = c.upload_lanes(R, c.J)
    z = torch.empty_like(r)
    work = c.mg_work(mixed=True)
    ens.ens_mg_setup(h, c.prob, S, c.E, c.rowptr, c.colidx, vals, work, mixed=True)
    ens.ens_mg_apply(h, c.prob, S, c.E, c.rowptr, c.colidx, vals, r, z, work, mixed=True)
    torch.cuda.synchronize()
    Z = c.lane_vec(z)
    for L in range(M):
        z32 = O.mg_apply32(n, rp, ci, V[L], R[L])
        z64 = O.mg_apply(n, rp, ci, V[L], R[L])
        assert elem_err(Z[L], z32) <= 1e-5, L
        assert elem_err(Z[L], z64) <= 1e-5, L
        assert not np.array_equal(Z[L], z64)  # the float path really ran


def _check(got, ref, lanes, bar):
    for j, L in enumerate(lanes):
        assert got["status"][L] == ref[j][2] == O.CONVERGED, L
        di = int(got["iters"][L]) - int(ref[j][1])
        assert abs(di) <= 1, (L, di)
        err = elem_err(got["x"][L], ref[j][0])
        assert err <= (bar if di == 0 else 1e-5), (L, err)


@pytest.mark.parametrize("S", [16, 1])
@pytest.mark.parametrize("kind", KINDS)
def test_mgpcg_matches_oracle_on_the_oracles_matrices(h, kind, S):
    """The solver alone (both sides from the oracle's matrices and loads):
    iterations within 1, x within 1e-9 when the counts agree.  The
    preconditioned operator is well conditioned, so rounding moves the iterate
    far less than in the Jacobi solve.  S = 1: 21 one-lane ensembles."""
    n, M = 15, 21
    c = Case(h, kind, n, 4, 0.0, S, draws(M, 13))
    rp, ci, V, B, vals, b = oracle_system(c, kind)
    got = c.solve_mg(1e-7, 500, vals=vals, b=b)
    ref = [O.mgpcg(n, rp, ci, V[L], B[L], 1e-7, 500) for L in range(M)]
    _check(got, ref, range(M), 1e-9)
    assert all(got["status"][M:] == ens.LANE_INACTIVE)


@pytest.mark.parametrize("S", [16, 1])
@pytest.mark.parametrize("kind", KINDS)
def test_mixed_mgpcg_matches_oracle_on_the_oracles_matrices(h, kind, S):
    """CG in FP64 with the float V-cycle, on the oracle's matrices and loads:
    iterations within 1 of the oracle's CG with its float V-cycle, x within 1e-6
    when the counts agree (the two float preconditioners differ at ~1e-7)."""
    n, M = 15, 21
    c = Case(h, kind, n, 4, 0.0, S, draws(M, 17))
    rp, ci, V, B, vals, b = oracle_system(c, kind)
    got = c.solve_mg(1e-7, 500, vals=vals, b=b, mixed=True)
    ref = [O.mgpcg32(n, rp, ci, V[L], B[L], 1e-7, 500) for L in range(M)]
    _check(got, ref, range(M), 1e-6)
    assert all(got["status"][M:] == ens.LANE_INACTIVE)


@pytest.mark.parametrize("shift", [-300, -140, 140, 300])
def test_mixed_mgpcg_is_homogeneous_in_the_load(h, shift):
    """Scaling the load by 2^shift scales every FP64 CG step and (through the
    per-lane power-of-two scaling before the rounding to float) every float
    V-cycle step exactly, so the mixed solve of b 2^shift returns the same
    iterations and x 2^shift bit for bit -- also where b 2^shift lies far
    outside float's range (2^-140 and 2^140 are about 1e-42 and 1e42)."""
    n, S, M = 7, 8, 12
    c = Case(h, "q1_3d_disc", n, 4, 0.0, S, draws(M, 18))
    ref = c.solve_mg(1e-8, 200, mixed=True)
    got = c.solve_mg(1e-8, 200, b=c.b * 2.0 ** shift, mixed=True)
    assert np.all(ref["status"][:M] == ens.LANE_CONVERGED)
    assert np.array_equal(got["status"], ref["status"]) and np.array_equal(got["iters"], ref["iters"])
    assert np.array_equal(got["x"], np.ldexp(ref["x"], shift))


def test_workspace_set_up_for_other_sizes_is_refused(h):
    """A workspace set up with one S, E or precision and then used with another
    is refused (its layout depends on them) instead of being read wrongly."""
    c = Case(h, "q1_3d_kl", 7, 4, 0.0, 8, draws(16, 19))
    work = c.mg_work(mixed=True)
    ens.ens_mg_setup(h, c.prob, 8, c.E, c.rowptr, c.colidx, c.vals, work, mixed=False)
    z = torch.empty_like(c.b)
    with pytest.raises(ens.EnsError, match="set up"):
        ens.ens_mg_apply(h, c.prob, 8, c.E, c.rowptr, c.colidx, c.vals, c.b, z, work, mixed=True)
    J, nnz = c.J, c.nnz
    with pytest.raises(ens.EnsError, match="set up"):
        ens.ens_mg_apply(h, c.prob, 8, 1, c.rowptr, c.colidx, c.vals[: nnz * 8], c.b[: J * 8], z[: J * 8], work,
                         mixed=False)
    ens.ens_mg_apply(h, c.prob, 8, c.E, c.rowptr, c.colidx, c.vals, c.b, z, work, mixed=False)  # as set up
    ens.ens_mg_setup(h, c.prob, 8, c.E, c.rowptr, c.colidx, c.vals, work, mixed=True)
    ens.ens_mg_apply(h, c.prob, 8, c.E, c.rowptr, c.colidx, c.vals, c.b, z, work, mixed=True)
    torch.cuda.synchronize()


@pytest.mark.parametrize("name,lanes", [("q1_32c_test1", [0, 19]), ("q1_32c_test2", [1, 30])])
def test_full_size_sampled_lanes(h, name, lanes):
    """32^3 cells, two ensembles of 16, GPU assembly: sampled lanes against the
    oracle's assembly and MG-PCG (the 1e-13 matrix differences times the
    operator's condition number bound x at 1e-7)."""
    wl = inputs.WORKLOADS[name]
    c = Case(h, wl.kind, wl.n, 4, 0.0, wl.S, draws(2 * wl.S, 14))
    got = c.solve_mg(wl.rtol, 500)
    rp, ci = O.pattern(OKIND[wl.kind], wl.n)
    ref = []
    for L in lanes:
        v, b = O.assemble(OKIND[wl.kind], wl.n, 4, 0.0, c.xi_h[L], rp, ci)
        ref.append(O.mgpcg(wl.n, rp, ci, v, b, wl.rtol, 500))
    _check(got, ref, lanes, 1e-7)


def test_status_codes_and_lane_independence(h):
    """A NaN parameter makes its lane BADINPUT (setup marks it), a zero load
    converges in 0 iterations, padding lanes are INACTIVE, maxit 0 stops every
    lane at once; and a sample's result is the same bit for bit wherever it
    sits (other lanes, other ensembles, another E, the same S)."""
    n, S = 7, 8
    xi = draws(12, 15)
    xi[3] = np.nan
    c = Case(h, "q1_3d_kl", n, 4, 0.0, S, xi)
    b = c.b.clone().view(c.E, c.J, S)
    b[0, :, 5] = 0.0
    got = c.solve_mg(1e-8, 200, b=b.reshape(-1))
    st = got["status"]
    assert st[3] == ens.LANE_BADINPUT and got["iters"][3] == 0
    assert st[5] == ens.LANE_CONVERGED and got["iters"][5] == 0 and got["relres"][5] == 0.0
    assert not got["x"][5].any()
    assert all(st[12:] == ens.LANE_INACTIVE)
    ok = [L for L in range(12) if L not in (3, 5)]
    assert all(st[ok] == ens.LANE_CONVERGED)
    # the same valid samples, reversed, at other lanes of other ensembles (same S:
    # the reduction order depends on J and S only)
    xi2 = xi[ok][::-1]
    c2 = Case(h, "q1_3d_kl", n, 4, 0.0, S, xi2)
    assert c2.E == 2
    got2 = c2.solve_mg(1e-8, 200)
    for j, L in enumerate(ok[::-1]):
        assert got2["iters"][j] == got["iters"][L] and np.array_equal(got2["x"][j], got["x"][L])
    z = c.solve_mg(1e-8, 0, b=b.reshape(-1))
    assert all(z["status"][ok] == ens.LANE_MAXIT) and all(z["iters"][ok] == 0) and all(z["relres"][ok] == 1.0)


@pytest.mark.parametrize("name", ["q1_32c_test1", "q1_32c_test2"])
def test_adaptive_loop_with_multigrid_matches_oracle(h, name):
    """The flowchart loop with the multigrid solver on a 16^3-cell version,
    capped at 200 points: the same grid and levels, G within 1e-7, iteration
    counts within one, surrogate groupings equal where the counts agree."""
    wl = dataclasses.replace(inputs.WORKLOADS[name], n=15, n_max=200, maxit=500)
    run = uq.Adaptive(h, wl, precond="mg").run("sur")

    def solve(y):
        o = O.solve_batch_mg(OKIND[wl.kind], wl.n, 4, 0.0, y, wl.rtol, wl.maxit, nthreads=os.cpu_count() or 4)
        return o["G"], o["iters"]

    ref = ouq.adaptive(solve, N=4, S=wl.S, tau=wl.tau, init_level=wl.init_level, max_level=wl.max_level,
                       n_max=wl.n_max)
    assert np.array_equal(run["lvl"], ref["lvl"]) and np.array_equal(run["idx"], ref["idx"])
    assert run["levels"] == ref["levels"] and len(run["levels"]) >= 2
    assert np.max(np.abs(run["I"] - ref["I"])) <= 1
    np.testing.assert_allclose(run["G"], ref["G"], rtol=1e-7)
    grouping_on_oracle_counts(h, ref)
    if np.array_equal(run["I"], ref["I"]):
        for p, po in zip(run["perms"][1:], ref["perms"]["sur"][1:]):
            assert np.array_equal(p, po)
