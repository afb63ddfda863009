"""GPU parity of the Section 4 problems (3-D trilinear FEM, exponential-
covariance KL field; Test 1 and Test 2) against the oracle: assembly, the
anisotropy indicator, ensemble PCG, full-size sampled lanes, and the adaptive
loop with surrogate grouping."""
import dataclasses
import os

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import OKIND, Case, elem_err, grouping_on_oracle_counts
from stopping import count_envelope
from oracle import uq as ouq
from paper_1705_02003_gb300 import ens, inputs, uq

pytestmark = pytest.mark.gpu
KINDS = ["q1_3d_kl", "q1_3d_disc"]


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


def draws_with_thresholds(M, seed):
    """Uniform draws plus dyadic points whose radius is exactly sqrt(3)/4 or
    sqrt(3)/2 (Test 2's jumps), as a sparse grid produces them."""
    xi = inputs.draws(M, 4, seed=seed)
    xi[0] = [0.25, 0.25, 0.25, 0.0]   # r = sqrt(3)/4
    xi[1] = [0.5, -0.5, 0.0, 0.5]     # r = sqrt(3)/2
    xi[2] = [0.0, 0.0, 0.0, 0.0]
    return xi


@pytest.mark.parametrize("kind", KINDS)
def test_assembly_matches_oracle(h, kind):
    n, S, M = 9, 8, 11
    xi = draws_with_thresholds(M, 7)
    c = Case(h, kind, n, 4, 0.0, S, xi)
    V, D, B = c.lane_vals(), c.lane_vec(c.dinv), c.lane_vec(c.b)
    rp, ci = O.pattern(OKIND[kind], n)
    for s in range(M):
        vals, b = O.assemble(OKIND[kind], n, 4, 0.0, xi[s], rp, ci)
        # face-neighbour entries nearly cancel (they vanish for an isotropic
        # tensor), so the bar is relative to the operator's scale
        np.testing.assert_allclose(V[s], vals, rtol=1e-13, atol=1e-13 * np.abs(vals).max())
        np.testing.assert_array_equal(B[s], b)
        np.testing.assert_allclose(D[s], O.jacobi(rp, ci, vals), rtol=1e-13, atol=0)


@pytest.mark.parametrize("kind", KINDS)
def test_indicator_matches_oracle(h, kind):
    n, M = 9, 13
    xi = draws_with_thresholds(M, 8)
    H = torch.empty(M, dtype=torch.float64, device="cuda")
    ens.ens_param_indicator(h, ens.problem(kind, n, 4, 0.0), torch.from_numpy(xi).cuda(), H)
    Ho = np.array([O.param_indicator(OKIND[kind], n, 4, 0.0, xi[m]) for m in range(M)])
    np.testing.assert_allclose(H.cpu().numpy(), Ho, rtol=1e-12)


def _check_solve(got, ref, lanes, rtol, bar):
    for j, L in enumerate(lanes):
        assert got["status"][L] == ref["status"][j] == O.CONVERGED
        di = int(got["iters"][L]) - int(ref["iters"][j])
        assert abs(di) <= 1
        err = elem_err(got["x"][L], ref["x"][j])
        assert err <= (bar if di == 0 else 1e-5), (L, err)


@pytest.mark.parametrize("kind", KINDS)
def test_pcg_matches_oracle_on_the_oracles_matrices(h, kind):
    """The solver alone: the oracle's assembled values, D^-1 and load are
    uploaded, so GPU and oracle solve the same systems and differ only in the
    PCG arithmetic (fused against separate multiply-adds).  On this 3-D operator
    (anisotropy up to ~400, condition number ~1e5 at 32^3 cells) that rounding
    difference moves the stopped iterate by up to ~2e-9 (measured; the 2-D
    problems stay below 1e-10), so the bar here is 1e-8 when the counts agree.
    Assembled on both sides the matrices also differ at 1e-13 (CUDA's and
    glibc's cos, sin, exp), which the condition number can lift to ~1e-8; the
    full-size test below uses 1e-7."""
    n, S, M = 15, 16, 21
    xi = draws_with_thresholds(M, 9)
    c = Case(h, kind, n, 4, 0.0, S, xi)
    rp, ci = O.pattern(OKIND[kind], n)
    E, nnz, J = c.E, c.nnz, c.J
    V = np.zeros((E, nnz, S))
    D = np.zeros((E, J, S))
    B = np.zeros((E, J, S))
    outs = []
    for L in range(E * S):
        vals, b = O.assemble(OKIND[kind], n, 4, 0.0, xi[min(L, M - 1)], rp, ci)
        V[L // S, :, L % S] = vals
        D[L // S, :, L % S] = O.jacobi(rp, ci, vals)
        B[L // S, :, L % S] = b
        if L < M:
            x, it, st, rr = O.pcg(rp, ci, vals, b, 1e-7, 50000)
            outs.append((x, it, st))
    c.vals.copy_(torch.from_numpy(V.ravel()))
    c.dinv.copy_(torch.from_numpy(D.ravel()))
    c.b.copy_(torch.from_numpy(B.ravel()))
    got = c.solve(1e-7, 50000)
    ref = {"x": [o[0] for o in outs], "iters": np.array([o[1] for o in outs]),
           "status": np.array([o[2] for o in outs])}
    _check_solve(got, ref, range(M), 1e-7, 1e-8)


@pytest.mark.parametrize("name,lanes", [("q1_32c_test1", [0, 19]), ("q1_32c_test2", [1, 30])])
def test_full_size_sampled_lanes(h, name, lanes):
    """The 32^3-cell problem of Section 4 in the bench's launch shape (two
    ensembles of 16), sampled lanes against the oracle."""
    wl = inputs.WORKLOADS[name]
    xi = draws_with_thresholds(2 * wl.S, 10)
    c = Case(h, wl.kind, wl.n, wl.nparam, wl.aniso, wl.S, xi)
    got = c.solve(wl.rtol, wl.maxit)
    ref = O.solve_batch(OKIND[wl.kind], wl.n, 4, 0.0, xi[lanes], wl.rtol, wl.maxit, nthreads=len(lanes),
                        want_x=True)
    # both sides assemble: 1e-13 matrix differences times the condition number (~1e5)
    _check_solve(got, ref, lanes, wl.rtol, 1e-7)


@pytest.mark.parametrize("name", ["q1_32c_test1", "q1_32c_test2"])
def test_adaptive_loop_matches_oracle(h, name):
    """The flowchart loop on a 16^3-cell version of the problem, capped at 200
    points: the same grid and levels, G within 1e-7, and the surrogate
    groupings equal wherever the counts agree.  Iteration counts within one,
    or, where a count differs by more, within one of the range of counts the
    oracle itself gives when its matrix is perturbed by the assembly bar (1e-13
    relative, random signs, twelve draws; tests/stopping.py count_envelope):
    each side assembles its own matrix, and Test 2's coefficient reaches 100 x
    the KL field, so condition numbers near 1e7 make the residual curve near
    the stop chaotic under such differences (with the same matrices the counts
    agree within one, test above)."""
    wl = dataclasses.replace(inputs.WORKLOADS[name], n=15, n_max=200)
    run = uq.Adaptive(h, wl).run("sur")

    def solve(y):
        o = O.solve_batch(OKIND[wl.kind], wl.n, 4, 0.0, y, wl.rtol, wl.maxit, nthreads=os.cpu_count() or 4)
        return o["G"], o["iters"]

    ref = ouq.adaptive(solve, N=4, S=wl.S, tau=wl.tau, init_level=wl.init_level, max_level=wl.max_level,
                       n_max=wl.n_max)
    assert np.array_equal(run["lvl"], ref["lvl"]) and np.array_equal(run["idx"], ref["idx"])
    assert run["levels"] == ref["levels"] and len(run["levels"]) >= 2
    Ig, Io = run["I"].astype(int), ref["I"].astype(int)
    rp, ci = O.pattern(OKIND[wl.kind], wl.n)
    for m in np.nonzero(np.abs(Ig - Io) > 1)[0]:
        vals, b = O.assemble(OKIND[wl.kind], wl.n, 4, 0.0, ref["y"][m], rp, ci)
        lo, hi = count_envelope(O, rp, ci, vals, b, wl.rtol, wl.maxit, 1e-13)
        assert lo - 1 <= Ig[m] <= hi + 1, (m, Io[m], Ig[m], lo, hi)
    np.testing.assert_allclose(run["G"], ref["G"], rtol=1e-7)  # assembled on both sides (see above)
    grouping_on_oracle_counts(h, ref)
    if np.array_equal(run["I"], ref["I"]):
        for p, po in zip(run["perms"][1:], ref["perms"]["sur"][1:]):
            assert np.array_equal(p, po)
