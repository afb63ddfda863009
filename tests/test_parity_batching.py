"""GPU parity of the batching layer (ens_solve_stream): continuous refill of
frozen lanes and re-packing of the drained pool change nothing about any
sample's solve -- its iteration count, status and residual are those of the
fixed-ensemble solve bit for bit, its QoI agrees to rounding, and both agree
with the oracle (iterations within one, G within 1e-10)."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import OKIND, Case
from paper_1705_02003_gb300 import batching, ens, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(ens_lib):
    return ens.Handle(0)


@pytest.mark.parametrize("kind,n,N,aniso,S,E,M,chunk", [("fd7", 10, 6, 3.0, 8, 2, 53, 8),
                                                        ("fd5", 24, 8, 3.0, 4, 3, 40, 5),
                                                        ("q1", 20, 4, 4.0, 16, 1, 37, 16),
                                                        ("fd5", 16, 2, 3.0, 1, 4, 9, 3)])
def test_stream_equals_fixed_ensembles_and_oracle(h, kind, n, N, aniso, S, E, M, chunk):
    xi = inputs.draws(M, N, seed=80 + n)
    order = torch.from_numpy(inputs.rand_perm(M, seed=3)).cuda()
    prob = ens.problem(kind, n, N, aniso)
    out = batching.solve_stream(h, prob, torch.from_numpy(xi).cuda(), S, E, 1e-8, 20000, chunk=chunk, order=order)
    it, st, rr, q = (out[k].cpu().numpy() for k in ("iters", "status", "relres", "qoi"))
    # the same samples in fixed ensembles of S
    c = Case(h, kind, n, N, aniso, S, xi)
    ref = c.solve(1e-8, 20000)
    assert np.array_equal(it, ref["iters"][:M])
    assert np.array_equal(st, ref["status"][:M])
    assert np.array_equal(rr, ref["relres"][:M])
    G = (ref["x"][:M] ** 2).sum(axis=1)
    np.testing.assert_allclose(q, G, rtol=1e-12)
    o = O.solve_batch(OKIND[kind], n, N, aniso, xi, 1e-8, 20000, nthreads=os.cpu_count() or 4)
    assert np.all(np.abs(it - o["iters"]) <= 1)
    np.testing.assert_allclose(q, o["G"], rtol=1e-9)


def test_stream_with_weights_and_a_bad_sample(h):
    n, N, S, E, M = 20, 8, 8, 2, 30
    xi = inputs.draws(M, N, seed=90)
    xi[11, 3] = np.nan
    w = torch.from_numpy(inputs.region_weights(n, 2)).cuda()
    prob = ens.problem("fd5", n, N, 3.0)
    out = batching.solve_stream(h, prob, torch.from_numpy(xi).cuda(), S, E, 1e-8, 20000, chunk=7, weights=w)
    st = out["status"].cpu().numpy()
    assert st[11] == ens.LANE_BADINPUT
    keep = [m for m in range(M) if m != 11]
    assert np.all(st[keep] == ens.LANE_CONVERGED)
    o = O.solve_batch(O.FD5_LOGKL, n, N, 3.0, xi[keep], 1e-8, 20000, nthreads=4, want_x=True)
    np.testing.assert_allclose(out["qoi"].cpu().numpy()[keep], o["x"] @ O.region_weights(n, 2), rtol=1e-9)


def test_stream_rejects_a_bad_order(h):
    prob = ens.problem("fd5", 8, 2, 3.0)
    xi = torch.from_numpy(inputs.draws(5, 2, seed=1)).cuda()
    bad = torch.tensor([0, 1, 1, 3, 4], dtype=torch.int32, device="cuda")
    with pytest.raises(ens.EnsError, match="permutation"):
        batching.solve_stream(h, prob, xi, 2, 1, 1e-8, 100, order=bad)


def test_autotune_returns_a_candidate(h):
    prob = ens.problem("fd7", 8, 6, 3.0)
    xi = torch.from_numpy(inputs.draws(64, 6, seed=2)).cuda()
    best, times = batching.autotune(h, prob, xi, lanes=32, rtol=1e-8, maxit=20000, chunk=16)
    assert best in (8, 16, 32) and set(times) == {8, 16, 32}
    c, ct = batching.autotune_chunk(h, prob, xi, 32, best, 1e-8, 20000, candidates=(4, 16))
    assert c in (4, 16) and set(ct) == {4, 16}


def test_adaptive_loop_with_repacked_levels_equals_fixed_levels(h):
    """The flowchart loop with every level solved through the batching layer
    (re-packing partly converged ensembles) visits the same grid with the same
    iteration counts as the fixed-ensemble loop, and G agrees to rounding."""
    from paper_1705_02003_gb300 import uq

    wl = inputs.WORKLOADS["fd5_32_adaptive"]
    fixed = uq.Adaptive(h, wl).run("sur")
    rp = uq.Adaptive(h, wl, repack=True, chunk=8).run("sur")
    assert np.array_equal(rp["lvl"], fixed["lvl"]) and np.array_equal(rp["idx"], fixed["idx"])
    assert np.array_equal(rp["I"], fixed["I"])
    np.testing.assert_allclose(rp["G"], fixed["G"], rtol=1e-12)
    for a, b in zip(rp["perms"], fixed["perms"]):
        assert np.array_equal(a, b)


def test_stream_full_batch_workload_sampled_against_oracle(h):
    """The batching workload at full size: all 4096 draws of the 64^3 7-point
    problem streamed through 64 lanes (S = 16, refills and re-packing), every
    sample converged, and sampled samples against the oracle's own solves."""
    wl = inputs.WORKLOADS["fd7_64_batch"]
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    xi_h = inputs.draws(wl.samples, wl.nparam, seed=wl.seed)
    out = batching.solve_stream(h, prob, torch.from_numpy(xi_h).cuda(), 16, 4, wl.rtol, wl.maxit, chunk=32)
    it, st, rr, q = (out[k].cpu().numpy() for k in ("iters", "status", "relres", "qoi"))
    assert np.all(st == ens.LANE_CONVERGED) and np.all(rr <= wl.rtol)
    assert it.max() > 1.4 * it.min()  # uneven counts: the refills and re-packs really happened
    pick = [0, 1234, 2047, 4095]
    o = O.solve_batch(O.FD7_AXIS, wl.n, wl.nparam, wl.aniso, xi_h[pick], wl.rtol, wl.maxit,
                      nthreads=os.cpu_count() or 4)
    assert np.all(np.abs(it[pick] - o["iters"]) <= 1)
    np.testing.assert_allclose(q[pick], o["G"], rtol=1e-9)
