"""Pins for the oracle's sparse grid, iteration surrogate, grouping and work
ratio R (CPU only): exact hierarchical identities, brute-force enumeration,
a library stable sort, brute-force optimal partitions and the conventions the
paper's printed tables fix."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import uq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def level_points_1d(l):
    """(l, i) pairs of one 1-D level: {0, 1} at level 0, odd i < 2^l above."""
    return [(0, 0), (0, 1)] if l == 0 else [(l, i) for i in range(1, 2**l, 2)]


def test_hat_partition_of_unity_at_level0():
    rng = np.random.default_rng(0)
    for y in rng.uniform(-1, 1, 200):
        s = O.hat(0, 0, y) + O.hat(0, 1, y)
        assert abs(s - 1.0) <= 2.3e-16
    assert O.hat(0, 0, -1.0) == 1.0 and O.hat(0, 1, 1.0) == 1.0
    assert O.sg_coord(0, 0) == -1.0 and O.sg_coord(0, 1) == 1.0 and O.sg_coord(1, 1) == 0.0
    assert O.sg_coord(3, 5) == 0.25  # i h_l - 1 with h_3 = 1/4


def test_hierarchical_triangularity_is_exact():
    pts = [p for l in range(7) for p in level_points_1d(l)]
    for (l, i) in pts:
        assert O.hat(l, i, O.sg_coord(l, i)) == 1.0
        for (l2, i2) in pts:
            if l2 <= l and (l2, i2) != (l, i):
                assert O.hat(l, i, O.sg_coord(l2, i2)) == 0.0


def test_hat_support_and_shape():
    # psi_{l,i} is a hat of half-width h_l centred at y_{l,i}
    for l, i in [(1, 1), (2, 3), (4, 5)]:
        c, h = O.sg_coord(l, i), 2.0 ** (1 - l)
        assert O.hat(l, i, c + h / 2) == 0.5 and O.hat(l, i, c - h / 4) == 0.75
        assert O.hat(l, i, c + h) == 0.0 and O.hat(l, i, c - 1.5 * h) == 0.0


def test_1d_square_has_surplus_minus_h_squared():
    lvl, idx = O.sg_initial(1, 7)
    y = O.sg_points(lvl, idx)[:, 0]
    c = uq.hierarchize(lvl, idx, y**2)
    for (l,), (i,), cv in zip(lvl, idx, c):
        if l == 0:
            assert cv == 1.0
        else:
            assert cv == -(2.0 ** (1 - l)) ** 2


def test_multilinear_functions_are_reproduced():
    rng = np.random.default_rng(1)
    N = 3
    lvl, idx = O.sg_initial(N, 4)
    coef = rng.integers(-8, 8, 2**N) / 8.0  # dyadic

    def f(Y):
        out = np.zeros(len(Y))
        for mask in range(2**N):
            term = np.full(len(Y), coef[mask])
            for n in range(N):
                if mask >> n & 1:
                    term = term * Y[:, n]
            out += term
        return out

    y = O.sg_points(lvl, idx)
    c = uq.hierarchize(lvl, idx, f(y))
    lev = lvl.sum(axis=1)
    assert np.all(c[lev >= 1] == 0.0)
    yq = rng.uniform(-1, 1, (300, N))
    np.testing.assert_allclose(O.sg_eval(lvl, idx, c, yq), f(yq), rtol=0, atol=1e-14)
    yd = rng.integers(-16, 17, (100, N)) / 16.0
    assert np.array_equal(O.sg_eval(lvl, idx, c, yd), f(yd))


def test_1d_interpolation_error_is_second_order():
    rng = np.random.default_rng(2)
    yq = rng.uniform(-1, 1, (2000, 1))
    errs = []
    for L in (4, 5, 6, 7):
        lvl, idx = O.sg_initial(1, L)
        y = O.sg_points(lvl, idx)
        c = uq.hierarchize(lvl, idx, np.exp(y[:, 0]))
        errs.append(np.abs(O.sg_eval(lvl, idx, c, yq) - np.exp(yq[:, 0])).max())
    ratios = [errs[k] / errs[k + 1] for k in range(3)]
    assert all(3.5 < r < 4.5 for r in ratios), ratios


@pytest.mark.parametrize("N,L", [(1, 5), (2, 3), (3, 3), (4, 2), (6, 2)])
def test_initial_grid_is_the_full_sparse_grid(N, L):
    lvl, idx = O.sg_initial(N, L)
    got = {tuple(zip(a.tolist(), b.tolist())) for a, b in zip(lvl, idx)}
    assert len(got) == len(lvl)  # no duplicates
    want = set()
    for ls in itertools.product(range(L + 1), repeat=N):
        if sum(ls) > L:
            continue
        for pts in itertools.product(*[level_points_1d(l) for l in ls]):
            want.add(tuple(pts))
    assert got == want
    levsum = lvl.sum(axis=1)
    assert np.all(np.diff(levsum) >= 0)  # generated in non-decreasing level order


def children(point):
    out = []
    for n, (l, i) in enumerate(point):
        opts = [(1, 1)] if l == 0 else [(l + 1, 2 * i - 1), (l + 1, 2 * i + 1)]
        for o in opts:
            out.append(tuple(o if k == n else point[k] for k in range(len(point))))
    return out


def test_refinement_follows_the_set_definition():
    rng = np.random.default_rng(4)
    N = 3
    lvl, idx = O.sg_initial(N, 2)
    first = int(np.argmax(lvl.sum(axis=1) == 2))
    surplus = rng.standard_normal(len(lvl))
    tau, max_level = 0.8, 3
    nl, ni = O.sg_refine(lvl, idx, first, surplus, tau, max_level)
    existing = [tuple(zip(a.tolist(), b.tolist())) for a, b in zip(lvl, idx)]
    want = []
    for m in range(first, len(lvl)):
        if abs(surplus[m]) >= tau and sum(l for l, _ in existing[m]) + 1 <= max_level:
            for ch in children(existing[m]):
                if ch not in existing and ch not in want:
                    want.append(ch)
    got = [tuple(zip(a.tolist(), b.tolist())) for a, b in zip(nl, ni)]
    assert got == want and len(got) > 0
    # level cap: nothing above max_level
    nl2, _ = O.sg_refine(lvl, idx, first, surplus, tau, 2)
    assert len(nl2) == 0


def test_sort_is_a_stable_ascending_sort():
    rng = np.random.default_rng(5)
    for M in (1, 7, 64, 500):
        keys = rng.integers(0, 12, M).astype(np.float64)  # many ties
        keys[rng.random(M) < 0.3] += 0.5
        perm = O.sort_perm(keys)
        assert perm.tolist() == sorted(range(M), key=lambda i: keys[i])


def brute_min_sum_max(iters, S):
    M = len(iters)
    best = math.inf
    for p in itertools.permutations(range(M)):
        s = sum(max(iters[j] for j in p[k:k + S]) for k in range(0, M, S))
        best = min(best, s)
    return best


def test_sorted_chunking_minimises_work():
    # With full ensembles (M a multiple of S) ascending sort-and-chunk is the
    # optimal partition; with a partial last ensemble it is not in general
    # (the remainder holds the largest counts), which the next test records.
    rng = np.random.default_rng(6)
    for M, S in [(8, 2), (6, 3), (8, 4), (9, 3)]:
        it = rng.integers(1, 50, M).astype(np.float64)
        perm = O.sort_perm(it)
        R = O.work_ratio(S, perm, it)
        assert R == pytest.approx(S * brute_min_sum_max(list(it), S) / it.sum(), rel=1e-15)
        for _ in range(20):
            assert O.work_ratio(S, rng.permutation(M).astype(np.int32), it) >= R


def test_padded_last_ensemble_holds_the_largest_counts():
    it = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0])
    perm = O.sort_perm(it)
    # chunks {1,2} {3,4} {5,6} {7}: S * (2 + 4 + 6 + 7) / 28
    assert O.work_ratio(2, perm, it) == 2.0 * 19.0 / 28.0
    assert brute_min_sum_max(list(it), 2) == 16.0  # {1} {2,3} {4,5} {6,7} would be cheaper


def test_work_ratio_conventions():
    # R = 1 for equal counts in full ensembles
    assert O.work_ratio(4, np.arange(12, dtype=np.int32), np.full(12, 9.0)) == 1.0
    rng = np.random.default_rng(8)
    for _ in range(20):
        it = rng.integers(1, 100, 37).astype(np.float64)
        assert O.work_ratio(8, rng.permutation(37).astype(np.int32), it) >= 1.0
    # padding lanes count only through S: one padded ensemble doubles when S doubles
    it = np.array([12.0, 40.0, 7.0, 33.0, 21.0, 9.0, 15.0, 18.0, 26.0])
    p = np.arange(9, dtype=np.int32)
    assert O.work_ratio(32, p, it) == 2.0 * O.work_ratio(16, p, it)
    assert O.work_ratio(16, p, it) == 16.0 * 40.0 / it.sum()


def read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            vals = [float("nan") if t == "-" else float(t) for t in tok[2:]]
            rows.append((tok[0], int(tok[1]), vals))
    return rows


@pytest.mark.parametrize("name,nlev", [("table2_test1_R.txt", 8), ("table3_test2_R.txt", 5)])
def test_paper_tables_fix_the_conventions(name, nlev):
    rows = read_table(name)
    by = {(m, S): v for m, S, v in rows}
    for (m, S), v in by.items():
        assert all(r >= 1.0 for r in v[:nlev + 1])  # R >= 1 everywhere
    for S in (4, 8, 16, 32):
        # the initial set is grouped in generation order by every method
        assert by[("sur", S)][0] == by[("par", S)][0] == by[("nat", S)][0]
        # sorting by actual iterations is optimal at every level
        for lev in range(nlev):
            for m in ("sur", "par", "nat"):
                assert by[("its", S)][lev] <= by[(m, S)][lev] + 1e-12
        # predicted speed-up = (iteration-independent speed-up) / R: the product
        # pred * R is the same for every method at a given S
        prods = [by[(m, S)][nlev + 2] * by[(m, S)][nlev] for m in ("its", "sur", "par", "nat")]
        assert max(prods) - min(prods) < 0.06
    # one padded ensemble in both cases: R_1(32) = 2 R_1(16) up to print rounding
    r16, r32 = by[("sur", 16)][0], by[("sur", 32)][0]
    assert abs(r32 - 2 * r16) <= 0.011


def test_adaptive_loop_on_the_small_workload():
    """The flowchart loop on the 32x32 5-point problem: level cap 4, tau 1e-3."""
    def solve(y):
        out = O.solve_batch(O.FD5_LOGKL, 32, 2, 3.0, y, 1e-8, 20000, nthreads=4)
        assert np.all(out["status"] == O.CONVERGED)
        return out["G"], out["iters"]

    run = uq.adaptive(solve, N=2, S=8, tau=1e-3, init_level=1, max_level=4, n_max=10**6)
    assert run["lvl"].sum(axis=1).max() <= 4
    assert len(run["levels"]) >= 3
    # surpluses of I at new points = I - prediction from the older points
    for (a, b), p in zip(run["levels"][1:], run["pred"][1:]):
        np.testing.assert_array_equal(run["cI"][a:b], run["I"][a:b] - p)
        # hierarchising the whole grid at once gives the same surpluses
    np.testing.assert_array_equal(uq.hierarchize(run["lvl"], run["idx"], run["I"]), run["cI"])
    # the surrogate interpolates the data at the grid points
    np.testing.assert_allclose(O.sg_eval(run["lvl"], run["idx"], run["cI"], run["y"]), run["I"],
                               rtol=0, atol=1e-9)
    R = uq.ratios(run)
    for lev, (a, b) in enumerate(run["levels"]):
        for m in ("its", "sur", "nat", "rand"):
            assert R[m][0][lev] >= 1.0
            if (b - a) % 8 == 0:  # full ensembles only: then sorting by I is optimal
                assert R["its"][0][lev] <= R[m][0][lev] + 1e-12
