"""Pins of the oracle's multigrid preconditioner (oracle/mg.c) against facts the
oracle does not compute itself: the trilinear FEM matrices of nested meshes
built here from 1-D Kronecker factors, scipy's trilinear interpolation, the
closed-form Chebyshev polynomial on known eigenpairs, dense eigenvalue and
direct solves, and textbook multigrid behaviour."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.interpolate import RegularGridInterpolator

import oracle as O

KL = O.Q1_3D_KL


def fem_1d(n):
    h = 1.0 / (n + 1)
    K = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h
    M = sp.diags([np.ones(n - 1), 4 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) * (h / 6)
    return K, M


def fem_3d(n, ax=1.0, ay=1.0, az=1.0):
    """Trilinear stiffness of -div(diag(ax, ay, az) grad u) on n^3 interior
    nodes (node index i + n j + n^2 l), from the 1-D stiffness and mass."""
    K, M = fem_1d(n)
    A = ax * sp.kron(M, sp.kron(M, K)) + ay * sp.kron(M, sp.kron(K, M)) + az * sp.kron(K, sp.kron(M, M))
    return A.toarray()


def in_pattern(n, dense):
    rp, ci = O.pattern(KL, n)
    rows = np.repeat(np.arange(n ** 3), np.diff(rp))
    return rp, ci, np.ascontiguousarray(dense[rows, ci])


def test_levels():
    assert O.mg_levels(31) == [31, 15, 7, 3]
    assert O.mg_levels(15) == [15, 7, 3]
    assert O.mg_levels(3) == [3]
    for bad in (1, 2, 5, 16, 30):
        with pytest.raises(ValueError):
            O.mg_levels(bad)


@pytest.mark.parametrize("aniso", [(1.0, 1.0, 1.0), (1.1, 1.0, 1.0), (7.0, 0.5, 2.0)])
def test_galerkin_operator_is_the_coarse_mesh_fem_matrix(aniso):
    """Nested trilinear spaces: P^T A_h P = A_2h for a constant tensor."""
    for nf in (7, 15):
        nc = (nf - 1) // 2
        rp, ci, vf = in_pattern(nf, fem_3d(nf, *aniso))
        _, _, vc_want = in_pattern(nc, fem_3d(nc, *aniso))
        vc = O.mg_galerkin(nf, rp, ci, vf, nc)
        np.testing.assert_allclose(vc, vc_want, rtol=0, atol=1e-14 * np.abs(vc_want).max())


def test_galerkin_of_the_section4_operator_at_the_mean_field():
    """At y = 0 the Section 4 field is the constant diag(1.1, 1, 1): the Galerkin
    operator equals the problem assembled on the coarse mesh, and the restricted
    load equals the coarse load exactly (h^3 is a power of two)."""
    nf, nc = 15, 7
    rp, ci = O.pattern(KL, nf)
    vf, bf = O.assemble(KL, nf, 4, 0.0, np.zeros(4), rp, ci)
    rpc, cic = O.pattern(KL, nc)
    vc_want, bc_want = O.assemble(KL, nc, 4, 0.0, np.zeros(4), rpc, cic)
    vc = O.mg_galerkin(nf, rp, ci, vf, nc)
    np.testing.assert_allclose(vc, vc_want, rtol=0, atol=1e-14 * np.abs(vc_want).max())
    np.testing.assert_array_equal(O.mg_restrict(nf, nc, bf), bc_want)


def test_prolongation_is_trilinear_interpolation_and_restriction_its_transpose():
    rng = np.random.default_rng(1)
    nf, nc = 15, 7
    ec = rng.standard_normal(nc ** 3)
    grid = np.zeros((nc + 2,) * 3)
    grid[1:-1, 1:-1, 1:-1] = ec.reshape(nc, nc, nc)  # [l][j][i]: z, y, x
    t = np.linspace(0.0, 1.0, nc + 2)
    f = RegularGridInterpolator((t, t, t), grid, method="linear")
    xf = np.arange(1, nf + 1) / (nf + 1)
    Z, Y, X = np.meshgrid(xf, xf, xf, indexing="ij")
    want = f(np.stack([Z.ravel(), Y.ravel(), X.ravel()], axis=1))
    np.testing.assert_allclose(O.mg_prolong(nf, nc, ec), want, rtol=0, atol=1e-14)
    rf = rng.standard_normal(nf ** 3)
    lhs = np.dot(O.mg_restrict(nf, nc, rf), ec)
    rhs = np.dot(rf, O.mg_prolong(nf, nc, ec))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0)


def test_gershgorin_bound():
    n = 7
    # isotropic trilinear stencil: off-diagonals <= 0, interior rows sum to 0 -> ratio 2
    rp, ci, v = in_pattern(n, fem_3d(n))
    assert O.gershgorin(rp, ci, v) == pytest.approx(2.0, rel=1e-14)
    # a bound on the spectrum of D^-1 A for a random Section 4 sample
    rng = np.random.default_rng(2)
    for kind in (O.Q1_3D_KL, O.Q1_3D_DISC):
        vals, _ = O.assemble(kind, n, 4, 0.0, rng.uniform(-1, 1, 4), rp, ci)
        A = np.zeros((n ** 3, n ** 3))
        A[np.repeat(np.arange(n ** 3), np.diff(rp)), ci] = vals
        d = np.sqrt(np.diag(A))
        lam = np.linalg.eigvalsh(A / d[:, None] / d[None, :]).max()
        g = O.gershgorin(rp, ci, vals)
        assert lam <= g <= 2.0 * lam
    bad = v.copy()
    bad[rp[5] + np.where(ci[rp[5]:rp[6]] == 5)[0][0]] = 0.0  # a zero diagonal
    assert np.isnan(O.gershgorin(rp, ci, bad))


@pytest.mark.parametrize("tensor", [(1.0, 1.0, 1.0), (1.1, 1.0, 1.0), (7.0, 0.5, 2.0)])
def test_chebyshev_smoother_applies_the_chebyshev_polynomial(tensor):
    """On A x = 0 from an eigenvector v of D^-1 A (constant diagonal: the tensor
    sines), the smoother returns p(mu) v with p(t) = T_2((theta - t)/delta) / T_2(theta/delta).
    diag(1.1, 1, 1) is the Section 4 field at y = 0."""
    n = 7
    h = 1.0 / (n + 1)
    ax, ay, az = tensor
    A = fem_3d(n, ax, ay, az)
    rp, ci, v = in_pattern(n, A)
    dinv = 1.0 / np.diag(A)
    lmax = O.gershgorin(rp, ci, v)
    lmin = lmax / 30.0
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    T2 = lambda u: 2 * u * u - 1
    x = np.arange(1, n + 1) * h
    for k, m, q in [(1, 1, 1), (2, 1, 3), (7, 7, 7), (4, 6, 2)]:
        sx, sy, sz = np.sin(k * np.pi * x), np.sin(m * np.pi * x), np.sin(q * np.pi * x)
        vec = np.einsum("l,j,i->lji", sz, sy, sx).ravel()
        kk = [(2 / h) * (1 - np.cos(w * np.pi * h)) for w in (k, m, q)]
        mm = [(h / 6) * (4 + 2 * np.cos(w * np.pi * h)) for w in (k, m, q)]
        lam = ax * kk[0] * mm[1] * mm[2] + ay * mm[0] * kk[1] * mm[2] + az * mm[0] * mm[1] * kk[2]
        np.testing.assert_allclose(A @ vec, lam * vec, atol=1e-12 * max(tensor))
        mu = lam * dinv[0]
        p = T2((theta - mu) / delta) / T2(theta / delta)
        out = O.cheb(rp, ci, v, dinv, lmax, np.zeros(n ** 3), vec)
        np.testing.assert_allclose(out, p * vec, rtol=0, atol=1e-13)


def test_coarsest_level_is_an_exact_solve():
    n = 3
    rp, ci = O.pattern(KL, n)
    rng = np.random.default_rng(3)
    vals, b = O.assemble(KL, n, 4, 0.0, rng.uniform(-1, 1, 4), rp, ci)
    A = np.zeros((27, 27))
    A[np.repeat(np.arange(27), np.diff(rp)), ci] = vals
    r = rng.standard_normal(27)
    np.testing.assert_allclose(O.mg_apply(n, rp, ci, vals, r), np.linalg.solve(A, r), rtol=1e-12)
    x, it, st, _ = O.mgpcg(n, rp, ci, vals, b, 1e-10, 10)
    assert st == O.CONVERGED and it == 1
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-12)


@pytest.mark.parametrize("kind", [O.Q1_3D_KL, O.Q1_3D_DISC])
def test_vcycle_is_symmetric_positive_definite(kind):
    n = 15
    rp, ci = O.pattern(kind, n)
    rng = np.random.default_rng(4)
    vals, _ = O.assemble(kind, n, 4, 0.0, rng.uniform(-1, 1, 4), rp, ci)
    us = [rng.standard_normal(n ** 3) for _ in range(3)]
    Mu = [O.mg_apply(n, rp, ci, vals, u) for u in us]
    for a in range(3):
        assert np.dot(us[a], Mu[a]) > 0
        for b in range(a + 1, 3):
            x, y = np.dot(us[a], Mu[b]), np.dot(us[b], Mu[a])
            assert abs(x - y) <= 1e-12 * abs(np.dot(us[a], Mu[a]))


def test_mgpcg_is_mesh_independent_and_solves_the_system():
    its = []
    for n in (7, 15, 31):
        rp, ci = O.pattern(KL, n)
        vals, b = O.assemble(KL, n, 4, 0.0, np.zeros(4), rp, ci)
        x, it, st, rr = O.mgpcg(n, rp, ci, vals, b, 1e-10, 200)
        assert st == O.CONVERGED and rr <= 1e-10
        its.append(it)
        if n == 15:
            A = sp.csr_matrix((vals, ci, rp), shape=(n ** 3, n ** 3))
            from scipy.sparse.linalg import spsolve
            xs = spsolve(A.tocsc(), b)
            assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    # n = 7 is a two-grid solve (exact 3^3 coarse level); 15 and 31 use three
    # and four levels: the count settles as the mesh is refined
    assert max(its) <= 20 and its[2] - its[1] <= 2 and its[1] >= its[0], its


def test_mgpcg_status_codes():
    n = 7
    rp, ci = O.pattern(KL, n)
    vals, b = O.assemble(KL, n, 4, 0.0, np.full(4, 0.3), rp, ci)
    x, it, st, rr = O.mgpcg(n, rp, ci, vals, np.zeros_like(b), 1e-8, 50)
    assert st == O.CONVERGED and it == 0 and rr == 0.0 and not x.any()
    bad = vals.copy()
    bad[17] = np.nan
    assert O.mgpcg(n, rp, ci, bad, b, 1e-8, 50)[2] == O.BADINPUT
    bnan = b.copy()
    bnan[3] = np.nan
    assert O.mgpcg(n, rp, ci, vals, bnan, 1e-8, 50)[2] == O.BADINPUT
    assert O.mgpcg(n, rp, ci, vals, b, 1e-14, 2)[2] == O.MAXIT


@pytest.mark.parametrize("kind", [O.Q1_3D_KL, O.Q1_3D_DISC])
def test_float_vcycle_is_the_vcycle_to_float_accuracy(kind):
    """The float V-cycle (hierarchy rounded to float) equals the FP64 V-cycle
    pinned above to float rounding, and is not the same computation (a dropped
    term or a wrong coefficient would differ at order one)."""
    n = 15
    rp, ci = O.pattern(kind, n)
    rng = np.random.default_rng(8)
    for _ in range(2):
        vals, _ = O.assemble(kind, n, 4, 0.0, rng.uniform(-1, 1, 4), rp, ci)
        r = rng.standard_normal(n ** 3)
        z64 = O.mg_apply(n, rp, ci, vals, r)
        z32 = O.mg_apply32(n, rp, ci, vals, r)
        rel = np.linalg.norm(z32 - z64) / np.linalg.norm(z64)
        assert 1e-9 < rel < 1e-6, rel


@pytest.mark.parametrize("kind", [O.Q1_3D_KL, O.Q1_3D_DISC])
def test_cg_with_the_float_vcycle_converges_like_fp64(kind):
    """CG stays in FP64; the float preconditioner changes neither the count
    (within one) nor the converged solution (1e-9 at rtol 1e-10)."""
    n = 15
    rp, ci = O.pattern(kind, n)
    rng = np.random.default_rng(9)
    for _ in range(3):
        vals, b = O.assemble(kind, n, 4, 0.0, rng.uniform(-1, 1, 4), rp, ci)
        x64, i64, s64, _ = O.mgpcg(n, rp, ci, vals, b, 1e-10, 300)
        x32, i32, s32, rr = O.mgpcg32(n, rp, ci, vals, b, 1e-10, 300)
        assert s64 == s32 == O.CONVERGED and rr <= 1e-10
        assert abs(i32 - i64) <= 1
        assert np.linalg.norm(x32 - x64) <= 1e-9 * np.linalg.norm(x64)
