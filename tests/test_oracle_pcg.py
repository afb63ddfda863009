"""Pins for the oracle's discretisation and per-sample Jacobi-PCG (CPU only).

Each check is independent of the oracle's own code: closed-form eigenpairs of
the constant-coefficient discrete operator, manufactured solutions whose
forcing is derived here by differentiating the field, dense LAPACK solves,
textbook stencils and the CG convergence bound.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def dense(rowptr, colidx, vals):
    J = len(rowptr) - 1
    A = np.zeros((J, J))
    for i in range(J):
        for k in range(rowptr[i], rowptr[i + 1]):
            A[i, colidx[k]] += vals[k]
    return A


def sine_matrix(n):
    """V[j-1, p] = sin(j pi x_p), x_p = (p+1)/(n+1): the Dirichlet eigenvectors."""
    h = 1.0 / (n + 1)
    j = np.arange(1, n + 1)[:, None]
    p = np.arange(1, n + 1)[None, :]
    return np.sin(j * np.pi * p * h)


def lam1d(n, j):
    h = 1.0 / (n + 1)
    return 4.0 / h**2 * np.sin(j * np.pi * h / 2) ** 2


# ---------------------------------------------------------------------------
# closed-form eigenpairs (constant tensor: the 2-D field at xi_2 = 0)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("xi1", [0.0, 0.5, -0.4])
def test_fd5_eigenvector_rhs_converges_in_one_iteration(xi1):
    n = 16
    k2 = 10.0 ** (3.0 * xi1)
    rp, ci = O.pattern(O.FD5_LOGKL, n)
    vals, _ = O.assemble(O.FD5_LOGKL, n, 2, 3.0, [xi1, 0.0], rp, ci)
    V = sine_matrix(n)
    for (j, k) in [(1, 1), (3, 2), (7, 11)]:
        v = np.outer(V[k - 1], V[j - 1]).ravel()  # [y][x] with x fastest
        lam = lam1d(n, j) + k2 * lam1d(n, k)
        x, it, st, rr = O.pcg(rp, ci, vals, v, 1e-10, 100)
        assert st == O.CONVERGED and it == 1
        np.testing.assert_allclose(x, v / lam, rtol=0, atol=1e-12 * np.abs(v / lam).max())


def test_fd5_m_distinct_eigenvalues_take_m_iterations():
    n = 16
    rp, ci = O.pattern(O.FD5_LOGKL, n)
    vals, _ = O.assemble(O.FD5_LOGKL, n, 2, 3.0, [0.5, 0.0], rp, ci)
    V = sine_matrix(n)
    for modes in ([(1, 1), (2, 3)], [(1, 1), (2, 3), (5, 2)], [(1, 2), (4, 4), (6, 1), (9, 3)]):
        b = sum(np.outer(V[k - 1], V[j - 1]).ravel() for j, k in modes)
        x, it, st, _ = O.pcg(rp, ci, vals, b, 1e-10, 100)
        assert st == O.CONVERGED and it == len(modes)


def test_fd5_unit_load_matches_sine_expansion():
    n = 24
    xi1 = 0.25
    k2 = 10.0 ** (3.0 * xi1)
    rp, ci = O.pattern(O.FD5_LOGKL, n)
    vals, b = O.assemble(O.FD5_LOGKL, n, 2, 3.0, [xi1, 0.0], rp, ci)
    assert np.all(b == 1.0)
    V = sine_matrix(n)
    norm2 = ((n + 1) / 2.0) ** 2
    B = V @ b.reshape(n, n) @ V.T  # [k][j]
    j = np.arange(1, n + 1)
    L = lam1d(n, j)[None, :] + k2 * lam1d(n, j)[:, None]
    u = (V.T @ (B / norm2 / L) @ V).ravel()
    x, it, st, _ = O.pcg(rp, ci, vals, b, 1e-14, 10000)
    assert st == O.CONVERGED
    assert np.linalg.norm(x - u) <= 1e-12 * np.linalg.norm(u)


def test_fd7_eigenvector_rhs_converges_in_one_iteration():
    n = 8
    xi = [0.5, -0.25, 0.0, 0.0, 0.0, 0.0]
    k2, k3 = 10.0 ** (3 * 0.5), 10.0 ** (3 * -0.25)
    rp, ci = O.pattern(O.FD7_AXIS, n)
    vals, b = O.assemble(O.FD7_AXIS, n, 6, 3.0, xi, rp, ci)
    V = sine_matrix(n)
    j, k, l = 2, 1, 3
    v = np.einsum("c,b,a->cba", V[l - 1], V[k - 1], V[j - 1]).ravel()  # [z][y][x]
    lam = lam1d(n, j) + k2 * lam1d(n, k) + k3 * lam1d(n, l)
    x, it, st, _ = O.pcg(rp, ci, vals, v, 1e-10, 100)
    assert st == O.CONVERGED and it == 1
    assert np.abs(x - v / lam).max() <= 1e-12 * np.abs(v / lam).max()


# ---------------------------------------------------------------------------
# manufactured solutions: second-order convergence with variable tensors
# ---------------------------------------------------------------------------
MODES2 = [(1, 1), (2, 1), (1, 2), (2, 2), (3, 1), (1, 3), (3, 2)]
MODES3 = [(1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2)]


def fd5_forcing(xi, aniso, X, Y):
    """-div(a diag(1, d) grad u*) for u* = sin(pi x) sin(pi y), derived by hand."""
    pi = np.pi
    d = 10.0 ** (aniso * xi[0])
    s = np.zeros_like(X)
    sx = np.zeros_like(X)
    sy = np.zeros_like(X)
    for k in range(1, len(xi)):
        m, q = MODES2[k - 1]
        c = 0.5 * xi[k] / k
        s += c * np.sin(m * pi * X) * np.sin(q * pi * Y)
        sx += c * m * pi * np.cos(m * pi * X) * np.sin(q * pi * Y)
        sy += c * q * pi * np.sin(m * pi * X) * np.cos(q * pi * Y)
    a = np.exp(s)
    u = np.sin(pi * X) * np.sin(pi * Y)
    ux = pi * np.cos(pi * X) * np.sin(pi * Y)
    uy = pi * np.sin(pi * X) * np.cos(pi * Y)
    return -(a * sx * ux - a * pi**2 * u) - d * (a * sy * uy - a * pi**2 * u), u


@pytest.mark.parametrize("xi", [[0.3, 0.9], [0.3, 0.4, -0.5, 0.6, -0.2, 0.3, 0.5, -0.4]])
def test_fd5_manufactured_second_order(xi):
    errs = []
    for n in (15, 31, 63):
        h = 1.0 / (n + 1)
        g = (np.arange(n) + 1) * h
        X, Y = np.meshgrid(g, g)  # [y][x]
        f, u = fd5_forcing(np.array(xi), 3.0, X, Y)
        rp, ci = O.pattern(O.FD5_LOGKL, n)
        vals, _ = O.assemble(O.FD5_LOGKL, n, len(xi), 3.0, xi, rp, ci)
        x, it, st, _ = O.pcg(rp, ci, vals, f.ravel(), 1e-13, 100000)
        assert st == O.CONVERGED
        errs.append(np.abs(x - u.ravel()).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o - 2.0) < 0.15 for o in orders), (errs, orders)


def test_fd7_manufactured_second_order():
    xi = np.array([0.2, -0.3, 0.5, -0.6, 0.4, 0.7])
    aniso = 3.0
    pi = np.pi
    errs = []
    for n in (7, 15, 31):
        h = 1.0 / (n + 1)
        g = (np.arange(n) + 1) * h
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        s = np.zeros_like(X)
        grad = [np.zeros_like(X) for _ in range(3)]
        for k, (a, b, c) in enumerate(MODES3):
            w = 0.3 * xi[2 + k]
            s += w * np.sin(a * pi * X) * np.sin(b * pi * Y) * np.sin(c * pi * Z)
            grad[0] += w * a * pi * np.cos(a * pi * X) * np.sin(b * pi * Y) * np.sin(c * pi * Z)
            grad[1] += w * b * pi * np.sin(a * pi * X) * np.cos(b * pi * Y) * np.sin(c * pi * Z)
            grad[2] += w * c * pi * np.sin(a * pi * X) * np.sin(b * pi * Y) * np.cos(c * pi * Z)
        e = np.exp(s)
        dd = [1.0, 10.0 ** (aniso * xi[0]), 10.0 ** (aniso * xi[1])]
        S = [np.sin(pi * X), np.sin(pi * Y), np.sin(pi * Z)]
        C = [np.cos(pi * X), np.cos(pi * Y), np.cos(pi * Z)]
        u = S[0] * S[1] * S[2]
        f = np.zeros_like(X)
        for ax in range(3):
            others = [S[o] for o in range(3) if o != ax]
            ua = pi * C[ax] * others[0] * others[1]
            f -= dd[ax] * (e * grad[ax] * ua - e * pi**2 * u)
        rp, ci = O.pattern(O.FD7_AXIS, n)
        vals, _ = O.assemble(O.FD7_AXIS, n, 6, aniso, xi, rp, ci)
        x, it, st, _ = O.pcg(rp, ci, vals, f.ravel(), 1e-13, 100000)
        assert st == O.CONVERGED
        errs.append(np.abs(x - u.ravel()).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o - 2.0) < 0.15 for o in orders), (errs, orders)


def q1_load(n, fun):
    """b_p = int f phi_p by 3x3 Gauss quadrature on every element (vectorised)."""
    h = 1.0 / (n + 1)
    gp = np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)])
    gw = np.array([5.0, 8.0, 5.0]) / 9.0
    t = (gp + 1) / 2  # on [0, 1]
    w = gw / 2
    b = np.zeros((n + 2, n + 2))  # node grid incl. boundary, [y][x]
    E = np.arange(n + 1)
    for a in range(3):
        for c in range(3):
            xs = (E[None, :] + t[a]) * h
            ys = (E[:, None] + t[c]) * h
            fv = fun(xs, ys) * w[a] * w[c] * h * h
            # bilinear shape functions of the element's 4 nodes
            b[:-1, :-1] += fv * (1 - t[a]) * (1 - t[c])
            b[:-1, 1:] += fv * t[a] * (1 - t[c])
            b[1:, :-1] += fv * (1 - t[a]) * t[c]
            b[1:, 1:] += fv * t[a] * t[c]
    return b[1:-1, 1:-1].ravel()


def test_q1_manufactured_second_order():
    xi = np.array([0.4, 0.7, -0.3, 0.8])
    aniso = 4.0
    pi = np.pi
    d = 10.0 ** (aniso * xi[0])
    th = pi / 4 * (1 + xi[2])
    c, s = math.cos(th), math.sin(th)
    T = np.array([[c * c + s * s * d, c * s * (1 - d)], [c * s * (1 - d), s * s + c * c * d]])

    def f(X, Y):
        lg = 0.5 * (xi[1] * np.sin(pi * X) * np.sin(pi * Y) + xi[3] / 2 * np.sin(2 * pi * X) * np.sin(pi * Y))
        ax = 0.5 * (xi[1] * pi * np.cos(pi * X) * np.sin(pi * Y) + xi[3] / 2 * 2 * pi * np.cos(2 * pi * X) * np.sin(pi * Y))
        ay = 0.5 * (xi[1] * pi * np.sin(pi * X) * np.cos(pi * Y) + xi[3] / 2 * pi * np.sin(2 * pi * X) * np.cos(pi * Y))
        a = np.exp(lg)
        ux = pi * np.cos(pi * X) * np.sin(pi * Y)
        uy = pi * np.sin(pi * X) * np.cos(pi * Y)
        uxx = -pi**2 * np.sin(pi * X) * np.sin(pi * Y)
        uyy = uxx
        uxy = pi**2 * np.cos(pi * X) * np.cos(pi * Y)
        flux_x = T[0, 0] * ux + T[0, 1] * uy
        flux_y = T[1, 0] * ux + T[1, 1] * uy
        div = T[0, 0] * uxx + 2 * T[0, 1] * uxy + T[1, 1] * uyy
        # ax, ay are the derivatives of log a, so grad a = a (ax, ay)
        return -(a * ax * flux_x + a * ay * flux_y + a * div)

    errs = []
    for n in (15, 31, 63):
        h = 1.0 / (n + 1)
        g = (np.arange(n) + 1) * h
        X, Y = np.meshgrid(g, g)
        u = np.sin(pi * X) * np.sin(pi * Y)
        rp, ci = O.pattern(O.Q1_ROT, n)
        vals, _ = O.assemble(O.Q1_ROT, n, 4, aniso, xi, rp, ci)
        b = q1_load(n, f)
        x, it, st, _ = O.pcg(rp, ci, vals, b, 1e-13, 200000)
        assert st == O.CONVERGED
        errs.append(np.abs(x - u.ravel()).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o - 2.0) < 0.2 for o in orders), (errs, orders)


def test_q1_isotropic_is_textbook_nine_point_stencil():
    n = 5
    rp, ci = O.pattern(O.Q1_ROT, n)
    vals, b = O.assemble(O.Q1_ROT, n, 4, 4.0, [0.0, 0.0, 0.37, 0.0], rp, ci)
    A = dense(rp, ci, vals)
    p = 2 + n * 2  # interior node
    row = A[p].reshape(n, n)
    assert abs(row[2, 2] - 8.0 / 3.0) < 1e-15
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            if di or dj:
                assert abs(row[2 + dj, 2 + di] + 1.0 / 3.0) < 1e-15
    assert np.allclose(b, 1.0 / (n + 1) ** 2, rtol=0, atol=1e-18)


# ---------------------------------------------------------------------------
# dense brute force, symmetry, SPD, CG bound
# ---------------------------------------------------------------------------
CASES = [
    (O.FD5_LOGKL, 6, 8, 3.0),
    (O.FD5_LOGKL, 7, 2, 3.0),
    (O.Q1_ROT, 6, 4, 4.0),
    (O.FD7_AXIS, 4, 6, 3.0),
    (O.FD7_AXIS, 4, 6, 2.0),
]


@pytest.mark.parametrize("kind,n,N,aniso", CASES)
def test_dense_bruteforce_and_structure(kind, n, N, aniso):
    rng = np.random.default_rng(7)
    for _ in range(3):
        xi = rng.uniform(-1, 1, N)
        rp, ci = O.pattern(kind, n)
        vals, b = O.assemble(kind, n, N, aniso, xi, rp, ci)
        A = dense(rp, ci, vals)
        assert np.array_equal(A, A.T)  # bit-symmetric
        assert np.linalg.eigvalsh(A).min() > 0
        xr = rng.standard_normal(len(b))
        np.testing.assert_allclose(O.spmv(rp, ci, vals, xr), A @ xr, rtol=1e-13, atol=1e-13 * np.abs(A).max())
        np.testing.assert_array_equal(O.jacobi(rp, ci, vals), 1.0 / np.diag(A))
        xd = np.linalg.solve(A, b)
        x, it, st, rr = O.pcg(rp, ci, vals, b, 1e-14, 10000)
        assert st == O.CONVERGED
        assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)
        # residual really is below the tolerance
        assert np.linalg.norm(b - A @ x) <= 1e-13 * np.linalg.norm(b)
        # Jacobi-PCG bound: k <= ceil(0.5 sqrt(kappa) ln(2/rtol))
        Dm = 1.0 / np.sqrt(np.diag(A))
        ev = np.linalg.eigvalsh(A * Dm[:, None] * Dm[None, :])
        kappa = ev.max() / ev.min()
        for rtol in (1e-6, 1e-8):
            _, k, st2, _ = O.pcg(rp, ci, vals, b, rtol, 10000)
            assert st2 == O.CONVERGED
            assert k <= math.ceil(0.5 * math.sqrt(kappa) * math.log(2.0 / rtol))


def test_pattern_sizes_and_sorted_rows():
    for kind, n in [(O.FD5_LOGKL, 32), (O.Q1_ROT, 256), (O.FD7_AXIS, 64), (O.FD5_LOGKL, 512)]:
        J, nnz = O.problem_size(kind, n)
        rp, ci = O.pattern(kind, n)
        assert rp[-1] == nnz and len(rp) == J + 1
        # rows sorted, diagonal present, neighbours within the stencil
        d = np.diff(ci.astype(np.int64))
        row_of = np.repeat(np.arange(J), np.diff(rp))
        same_row = row_of[1:] == row_of[:-1]
        assert np.all(d[same_row] > 0)
    # the sizes quoted for the five workloads
    assert O.problem_size(O.FD5_LOGKL, 32) == (1024, 4992)
    assert O.problem_size(O.Q1_ROT, 256) == (65536, 586756)
    assert O.problem_size(O.FD7_AXIS, 64) == (262144, 1810432)
    assert O.problem_size(O.FD7_AXIS, 128) == (2097152, 14581760)
    assert O.problem_size(O.FD5_LOGKL, 512) == (262144, 1308672)


# ---------------------------------------------------------------------------
# status codes and degenerate cases
# ---------------------------------------------------------------------------
def _small():
    rp, ci = O.pattern(O.FD5_LOGKL, 8)
    vals, b = O.assemble(O.FD5_LOGKL, 8, 2, 3.0, [0.1, 0.2], rp, ci)
    return rp, ci, vals, b


def test_breakdown_guard_keeps_x():
    rp, ci, vals, b = _small()
    x, it, st, _ = O.pcg(rp, ci, -vals, b, 1e-8, 100)  # p^T A p < 0 at once
    assert st == O.BREAKDOWN and it == 0 and np.all(x == 0)


def test_maxit_and_zero_and_nonfinite():
    rp, ci, vals, b = _small()
    x, it, st, rr = O.pcg(rp, ci, vals, b, 1e-8, 1)
    assert st == O.MAXIT and it == 1 and rr > 1e-8
    x, it, st, rr = O.pcg(rp, ci, vals, 0 * b, 1e-8, 100)
    assert st == O.CONVERGED and it == 0 and np.all(x == 0)
    bn = b.copy()
    bn[3] = np.nan
    x, it, st, _ = O.pcg(rp, ci, vals, bn, 1e-8, 100)
    assert st == O.BADINPUT and it == 0
    vn = vals.copy()
    vn[:] = np.nan
    x, it, st, _ = O.pcg(rp, ci, vn, b, 1e-8, 100)
    assert st == O.BADINPUT


def test_batch_equals_individual_and_is_order_free():
    rng = np.random.default_rng(3)
    xi = rng.uniform(-1, 1, (12, 2))
    out = O.solve_batch(O.FD5_LOGKL, 16, 2, 3.0, xi, 1e-8, 10000, nthreads=3, want_x=True)
    perm = rng.permutation(12)
    out2 = O.solve_batch(O.FD5_LOGKL, 16, 2, 3.0, xi[perm], 1e-8, 10000, nthreads=5, want_x=True)
    np.testing.assert_array_equal(out["x"][perm], out2["x"])
    np.testing.assert_array_equal(out["iters"][perm], out2["iters"])
    rp, ci = O.pattern(O.FD5_LOGKL, 16)
    for m in (0, 7):
        vals, b = O.assemble(O.FD5_LOGKL, 16, 2, 3.0, xi[m], rp, ci)
        x, it, st, _ = O.pcg(rp, ci, vals, b, 1e-8, 10000)
        np.testing.assert_array_equal(x, out["x"][m])
        assert it == out["iters"][m]
        assert out["G"][m] == pytest.approx(float(x @ x), rel=1e-15)


# ---------------------------------------------------------------------------
# parameter-based grouping indicator: closed forms of the eigenvalue ratio
# ---------------------------------------------------------------------------
def test_param_indicator_closed_forms():
    rng = np.random.default_rng(13)
    for _ in range(5):
        xi = rng.uniform(-1, 1, 8)
        # 2-D fields: a scalar field times diag(1, d) (or a rotation of it): ratio 10^(aniso |xi_1|)
        assert O.param_indicator(O.FD5_LOGKL, 9, 8, 3.0, xi) == pytest.approx(10 ** (3 * abs(xi[0])), rel=1e-12)
        assert O.param_indicator(O.Q1_ROT, 9, 4, 4.0, xi[:4]) == pytest.approx(10 ** (4 * abs(xi[0])), rel=1e-10)
        # 3-D: diag(1, 10^(a xi_1), 10^(a xi_2)) times a scalar
        e = np.array([0.0, xi[0], xi[1]])
        want = 10 ** (2.0 * (e.max() - e.min()))
        assert O.param_indicator(O.FD7_AXIS, 5, 6, 2.0, xi[:6]) == pytest.approx(want, rel=1e-12)
