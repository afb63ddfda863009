"""Pins of the oracle's Section 4 problems (3-D trilinear FEM, exponential-
covariance KL field, Test 1 / Test 2), none of which re-types the oracle:

- the 1-D eigenvalues against an independent Nystrom eigen-solve of the
  kernel exp(-|s - t| / delta) (Gauss-Legendre, numpy eigh), and the choice of
  the four largest 3-D products against that spectrum;
- the mode shapes against the integral equation itself (adaptive quadrature),
  orthonormality in [0, 1]^3;
- the assembled operator: for the constant tensor at xi = 0 every interior row
  is the closed-form 27-point stencil a_x K1(x)M1(x)M1 + ... of the assembled 1-D
  stiffness K1 = [-1, 2, -1] / h and mass M1 = h [1, 4, 1] / 6; for a variable
  field the matrix is symmetric, positive definite and its rows away from the
  boundary sum to zero; the load is h^3;
- Test 2's coefficient jumps by 100 and by 1/10 where r(xi) crosses d/4 and d/2."""
import numpy as np
import pytest

import oracle as O

DELTA, SIGMA0 = 0.25, np.sqrt(300.0)


def nystrom_eigs(m):
    t, w = np.polynomial.legendre.leggauss(m)
    s, w = 0.5 * (t + 1.0), 0.5 * w
    K = np.exp(-np.abs(s[:, None] - s[None, :]) / DELTA)
    sw = np.sqrt(w)
    return np.sort(np.linalg.eigvalsh(sw[:, None] * K * sw[None, :]))[::-1]


def test_kl_eigenvalues_match_a_nystrom_solve():
    # the kernel has a kink on s = t, so the Nystrom error falls as 1/m^2:
    # Richardson-extrapolate two solves
    l1, l2 = nystrom_eigs(400)[:8], nystrom_eigs(800)[:8]
    lam = (4.0 * l2 - l1) / 3.0
    we, le = O.kl_1d(0)
    wo, lo = O.kl_1d(1)
    assert 0 < we < np.pi < wo < 2 * np.pi
    assert abs(le - lam[0]) <= 1e-8 and abs(lo - lam[1]) <= 1e-8
    # the four largest 3-D products of the 1-D spectrum are the oracle's four parameters
    prods = sorted((lam[i] * lam[j] * lam[k] for i in range(4) for j in range(4) for k in range(4)), reverse=True)
    got = sorted((O.kl_lambda(k) / SIGMA0 for k in range(1, 5)), reverse=True)
    np.testing.assert_allclose(got, prods[:4], rtol=1e-7)
    assert prods[4] < prods[3] * (1 - 1e-3)  # no tie at the cut


def test_kl_modes_solve_the_integral_equation_and_are_orthonormal():
    quad = pytest.importorskip("scipy.integrate").quad
    we, le = O.kl_1d(0)
    wo, lo = O.kl_1d(1)
    y, z = 0.31, 0.77
    for k, lam1 in ((1, le), (2, lo)):  # the x-factor of mode 1 is even, of mode 2 odd
        g = lambda t: O.kl_mode(k, [t, y, z])
        for s in (0.05, 0.4, 0.5, 0.83):
            lhs = quad(lambda t: np.exp(-abs(s - t) / DELTA) * g(t), 0.0, 1.0, points=[s], limit=200)[0]
            assert abs(lhs - lam1 * g(s)) <= 1e-8 * max(1.0, abs(g(s))), (k, s)
    t, w = np.polynomial.legendre.leggauss(24)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    X = np.array([[a, b, c] for a in t for b in t for c in t])
    W = np.array([wa * wb * wc for wa in w for wb in w for wc in w])
    B = np.array([[O.kl_mode(k, x) for x in X] for k in range(1, 5)])
    G = (B * W) @ B.T
    np.testing.assert_allclose(G, np.eye(4), atol=1e-9)


def stencil_closed_form(a, h):
    K1 = np.array([-1.0, 2.0, -1.0]) / h
    M1 = h * np.array([1.0, 4.0, 1.0]) / 6.0
    return (a[0] * np.einsum("k,j,i->kji", M1, M1, K1) + a[1] * np.einsum("k,j,i->kji", M1, K1, M1)
            + a[2] * np.einsum("k,j,i->kji", K1, M1, M1))


@pytest.mark.parametrize("kind", [O.Q1_3D_KL, O.Q1_3D_DISC])
def test_constant_tensor_gives_the_closed_form_stencil(kind):
    n = 6
    h = 1.0 / (n + 1)
    rp, ci = O.pattern(kind, n)
    vals, b = O.assemble(kind, n, 4, 0.0, np.zeros(4), rp, ci)
    assert np.all(b == h ** 3)
    # xi = 0: a = a_min + ahat(0) = 0.1 + 1 everywhere
    want = stencil_closed_form((1.1, 1.0, 1.0), h)
    for p in range(n ** 3):
        i, j, l = p % n, (p // n) % n, p // (n * n)
        if min(i, j, l) == 0 or max(i, j, l) == n - 1:
            continue
        row = {int(c): v for c, v in zip(ci[rp[p]:rp[p + 1]], vals[rp[p]:rp[p + 1]])}
        assert len(row) == 27
        for dl in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    q = p + di + n * dj + n * n * dl
                    assert abs(row[q] - want[dl + 1, dj + 1, di + 1]) <= 1e-15 * 10, (p, di, dj, dl)


@pytest.mark.parametrize("kind", [O.Q1_3D_KL, O.Q1_3D_DISC])
def test_variable_field_operator_is_symmetric_spd_with_zero_interior_row_sums(kind):
    n = 5
    rp, ci = O.pattern(kind, n)
    xi = np.array([0.8, -0.6, 0.3, -0.9])
    vals, _ = O.assemble(kind, n, 4, 0.0, xi, rp, ci)
    J = n ** 3
    A = np.zeros((J, J))
    for p in range(J):
        A[p, ci[rp[p]:rp[p + 1]]] = vals[rp[p]:rp[p + 1]]
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    for p in range(J):
        i, j, l = p % n, (p // n) % n, p // (n * n)
        if 0 < i < n - 1 and 0 < j < n - 1 and 0 < l < n - 1:
            assert abs(A[p].sum()) <= 1e-13 * np.abs(A[p]).sum()


def test_test2_coefficient_jumps_where_the_radius_crosses_d4_and_d2():
    d = np.sqrt(3.0)
    x = [0.3, 0.6, 0.45]
    u = np.ones(4) / 2.0  # unit vector: r(t u) = t
    amin = 0.1
    for r0, ratio in ((d / 4, 100.0), (d / 2, 0.1)):
        lo = O.tensor(O.Q1_3D_DISC, 4, 0.0, (r0 - 1e-12) * u, x)[0, 0] - amin
        hi = O.tensor(O.Q1_3D_DISC, 4, 0.0, (r0 + 1e-12) * u, x)[0, 0] - amin
        assert hi / lo == pytest.approx(ratio, rel=1e-9)
        cont = O.tensor(O.Q1_3D_KL, 4, 0.0, (r0 + 1e-12) * u, x)[0, 0] - amin
        base = O.tensor(O.Q1_3D_KL, 4, 0.0, (r0 - 1e-12) * u, x)[0, 0] - amin
        assert cont / base == pytest.approx(1.0, rel=1e-9)  # Test 1 has no jump
