"""Pins for the oracle's mixed-precision and adjoint layers (CPU only):
iterative refinement against the FP64 solve and the residual bound, and the
adjoint gradient against central finite differences of the forward map."""
import numpy as np
import pytest

import oracle as O
from paper_1705_02003_gb300 import inputs


@pytest.mark.parametrize("kind,n,N,aniso", [(O.FD7_AXIS, 10, 6, 2.0), (O.FD5_LOGKL, 24, 8, 3.0)])
def test_ir_matches_fp64_solution(kind, n, N, aniso):
    rng = np.random.default_rng(11)
    rp, ci = O.pattern(kind, n)
    for _ in range(3):
        xi = rng.uniform(-1, 1, N)
        vals, b = O.assemble(kind, n, N, aniso, xi, rp, ci)
        x64, _, st, _ = O.pcg(rp, ci, vals, b, 1e-13, 100000)
        assert st == O.CONVERGED
        x, outer, inner, st, rr = O.pcg_ir(rp, ci, vals, b, 1e-10, 1e-6, 100000, 50)
        assert st == O.CONVERGED and outer >= 2
        r = b - O.spmv(rp, ci, vals, x)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
        assert np.linalg.norm(x - x64) <= 1e-8 * np.linalg.norm(x64)


@pytest.mark.parametrize("kind,n,N,aniso", [(O.FD5_LOGKL, 15, 8, 3.0), (O.FD7_AXIS, 6, 6, 3.0)])
def test_adjoint_gradient_matches_central_differences(kind, n, N, aniso):
    rng = np.random.default_rng(12)
    w = O.region_weights(n, 3 if kind == O.FD7_AXIS else 2)
    assert w.sum() == pytest.approx(1.0)
    for _ in range(2):
        xi = rng.uniform(-0.9, 0.9, N)
        Q, g, itf, ita, st = O.adjoint_grad(kind, n, N, aniso, xi, w, 1e-13, 100000)
        assert st == O.CONVERGED
        h = 1e-6
        pts = []
        for k in range(N):
            for s in (1, -1):
                e = xi.copy()
                e[k] += s * h
                pts.append(e)
        out = O.solve_batch(kind, n, N, aniso, np.array(pts), 1e-13, 100000, nthreads=4, want_x=True)
        Qs = out["x"] @ w
        gfd = (Qs[0::2] - Qs[1::2]) / (2 * h)
        assert np.all(np.abs(g - gfd) <= 1e-6 * np.maximum(1.0, np.abs(gfd))), (g, gfd)
        # the region mean really is Q
        out0 = O.solve_batch(kind, n, N, aniso, xi[None], 1e-13, 100000, want_x=True)
        assert Q == pytest.approx(float(out0["x"][0] @ w), rel=1e-12)


def test_region_weights_select_the_square():
    """The oracle's weights: the support is the set of nodes in [0.4, 0.6]^d by
    exact rational coordinates (checked here with fractions, including meshes
    where a node sits exactly on 0.4 or 0.6), the weights sum to one, and the
    input module's weights, which the GPU side receives, are the same bits."""
    from fractions import Fraction

    for n, dim in ((49, 2), (24, 2), (9, 3), (14, 3), (512, 2)):
        w = O.region_weights(n, dim)
        x = [Fraction(i, n + 1) for i in range(1, n + 1)]
        inside = np.array([Fraction(2, 5) <= xi <= Fraction(3, 5) for xi in x])
        want = np.outer(inside, inside) if dim == 2 else np.einsum("a,b,c->abc", inside, inside, inside)
        # node order x fastest: w[j] with j = i0 + n i1 (+ n^2 i2) -> array index [i_last, ..., i0]
        assert np.array_equal(w.reshape((n,) * dim) > 0, want.T if dim == 2 else want.transpose(2, 1, 0))
        assert abs(w.sum() - 1.0) < 1e-12
        assert np.array_equal(w, inputs.region_weights(n, dim))
    assert 5 * 4 == 2 * (9 + 1) and 5 * 6 == 3 * (9 + 1)  # n = 9: nodes 4 and 6 sit on 0.4 and 0.6
