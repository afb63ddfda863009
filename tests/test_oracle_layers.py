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
    w = inputs.region_weights(n, 3 if kind == O.FD7_AXIS else 2)
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
    n = 49
    w = inputs.region_weights(n, 2).reshape(n, n)
    x = (np.arange(n) + 1) / (n + 1)
    inside = (x >= 0.4 - 1e-12) & (x <= 0.6 + 1e-12)
    assert np.array_equal(w > 0, np.outer(inside, inside))
