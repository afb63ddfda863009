"""CPU pins of the stopping-decision check (tests/stopping.py) and of the
oracle's residual history it reads."""
import numpy as np

import oracle as O
from paper_1705_02003_gb300 import inputs
from stopping import PERTURBATION_SEEDS, oracle_check, perturb, rounding_drift, stop_consistent

RTOL = 1e-8


def test_history_is_the_convergence_record():
    """The history ends where the solve stops, its last entry is the returned
    relative residual, the run is the same as or_pcg's, and with rtol = 0 the
    iteration continues past the stop with the same prefix."""
    rp, ci = O.pattern(O.FD5_LOGKL, 24)
    vals, b = O.assemble(O.FD5_LOGKL, 24, 2, 3.0, np.array([0.4, -0.7]), rp, ci)
    x0, it0, st0, rr0 = O.pcg(rp, ci, vals, b, RTOL, 5000)
    x, it, st, rr, hist = O.pcg_history(rp, ci, vals, b, RTOL, 5000)
    assert (it, st, rr) == (it0, st0, rr0) and np.array_equal(x, x0)
    assert len(hist) == it and hist[-1] == rr
    assert hist[-1] <= RTOL and np.all(hist[:-1] > RTOL)
    _, it2, st2, _, hist2 = O.pcg_history(rp, ci, vals, b, 0.0, it + 7)
    assert it2 == it + 7 and st2 == O.MAXIT
    assert np.array_equal(hist2[:it], hist)


def test_history_of_an_eigenvector_rhs_drops_to_rounding_in_one_step():
    """Constant coefficients, b = a discrete sine mode: Jacobi-PCG is exact after
    one update (the diagonal is constant), so rho_1 is at rounding level."""
    n = 16
    rp, ci = O.pattern(O.FD5_LOGKL, n)
    vals, _ = O.assemble(O.FD5_LOGKL, n, 2, 3.0, np.zeros(2), rp, ci)
    p = np.arange(1, n + 1) / (n + 1)
    b = np.outer(np.sin(2 * np.pi * p), np.sin(3 * np.pi * p)).ravel()
    _, it, st, _, hist = O.pcg_history(rp, ci, vals, b, 1e-12, 10)
    assert it == 1 and st == O.CONVERGED and hist[0] < 1e-13


def test_check_accepts_exact_and_marginal_stops_and_rejects_others():
    d = 1e-3
    # a geometric decay crossing the threshold cleanly between k = 10 and 11
    hist = RTOL * 1.5 ** (10.5 - np.arange(1, 16))
    assert stop_consistent(11, hist, RTOL, d)
    assert not stop_consistent(12, hist, RTOL, d)   # went on past a clear stop
    assert not stop_consistent(10, hist, RTOL, d)   # stopped 22 % above the threshold
    assert not stop_consistent(13, hist, RTOL, d)
    # a residual that touches the threshold within d at k = 5, rises, and
    # crosses for good at k = 8: stopping at 5 or at 8 are both consistent
    hist = RTOL * np.array([3.0, 2.0, 1.5, 1.2, 1 - d / 3, 1.015, 1.011, 0.99, 0.995, 0.9])
    assert stop_consistent(5, hist, RTOL, d)
    assert stop_consistent(8, hist, RTOL, d)
    assert not stop_consistent(6, hist, RTOL, d)    # 1.5 % above
    assert not stop_consistent(9, hist, RTOL, d)    # went on past 0.99
    assert stop_consistent(0, hist, RTOL, d)
    # with delta = 0 only the oracle's own count passes
    assert stop_consistent(5, hist, RTOL, 0.0) and not stop_consistent(8, hist, RTOL, 0.0)


def test_rounding_drift_is_small_early_and_grows():
    """The drift the check allows is measured, not chosen: one-ulp perturbations
    change the first residuals at rounding level and later ones more."""
    rp, ci = O.pattern(O.FD5_LOGKL, 32)
    vals, b = O.assemble(O.FD5_LOGKL, 32, 2, 3.0, np.array([0.9, 0.5]), rp, ci)
    hist = O.pcg_history(rp, ci, vals, b, 0.0, 120)[4]
    pert = [O.pcg_history(rp, ci, perturb(vals, s), b, 0.0, 120)[4] for s in PERTURBATION_SEEDS]
    d = rounding_drift(hist, pert)
    assert d.shape == hist.shape
    assert d[:3].max() < 1e-13 and d.max() > 1e3 * d[:3].max()
    assert np.all(rounding_drift(hist, [hist]) == 0.0)


def test_check_accepts_the_oracles_own_perturbed_runs():
    """One-ulp random perturbations of the matrix move the oracle's own count on
    some samples.  Every count of perturbations other than the ones delta is
    measured from passes the check; a count one or two off where the stop is
    clear does not."""
    wl = inputs.WORKLOADS["fd5_32_adaptive"]
    rp, ci = O.pattern(O.FD5_LOGKL, wl.n)
    xi = inputs.draws(24, wl.nparam, seed=11)
    moved = clear = 0
    for m in range(len(xi)):
        vals, b = O.assemble(O.FD5_LOGKL, wl.n, wl.nparam, wl.aniso, xi[m], rp, ci)
        _, it, _, _ = O.pcg(rp, ci, vals, b, RTOL, 20000)
        its = []
        for seed in (10, 11, 12):
            _, itp, stp, _ = O.pcg(rp, ci, perturb(vals, seed), b, RTOL, 20000)
            assert stp == O.CONVERGED
            its.append(itp)
        for itp in its:
            moved += itp != it
            ok, delta, hist = oracle_check(O, rp, ci, vals, b, RTOL, itp, it)
            assert ok, (m, it, itp, delta)
        # a count one or two off where the oracle's stop is clear is rejected
        ok, delta, hist = oracle_check(O, rp, ci, vals, b, RTOL, it + 2, it)
        if hist[it - 1] < RTOL * (1 - delta[it - 1]):
            clear += 1
            assert not ok
            for d in (-1, 1):
                assert not oracle_check(O, rp, ci, vals, b, RTOL, it + d, it)[0]
    assert moved >= 1 and clear >= len(xi) - 2


def test_count_envelope_is_narrow_on_clear_stops_and_holds_the_oracles_count():
    """The envelope always holds the unperturbed count; on a sample whose stop
    is clear it is that count alone at one ulp, and it widens with the size of
    the perturbation only where the residual near the stop is flat."""
    from stopping import count_envelope

    rp, ci = O.pattern(O.FD5_LOGKL, 32)
    for xi in (np.array([0.3, -0.2]), np.array([-0.8, 0.6])):
        vals, b = O.assemble(O.FD5_LOGKL, 32, 2, 3.0, xi, rp, ci)
        _, it, _, _ = O.pcg(rp, ci, vals, b, RTOL, 20000)
        lo, hi = count_envelope(O, rp, ci, vals, b, RTOL, 20000, 2.0 ** -52)
        assert lo <= it <= hi
        hist = O.pcg_history(rp, ci, vals, b, 0.0, it + 1)[4]
        if hist[it - 1] < 0.9 * RTOL and hist[it - 2] > 1.1 * RTOL:
            assert lo == hi == it
