"""Stopping decisions of a CG run checked against the oracle's residual history.

Section 4 records for every sample the iteration at which its residual first
meets the tolerance.  On hard samples the unpreconditioned residual ||r_k||
is not monotone near the threshold: it can dip just below rtol ||b||, rise
above it and dip again a few iterations later.  Two FP64 runs whose roundings
differ (fused multiply-adds, another summation tree) then stop at different
iterations although their residual histories agree closely; a random one-ulp
perturbation of the matrix moves the oracle itself by the same amount on
such samples.

So where a run's count differs from the oracle's, each stopping decision the
run made is checked against the oracle's residual history
rho_k = ||r_k|| / ||b||, to within the drift that FP64 rounding itself causes:
  - delta_k = DRIFT_FACTOR x the largest relative change of rho_k that
    one-ulp random perturbations of the matrix cause in the oracle's own
    history at iteration k (rounding_drift);
  - not stopping at k is consistent when rho_k >= rtol (1 - delta_k),
    stopping at k when rho_k <= rtol (1 + delta_k).
Where the counts agree nothing is relaxed."""
from __future__ import annotations

import numpy as np

DRIFT_FACTOR = 4.0
PERTURBATION_SEEDS = (0, 1, 2, 3)


def perturb(vals: np.ndarray, seed: int) -> np.ndarray:
    """vals with every entry moved by one unit in the last place (relative
    2^-52), up or down at random."""
    sgn = np.random.default_rng(seed).choice([-1.0, 1.0], len(vals))
    return vals * (1.0 + sgn * 2.0 ** -52)


def rounding_drift(hist: np.ndarray, perturbed) -> np.ndarray:
    """Per iteration k, max |rho'_k / rho_k - 1| over the perturbed histories
    rho' (each at least as long as hist)."""
    hist = np.asarray(hist, np.float64)
    return np.max([np.abs(np.asarray(p[: len(hist)]) / hist - 1.0) for p in perturbed], axis=0)


def stop_consistent(iters: int, hist: np.ndarray, rtol: float, delta) -> bool:
    """True when a run that stopped (converged) after `iters` updates made every
    stopping decision the oracle's residual history hist[k - 1] = rho_k
    (k = 1..len(hist), len(hist) >= iters) allows within a relative delta
    (a number, or one per iteration)."""
    hist = np.asarray(hist, np.float64)
    if iters > len(hist):
        raise ValueError("the history must reach the run's count")
    delta = np.broadcast_to(np.asarray(delta, np.float64), hist.shape)
    n = max(iters - 1, 0)
    went_on = bool(np.all(hist[:n] >= rtol * (1.0 - delta[:n])))
    stopped = iters == 0 or bool(hist[iters - 1] <= rtol * (1.0 + delta[iters - 1]))
    return went_on and stopped


def oracle_check(O, rowptr, colidx, vals, b, rtol: float, iters: int, iters_oracle: int):
    """(consistent, delta, history) of a run's count against the oracle's solve
    of the same system (vals, b), with delta[k - 1] = DRIFT_FACTOR x the
    oracle's own rounding drift at iteration k, up to the later of the two stops."""
    k = max(iters, iters_oracle)
    hist = O.pcg_history(rowptr, colidx, vals, b, 0.0, k)[4]
    pert = [O.pcg_history(rowptr, colidx, perturb(vals, s), b, 0.0, k)[4] for s in PERTURBATION_SEEDS]
    delta = DRIFT_FACTOR * rounding_drift(hist, pert)
    return stop_consistent(iters, hist, rtol, delta), delta, hist
