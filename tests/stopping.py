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
PERTURBATION_SEEDS = (0, 1, 2, 3, 4, 5)


def perturb(vals: np.ndarray, seed: int, scale: float = 2.0 ** -52) -> np.ndarray:
    """vals with every entry moved by the relative amount scale (by default one
    unit in the last place), up or down at random."""
    sgn = np.random.default_rng(seed).choice([-1.0, 1.0], len(vals))
    return vals * (1.0 + sgn * scale)


def rounding_drift(hist: np.ndarray, perturbed) -> np.ndarray:
    """Per iteration k, max |rho'_k / rho_k - 1| over the perturbed histories
    rho' (each at least as long as hist)."""
    hist = np.asarray(hist, np.float64)
    if any(len(p) < len(hist) for p in perturbed):
        raise ValueError("a perturbed run stopped early (breakdown): no drift to measure")
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


def oracle_check(O, rowptr, colidx, vals, b, rtol: float, iters: int, iters_oracle: int,
                 scale: float = 2.0 ** -52):
    """(consistent, delta, history) of a run's count against the oracle's solve
    of the same system (vals, b), with delta[k - 1] = DRIFT_FACTOR x the drift
    that perturbations of the matrix by the relative amount scale (one ulp when
    both sides solve the same matrix; the assembly bar when each side assembles
    its own) cause in the oracle's history at iteration k, up to the later of
    the two stops."""
    k = max(iters, iters_oracle)
    hist = O.pcg_history(rowptr, colidx, vals, b, 0.0, k)[4]
    pert = [O.pcg_history(rowptr, colidx, perturb(vals, s, scale), b, 0.0, k)[4] for s in PERTURBATION_SEEDS]
    delta = DRIFT_FACTOR * rounding_drift(hist, pert)
    return stop_consistent(iters, hist, rtol, delta), delta, hist


def count_envelope(O, rowptr, colidx, vals, b, rtol: float, maxit: int, scale: float,
                   seeds=tuple(range(10, 22))):
    """(lowest, highest) count of the oracle's solve of (vals, b) and of its
    solves of the matrix perturbed by the relative amount scale, one per seed.
    Where each side assembles its own matrix (differences up to the assembly
    bar) and the residual near the stop is chaotic, a count inside this
    envelope widened by one is what the oracle itself would give for a matrix
    that close to its own."""
    counts = [O.pcg(rowptr, colidx, vals, b, rtol, maxit)[1]]
    counts += [O.pcg(rowptr, colidx, perturb(vals, s, scale), b, rtol, maxit)[1] for s in seeds]
    return min(counts), max(counts)
