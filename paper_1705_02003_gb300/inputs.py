"""Seeded synthetic inputs and workload presets.

This module holds no arithmetic of the method: only the sizes of the five
workloads, seeded parameter draws, the random-grouping permutation and the
quantity-of-interest region.  Both the CUDA path's tests/bench and the CPU
oracle take their inputs from here.

Workloads (stand-ins for the paper's 3-D 32^3 / N = 4 anisotropic runs of
Section 4, which used no public dataset):
  fd5_32_adaptive   2-D 5-point FD, 32 x 32, N = 2, adaptive sparse grid to
                    level 4 (tau = 1e-3), S = 8
  q1_256_adaptive   2-D Q1 9-point FEM, 256 x 256, N = 4, rotated anisotropy
                    up to 10^4, adaptive sparse grid of at most 512 points, S = 16
  fd7_64_batch      3-D 7-point FD, 64^3, N = 6, 4096 uniform draws
  fd7_128_mixed     3-D 7-point FD, 128^3, N = 6, anisotropy up to 10^4,
                    1024 uniform draws, S = 32, FP32-in-FP64 refinement
  fd5_512_adjoint   2-D 5-point FD, 512 x 512, N = 8, 1024 uniform draws,
                    S = 32, QoI = mean of u over [0.4, 0.6]^2
  q1_32c_test1      the paper's own problem (Section 4, Test 1): 3-D trilinear FEM on
                    32^3 cells, exponential-covariance KL field, N = 4, adaptive
                    sparse grid from level 1, tau = 1e-3, N_max = 2000, rtol 1e-7, S = 16
  q1_32c_test2      the same with Test 2's discontinuous coefficient
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    kind: str          # "fd5" | "q1" | "fd7"
    n: int             # interior nodes per axis
    nparam: int        # N, the number of random parameters
    aniso: float       # exponent scale of the axis anisotropy 10^(aniso xi)
    S: int             # ensemble size
    rtol: float
    maxit: int
    # adaptive sparse grid (tau, initial level, level cap, sample budget)
    tau: float = 1e-3
    init_level: int = 1
    max_level: int = 64
    n_max: int = 1 << 30
    samples: int = 0   # number of uniform draws for the non-adaptive workloads
    seed: int = 0


WORKLOADS = {
    "fd5_32_adaptive": Workload("fd5_32_adaptive", "fd5", 32, 2, 3.0, 8, 1e-8, 20000,
                                tau=1e-3, init_level=1, max_level=4),
    "q1_256_adaptive": Workload("q1_256_adaptive", "q1", 256, 4, 4.0, 16, 1e-8, 50000,
                                tau=1e-3, init_level=1, n_max=512),
    "fd7_64_batch": Workload("fd7_64_batch", "fd7", 64, 6, 3.0, 32, 1e-8, 50000, samples=4096),
    "fd7_128_mixed": Workload("fd7_128_mixed", "fd7", 128, 6, 2.0, 32, 1e-10, 50000, samples=1024),
    "fd5_512_adjoint": Workload("fd5_512_adjoint", "fd5", 512, 8, 3.0, 32, 1e-8, 50000, samples=1024),
    "q1_32c_test1": Workload("q1_32c_test1", "q1_3d_kl", 31, 4, 0.0, 16, 1e-7, 50000,
                             tau=1e-3, init_level=1, n_max=2000),
    "q1_32c_test2": Workload("q1_32c_test2", "q1_3d_disc", 31, 4, 0.0, 16, 1e-7, 50000,
                             tau=1e-3, init_level=1, n_max=2000),
}


def draws(M: int, N: int, seed: int = 0) -> np.ndarray:
    """M parameter vectors xi ~ U[-1, 1]^N (numpy default_rng(seed))."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (M, N))


def rand_perm(M: int, seed: int = 0) -> np.ndarray:
    """The random-grouping permutation of M points."""
    return np.random.default_rng(seed).permutation(M).astype(np.int32)


def region_weights(n: int, dim: int) -> np.ndarray:
    """w_p = 1/|R| on the interior nodes inside R = [0.4, 0.6]^dim, else 0.

    Node p (1-based, x = p/(n+1)) is inside when 5p >= 2(n+1) and
    5p <= 3(n+1): an integer test with no rounding at the edges."""
    p = np.arange(1, n + 1)
    inside = (5 * p >= 2 * (n + 1)) & (5 * p <= 3 * (n + 1))
    m = inside.astype(np.float64)
    if dim == 2:
        w = np.outer(m, m)
    else:
        w = np.einsum("a,b,c->abc", m, m, m)
    cnt = w.sum()
    return (w / cnt).ravel()
