"""The C ABI builds, loads and exports every entry point include/ens.h declares,
and its host-only routines (grid bookkeeping, sizes) agree with the oracle.
CPU only: no compute call touches a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1705_02003_gb300 import build, ens, inputs, uq

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ens.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ens_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = ens.load()
    names = declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(ens.EXPORTS)


def test_build_is_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.build())


def test_create_without_gpu_fails_cleanly():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = ens.load().ens_create(ctypes.byref(h), 0)
    assert rc in (ens.ECUDA, ens.EINVAL) and not h.value


@pytest.mark.parametrize("wl", list(inputs.WORKLOADS.values()), ids=lambda w: w.name)
def test_problem_sizes_match_oracle(wl):
    p = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    kind = {"fd5": O.FD5_LOGKL, "q1": O.Q1_ROT, "fd7": O.FD7_AXIS, "q1_3d_kl": O.Q1_3D_KL,
            "q1_3d_disc": O.Q1_3D_DISC}[wl.kind]
    assert ens.ens_problem_size(p) == O.problem_size(kind, wl.n)


def test_problem_validation():
    with pytest.raises(ens.EnsError):
        ens.ens_problem_size(ens.problem("q1", 16, 3, 4.0))  # Q1 needs N = 4
    with pytest.raises(ens.EnsError):
        ens.ens_problem_size(ens.problem("fd5", 1, 2, 3.0))
    with pytest.raises(ens.EnsError):
        ens.ens_problem_size(ens.problem(9, 16, 2, 3.0))
    assert ens.load().ens_pcg_workspace_size(1024, 4992, 3, 1) == 0  # S must be a power of two


@pytest.mark.parametrize("N,L", [(1, 6), (2, 4), (4, 2), (6, 2), (8, 1)])
def test_initial_grid_bit_exact(N, L):
    a = ens.ens_sg_initial(N, L)
    b = O.sg_initial(N, L)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    np.testing.assert_array_equal(uq.coords(*a), O.sg_points(*b))


def test_grid_points_bit_exact_and_checked():
    """ens_sg_points gives the oracle's coordinates bit for bit on refined grids
    of every dimension, and refuses levels outside [0, 62]."""
    rng = np.random.default_rng(12)
    for N in (1, 2, 4, 6, 8):
        lvl, idx = O.sg_initial(N, 3 if N <= 4 else 1)
        first = 0
        for _ in range(2):
            nl, ni = O.sg_refine(lvl, idx, first, rng.standard_normal(len(lvl)), 1.0, 40)
            first = len(lvl)
            lvl, idx = np.concatenate([lvl, nl]), np.concatenate([idx, ni])
        assert np.array_equal(ens.ens_sg_points(lvl, idx), O.sg_points(lvl, idx))
    assert ens.ens_sg_points(np.zeros((0, 3), np.int8), np.zeros((0, 3), np.int32)).shape == (0, 3)
    with pytest.raises(ens.EnsError):
        ens.ens_sg_points(np.full((1, 2), -1, np.int8), np.ones((1, 2), np.int32))


def test_fp64_peak_flop_count():
    """The throughput kernel's operation count: 2 flops x 8 chains per thread
    and step, 256 threads per block."""
    assert ens.load().ens_fp64_peak_flops(3, 5) == 2 * 8 * 5 * 3 * 256


def test_refinement_bit_exact():
    rng = np.random.default_rng(9)
    for N in (2, 3, 4, 6):
        lvl, idx = O.sg_initial(N, 2)
        for trial in range(3):
            sur = rng.standard_normal(len(lvl))
            first = int(rng.integers(0, len(lvl)))
            for tau, cap in [(0.5, 10), (0.0, 3), (2.0, 10)]:
                got = ens.ens_sg_refine(lvl, idx, first, sur, tau, cap)
                want = O.sg_refine(lvl, idx, first, sur, tau, cap)
                assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_work_ratio_matches_oracle():
    rng = np.random.default_rng(10)
    for S in (1, 4, 8, 16):
        it = rng.integers(1, 500, 77).astype(np.float64)
        p = rng.permutation(77).astype(np.int32)
        assert uq.work_ratio(S, p, it) == pytest.approx(O.work_ratio(S, p, it), rel=1e-14)


def test_run_checkpoint_round_trip(tmp_path):
    """save_run / load_run keep every array bit for bit and the loop metadata."""
    from paper_1705_02003_gb300 import uq

    rng = np.random.default_rng(0)
    run = {"lvl": rng.integers(0, 4, (7, 2)).astype(np.int8), "idx": rng.integers(0, 9, (7, 2)).astype(np.int32),
           "y": rng.uniform(-1, 1, (7, 2)), "G": rng.random(7), "I": rng.integers(1, 99, 7).astype(np.float64),
           "cG": rng.standard_normal(7), "cI": rng.standard_normal(7), "levels": [(0, 4), (4, 7)],
           "perms": [np.arange(4, dtype=np.int32), np.array([2, 0, 1], np.int32)],
           "preds": [np.zeros(4), rng.random(3)], "S": 8, "grouping": "rand", "rng_seed": 5, "done": False}
    path = str(tmp_path / "ck.npz")
    uq.save_run(run, path)
    back = uq.load_run(path)
    for k in ("lvl", "idx", "y", "G", "I", "cG", "cI"):
        assert back[k].dtype == run[k].dtype and np.array_equal(back[k], run[k])
    for a, b in zip(back["perms"] + back["preds"], run["perms"] + run["preds"]):
        assert np.array_equal(a, b)
    assert back["levels"] == run["levels"] and back["S"] == 8 and back["grouping"] == "rand"
    assert back["rng_seed"] == 5 and back["done"] is False


def test_entry_points_refuse_null_arguments_without_crashing():
    """Every entry point called with a NULL handle, NULL arrays and zero sizes
    returns an error code (ens_pcg_branches and ens_pcg_cluster_size return 0
    as documented); none
    dereferences the handle or an array before checking it.  Runs on a machine
    without a GPU: the argument checks come before any CUDA call."""
    import ctypes as c

    L = ens.load()
    skip = {"ens_create", "ens_last_error", "ens_problem_size", "ens_pcg_workspace_size",
            "ens_pcg_ir_workspace_size", "ens_stream_workspace_size", "ens_adjoint_workspace_size",
            "ens_sg_refine", "ens_sg_initial", "ens_mg_workspace_size", "ens_adjoint_solve_workspace_size",
            "ens_sg_points", "ens_fp64_peak_flops"}
    for name in ens.EXPORTS:
        if name in skip:
            continue
        f = getattr(L, name)
        args = []
        for t in f.argtypes:
            if t in (c.c_int, c.c_int64, c.c_size_t):
                args.append(0)
            elif t is c.c_double:
                args.append(0.0)
            else:
                args.append(None)
        rc = f(*args)
        if name in ("ens_pcg_branches", "ens_pcg_cluster_size"):
            assert rc == 0
        else:
            assert rc < 0, name


def test_multigrid_workspace_only_for_the_trilinear_hierarchies():
    """The hierarchy exists for the trilinear problems with n = 2^k - 1; the
    size grows with the ensembles and is 0 (unsupported) otherwise."""
    f = ens.ens_mg_workspace_size
    a = f(ens.problem("q1_3d_kl", 31, 4, 0.0), 16, 2)
    assert a > 0 and f(ens.problem("q1_3d_disc", 31, 4, 0.0), 16, 2) == a
    assert f(ens.problem("q1_3d_kl", 31, 4, 0.0), 16, 4) > a
    assert f(ens.problem("q1_3d_kl", 15, 4, 0.0), 16, 2) < a
    assert f(ens.problem("q1_3d_kl", 3, 4, 0.0), 1, 1) > 0
    for bad in (ens.problem("q1_3d_kl", 30, 4, 0.0), ens.problem("q1_3d_kl", 16, 4, 0.0),
                ens.problem("fd7", 31, 6, 3.0), ens.problem("q1", 31, 4, 4.0)):
        assert f(bad, 16, 2) == 0
    assert f(ens.problem("q1_3d_kl", 31, 4, 0.0), 3, 2) == 0  # S must be a power of two
    assert f(ens.problem("q1_3d_kl", 31, 4, 0.0), 16, 2, mixed=True) > a  # plus the float copy
