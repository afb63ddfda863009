"""Benchmark: sample-solves/s of the surrogate-grouped ensemble PCG.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload q1_256_adaptive] [--no-arms] [--no-cpu]
                    [--suite layers,configs,c1,pilot,paper,mixed-mg | all]
                    [--detail-out PATH]
                    [--kernel-only [--kernel-ensembles E]] [--mg-once mg|mg32] [--ir-once]

A step is one pass of the whole path over the workload: the grid-generation
and grouping loop of the paper's flowchart (initial sparse grid, then per
level: surrogate grouping (K6, K7), ensemble assembly (K1), ensemble Jacobi-PCG
(K2-K4) to rel. residual 1e-8, QoI, surpluses and host refinement) until the
sample budget is reached.  value = samples solved / device time (CUDA events
around K steps, max over ranks).

The LAST line on stdout is one compact JSON object: metric, value, config,
roofline of the dominant kernel (K2, against the FP64 issue rate measured in
the same run, with the HBM view beside it), cpu_baseline, e2e, clocks and the
speed-up over per-sample PCG, both one sample at a time and as a batch of
one-lane ensembles (on this problem the batch is the faster of the two, and
faster than the ensemble: the path is bound by FP64 issue, not by memory).
Everything else goes to the detail
file (--detail-out, default <tmpdir>/ens_bench_detail.json):
  arms            parameter-based, natural and random grouping; one sample per
                  call (serial) and all samples of a level in one call at S = 1
                  (batched); the surrogate groups with lane re-packing -- each
                  as sample-solves/s and as a fraction of its HBM roofline and
                  of its path roofline (HBM and FP64)
  R, R_levels     the work ratio of Eq. (R) overall and per level
  level_calls     each level's solve call: size, ensembles, branches, time
and, with --suite:
  layers          FP32-in-FP64 refinement on 1024 draws of 128^3, streamed
                  batching of all 4096 draws of 64^3, the adjoint gradient of
                  1024 draws of 512^2, each with per-sample errors against the
                  oracle on a stated subset
  configs         K2 on the 7-point 64^3 / 128^3 and 5-point 512^2 problems
  c1              the 32^2 5-point workload with its four arms
  pilot           surrogate grouping of a non-adaptive sample set (Section 5)
  paper           Section 4's Test 1 / Test 2 (32^3 trilinear FEM, N = 4) with
                  the Jacobi and the multigrid preconditioner
  mixed-mg        the multigrid solve with a float V-cycle on Test 1 / Test 2

--kernel-only times K2 alone, --mg-once runs one multigrid solve and --ir-once
one mixed-precision refinement solve (the cases the Nsight Compute summaries use).
--impl reference times the CPU oracle (the reference arm of this project) on
the host cores for the same metric.  Multi-GPU runs are independent replicas
that time the loop only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sample-solves/s at rel-res 1e-8: ensemble PCG vs per-sample PCG; SpMV HBM GB/s"

# The FP64 roof from unit counts (context beside the measured one): 152 SMs x
# 2 FP64 fused multiply-adds per clock x 2.07 GHz.
FP64_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# DRAM bytes (read + write) of one K2 launch on the Q1 256^2 problem at S = 16,
# per ensemble, from an Nsight Compute capture of E = 8 ensembles (0.674 GB
# read, 0.038 GB written); a full-capacity launch scales it by E.
SPMV_TRAFFIC_PER_ENSEMBLE = {"q1_256_adaptive": (673.564160e6 + 38.298368e6) / 8}

N_MAX_READING = ("levels of 48, 58 and 159 points; a level that would take the grid past N_max = 512 "
                 "is not admitted (the fourth would)")


def spmv_traffic(wl, E):
    t = SPMV_TRAFFIC_PER_ENSEMBLE.get(wl.name)
    return None if t is None else t * E


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def replica_rate(pg, world: int, samples: int, t_local: float):
    """Whole-job rate of `world` independent replicas, each of which solved
    `samples` samples in t_local seconds: the slowest rank bounds the job.
    Returns (samples per second over all ranks, the slowest rank's seconds)."""
    tmax = allmax(pg, t_local)
    return world * samples / tmax, tmax


def allmax(pg, v):
    if pg is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def timed(stream, fn):
    """(fn(), seconds) with CUDA events on `stream`, synchronised on both sides."""
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1) / 1e3


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
OKINDS = {"fd5": 1, "q1": 2, "fd7": 3}


def oracle_rate(wl, points: np.ndarray, threads: int):
    import oracle as O

    t0 = time.perf_counter()
    out = O.solve_batch(OKINDS[wl.kind], wl.n, wl.nparam, wl.aniso, points, wl.rtol, wl.maxit, nthreads=threads)
    dt = time.perf_counter() - t0
    assert np.all(out["status"] == O.CONVERGED)
    return len(points) / dt, dt, out


def oracle_sample_points(wl, count: int):
    """A bounded, deterministic sample of the workload's points: every k-th
    point of the full sparse grid of the workload's dimension (levels 0..3),
    generated by the oracle's own sparse-grid routines."""
    import oracle as O

    lvl, idx = O.sg_initial(wl.nparam, 3)
    y = O.sg_points(lvl, idx)
    step = max(1, len(y) // count)
    return y[::step][:count]


def run_reference(args, wl):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    pts = oracle_sample_points(wl, args.ref_samples)
    for _ in range(args.warmup):
        oracle_rate(wl, pts[: max(1, threads)], threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rate(wl, pts, threads)
    dt = time.perf_counter() - t0
    value = len(pts) * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sample-solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "kind": wl.kind, "n": wl.n, "N": wl.nparam, "rtol": wl.rtol,
                   "sample": f"{len(pts)} sparse-grid points per step"},
        "cpu_baseline": {"value": value, "unit": "sample-solves/s", "cores": threads, "kind": "oracle",
                         "sample": f"{len(pts)} points of the level-3 sparse grid, one sample per thread"},
        "e2e": {"value": value, "unit": "sample-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm: roofline helpers
# ---------------------------------------------------------------------------
def measure_fp64_peak(h, stream, reps: int = 5):
    """The FP64 fused multiply-add rate of this GPU (TFLOP/s, best of reps),
    from the throughput kernel ens_fp64_peak on every SM at full occupancy."""
    import torch

    from paper_1705_02003_gb300 import ens

    blocks, iters = 152 * 8, 4096
    sink = torch.zeros(blocks, dtype=torch.float64, device="cuda")
    for _ in range(2):
        ens.ens_fp64_peak(h, blocks, iters, sink, stream)
    best = float("inf")
    flops = 0.0
    for _ in range(reps):
        flops, t = timed(stream, lambda: ens.ens_fp64_peak(h, blocks, iters, sink, stream))
        best = min(best, t)
    return flops / best / 1e12


def b_alg(nnz: int, J: int, S: int) -> float:
    """Algorithmic bytes per sample per FP64 Jacobi-PCG iteration: values,
    nine vector streams (x r/w, r r/w, p r/w, q w+r, D^-1 r) and the graph
    shared by the S lanes of an ensemble."""
    return 8 * nnz + 72 * J + (4 * nnz + 4 * (J + 1)) / S


def charged_iterations(I: np.ndarray, groups) -> float:
    """Sample-iterations an ensemble schedule streams: every lane of an
    ensemble runs until its slowest lane stops.  groups = list of index arrays."""
    return float(sum(len(g_) and I[g_].max() * len(g_) for g_ in groups))


def roof_fracs(value, M, charged, nnz, J, S, hbm_gbs, fp64_tflops):
    """value as a fraction of the HBM roofline M / (charged B_alg / HBM) and of
    the path roofline, which also bounds each sample-iteration by its FP64
    work (nnz + 7 J fused multiply-adds: K2 nnz + J, K3 5 J, K4 J)."""
    ba = b_alg(nnz, J, S)
    t_hbm = ba / (hbm_gbs * 1e9)
    t_fp = 2.0 * (nnz + 7 * J) / (fp64_tflops * 1e12)
    hbm_roof = M / (charged * t_hbm)
    path_roof = M / (charged * max(t_hbm, t_fp))
    return {"hbm_roof": hbm_roof, "hbm_frac": value / hbm_roof, "path_roof": path_roof,
            "path_frac": value / path_roof, "sample_iterations_charged": charged, "bytes_per_sample_iteration": ba}


def level_groups(run, S):
    """Index arrays of the ensembles of every level of a run (global point indices)."""
    out = []
    for (a, b), perm in zip(run["levels"], run["perms"]):
        perm = np.asarray(perm)
        for k in range(0, b - a, S):
            out.append(a + perm[k:k + S])
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_arms(h, wl, ad, run, value, stream, hbm, fp64):
    """The comparison arms of the headline workload, one step each."""
    from paper_1705_02003_gb300.uq import Adaptive, ratios

    sol = ad.solver
    M = len(run["I"])
    J, nnz, S = sol.J, sol.nnz, sol.S
    arms = {"sur": {"value": value, "R": ratios(run)["run"][1],
                    **roof_fracs(value, M, charged_iterations(run["I"], level_groups(run, S)), nnz, J, S, hbm, fp64)}}
    for arm in ("par", "nat", "rand"):
        r2, ta = timed(stream, lambda: ad.run(arm, seed=0))
        Ra = ratios(r2)["run"]
        v = M / ta
        arms[arm] = {"value": v, "R": Ra[1], "R_levels": Ra[0],
                     **roof_fracs(v, M, charged_iterations(r2["I"], level_groups(r2, S)), nnz, J, S, hbm, fp64)}
    # one sample per call (S = 1, E = 1), serially: the same kernels, one solve at a time
    ps = Adaptive(h, wl, per_sample=True)
    ps.run("nat")  # warm-up (graph instantiation)
    r3, tp = timed(stream, lambda: ps.run("nat"))
    v = M / tp
    arms["per_sample_serial"] = {
        "value": v, "max_iter_diff_vs_ensemble": int(np.max(np.abs(r3["I"] - run["I"]))),
        **roof_fracs(v, M, float(r3["I"].sum()), nnz, J, 1, hbm, fp64)}
    del ps
    # one sample per lane, all samples of a level in one call (S = 1, E = M)
    pb = Adaptive(h, wl, S=1)
    pb.run("nat")  # warm-up
    r5, tb = timed(stream, lambda: pb.run("nat"))
    v = M / tb
    arms["per_sample_batched"] = {
        "value": v, "max_iter_diff_vs_ensemble": int(np.max(np.abs(r5["I"] - run["I"]))),
        "max_iter_diff_vs_serial": int(np.max(np.abs(r5["I"] - r3["I"]))),
        **roof_fracs(v, M, float(r5["I"].sum()), nnz, J, 1, hbm, fp64)}
    del pb
    # the same surrogate groups, each level solved through the batching layer
    # (live lanes of partly converged ensembles re-packed every 64 trips)
    rp = Adaptive(h, wl, solver=ad.solver, repack=True)
    rp.run("sur")  # warm-up
    r4, tr = timed(stream, lambda: rp.run("sur"))
    arms["sur_repack"] = {"value": M / tr, "same_grid": bool(np.array_equal(r4["lvl"], run["lvl"])),
                          "same_iterations": bool(np.array_equal(r4["I"], run["I"]))}
    del rp
    for k in ("per_sample_serial", "per_sample_batched"):
        arms["sur"][f"speedup_vs_{k}"] = value / arms[k]["value"]
    return arms


def spmv_launch(h, sol, E, xi_all, stream, reps=20):
    """CUDA-event time of one K2 launch (ens_spmv) on E ensembles of the solver's
    problem, inputs larger than L2."""
    import torch

    from paper_1705_02003_gb300 import ens

    ens.ens_assemble(h, sol.prob, sol.S, E, xi_all.reshape(-1).contiguous(), sol.rowptr, sol.colidx, sol.vals,
                     sol.dinv, sol.b)
    q = torch.empty_like(sol.x)
    pq = torch.empty(E * sol.S, dtype=torch.float64, device="cuda")
    call = lambda: ens.ens_spmv(h, sol.J, sol.nnz, sol.S, E, sol.rowptr, sol.colidx, sol.vals, sol.b, q, pq,
                                sol.work, stream)
    for _ in range(3):
        call()

    def many():
        for _ in range(reps):
            call()

    _, t = timed(stream, many)
    del q, pq
    return t / reps


def run_ours(args, wl):
    import torch

    from paper_1705_02003_gb300 import ens
    from paper_1705_02003_gb300.uq import Adaptive, ratios

    world, rank, local, pg = dist_setup(args)
    if world > 1:
        # N independent replicas: only the timed loop runs on every GPU; the
        # single-GPU diagnostics (arms, suites) are N = 1 work
        args.no_arms = True
        args.suite = ""
    torch.cuda.set_device(local)
    h = ens.Handle(local)
    stream = torch.cuda.current_stream()
    ad = Adaptive(h, wl)

    # warm-up (also fixes the grid: it does not depend on the grouping)
    for _ in range(max(args.warmup, 1)):
        run = ad.run("sur")
    torch.cuda.synchronize()
    M = len(run["I"])
    launches_per_step = ad.kernel_launches(run["I"])

    clocks = ClockSampler(local)
    clocks.start()
    barrier(pg)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        run = ad.run("sur")
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    clk = clocks.stop()
    t = ev0.elapsed_time(ev1) / 1e3
    value, tmax = replica_rate(pg, world, M * args.steps, t)
    R = ratios(run)
    sol = ad.solver
    hbm, hbm_kind = peaks()
    fp64 = measure_fp64_peak(h, stream)

    detail = {"workload": wl.name, "value": value, "unit": "sample-solves/s",
              "R": {"sur": R["run"][1], "its": R["its"][1]},
              "R_levels": {"sur": R["run"][0], "its": R["its"][0], "points": [b - a for a, b in run["levels"]]},
              "peaks": {"hbm_gbs": hbm, "hbm_source": hbm_kind, "fp64_tflops_measured": fp64,
                        "fp64_tflops_derived": FP64_DERIVED_TFLOPS}}
    if not args.no_arms:
        detail["arms"] = run_arms(h, wl, ad, run, value, stream, hbm, fp64)

    # per solve call (one per level): size, branches and time, from one more step
    ad.time_calls = True
    rl = ad.run("sur")
    ad.time_calls = False
    level_calls = []
    for (M_c, ms), pts in zip(ad.call_times(), ad.solve_sets):
        it = rl["I"][pts]
        E_c = -(-M_c // ad.S)
        charged_c = ad.S * sum(float(it[k:k + ad.S].max()) for k in range(0, M_c, ad.S))
        level_calls.append({"M": M_c, "E": E_c, "branches": ens.ens_pcg_branches(h, E_c),
                            "max_iters": int(it.max()), "ms": ms,
                            "ps_per_row_lane_iteration": ms * 1e9 / (charged_c * sol.J)})
    detail["level_calls"] = level_calls

    # dominant kernel: the ensemble SpMV (K2) on a full-capacity batch
    E = sol.Emax
    L = E * sol.S
    xi_all = torch.from_numpy(run["y"][:L] if len(run["y"]) >= L else np.resize(run["y"], (L, wl.nparam))).to("cuda")
    t_spmv = spmv_launch(h, sol, E, xi_all, stream)
    spmv_bytes = E * (8 * sol.nnz * sol.S + 4 * sol.nnz + 4 * (sol.J + 1) + 16 * sol.J * sol.S)
    spmv_fma = E * sol.S * (sol.nnz + sol.J)  # one fused multiply-add per nonzero-lane, one per row-lane for p^T q
    achieved = spmv_bytes / t_spmv / 1e9
    tflops = 2.0 * spmv_fma / t_spmv / 1e12
    roofline = {"bound": "alu", "achieved": tflops, "peak": fp64, "unit": "TFLOP/s", "frac": tflops / fp64,
                "traffic": spmv_traffic(wl, E), "kernel": f"k_spmv (K2), FP64, E={E} S={sol.S}",
                "peak_source": "measured FP64 FMA rate (ens_fp64_peak, this run)",
                "hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "peak_source": hbm_kind}}
    detail["spmv"] = {"E": E, "bytes_per_launch": spmv_bytes, "fma_per_launch": spmv_fma, "launch_ms": t_spmv * 1e3,
                      "fp64_frac_of_derived": tflops / FP64_DERIVED_TFLOPS}
    path = roof_fracs(value, M, charged_iterations(run["I"], level_groups(run, sol.S)), sol.nnz, sol.J, sol.S,
                      hbm, fp64)
    detail["path"] = path

    # end to end through the public API with host buffers: the loop copies each
    # level's points in and its surpluses out; in addition every solve's
    # solution fields u (all samples) go to pinned host memory, and the
    # per-sample G, I and surpluses come back at the end of the step
    host_u = torch.empty(max(M, sol.S) * sol.J + sol.Emax * sol.S * sol.J, dtype=torch.float64, pin_memory=True)
    moved = {"d2h": 0}
    cursor = {"at": 0}

    def sink(s_, m):
        E_ = math.ceil(m / s_.S)
        n = E_ * s_.J * s_.S
        if cursor["at"] + n > host_u.numel():
            cursor["at"] = 0
        host_u[cursor["at"]:cursor["at"] + n].copy_(s_.x[:n], non_blocking=True)
        cursor["at"] += n
        moved["d2h"] += 8 * n

    ad.sink = sink
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cursor["at"] = 0
        ad.run("sur")
        torch.cuda.synchronize()
    te = time.perf_counter() - t0
    ad.sink = None
    N_ = wl.nparam
    h2d = int(M * N_ * (8 + 1 + 4))                      # point coordinates, levels, indices
    d2h = int(moved["d2h"] / args.steps) + int(M * 8 * 2 + M * 8 * 4)  # u fields, surpluses, G/I/cG/cI
    e2e = {"value": world * M * args.steps / allmax(pg, te), "unit": "sample-solves/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        pts = run["y"][:: max(1, M // args.cpu_samples)][: args.cpu_samples]
        rate, dt, _ = oracle_rate(wl, pts, threads)
        rate1, dt1, _ = oracle_rate(wl, pts[:2], 1)  # the same solver on one core
        cpu = {"value": rate, "unit": "sample-solves/s", "cores": threads, "kind": "oracle",
               "sample": f"{len(pts)} of the {M} grid points, one per thread, {dt:.1f} s"}
        detail["cpu_baseline"] = dict(cpu, single_core_value=rate1,
                                      single_core_sample=f"the first 2 of those points, {dt1:.1f} s")

    if rank == 0 and args.suite:
        detail["suites"] = run_suites(h, stream, args.suite, hbm, fp64)

    h.close()
    if rank == 0:
        detail_path = args.detail_out or os.path.join(tempfile.gettempdir(), "ens_bench_detail.json")
        try:
            os.makedirs(os.path.dirname(os.path.abspath(detail_path)), exist_ok=True)
            with open(detail_path, "w") as fh:
                json.dump(detail, fh, indent=1, default=float)
        except OSError as e:
            detail_path = f"not written ({e})"
        line = compact_line(value=value, world=world, args=args, tmax=tmax, wl=wl, sol=sol, M=M,
                            levels=len(run["levels"]), roofline=roofline, cpu=cpu, e2e=e2e,
                            launches=launches_per_step * args.steps, clocks=clk, path_frac=path["path_frac"],
                            arms=detail.get("arms", {}), detail_path=detail_path)
        print(json.dumps(line, separators=(",", ":")))
    return 0


def compact_line(value, world, args, tmax, wl, sol, M, levels, roofline, cpu, e2e, launches, clocks, path_frac,
                 arms, detail_path):
    """The one JSON object printed last: the measured metric with its config,
    the dominant kernel's roofline, the CPU baseline, the end-to-end figure and
    the clocks (everything else is in the detail file)."""
    return {
        "metric": METRIC, "value": value, "unit": "sample-solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "problem": "Q1 9-point FEM 256x256, N=4, rotated anisotropy",
                   "J": sol.J, "nnz": sol.nnz, "S": sol.S, "samples_per_step": M,
                   "levels": levels, "n_max": wl.n_max, "n_max_reading": N_MAX_READING,
                   "rtol": wl.rtol, "grouping": "sur", "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (each level's values >= 225 MB)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clocks,
        "path_frac": path_frac,
        "speedup_vs_per_sample": {k: arms["sur"][f"speedup_vs_{k}"]
                                  for k in ("per_sample_serial", "per_sample_batched")} if arms else None,
        "detail": detail_path,
    }


def run_suites(h, stream, suite: str, hbm: float, fp64: float):
    names = ["layers", "configs", "c1", "pilot", "paper", "mixed-mg"] if suite == "all" else \
        [s for s in suite.split(",") if s]
    out = {}
    for name in names:
        t0 = time.perf_counter()
        if name == "layers":
            out[name] = run_layers(h, stream)
        elif name == "configs":
            out[name] = run_configs(h, stream, hbm, fp64)
        elif name == "c1":
            out[name] = run_c1(h, stream, hbm, fp64)
        elif name == "pilot":
            out[name] = run_pilot(h, stream)
        elif name == "paper":
            out[name] = run_paper(h, stream)
        elif name == "mixed-mg":
            out[name] = run_mixed_mg(h, stream)
        else:
            raise ValueError(f"unknown suite {name}")
        out[name]["suite_seconds"] = time.perf_counter() - t0
        sys.stderr.write(f"suite {name}: {out[name]['suite_seconds']:.1f} s\n")
    return out


def run_configs(h, stream, hbm: float, fp64: float):
    """The ensemble SpMV (K2) on the other problem configurations, in the launch
    shapes of their layers (the 64^3 and 512^2 problems with 1024 lanes, the
    128^3 problem with 8 ensembles per call) and with one ensemble, each with
    inputs larger than L2: algorithmic GB/s and FP64 rate per launch."""
    import torch

    from paper_1705_02003_gb300 import ens, inputs
    from paper_1705_02003_gb300.solver import EnsembleSolver

    out = {}
    for name, E in (("fd7_64_batch", 32), ("fd7_128_mixed", 8), ("fd5_512_adjoint", 32), ("fd7_64_batch", 1),
                    ("fd7_128_mixed", 1), ("fd5_512_adjoint", 1)):
        wl = inputs.WORKLOADS[name]
        prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
        S = 32
        sol = EnsembleSolver(h, prob, S, E * S, wl.rtol, wl.maxit)
        xi = torch.from_numpy(inputs.draws(E * S, wl.nparam, seed=wl.seed)).cuda()
        t = spmv_launch(h, sol, E, xi, stream, reps=10)
        byts = E * (8 * sol.nnz * S + 4 * sol.nnz + 4 * (sol.J + 1) + 16 * sol.J * S)
        fma = E * S * (sol.nnz + sol.J)
        out[f"{name}_E{E}"] = {"E": E, "S": S, "bytes_per_launch": byts, "launch_ms": t * 1e3,
                     "hbm_gbs": byts / t / 1e9, "hbm_frac": byts / t / 1e9 / hbm,
                     "fp64_tflops": 2 * fma / t / 1e12, "fp64_frac": 2 * fma / t / 1e12 / fp64}
        del sol
        torch.cuda.empty_cache()
    out["peaks"] = {"hbm_gbs": hbm, "fp64_tflops_measured": fp64}
    return out


def run_c1(h, stream, hbm: float, fp64: float):
    """The 32 x 32 5-point workload (adaptive grid to level 4, S = 8): its four
    arms (surrogate, natural, random grouping, one sample per call) and R."""
    from paper_1705_02003_gb300 import inputs
    from paper_1705_02003_gb300.uq import Adaptive, ratios

    wl = inputs.WORKLOADS["fd5_32_adaptive"]
    ad = Adaptive(h, wl)
    ad.run("sur")
    out = {"workload": wl.name}
    ref = None
    for arm in ("sur", "nat", "rand"):
        ad.run(arm, seed=0)  # warm-up
        r, t = timed(stream, lambda: ad.run(arm, seed=0))
        ref = r if ref is None else ref
        M = len(r["I"])
        out[arm] = {"value": M / t, "R": ratios(r)["run"][1],
                    **roof_fracs(M / t, M, charged_iterations(r["I"], level_groups(r, wl.S)), ad.solver.nnz,
                                 ad.solver.J, wl.S, hbm, fp64)}
    ps = Adaptive(h, wl, per_sample=True)
    ps.run("nat")
    r, t = timed(stream, lambda: ps.run("nat"))
    M = len(r["I"])
    out["per_sample_serial"] = {"value": M / t, "max_iter_diff_vs_ensemble": int(np.max(np.abs(r["I"] - ref["I"]))),
                                **roof_fracs(M / t, M, float(r["I"].sum()), ad.solver.nnz, ad.solver.J, 1, hbm, fp64)}
    pb = Adaptive(h, wl, S=1)  # one sample per lane, a level per call
    pb.run("nat")
    r, t = timed(stream, lambda: pb.run("nat"))
    out["per_sample_batched"] = {"value": M / t, "max_iter_diff_vs_ensemble": int(np.max(np.abs(r["I"] - ref["I"]))),
                                 **roof_fracs(M / t, M, float(r["I"].sum()), ad.solver.nnz, ad.solver.J, 1, hbm,
                                              fp64)}
    # the same surrogate arm with every solve on the three-kernel graph loop
    # instead of the one-launch cluster schedule (identical results)
    import torch

    from paper_1705_02003_gb300 import ens

    out["cluster_ctas"] = ens.ens_pcg_cluster_size(h, ad.solver.J, ad.solver.nnz, wl.S, 4)
    prev = os.environ.get("ENS_PCG_FUSED")
    os.environ["ENS_PCG_FUSED"] = "0"
    try:
        hl = ens.Handle(torch.cuda.current_device())
    finally:
        if prev is None:
            del os.environ["ENS_PCG_FUSED"]
        else:
            os.environ["ENS_PCG_FUSED"] = prev
    al = Adaptive(hl, wl)
    al.run("sur")
    rl, tl = timed(stream, lambda: al.run("sur"))
    out["sur_graph_loop"] = {"value": len(rl["I"]) / tl, "same_counts": bool(np.array_equal(rl["I"], ref["I"])),
                             "same_G": bool(np.array_equal(rl["G"], ref["G"]))}
    hl.close()
    out["points"] = M
    out["note"] = ("each solve is one cluster launch with its state in shared memory: latency-bound, roofline "
                   "fractions are HBM's")
    return out


def run_pilot(h, stream):
    """Surrogate grouping of a non-adaptive sample set (Section 5): the level-1
    sparse grid of the 64^3 problem (256 points) is solved and its iteration
    surrogate groups 512 of the 4096 uniform draws; surrogate order against
    generation order, and R for S = 8..64 from the draws' iteration counts."""
    import torch

    from paper_1705_02003_gb300 import ens, inputs, uq
    from paper_1705_02003_gb300.solver import EnsembleSolver

    wl = inputs.WORKLOADS["fd7_64_batch"]
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    S, M = 32, 512
    sol = EnsembleSolver(h, prob, S, M, wl.rtol, wl.maxit)
    pg = uq.PilotGrouping(h, sol, level=1)
    _, t_pilot = timed(stream, pg.build)
    xi = torch.from_numpy(inputs.draws(wl.samples, wl.nparam, seed=wl.seed)[:M]).cuda()
    (pred, perm, _), t_group = timed(stream, lambda: pg.group(xi, S))
    order = perm.to(torch.int64)
    sol.solve(xi)  # warm-up (graph instantiation)
    (it_nat, *_), t_nat = timed(stream, lambda: sol.solve(xi))
    it_nat = it_nat.cpu().numpy().astype(np.float64)
    (it_sur, *_), t_sur = timed(stream, lambda: sol.solve(xi.index_select(0, order)))
    p = perm.cpu().numpy()
    R = {}
    for s_ in (8, 16, 32, 64):
        R[s_] = {"sur": uq.work_ratio(s_, p, it_nat), "nat": uq.work_ratio(s_, np.arange(M), it_nat),
                 "its": uq.work_ratio(s_, np.argsort(it_nat, kind="stable"), it_nat)}
    return {"workload": wl.name, "pilot_points": len(pg.lvl), "draws": M, "S": S,
            "pilot_seconds": t_pilot, "group_seconds": t_group,
            "sur_value": M / t_sur, "nat_value": M / t_nat, "unit": "sample-solves/s",
            "speedup_sur_vs_nat": t_nat / t_sur, "R": R,
            "same_iterations": bool(np.array_equal(np.sort(it_sur.cpu().numpy()), np.sort(it_nat)))}


def run_paper(h, stream, S_list=(4, 8, 16, 32)):
    """Section 4's Tables 2 and 3 on the GPU path.  For Test 1 and Test 2
    (32^3 trilinear FEM, N = 4, adaptive grid from level 1, tau = 1e-3,
    N_max = 2000, CG to a relative residual of 1e-7), each with the Jacobi
    preconditioner and with the multigrid V-cycle (ens_mgpcg_solve): R_l per
    level and R (Eqs. Rl and R) of the surrogate (sur), parameter (par),
    generation-order (nat) and iteration-sorted (its) groupings at S = 4..32;
    the measured speed-up = the time of all solve calls made one sample at a
    time / the time of all ensemble solve calls; and the predicted speed-up =
    sigma(S) / R, where sigma(S) is the speed-up the same kernels reach when
    every sample takes the same iterations (512 copies of the median-iteration
    sample in one call against one solve of it, times 512)."""
    import torch

    from paper_1705_02003_gb300 import inputs
    from paper_1705_02003_gb300.uq import Adaptive, ratios

    def solve_ms(ad):
        return sum(ms for _, ms in ad.call_times())

    out = {}
    for name in ("q1_32c_test1", "q1_32c_test2"):
        wl = inputs.WORKLOADS[name]
        out[name] = {}
        for pc in ("jacobi", "mg"):
            seq = Adaptive(h, wl, per_sample=True, precond=pc)
            y0 = torch.zeros(1, wl.nparam, dtype=torch.float64, device="cuda")
            seq.solver.solve(y0)  # warm-up (graph instantiation)
            seq.time_calls = True
            r0 = seq.run("nat")
            t_seq = solve_ms(seq)
            # the equal-iteration case uses the sample of median iteration count,
            # so that its fixed per-call cost weighs as in a typical solve
            j_med = int(np.argsort(r0["I"], kind="stable")[len(r0["I"]) // 2])
            y_med = torch.from_numpy(r0["y"][j_med:j_med + 1].copy()).to("cuda")
            seq.call_events = []
            for _ in range(5):
                seq._call(y_med)
            t1 = float(np.median([ms for _, ms in seq.call_times()]))
            del seq
            res = {"points": len(r0["I"]), "levels": [b - a for a, b in r0["levels"]],
                   "iters_min": int(r0["I"].min()), "iters_max": int(r0["I"].max()),
                   "iters_mean": float(r0["I"].mean()), "sequential_solve_ms": t_seq,
                   "sigma_sample_iters": int(r0["I"][j_med]), "sigma_one_solve_ms": t1, "S": {}}
            # one sample per lane, a level per call (S = 1): independent per-sample
            # solves batched, against which the ensembles' speed-up is also quoted
            one = Adaptive(h, wl, S=1, precond=pc)
            one.run("nat")  # warm-up
            one.time_calls = True
            r1 = one.run("nat")
            t_one = solve_ms(one)
            res["one_lane_batch"] = {"solve_ms": t_one, "speedup": t_seq / t_one,
                                     "same_grid": bool(np.array_equal(r1["lvl"], r0["lvl"])),
                                     "max_iter_diff_vs_sequential": int(np.max(np.abs(r1["I"] - r0["I"])))}
            del one
            torch.cuda.empty_cache()
            for S in S_list:
                ad = Adaptive(h, wl, S=S, precond=pc)
                ad.run("nat")  # warm-up: instantiates every level's loop graph
                Ms = min(512, ad.solver.Emax * S)
                ys = y_med.expand(Ms, -1).contiguous()
                ad.solver.solve(ys)
                ad.time_calls = True
                ad.call_events = []
                ad._call(ys)
                sigma = Ms * t1 / ad.call_times()[0][1]
                row = {"sigma": sigma}
                same_grid = True
                for g in ("sur", "par", "nat"):
                    r = ad.run(g)
                    t = solve_ms(ad)
                    same_grid &= bool(np.array_equal(r["lvl"], r0["lvl"]))
                    R = ratios(r)
                    row[g] = {"R_levels": R["run"][0], "R": R["run"][1], "speedup": t_seq / t,
                              "pred_speedup": sigma / R["run"][1], "solve_ms": t,
                              "vs_one_lane_batch": t_one / t}
                    if g == "sur":
                        row["its"] = {"R_levels": R["its"][0], "R": R["its"][1],
                                      "pred_speedup": sigma / R["its"][1]}
                        row["sur_pred_rel_err"] = [
                            float(np.mean(np.abs(pr - r["I"][a:b])) / np.mean(r["I"][a:b]))
                            for (a, b), pr in list(zip(r["levels"], r["preds"]))[1:]]
                        row["max_iter_diff_vs_sequential"] = int(np.max(np.abs(r["I"] - r0["I"])))
                row["same_grid_as_sequential"] = same_grid
                res["S"][S] = row
                del ad
                torch.cuda.empty_cache()
            out[name][pc] = res
    return out


def run_mixed_mg(h, stream):
    """The multigrid preconditioner with its V-cycle in float (CG in double)
    against the FP64 V-cycle, on Section 4's Test 1 and Test 2: one full
    adaptive grid each, surrogate grouping, S = 16; solve-call time, R and the
    iteration counts (the grid is the same: it depends on G only); and every
    solution of 64 draws in one call against the FP64 V-cycle's solution of the
    same draws (max over samples of max_j |x32_j - x64_j| / max_j |x64_j|)."""
    import torch

    from paper_1705_02003_gb300 import ens, inputs
    from paper_1705_02003_gb300.solver import EnsembleSolver
    from paper_1705_02003_gb300.uq import Adaptive, ratios

    out = {}
    for name in ("q1_32c_test1", "q1_32c_test2"):
        wl = inputs.WORKLOADS[name]
        res = {}
        for pc in ("mg", "mg32"):
            ad = Adaptive(h, wl, S=16, precond=pc)
            ad.run("sur")  # warm-up
            ad.time_calls = True
            r = ad.run("sur")
            res[pc] = {"solve_ms": sum(ms for _, ms in ad.call_times()), "R": ratios(r)["run"][1],
                       "iters_mean": float(r["I"].mean()), "iters_max": int(r["I"].max()), "I": r["I"]}
            del ad
        res["max_iter_diff"] = int(np.max(np.abs(res["mg32"].pop("I") - res["mg"].pop("I"))))
        res["speedup_mg32_vs_mg"] = res["mg"]["solve_ms"] / res["mg32"]["solve_ms"]
        prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
        xi = torch.from_numpy(inputs.draws(64, wl.nparam, seed=5)).cuda()
        xs = {}
        for pc in ("mg", "mg32"):
            sol = EnsembleSolver(h, prob, 16, 64, wl.rtol, wl.maxit, precond=pc)
            it, st, _, _ = sol.solve(xi)
            assert bool((st == ens.LANE_CONVERGED).all().item())
            xs[pc] = sol.solution(64).permute(0, 2, 1).reshape(64, sol.J).clone()
            del sol
        err = ((xs["mg32"] - xs["mg"]).abs().amax(dim=1) / xs["mg"].abs().amax(dim=1)).max().item()
        res["max_rel_error_vs_fp64_vcycle"] = err
        res["error_sample"] = "64 draws (seed 5) at rtol 1e-7, one call of 4 ensembles of 16"
        out[name] = res
        torch.cuda.empty_cache()
    return out


def _lanes_to_rows(x, E, J, S):
    """[E][J][S] device vector -> [E*S][J]."""
    return x[: E * J * S].view(E, J, S).permute(0, 2, 1).reshape(E * S, J)


def run_layers(h, stream):
    """The three system layers at their configurations' sizes, each with
    per-sample results against the oracle on a stated subset (timed on all
    host cores):
      precision       1024 draws of the 128^3 7-point problem, S = 32, FP32
                      values and inner Jacobi-PCG inside FP64 refinement to
                      1e-10, in calls of 8 ensembles, against the FP64 solve;
      batching        all 4096 draws of the 64^3 problem through a pool of 1024
                      lanes, S autotuned over {8, 16, 32, 64}, against fixed
                      batches of 1024 draws;
      differentiation 1024 draws of the 512^2 5-point problem, S = 32: Q and
                      dQ/dxi from the forward and adjoint ensemble solves."""
    import torch

    import oracle as O
    from paper_1705_02003_gb300 import adjoint, batching, ens, inputs
    from paper_1705_02003_gb300.solver import EnsembleSolver

    threads = os.cpu_count() or 1
    out = {}

    # ---- precision layer --------------------------------------------------
    wl = inputs.WORKLOADS["fd7_128_mixed"]
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    S, M, Ec = wl.S, wl.samples, 8
    xi_all = inputs.draws(M, wl.nparam, seed=wl.seed)
    sub = np.arange(0, M, M // 16)  # 16 samples checked against the oracle
    sol = EnsembleSolver(h, prob, S, Ec * S, wl.rtol, wl.maxit)
    J, nnz = sol.J, sol.nnz
    v32 = torch.empty(Ec * nnz * S, dtype=torch.float32, device="cuda")
    xir = torch.empty(Ec * J * S, dtype=torch.float64, device="cuda")
    L = Ec * S
    itir = torch.empty(L, dtype=torch.int32, device="cuda")
    oit, stir = torch.empty_like(itir), torch.empty_like(itir)
    rrir = torch.empty(L, dtype=torch.float64, device="cuda")
    wir = torch.empty(ens.ens_pcg_ir_workspace_size(J, nnz, S, Ec), dtype=torch.uint8, device="cuda")

    def assemble(c0, E):
        xi = torch.from_numpy(xi_all[c0:c0 + E * S]).cuda()
        ens.ens_assemble(h, prob, S, E, xi.reshape(-1), sol.rowptr, sol.colidx, sol.vals[: E * nnz * S],
                         sol.dinv[: E * J * S], sol.b[: E * J * S])
        ens.ens_assemble(h, prob, S, E, xi.reshape(-1), sol.rowptr, sol.colidx, v32[: E * nnz * S])

    def ir(E, tin):
        ens.ens_pcg_solve_ir(h, J, nnz, S, E, sol.rowptr, sol.colidx, sol.vals[: E * nnz * S], v32[: E * nnz * S],
                             sol.dinv[: E * J * S], sol.b[: E * J * S], xir[: E * J * S], None, wl.rtol, tin,
                             wl.maxit, 50, itir[: E * S], oit[: E * S], rrir[: E * S], stir[: E * S], wir)

    def fp64(E):
        ens.ens_pcg_solve(h, J, nnz, S, E, sol.rowptr, sol.colidx, sol.vals[: E * nnz * S], sol.dinv[: E * J * S],
                          sol.b[: E * J * S], sol.x[: E * J * S], None, wl.rtol, wl.maxit, sol.iters[: E * S],
                          sol.relres[: E * S], sol.status[: E * S], sol.work)

    # the inner tolerance trades FP32 iterations per correction against
    # corrections: time each candidate on the first ensemble, keep the fastest
    assemble(0, 1)
    tune = {tin: timed(stream, lambda: ir(1, tin))[1] for tin in (1e-3, 1e-4, 1e-5, 1e-6)}
    best = min(tune, key=tune.get)
    t64 = tir = 0.0
    its64, itsir, outer, relres, conv = [], [], [], [], True
    err_fp64, gpu_sub = [], {}
    for c0 in range(0, M, Ec * S):
        assemble(c0, Ec)
        _, t = timed(stream, lambda: fp64(Ec))
        t64 += t
        _, t = timed(stream, lambda: ir(Ec, best))
        tir += t
        conv &= bool((stir == 0).all().item() and (sol.status[:L] == 0).all().item())
        its64.append(sol.iters[:L].cpu().numpy())
        itsir.append(itir.cpu().numpy())
        outer.append(oit.cpu().numpy())
        relres.append(rrir.cpu().numpy())
        x64r = _lanes_to_rows(sol.x, Ec, J, S)
        xirr = _lanes_to_rows(xir, Ec, J, S)
        err_fp64.append(((xirr - x64r).abs().amax(dim=1) / x64r.abs().amax(dim=1)).cpu().numpy())
        for m in sub[(sub >= c0) & (sub < c0 + L)]:
            gpu_sub[int(m)] = (xirr[m - c0].cpu().numpy(), x64r[m - c0].cpu().numpy(), int(sol.iters[m - c0].item()))
    del sol, v32, wir, xir
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    ref = O.solve_batch(O.FD7_AXIS, wl.n, wl.nparam, wl.aniso, xi_all[sub], wl.rtol, wl.maxit, nthreads=threads,
                        want_x=True)
    t_or = time.perf_counter() - t0
    e_ir = [np.abs(gpu_sub[int(m)][0] - ref["x"][k]).max() / np.abs(ref["x"][k]).max() for k, m in enumerate(sub)]
    e_64 = [np.abs(gpu_sub[int(m)][1] - ref["x"][k]).max() / np.abs(ref["x"][k]).max() for k, m in enumerate(sub)]
    d_it = [gpu_sub[int(m)][2] - int(ref["iters"][k]) for k, m in enumerate(sub)]
    out["precision"] = {
        "workload": wl.name, "samples": M, "S": S, "ensembles_per_call": Ec,
        "fp64_value": M / t64, "ir_value": M / tir, "unit": "sample-solves/s", "speedup": t64 / tir,
        "rtol_inner": best, "rtol_inner_seconds_one_ensemble": {f"{k:g}": v for k, v in tune.items()},
        "fp64_iters_min_max": [int(np.min(its64)), int(np.max(its64))],
        "ir_inner_iters_max": int(np.max(itsir)), "ir_outer_max": int(np.max(outer)),
        "max_relres_fp64_residual": float(np.max(relres)), "all_converged": conv,
        "max_rel_error_ir_vs_fp64_gpu_all_samples": float(np.max(err_fp64)),
        "oracle_subset": f"{len(sub)} samples (every {M // len(sub)}th), FP64 oracle, {threads} threads, {t_or:.0f} s",
        "max_rel_error_ir_vs_oracle": float(np.max(e_ir)), "max_rel_error_fp64_vs_oracle": float(np.max(e_64)),
        "fp64_iter_diff_vs_oracle": d_it, "error_norm": "max_j |x_j - x_oracle_j| / max_j |x_oracle_j|"}

    # ---- batching layer ---------------------------------------------------
    wl = inputs.WORKLOADS["fd7_64_batch"]
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    M, lanes = wl.samples, 1024
    xi_h = inputs.draws(M, wl.nparam, seed=wl.seed)
    xi = torch.from_numpy(xi_h).cuda()
    S, tune = batching.autotune(h, prob, xi[:512], lanes=256, rtol=wl.rtol, maxit=wl.maxit, chunk=32, stream=stream)
    chunk, ctune = batching.autotune_chunk(h, prob, xi[:512], 256, S, wl.rtol, wl.maxit, stream=stream)
    E = lanes // S
    work = torch.empty(ens.ens_stream_workspace_size(prob, S, E), dtype=torch.uint8, device="cuda")
    batching.solve_stream(h, prob, xi[:lanes], S, E, wl.rtol, wl.maxit, chunk=chunk, work=work)  # warm-up
    res, tstream = timed(stream, lambda: batching.solve_stream(h, prob, xi, S, E, wl.rtol, wl.maxit, chunk=chunk,
                                                               work=work))
    del work
    fsol = EnsembleSolver(h, prob, S, lanes, wl.rtol, wl.maxit)
    fsol.solve(xi[:lanes])  # warm-up

    def fixed():
        its, qs = [], []
        for a0 in range(0, M, lanes):
            it, _, _, q = fsol.solve(xi[a0:a0 + lanes])
            its.append(it.clone())
            qs.append(q.clone())
        return torch.cat(its), torch.cat(qs)

    (fits, fq), tfixed = timed(stream, fixed)
    del fsol
    torch.cuda.empty_cache()
    sub = np.arange(0, M, M // 16)
    t0 = time.perf_counter()
    ref = O.solve_batch(O.FD7_AXIS, wl.n, wl.nparam, wl.aniso, xi_h[sub], wl.rtol, wl.maxit, nthreads=threads)
    t_or = time.perf_counter() - t0
    it_s = res["iters"].cpu().numpy()
    q_s = res["qoi"].cpu().numpy()
    out["batching"] = {
        "workload": wl.name, "samples": M, "lanes": lanes, "S": S, "S_autotune_seconds": {str(k): v for k, v in tune.items()},
        "chunk": chunk, "chunk_autotune_seconds": {str(k): v for k, v in ctune.items()},
        "autotune_sample": "the first 512 draws through 256 lanes",
        "stream_value": M / tstream, "fixed_batches_value": M / tfixed, "unit": "sample-solves/s",
        "speedup": tfixed / tstream, "iters_min_max": [int(it_s.min()), int(it_s.max())],
        "same_iterations_as_fixed": bool(np.array_equal(it_s, fits.cpu().numpy())),
        "all_converged": bool((res["status"] == 0).all().item()),
        "oracle_subset": f"{len(sub)} draws (every {M // len(sub)}th), {threads} threads, {t_or:.0f} s",
        "iter_diff_vs_oracle": (it_s[sub] - ref["iters"]).astype(int).tolist(),
        "max_G_rel_error_vs_oracle": float(np.max(np.abs(q_s[sub] - ref["G"]) / ref["G"]))}
    del xi

    # ---- differentiation layer --------------------------------------------
    wl = inputs.WORKLOADS["fd5_512_adjoint"]
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    M = wl.samples
    w_h = inputs.region_weights(wl.n, 2)
    asol = adjoint.AdjointSolver(h, prob, wl.S, M, torch.from_numpy(w_h), wl.rtol, wl.maxit)
    xi_h = inputs.draws(M, wl.nparam, seed=wl.seed)
    xi = torch.from_numpy(xi_h).cuda()
    asol.forward(xi[: wl.S])  # warm-up
    Q, tf = timed(stream, lambda: asol.forward(xi))
    g, tg = timed(stream, lambda: asol.gradient(xi, recompute_forward=False))
    fit = asol.last["forward_iters"].cpu().numpy()
    ait = asol.last["adjoint_iters"].cpu().numpy()
    conv = bool((asol.last["forward_status"] == 0).all().item() and (asol.last["adjoint_status"] == 0).all().item())
    Qh, gh = Q.cpu().numpy(), g.cpu().numpy()
    del asol
    torch.cuda.empty_cache()
    sub = np.arange(0, M, M // 16)
    from concurrent.futures import ThreadPoolExecutor

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        w_o = O.region_weights(wl.n, 2)
        refs = list(ex.map(lambda m: O.adjoint_grad(O.FD5_LOGKL, wl.n, wl.nparam, wl.aniso, xi_h[m], w_o, wl.rtol,
                                                    wl.maxit), sub))
    t_or = time.perf_counter() - t0
    gerr = [np.abs(gh[m] - r[1]).max() / np.abs(r[1]).max() for m, r in zip(sub, refs)]
    qerr = [abs(Qh[m] - r[0]) / abs(r[0]) for m, r in zip(sub, refs)]
    out["differentiation"] = {
        "workload": wl.name, "samples": M, "S": wl.S, "ensembles_per_call": M // wl.S,
        "forward_value": M / tf, "gradient_value": M / (tf + tg), "unit": "samples/s (Q, and Q with dQ/dxi)",
        "forward_iters_max": int(fit.max()), "adjoint_iters_max": int(ait.max()), "all_converged": conv,
        "oracle_subset": f"{len(sub)} draws (every {M // len(sub)}th), oracle adjoint at the same rtol, "
                         f"{threads} threads, {t_or:.0f} s",
        "max_rel_error_Q_vs_oracle": float(np.max(qerr)), "max_rel_error_grad_vs_oracle": float(np.max(gerr)),
        "error_norm": "max_k |g_k - g_oracle_k| / max_k |g_oracle_k| per sample"}
    return out


def run_kernel_only(args, wl):
    """A small case of the dominant kernel for profilers: E ensembles of the
    workload's problem (inputs larger than L2, a few GB at most), assembled once,
    then ens_spmv launched --steps times."""
    import torch

    from paper_1705_02003_gb300 import ens, inputs
    from paper_1705_02003_gb300.solver import EnsembleSolver

    h = ens.Handle(0)
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    S = args.kernel_s or wl.S
    E = args.kernel_ensembles
    sol = EnsembleSolver(h, prob, S, E * S, wl.rtol, wl.maxit)
    xi = torch.from_numpy(inputs.draws(E * S, wl.nparam, seed=1)).cuda()
    ens.ens_assemble(h, prob, S, E, xi.reshape(-1), sol.rowptr, sol.colidx, sol.vals, sol.dinv, sol.b)
    q = torch.empty_like(sol.x)
    pq = torch.empty(E * S, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ens.ens_spmv(h, sol.J, sol.nnz, S, E, sol.rowptr, sol.colidx, sol.vals, sol.b, q, pq, sol.work)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ens.ens_spmv(h, sol.J, sol.nnz, S, E, sol.rowptr, sol.colidx, sol.vals, sol.b, q, pq, sol.work)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    byts = E * (8 * sol.nnz * S + 4 * sol.nnz + 4 * (sol.J + 1) + 16 * sol.J * S)
    fma = E * S * (sol.nnz + sol.J)
    peak, _ = peaks()
    print(json.dumps({"kernel": "k_spmv", "workload": wl.name, "E": E, "S": S, "ms": t * 1e3,
                      "bytes": byts, "GBps": byts / t / 1e9, "frac": byts / t / 1e9 / peak,
                      "fp64_tflops": 2 * fma / t / 1e12}))
    h.close()
    return 0


def run_mg_once(args):
    """One multigrid-preconditioned ensemble solve of 64 draws of Section 4's
    Test 1 (4 ensembles of 16; the CG loop is launched from the host, so a
    kernel profiler lists every launch)."""
    import torch

    from paper_1705_02003_gb300 import ens, inputs
    from paper_1705_02003_gb300.solver import EnsembleSolver

    h = ens.Handle(0)
    wl = inputs.WORKLOADS["q1_32c_test1"]
    sol = EnsembleSolver(h, ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso), 16, 64, wl.rtol, 2000,
                         precond="mg32" if args.mg_once == "mg32" else "mg")
    it, st, _, _ = sol.solve(torch.from_numpy(inputs.draws(64, 4, seed=1)).cuda())
    torch.cuda.synchronize()
    print(json.dumps({"mg_once": args.mg_once, "iters_max": int(it.max().item()),
                      "converged": bool((st == ens.LANE_CONVERGED).all().item())}))
    h.close()
    return 0


def run_loop_once(args, wl):
    """The Section 3.1 loop of the workload --workload names (surrogate
    grouping), run twice: one pass to build and warm up, one to profile.  On
    the 32^2 workload every solve takes the one-launch cluster schedule, so a
    kernel profiler lists each solve as one launch."""
    import torch

    from paper_1705_02003_gb300 import ens
    from paper_1705_02003_gb300.uq import Adaptive

    h = ens.Handle(0)
    ad = Adaptive(h, wl)
    for _ in range(2):
        r = ad.run("sur")
    torch.cuda.synchronize()
    print(json.dumps({"loop_once": wl.name, "points": int(len(r["I"])), "iters_max": int(r["I"].max()),
                      "cluster_ctas": ens.ens_pcg_cluster_size(h, ad.solver.J, ad.solver.nnz, wl.S, 1)}))
    h.close()
    return 0


def run_ir_once(args):
    """One FP32-in-FP64 refinement solve of one ensemble of 32 draws (inner rtol
    1e-4, outer 1e-10) of the 128^3 7-point problem, or of the FD workload
    --workload names (profiling case)."""
    import torch

    from paper_1705_02003_gb300 import ens, inputs
    from paper_1705_02003_gb300.solver import EnsembleSolver

    h = ens.Handle(0)
    wl = inputs.WORKLOADS[args.workload if args.workload.startswith("fd") else "fd7_128_mixed"]
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    S = 32
    sol = EnsembleSolver(h, prob, S, S, 1e-10, wl.maxit)
    J, nnz = sol.J, sol.nnz
    xi = torch.from_numpy(inputs.draws(S, wl.nparam, seed=wl.seed)).cuda()
    ens.ens_assemble(h, prob, S, 1, xi.reshape(-1), sol.rowptr, sol.colidx, sol.vals, sol.dinv, sol.b)
    v32 = torch.empty(nnz * S, dtype=torch.float32, device="cuda")  # the same values rounded to float
    ens.ens_assemble(h, prob, S, 1, xi.reshape(-1), sol.rowptr, sol.colidx, v32)
    x = torch.empty(J * S, dtype=torch.float64, device="cuda")
    it = torch.empty(S, dtype=torch.int32, device="cuda")
    oit, st = torch.empty_like(it), torch.empty_like(it)
    rr = torch.empty(S, dtype=torch.float64, device="cuda")
    work = torch.empty(ens.ens_pcg_ir_workspace_size(J, nnz, S, 1), dtype=torch.uint8, device="cuda")
    _, t = timed(torch.cuda.current_stream(), lambda: ens.ens_pcg_solve_ir(
        h, J, nnz, S, 1, sol.rowptr, sol.colidx, sol.vals, v32, sol.dinv, sol.b, x, None, 1e-10, 1e-4, wl.maxit, 50,
        it, oit, rr, st, work))
    print(json.dumps({"ir_once": wl.name, "seconds": t, "inner_iters_max": int(it.max().item()),
                      "outer_max": int(oit.max().item()), "converged": bool((st == 0).all().item())}))
    h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="q1_256_adaptive")
    ap.add_argument("--no-arms", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--suite", default="", help="comma-separated: layers, configs, c1, pilot, paper, mixed-mg; or all")
    ap.add_argument("--detail-out", default=None, help="where to write the detail JSON")
    ap.add_argument("--cpu-samples", type=int, default=32)
    ap.add_argument("--ref-samples", type=int, default=32)
    ap.add_argument("--kernel-only", action="store_true", help="time the ensemble SpMV alone (profiling)")
    ap.add_argument("--kernel-ensembles", type=int, default=8)
    ap.add_argument("--kernel-s", type=int, default=0, help="lanes per ensemble for --kernel-only (0: the workload's)")
    ap.add_argument("--mg-once", choices=["mg", "mg32"], default=None,
                    help="one multigrid solve of 64 draws of Section 4's Test 1 (profiling)")
    ap.add_argument("--loop-once", action="store_true",
                    help="two passes of the adaptive loop of --workload, surrogate grouping (profiling)")
    ap.add_argument("--ir-once", action="store_true",
                    help="one FP32-in-FP64 refinement solve of 32 draws of the 128^3 problem (profiling)")
    args = ap.parse_args()
    from paper_1705_02003_gb300 import inputs

    wl = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.kernel_only:
        return run_kernel_only(args, wl)
    if args.mg_once:
        return run_mg_once(args)
    if args.ir_once:
        return run_ir_once(args)
    if args.loop_once:
        return run_loop_once(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
