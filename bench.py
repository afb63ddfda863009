"""Benchmark: sample-solves/s of the surrogate-grouped ensemble PCG.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload q1_256_adaptive] [--no-arms] [--no-layers] [--no-paper] [--no-cpu]
                    [--mixed-mg]
                    [--kernel-only [--kernel-ensembles E]]

A step is one pass of the whole path over the workload: the grid-generation
and grouping loop of the paper's flowchart (initial sparse grid, then per
level: surrogate grouping (K6, K7), ensemble assembly (K1), ensemble Jacobi-PCG
(K2-K4) to rel. residual 1e-8, QoI, surpluses and host refinement) until the
sample budget is reached.  value = samples solved / device time (CUDA events
around K steps, max over ranks).

The same run (one GPU) also reports:
  arms            parameter-based, natural and random grouping; one sample at a
                  time on the same GPU; the surrogate groups with lane re-packing
  R, R_levels     the work ratio of Eq. (R) overall and per level
  level_calls     each level's solve call: size, ensembles, branches, time
  roofline        the ensemble SpMV (K2) against the FP64 and HBM roofs, and
                  the whole path against its roofline
  e2e             the same metric through the public API with host buffers
  layers          FP32-in-FP64 refinement, batching (two iteration spreads),
                  the adjoint gradient, each on a bounded sample
  spmv_configs    K2 on the 7-point 64^3 / 128^3 and 5-point 512^2 problems
  pilot_grouping  surrogate grouping of a non-adaptive sample set (Section 5)
  paper_tables    Section 4's Test 1 / Test 2 (32^3 trilinear FEM, N = 4), with
                  the Jacobi and the multigrid preconditioner: R_l, R,
                  measured and predicted speed-up for S = 4..32
                  (--mixed-mg adds the multigrid solve with a float V-cycle)
  cpu_baseline    the CPU oracle on a bounded sample of the same points

--kernel-only times K2 alone (the case the Nsight Compute summaries use).
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sample-solves/s at rel-res 1e-8: ensemble PCG vs per-sample PCG; SpMV HBM GB/s"


# FP64 roof of GB300: the FP64 pipe retires two lanes per clock per SM (the
# pipe-activity counter of K2 gives 1.67 per active cycle at 84 % activity),
# so 152 SMs x 2 FMA x 2.07 GHz = 630 G FMA/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PEAK_SOURCE = "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz (nominal 1.25 TFLOP/s)"

# DRAM bytes of one K2 launch measured by ncu on the E = 8 case of the same
# kernel (profiles/k_spmv_q1_256_E8.md), scaled by the units a launch processes.
SPMV_TRAFFIC_PER_ENSEMBLE = {"q1_256_adaptive": (673.661696e6 + 37.994240e6) / 8}


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
    point of the full sparse grid of the workload's dimension (levels 0..3)."""
    from paper_1705_02003_gb300 import ens, uq

    lvl, idx = ens.ens_sg_initial(wl.nparam, 3)
    y = uq.coords(lvl, idx)
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
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, wl):
    import torch

    from paper_1705_02003_gb300 import ens
    from paper_1705_02003_gb300.uq import Adaptive, ratios

    world, rank, local, pg = dist_setup(args)
    if world > 1:
        # N independent replicas: only the timed loop runs on every GPU; the
        # single-GPU diagnostics (arms, layers, per-problem SpMV) are N = 1 work
        args.no_arms = args.no_layers = args.no_paper = True
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

    extra = {}
    if not args.no_arms:
        # the other groupings and one-sample-at-a-time PCG, one step each
        for arm in ("par", "nat", "rand"):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r2 = ad.run(arm, seed=0)
            e1.record(stream)
            torch.cuda.synchronize()
            ta = e0.elapsed_time(e1) / 1e3
            Ra = ratios(r2)["run"]
            extra[arm] = {"value": M / ta, "R": Ra[1], "R_levels": Ra[0]}
        ps = Adaptive(h, wl, per_sample=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ps.run("nat")  # warm-up (graph instantiation)
        torch.cuda.synchronize()
        e0.record(stream)
        r3 = ps.run("nat")
        e1.record(stream)
        torch.cuda.synchronize()
        tp = e0.elapsed_time(e1) / 1e3
        extra["per_sample"] = {"value": M / tp, "max_iter_diff_vs_ensemble": int(np.max(np.abs(r3["I"] - run["I"])))}
        # the same surrogate groups, each level solved through the batching layer
        # (live lanes of partly converged ensembles re-packed every 64 trips)
        rp = Adaptive(h, wl, solver=ad.solver, repack=True)
        rp.run("sur")  # warm-up
        torch.cuda.synchronize()
        e0.record(stream)
        r4 = rp.run("sur")
        e1.record(stream)
        torch.cuda.synchronize()
        tr = e0.elapsed_time(e1) / 1e3
        extra["sur_repack"] = {"value": M / tr, "same_grid": bool(np.array_equal(r4["lvl"], run["lvl"])),
                               "same_iterations": bool(np.array_equal(r4["I"], run["I"]))}
        del rp

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
                            "ps_per_row_lane_iteration": ms * 1e9 / (charged_c * ad.solver.J)})

    layers = {} if args.no_layers else run_layers(h, stream)
    configs = {} if args.no_layers else run_configs(h, stream)
    pilot = {} if args.no_layers else run_pilot(h, stream)
    paper = {} if args.no_paper else run_paper(h, stream)
    if args.mixed_mg:
        paper["mixed_multigrid"] = run_mixed_mg(h, stream)

    # dominant kernel: the ensemble SpMV (K2) on a full-capacity batch
    sol = ad.solver
    E = sol.Emax
    L = E * sol.S
    xi_all = torch.from_numpy(run["y"][:L] if len(run["y"]) >= L else
                              np.resize(run["y"], (L, wl.nparam))).to("cuda")
    ens.ens_assemble(h, sol.prob, sol.S, E, xi_all.reshape(-1).contiguous(), sol.rowptr, sol.colidx, sol.vals,
                     sol.dinv, sol.b)
    p = sol.b
    q = torch.empty_like(sol.x)
    pq = torch.empty(L, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ens.ens_spmv(h, sol.J, sol.nnz, sol.S, E, sol.rowptr, sol.colidx, sol.vals, p, q, pq, sol.work)
    reps = 20
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ens.ens_spmv(h, sol.J, sol.nnz, sol.S, E, sol.rowptr, sol.colidx, sol.vals, p, q, pq, sol.work)
    e1.record(stream)
    torch.cuda.synchronize()
    t_spmv = e0.elapsed_time(e1) / 1e3 / reps
    spmv_bytes = E * (8 * sol.nnz * sol.S + 4 * sol.nnz + 4 * (sol.J + 1) + 16 * sol.J * sol.S)
    spmv_fma = E * sol.S * (sol.nnz + sol.J)  # one fused multiply-add per nonzero-lane, one per row-lane for p^T q
    peak, peak_kind = peaks()
    achieved = spmv_bytes / t_spmv / 1e9
    tflops = 2.0 * spmv_fma / t_spmv / 1e12
    roofline = {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tflops / FP64_PEAK_TFLOPS, "traffic": spmv_traffic(wl, E),
                "kernel": "k_spmv (K2), FP64", "peak_source": FP64_PEAK_SOURCE,
                "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_source": peak_kind},
                "bytes_per_launch": spmv_bytes, "fma_per_launch": spmv_fma, "launch_ms": t_spmv * 1e3}
    # the whole path: every lane of an ensemble streams until the slowest lane stops
    charged = sum(float(np.max(run["I"][a + perm[k:k + sol.S]]))
                  for (a, b), perm in zip(run["levels"], run["perms"]) for k in range(0, b - a, sol.S)) * sol.S
    b_alg = 8 * sol.nnz + 72 * sol.J + (4 * sol.nnz + 4 * (sol.J + 1)) / sol.S
    fma_it = sol.nnz + 7 * sol.J  # K2: nnz + J, K3: 5 J (z = D^-1 r stored), K4: J per sample-iteration
    t_it = max(b_alg / (peak * 1e9), 2.0 * fma_it / (FP64_PEAK_TFLOPS * 1e12))
    path_roof = M / (charged * t_it)
    roofline["path"] = {"value": path_roof, "unit": "sample-solves/s", "frac": value / path_roof,
                        "sample_iterations_charged": charged, "bytes_per_sample_iteration": b_alg,
                        "fma_per_sample_iteration": fma_it}

    # end to end through the public API with host buffers: the loop copies each
    # level's points in and its surpluses out; in addition every solve's
    # solution fields u (all samples) go to pinned host memory, and the
    # per-sample G, I and surpluses come back at the end of the step
    host_u = torch.empty(max(M, sol.S) * sol.J + sol.Emax * sol.S * sol.J, dtype=torch.float64,
                         pin_memory=True)
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
        r4 = ad.run("sur")
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
               "sample": f"{len(pts)} of the {M} grid points (every {max(1, M // args.cpu_samples)}-th), "
                         f"FP64 per-sample Jacobi-PCG, one sample per thread, {dt:.1f} s",
               "single_core_value": rate1, "single_core_sample": f"the first 2 of those points, {dt1:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "sample-solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "kind": wl.kind, "n": wl.n, "J": sol.J, "nnz": sol.nnz,
                       "N": wl.nparam, "S": sol.S, "samples_per_step": M, "levels": len(run["levels"]),
                       "rtol": wl.rtol, "grouping": "sur", "parallelism": "replicas" if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (vals of one level >= 225 MB)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "R": {"sur": R["run"][1], "its": R["its"][1]},
            "R_levels": {"sur": R["run"][0], "its": R["its"][0],
                         "points": [b - a for a, b in run["levels"]]},
            "arms": extra,
            "level_calls": level_calls,
            "layers": layers,
            "spmv_configs": configs,
            "pilot_grouping": pilot,
            "paper_tables": paper,
        }
        if "per_sample" in extra:
            line["speedup_vs_per_sample"] = value / extra["per_sample"]["value"]
        print(json.dumps(line))
    h.close()
    return 0


def run_configs(h, stream):
    """The ensemble SpMV (K2) on the other problem configurations, each with
    inputs larger than L2: algorithmic GB/s and FP64 rate per launch."""
    import torch

    from paper_1705_02003_gb300 import ens, inputs
    from paper_1705_02003_gb300.solver import EnsembleSolver

    peak, peak_kind = peaks()
    out = {}
    for name, E in (("fd7_64_batch", 4), ("fd7_128_mixed", 1), ("fd5_512_adjoint", 4)):
        wl = inputs.WORKLOADS[name]
        prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
        S = 32
        sol = EnsembleSolver(h, prob, S, E * S, wl.rtol, wl.maxit)
        xi = torch.from_numpy(inputs.draws(E * S, wl.nparam, seed=wl.seed)).cuda()
        ens.ens_assemble(h, prob, S, E, xi.reshape(-1), sol.rowptr, sol.colidx, sol.vals, sol.dinv, sol.b)
        q = torch.empty_like(sol.x)
        pq = torch.empty(E * S, dtype=torch.float64, device="cuda")
        call = lambda: ens.ens_spmv(h, sol.J, sol.nnz, S, E, sol.rowptr, sol.colidx, sol.vals, sol.b, q, pq,
                                    sol.work)
        for _ in range(3):
            call()
        reps = 10
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            call()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        byts = E * (8 * sol.nnz * S + 4 * sol.nnz + 4 * (sol.J + 1) + 16 * sol.J * S)
        fma = E * S * (sol.nnz + sol.J)
        out[name] = {"E": E, "S": S, "bytes_per_launch": byts, "launch_ms": t * 1e3,
                     "hbm_gbs": byts / t / 1e9, "hbm_frac": byts / t / 1e9 / peak,
                     "fp64_tflops": 2 * fma / t / 1e12, "fp64_frac": 2 * fma / t / 1e12 / FP64_PEAK_TFLOPS}
        del sol, q
    out["peaks"] = {"hbm_gbs": peak, "hbm_source": peak_kind, "fp64_tflops": FP64_PEAK_TFLOPS}
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

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    pg = uq.PilotGrouping(h, sol, level=1)
    _, t_pilot = timed(pg.build)
    xi = torch.from_numpy(inputs.draws(wl.samples, wl.nparam, seed=wl.seed)[:M]).cuda()
    (pred, perm, _), t_group = timed(lambda: pg.group(xi, S))
    order = perm.to(torch.int64)
    sol.solve(xi)  # warm-up (graph instantiation)
    (it_nat, *_), t_nat = timed(lambda: sol.solve(xi))
    it_nat = it_nat.cpu().numpy().astype(np.float64)
    (it_sur, *_), t_sur = timed(lambda: sol.solve(xi.index_select(0, order)))
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
                              "pred_speedup": sigma / R["run"][1], "solve_ms": t}
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
    iteration counts (the grid is the same: it depends on G only)."""
    from paper_1705_02003_gb300 import inputs
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
        out[name] = res
    return out


def run_layers(h, stream):
    """The three system layers on bounded samples of their workloads:
    FP32-in-FP64 refinement vs the FP64 solve on the 128^3 problem (one
    ensemble), continuous batching with an autotuned S vs fixed batches on the
    64^3 problem, the adjoint gradient on the 512^2 problem (one ensemble)."""
    import torch

    from paper_1705_02003_gb300 import adjoint, ens, inputs
    from paper_1705_02003_gb300.solver import EnsembleSolver

    out = {}

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    # precision layer
    wl = inputs.WORKLOADS["fd7_128_mixed"]
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    sol = EnsembleSolver(h, prob, wl.S, wl.S, wl.rtol, wl.maxit)
    xi = torch.from_numpy(inputs.draws(wl.S, wl.nparam, seed=wl.seed)).cuda()
    J, nnz, S = sol.J, sol.nnz, sol.S
    ens.ens_assemble(h, prob, S, 1, xi.reshape(-1), sol.rowptr, sol.colidx, sol.vals, sol.dinv, sol.b)
    v32 = torch.empty(nnz * S, dtype=torch.float32, device="cuda")
    ens.ens_assemble(h, prob, S, 1, xi.reshape(-1), sol.rowptr, sol.colidx, v32)
    x64 = torch.empty(J * S, dtype=torch.float64, device="cuda")
    it64 = torch.empty(S, dtype=torch.int32, device="cuda")
    st64 = torch.empty_like(it64)
    rr64 = torch.empty(S, dtype=torch.float64, device="cuda")
    _, t64 = timed(lambda: ens.ens_pcg_solve(h, J, nnz, S, 1, sol.rowptr, sol.colidx, sol.vals, sol.dinv, sol.b,
                                             x64, None, wl.rtol, wl.maxit, it64, rr64, st64, sol.work))
    xir = torch.empty(J * S, dtype=torch.float64, device="cuda")
    itir = torch.empty(S, dtype=torch.int32, device="cuda")
    oit = torch.empty_like(itir)
    stir = torch.empty_like(itir)
    rrir = torch.empty(S, dtype=torch.float64, device="cuda")
    wir = torch.empty(ens.ens_pcg_ir_workspace_size(J, nnz, S, 1), dtype=torch.uint8, device="cuda")
    # the inner tolerance trades FP32 iterations per correction against corrections:
    # time each candidate once and keep the fastest (the last run's results are reported)
    tune = {}
    for tin in (1e-3, 1e-4, 1e-5, 1e-6):
        _, tt = timed(lambda: ens.ens_pcg_solve_ir(h, J, nnz, S, 1, sol.rowptr, sol.colidx, sol.vals, v32,
                                                   sol.dinv, sol.b, xir, None, wl.rtol, tin, wl.maxit, 50, itir,
                                                   oit, rrir, stir, wir))
        tune[tin] = tt
    best = min(tune, key=tune.get)
    _, tir = timed(lambda: ens.ens_pcg_solve_ir(h, J, nnz, S, 1, sol.rowptr, sol.colidx, sol.vals, v32, sol.dinv,
                                                sol.b, xir, None, wl.rtol, best, wl.maxit, 50, itir, oit, rrir,
                                                stir, wir))
    d = (xir - x64).view(J, S)
    err = (d.norm(dim=0) / x64.view(J, S).norm(dim=0)).max().item()
    out["precision"] = {
        "workload": wl.name, "sample": f"one ensemble of {S} draws",
        "fp64_value": S / t64, "ir_value": S / tir, "unit": "sample-solves/s", "speedup": t64 / tir,
        "fp64_max_iters": int(it64.max().item()), "ir_inner_iters_max": int(itir.max().item()),
        "ir_outer_max": int(oit.max().item()), "max_relres": float(rrir.max().item()),
        "max_rel_error_vs_fp64": err, "rtol_inner": best,
        "rtol_inner_seconds": {f"{k:g}": v for k, v in tune.items()},
        "all_converged": bool((stir == 0).all().item() and (st64 == 0).all().item())}
    del sol, v32, wir, x64, xir
    torch.cuda.empty_cache()

    # batching layer: the same samples through a fixed lane capacity, as fixed
    # batches solved to completion one after another vs continuous refill
    from paper_1705_02003_gb300 import batching

    def batching_case(name, M, lanes, S=None, order_note="the first"):
        wl = inputs.WORKLOADS[name]
        prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
        total = wl.samples if wl.samples else M
        xi = torch.from_numpy(inputs.draws(total, wl.nparam, seed=wl.seed)[:M]).cuda()
        tune, ctune, chunk = {}, {}, 32
        if S is None:
            S, tune = batching.autotune(h, prob, xi, lanes=lanes, rtol=wl.rtol, maxit=wl.maxit, chunk=32,
                                        stream=stream)
            chunk, ctune = batching.autotune_chunk(h, prob, xi, lanes, S, wl.rtol, wl.maxit, stream=stream)
        E = lanes // S
        work = torch.empty(ens.ens_stream_workspace_size(prob, S, E), dtype=torch.uint8, device="cuda")
        batching.solve_stream(h, prob, xi[:lanes], S, E, wl.rtol, wl.maxit, chunk=chunk, work=work)  # warm-up
        # the streamed solve syncs with the host every `chunk` trips: best of two runs
        runs_s = [timed(lambda: batching.solve_stream(h, prob, xi, S, E, wl.rtol, wl.maxit, chunk=chunk,
                                                      work=work)) for _ in range(2)]
        res, tstream = min(runs_s, key=lambda rt: rt[1])
        del work
        fsol = EnsembleSolver(h, prob, S, lanes, wl.rtol, wl.maxit)
        fsol.solve(xi[:lanes])  # warm-up

        def fixed():
            its = []
            for a0 in range(0, M, lanes):
                it, _, _, _ = fsol.solve(xi[a0:a0 + lanes])
                its.append(it.clone())
            return torch.cat(its)

        runs_f = [timed(fixed) for _ in range(2)]
        fits, tfixed = min(runs_f, key=lambda rt: rt[1])
        del fsol
        torch.cuda.empty_cache()
        return {"workload": name, "sample": f"{M} uniform draws ({order_note}), {lanes} lanes", "S": S,
                "S_autotuned": bool(tune), "autotune_seconds": {str(k): v for k, v in tune.items()},
                "chunk": chunk, "chunk_autotune_seconds": {str(k): v for k, v in ctune.items()},
                "stream_value": M / tstream, "fixed_batches_value": M / tfixed, "unit": "sample-solves/s",
                "timing": "best of 2 runs each", "stream_seconds": [t for _, t in runs_s],
                "fixed_seconds": [t for _, t in runs_f], "speedup": tfixed / tstream,
                "iters_min_max": [int(res["iters"].min().item()), int(res["iters"].max().item())],
                "same_iterations_as_fixed": bool(torch.equal(res["iters"], fits))}

    out["batching"] = batching_case("fd7_64_batch", 256, 64, order_note="the first of the 4096")
    # the same comparison where the counts spread widely (10^(4 xi_1) anisotropy)
    out["batching_wide_spread"] = batching_case("q1_256_adaptive", 128, 64, S=16, order_note="seed 0")

    # differentiation layer
    wl = inputs.WORKLOADS["fd5_512_adjoint"]
    prob = ens.problem(wl.kind, wl.n, wl.nparam, wl.aniso)
    w = torch.from_numpy(inputs.region_weights(wl.n, 2))
    asol = adjoint.AdjointSolver(h, prob, wl.S, wl.S, w, wl.rtol, wl.maxit)
    xi = torch.from_numpy(inputs.draws(wl.S, wl.nparam, seed=wl.seed)).cuda()
    _, tf = timed(lambda: asol.forward(xi))
    _, tg = timed(lambda: asol.gradient(xi, recompute_forward=False))
    out["differentiation"] = {
        "workload": wl.name, "sample": f"one ensemble of {wl.S} draws",
        "forward_value": wl.S / tf, "gradient_value": wl.S / (tf + tg), "unit": "samples/s (Q and dQ/dxi)",
        "forward_max_iters": int(asol.last["forward_iters"].max().item()),
        "adjoint_max_iters": int(asol.last["adjoint_iters"].max().item())}
    del asol
    torch.cuda.empty_cache()
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
    S = wl.S
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
    peak, _ = peaks()
    print(json.dumps({"kernel": "k_spmv", "workload": wl.name, "E": E, "S": S, "ms": t * 1e3,
                      "bytes": byts, "GBps": byts / t / 1e9, "frac": byts / t / 1e9 / peak}))
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
    ap.add_argument("--no-layers", action="store_true")
    ap.add_argument("--no-paper", action="store_true", help="skip the Section 4 tables (Test 1 / Test 2)")
    ap.add_argument("--mixed-mg", action="store_true",
                    help="also time the multigrid solve with its V-cycle in float on Test 1 / Test 2")
    ap.add_argument("--cpu-samples", type=int, default=32)
    ap.add_argument("--ref-samples", type=int, default=32)
    ap.add_argument("--kernel-only", action="store_true", help="time the ensemble SpMV alone (profiling)")
    ap.add_argument("--kernel-ensembles", type=int, default=8)
    args = ap.parse_args()
    from paper_1705_02003_gb300 import inputs

    wl = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.kernel_only:
        return run_kernel_only(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
