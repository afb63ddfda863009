"""The benchmark's last stdout line: one compact JSON object with the keys the
measurement contract asks for (CPU only: built from representative values)."""
import json
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1705_02003_gb300 import inputs  # noqa: E402


def test_compact_line_keys_and_size():
    wl = inputs.WORKLOADS["q1_256_adaptive"]
    args = types.SimpleNamespace(steps=20, warmup=5)
    sol = types.SimpleNamespace(J=65536, nnz=586756, S=16)
    roofline = {"bound": "alu", "achieved": 1.041, "peak": 1.056, "unit": "TFLOP/s", "frac": 0.986,
                "traffic": 2.85e9, "kernel": "k_spmv (K2), FP64, E=32 S=16",
                "peak_source": "measured FP64 FMA rate (ens_fp64_peak, this run)",
                "hbm": {"achieved": 4712.3, "peak": 6752.8, "unit": "GB/s", "frac": 0.698, "peak_source": "measured"}}
    cpu = {"value": 16.1, "unit": "sample-solves/s", "cores": 16, "kind": "oracle",
           "sample": "32 of the 265 grid points, one per thread, 2.0 s"}
    e2e = {"value": 280.3, "unit": "sample-solves/s", "h2d_bytes_per_step": 13780, "d2h_bytes_per_step": 142619056}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 80}
    arms = {"sur": {"speedup_vs_per_sample_serial": 8.8, "speedup_vs_per_sample_batched": 2.16}}
    line = bench.compact_line(value=281.3, world=1, args=args, tmax=18.8, wl=wl, sol=sol, M=265, levels=3,
                              roofline=roofline, cpu=cpu, e2e=e2e, launches=1574460, clocks=clocks, path_frac=0.85,
                              arms=arms, detail_path="/tmp/ens_bench_detail.json")
    text = json.dumps(line, separators=(",", ":"))
    assert "\n" not in text and len(text) < 2500
    back = json.loads(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in back, k
    assert back["config"]["workload"] == "q1_256_adaptive" and back["config"]["samples_per_step"] == 265
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in back["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in back["e2e"], k
    assert back["cpu_baseline"]["kind"] == "oracle" and back["cpu_baseline"]["cores"] == 16
    assert back["higher_is_better"] is True and back["ms_per_step"] == 18.8e3 / 20
