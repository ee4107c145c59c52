#!/usr/bin/env python3
"""Benchmark of the domain-wall hot path on GB300.

Metric: DWF solve time to a 1e-10 true residual (MADWF + mixed precision, or
mixed-precision CG), with plain FP64 CG on the same GPU as the comparison and
the Wilson hop (Dslash) kernel's achieved HBM bandwidth against the measured
copy peak.

A step is one solve of D(m) x = b from a zero guess on seeded synthetic
inputs already resident in HBM.  Defaults finish in a few minutes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload mixed|madwf]
                  [--impl native|reference] [--no-fp64] [--no-cpu-baseline]

Under torchrun (N > 1) every rank solves its own replica (no collective on
the data path); rank 0 prints the JSON line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0

WORKLOADS = {
    # 16^3 x 32 x Ls=16 Shamir, m_f = 0.01, eps = 0.5: mixed-precision CG vs FP64 CG
    "mixed": dict(name="shamir-16^3x32-Ls16-mixedCG", dims=(16, 16, 16, 32), Ls=16, M5=1.8, m=0.01,
                  eps=0.5, seed=2, inner="f32",
                  # FP64 CG iterations to 1e-10 on this input (GB300, dwf_cg inner=f64); scales the
                  # per-iteration oracle time of the reference arm and the cpu_baseline
                  fp64_iters=260),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="mixed", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 CG comparison solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-10)
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- oracle timing


def oracle_iteration_seconds(w, n_iter=1):
    """Seconds per CG iteration of the FP64 oracle (M_pc and M_pc^+ once each) on
    the full workload lattice, on this host's cores."""
    import numpy as np

    from oracle import dwf_oracle as O
    from paper_1111_5059_gb300 import inputs

    U = inputs.gauge_field(w["seed"], w["dims"], w["eps"])
    b = inputs.gaussian_spinor(w["seed"], w["dims"], w["Ls"])
    eo = O.EO(U, w["m"], w["M5"], w["Ls"])
    v = b * eo.even
    t0 = time.perf_counter()
    for _ in range(n_iter):
        q = eo.Mpc(v)
        v = eo.Mpc(q, True)
        v = v / np.sqrt(O.norm2(v))
    return (time.perf_counter() - t0) / n_iter


def run_reference(args, w):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_iteration_seconds(w)
    times = [oracle_iteration_seconds(w) for _ in range(args.steps)]
    per_it = statistics.mean(times)
    value = per_it * w["fp64_iters"]
    sample = (f"1 oracle CG iteration (M_pc then M_pc^+) on the full {w['name']} lattice per step, "
              f"scaled by the {w['fp64_iters']} FP64 CG iterations the solve takes")
    line = {"impl": "reference", "metric": metric_name(w), "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_it * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w),
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def metric_name(w):
    return "DWF solve time @1e-10 (" + ("MADWF+mixed" if w.get("madwf") else "mixed-precision CG") + ")"


def config_of(w):
    X, Y, Z, T = w["dims"]
    c = {"workload": w["name"], "lattice": f"{X}x{Y}x{Z}x{T}", "Ls": w["Ls"], "M5": w["M5"], "m_f": w["m"],
         "eps": w["eps"], "seed": w["seed"], "tol": 1e-10, "inner": w["inner"],
         "l2": "inputs larger than L2 between steps (working set > 129 MB) plus a 512 MB L2 flush write"}
    if w.get("madwf"):
        c.update({"Ls_inner": w["inner_Ls"], "b_inner": w["b"], "c_inner": w["c"], "n_dc": w["n_dc"]})
    return c


# --------------------------------------------------------------------------- native arm


def main():
    args = parse()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
        return
    import numpy as np
    import torch

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1111_5059_gb300 import dwf, inputs

    if not os.path.exists(dwf.LIB_PATH):
        from paper_1111_5059_gb300 import build

        build.build()
    hbm_peak, peak_src = measured_peaks()

    U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], w["eps"])).to(dev)
    b_host = torch.from_numpy(inputs.gaussian_spinor(w["seed"], w["dims"], w["Ls"])).pin_memory()
    b = b_host.to(dev)
    x_host = torch.empty_like(b_host).pin_memory()
    stream = torch.cuda.current_stream(dev)
    lat = dwf.Lattice(w["dims"], w["Ls"], w["M5"], 1.0, 0.0, 1, stream=stream, device=dev)
    lat.set_gauge(U)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def solve(bb):
        return lat.cg(w["m"], bb, tol=args.tol, inner=w["inner"], delta=0.1, check_every=10)

    for _ in range(args.warmup):
        r = solve(b)
    torch.cuda.synchronize()

    # ---- timed region: K solves, inputs resident in HBM
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat.set_kernel_timing(True)
    n0 = lat.launch_count()
    step_ms, stats = [], []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = solve(b)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            stats.append(r.stats)
    torch.cuda.synchronize()
    barrier(world)
    launches = lat.launch_count() - n0
    kt = lat.kernel_time(w["inner"])
    lat.set_kernel_timing(False)
    total_ms = max_over_ranks(world, sum(step_ms), dev)
    ms_step = total_ms / args.steps
    value = ms_step / 1e3 / world  # seconds per solve, whole job (replicas solve concurrently)

    x = r.x.cpu().numpy()
    true_res = r.stats["true_resid"]

    # ---- e2e through the C ABI with host buffers
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bd = b_host.to(dev, non_blocking=True)
        rr = solve(bd)
        x_host.copy_(rr.x, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(world, statistics.mean(e2e_ms), dev)

    # ---- FP64 CG comparison on the same GPU
    fp64 = None
    if not args.no_fp64:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rf = lat.cg(w["m"], b, tol=args.tol, inner="f64", check_every=10)
        torch.cuda.synchronize()
        fp64 = {"seconds": time.perf_counter() - t0, "iters": rf.stats["iters"], "op_count": rf.stats["op_count"],
                "true_resid": rf.stats["true_resid"]}
        fp64["speedup_of_headline"] = fp64["seconds"] / (ms_step / 1e3)

    achieved = kt["bytes"] / (kt["ms"] / 1e3) / 1e9 if kt["ms"] > 0 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": (achieved / hbm_peak) if achieved else None, "traffic": None,
            "kernel": f"hop_kernel<{w['inner']}> (Wilson hop x Ls with fused s-local epilogues)",
            "launches": kt["launches"], "avg_launch_us": kt["ms"] / max(1, kt["launches"]) * 1e3,
            "bytes_per_launch": kt["bytes"] / max(1, kt["launches"]),
            "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured" else "fallback"}

    line = {"metric": metric_name(w), "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": config_of(w),
            "roofline": roof,
            "e2e": {"value": e2e_ms / 1e3 / world, "unit": "s", "h2d_bytes_per_step": b_host.numel() * 16,
                    "d2h_bytes_per_step": x_host.numel() * 16},
            "gpu_launches": launches,
            "solve": {"iters": stats[-1]["iters"], "reliable_updates": stats[-1]["reliable_updates"],
                      "op_count": stats[-1]["op_count"], "true_resid": true_res,
                      "step_ms": step_ms},
            "fp64_cg": fp64}
    if rank == 0:
        with ClockSampler(local):
            pass
        line["clocks"] = clk.summary()
        if not args.no_cpu_baseline:
            per_it = oracle_iteration_seconds(w)
            line["cpu_baseline"] = {
                "value": per_it * w["fp64_iters"], "unit": "s", "cores": 1, "kind": "oracle",
                "sample": (f"1 FP64 oracle CG iteration (M_pc, M_pc^+) on the full {w['name']} lattice "
                           f"({per_it:.1f} s), scaled by the {w['fp64_iters']} iterations of the FP64 solve")}
        print(json.dumps(line), flush=True)
    del x
    lat.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
