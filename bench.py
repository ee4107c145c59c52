#!/usr/bin/env python3
"""Benchmark of the domain-wall hot path on GB300.

Metric: DWF solve time to a 1e-10 true residual |b - D(m) x| / |b|.  The
headline workload is the Moebius-accelerated solve (MADWF, FP32 inner solves
with FP64 reliable updates and FP64 defect correction) of Shamir DWF on
24^3 x 64 x Ls=32 through a Moebius operator at Ls'=12; plain FP64 CG on the
same GPU and input is measured beside it, and the Wilson hop (Dslash) kernel's
achieved HBM bandwidth is reported against the measured copy peak.

A step is one solve from a zero guess on seeded synthetic inputs already
resident in HBM (timed with CUDA events on the solve's stream).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload madwf|mixed|hopprof|ladder]
                  [--impl native|reference] [--no-fp64] [--no-cpu-baseline]

Under torchrun (N > 1) every rank solves its own replica (no collective on
the data path, "replicas only"); rank 0 prints the JSON line with the max
time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e data-sheet bandwidth, reported beside the measured peak

# reliable-update threshold of the mixed-precision solves: the FP64 residual is
# recomputed when the iterated one has dropped by this factor
DELTA = 0.01

# DRAM traffic per algorithmic byte of the FP32 hop kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum of two launches on the
# 24^3x48x16 Ls=16 case); it applies only to the kernel source it was taken on.
HOP_TRAFFIC = {"source_sha256_prefix": "dc5de73caaafee4b", "ratio": 1.105}

WORKLOADS = {
    # MADWF: Shamir 24^3 x 64 x Ls=32, m_f = 0.002, eps = 0.6, through Moebius Ls' = 12 with
    # b - c = 1 and b + c = Ls / Ls' (b = 11/6, c = 5/6); 3 defect-correction passes.
    "madwf": dict(name="madwf-shamir-24^3x64-Ls32-via-mobius-Ls12", dims=(24, 24, 24, 64), Ls=32, M5=1.8,
                  m=0.002, eps=0.6, seed=3, inner="f32", madwf=True, inner_Ls=12, b=11 / 6, c=5 / 6, n_dc=3,
                  tol_pv=1e-6, tol_mob=1e-5, sample_T=2),
    # 16^3 x 32 x Ls=16 Shamir, m_f = 0.01, eps = 0.5: mixed-precision CG
    "mixed": dict(name="shamir-16^3x32-Ls16-mixedCG", dims=(16, 16, 16, 32), Ls=16, M5=1.8, m=0.01, eps=0.5,
                  seed=2, inner="f32", madwf=False, sample_T=4),
    # the kernel-profiling case: every FP32 half-lattice field (509 MB) is larger than L2
    "hopprof": dict(name="shamir-24^3x48-Ls16-mixedCG", dims=(24, 24, 24, 48), Ls=16, M5=1.8, m=0.01, eps=0.5,
                    seed=2, inner="f32", madwf=False, sample_T=2),
    # Hasenbusch ladder: Moebius 32^3 x 64 x Ls=16 (b = 1.5, c = 0.5), four Gaussian sources at the
    # masses {0.001, 0.01, 0.05, 0.2}, solved together by the multi-right-hand-side CG
    "ladder": dict(name="ladder-mobius-32^3x64-Ls16-4rhs", dims=(32, 32, 32, 64), Ls=16, M5=1.8,
                   masses=(0.001, 0.01, 0.05, 0.2), m=0.001, b5=1.5, c5=0.5, eps=0.6, seed=5, inner="f32",
                   madwf=False, ladder=True, sample_T=2),
}
# FP64 CG iterations to 1e-10 on each input (GB300, dwf_cg inner=f64; for the ladder
# the summed iterations of its four mixed-precision solves); they scale the
# per-iteration oracle time of the reference arm when the FP64 solve is not run.
FP64_ITERS = {"madwf": 300, "mixed": 250, "hopprof": 260, "ladder": 1180}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="madwf", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--inner", default=None, choices=["f32", "f16"], help="inner precision (default per workload)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 CG comparison solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-10)
    return ap.parse_args()


def hop_traffic(bytes_per_launch):
    """DRAM bytes per launch of the FP32 hop (scaled from the ncu capture), or
    None if the kernel source differs from the one that was measured."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "paper_1111_5059_gb300", "csrc", "hop2.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    if sha != HOP_TRAFFIC["source_sha256_prefix"]:
        return None
    return bytes_per_launch * HOP_TRAFFIC["ratio"]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu, self.proc, self.lines = gpu_index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
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
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(self.NAMES, parts[5:9]):
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


def metric_name(w):
    if w.get("ladder"):
        return "DWF solve time @1e-10 (4-mass ladder, multi-RHS mixed CG)"
    return "DWF solve time @1e-10 (" + ("MADWF+mixed" if w["madwf"] else "mixed-precision CG") + ")"


def config_of(w, inner):
    X, Y, Z, T = w["dims"]
    c = {"workload": w["name"], "lattice": f"{X}x{Y}x{Z}x{T}", "Ls": w["Ls"], "M5": w["M5"], "m_f": w["m"],
         "eps": w["eps"], "seed": w["seed"], "tol": 1e-10, "inner": inner, "reliable_update_delta": DELTA,
         "l2": "inputs larger than L2 (each FP32 half-lattice field > 129 MB) plus a 512 MB write between steps"}
    if w["madwf"]:
        c.update({"Ls_inner": w["inner_Ls"], "b_inner": w["b"], "c_inner": w["c"], "n_dc": w["n_dc"],
                  "tol_pv": w["tol_pv"], "tol_mob": w["tol_mob"]})
        if inner == "f32":  # the library's trigger for the FP32 intermediate solves (include/dwf.h)
            c.update({"reliable_update_delta_pv": min(DELTA, max(math.sqrt(w["tol_pv"]), 1e-3)),
                      "reliable_update_delta_mob": min(DELTA, max(math.sqrt(w["tol_mob"]), 1e-3))})
    if w.get("ladder"):
        c.update({"m_f": list(w["masses"]), "b": w["b5"], "c": w["c5"], "nrhs": len(w["masses"]),
                  "sources": f"Gaussian, seeds {w['seed']}..{w['seed'] + len(w['masses']) - 1}"})
    return c


# --------------------------------------------------------------------------- oracle timing


def oracle_iteration_seconds(w):
    """Seconds per FP64 oracle CG iteration (M_pc then M_pc^+) on the workload,
    measured on a t-slab of sample_T timeslices and scaled to the full volume
    (the oracle's work per site does not depend on the lattice extent), and the
    host cores it kept busy: process CPU time over wall time of the timed part,
    rounded (numpy may run its array operations on several threads)."""
    import numpy as np

    from oracle import dwf_oracle as O
    from paper_1111_5059_gb300 import inputs

    X, Y, Z, T = w["dims"]
    dims = (X, Y, Z, w["sample_T"])
    U = inputs.gauge_field(w["seed"], dims, w["eps"])
    b = inputs.gaussian_spinor(w["seed"], dims, w["Ls"])
    eo = O.EO(U, w["m"], w["M5"], w["Ls"], w.get("b5", 1.0), w.get("c5", 0.0))
    v = b * eo.even
    t0, c0 = time.perf_counter(), time.process_time()
    q = eo.Mpc(v)
    v = eo.Mpc(q, True)
    v = v / np.sqrt(O.norm2(v))
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    return wall * (T / w["sample_T"]), max(1, round(cpu / wall))


def oracle_rates(w, per_it):
    """The oracle's rates from its time per full-volume CG iteration, which
    applies the Wilson hop four times (M_pc and M_pc^+, two hops each): hops
    per second over the whole 5D half lattice, and algorithmic FP64 GB/s (each
    spinor read or written once and the 8 links once per 4D site:
    48*8 + 144*8/Ls bytes per 5D half site and hop)."""
    X, Y, Z, T = w["dims"]
    sites = X * Y * Z * T // 2 * w["Ls"]
    bytes_per_hop = (48 * 8 + 144 * 8 / w["Ls"]) * sites
    return {"hops_per_s": 4.0 / per_it, "algorithmic_gbs": 4.0 * bytes_per_hop / per_it / 1e9}


def sample_text(w, iters, per_it):
    X, Y, Z, T = w["dims"]
    slab = f"a {X}x{Y}x{Z}x{w['sample_T']} t-slab scaled by {T // w['sample_T']}" if w["sample_T"] < T \
        else "the full lattice"
    what = "the summed iterations of the FP64 CG solves of the ladder's masses" if w.get("ladder") \
        else "the iterations of the FP64 CG solve of this input"
    return (f"one FP64 oracle CG iteration (M_pc then M_pc^+) on {slab} ({per_it:.1f} s per full-volume "
            f"iteration), times {iters}, {what}; numpy on a host with {os.cpu_count()} CPUs")


def run_reference(args, w):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    for _ in range(args.warmup):
        oracle_iteration_seconds(w)
    runs = [oracle_iteration_seconds(w) for _ in range(args.steps)]
    per_it = statistics.mean(t for t, _ in runs)
    cores = max(c for _, c in runs)
    iters = FP64_ITERS[args.workload]
    value = per_it * iters
    line = {"impl": "reference", "metric": metric_name(w), "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_it * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, "f64"),
            "cpu_baseline": dict({"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                                  "sample": sample_text(w, iters, per_it)}, **oracle_rates(w, per_it)),
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- native arm


def run_ladder(args, w, inner, world, rank, local, dev, hbm_peak, peak_src):
    """The mass ladder: one step is one dwf_cg_multi call over all masses (CUDA
    graphs on, launch shapes from the autotuner, tuned during warm-up)."""
    import torch

    from paper_1111_5059_gb300 import dwf, inputs

    masses = w["masses"]
    n = len(masses)
    U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], w["eps"])).to(dev)
    b_host = [torch.from_numpy(inputs.gaussian_spinor(w["seed"] + r, w["dims"], w["Ls"])).pin_memory()
              for r in range(n)]
    bs = [h.to(dev) for h in b_host]
    x_host = [torch.empty_like(h).pin_memory() for h in b_host]
    stream = torch.cuda.current_stream(dev)
    lat = dwf.Lattice(w["dims"], w["Ls"], w["M5"], w["b5"], w["c5"], 1, stream=stream, device=dev)
    lat.set_gauge(U)
    del U
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def solve(srcs):
        return lat.cg_multi(masses, srcs, tol=args.tol, inner=inner, delta=DELTA, check_every=10)

    tune_s = 0.0
    for _ in range(args.warmup):
        _, _, info, _ = solve(bs)
        tune_s += info["tune_seconds"]
    torch.cuda.synchronize()

    lat.set_kernel_timing(True)
    n0 = lat.launch_count()
    step_ms, infos, stats = [], [], []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            xs, st, info, _ = solve(bs)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            infos.append(info)
            stats.append(st)
            del xs
    torch.cuda.synchronize()
    barrier(world)
    launches = lat.launch_count() - n0
    kt = lat.kernel_time(inner)
    lat.set_kernel_timing(False)
    total_ms = max_over_ranks(world, sum(step_ms), dev)
    ms_step = total_ms / args.steps
    value = ms_step / 1e3 / world

    # ---- e2e: sources from pinned host memory in, solutions back out, inside the timed region
    e2e = []
    for _ in range(max(1, min(args.steps, 2))):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bd = [h.to(dev, non_blocking=True) for h in b_host]
        xs, _, _, _ = solve(bd)
        for xh, xd in zip(x_host, xs):
            xh.copy_(xd, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e.append(e0.elapsed_time(e1))
        del bd, xs
    e2e_ms = max_over_ranks(world, statistics.mean(e2e), dev)

    # ---- the same ladder with every right-hand side in one hop launch (no autotuning)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, _, info_all, _ = lat.cg_multi(masses, bs, tol=args.tol, inner=inner, delta=DELTA, check_every=10,
                                     autotune=False)
    e1.record(stream)
    e1.synchronize()
    one_launch = {"seconds": e0.elapsed_time(e1) / 1e3, "batch": info_all["batch"]}

    # ---- the same four solves one after the other (single-RHS mixed CG)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    seq = [lat.cg(m, bb, tol=args.tol, inner=inner, delta=DELTA, check_every=10) for m, bb in zip(masses, bs)]
    e1.record(stream)
    e1.synchronize()
    seq_s = e0.elapsed_time(e1) / 1e3
    sequential = {"seconds": seq_s, "iters": [r.stats["iters"] for r in seq],
                  "true_resid": [r.stats["true_resid"] for r in seq], "speedup_of_headline": seq_s / (ms_step / 1e3)}
    del seq

    st, info = stats[-1], infos[-1]
    achieved = kt["bytes"] / (kt["ms"] / 1e3) / 1e9 if kt["ms"] > 0 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": (achieved / hbm_peak) if achieved else None,
            "frac_of_nominal_7900_gbs": (achieved / HBM_NOMINAL_GBS) if achieved else None,
            "traffic": hop_traffic(kt["bytes"] / max(1, kt["launches"])) if inner == "f32" else None,
            "kernel": f"hop3_kernel<{inner}> batched over right-hand sides (Wilson hop at every s, fused "
                      "fifth-dimension epilogues per mass)",
            "launches": kt["launches"], "avg_launch_us": kt["ms"] / max(1, kt["launches"]) * 1e3,
            "bytes_per_launch": kt["bytes"] / max(1, kt["launches"]),
            "timed_launches": "the eager first iteration of each batch (graph replays are not bracketed by events)",
            "peak_source": ("of measured hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                            else "of fallback 6.8 TB/s")}
    solve_info = {"iters": [s["iters"] for s in st], "reliable_updates": [s["reliable_updates"] for s in st],
                  "op_count": [s["op_count"] for s in st], "true_resid": [s["true_resid"] for s in st],
                  "joint_iterations": info["iterations"], "batch": info["batch"], "ctas_per_sm": info["ctas_per_sm"],
                  "graphs": info["graphs"], "replays": info["replays"], "autotune_seconds_warmup": tune_s,
                  "step_ms": step_ms}
    line = {"metric": metric_name(w), "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if inner == "f32" else "f16-storage/f32+f64",
            "data": "synthetic", "config": config_of(w, inner), "roofline": roof,
            "e2e": {"value": e2e_ms / 1e3 / world, "unit": "s",
                    "h2d_bytes_per_step": sum(h.numel() * 16 for h in b_host),
                    "d2h_bytes_per_step": sum(h.numel() * 16 for h in x_host)},
            "gpu_launches": launches, "solve": solve_info, "sequential_cg": sequential,
            "all_rhs_one_launch": one_launch, "clocks": clk.summary()}
    if rank == 0:
        if not args.no_cpu_baseline:
            iters = sum(s["iters"] for s in st)
            per_it, cores = oracle_iteration_seconds(w)
            line["cpu_baseline"] = {"value": per_it * iters, "unit": "s", "cores": cores, "kind": "oracle",
                                    "sample": sample_text(w, iters, per_it)
                                    + " (the mixed solves' iteration counts stand in for FP64 CG's)"}
            line["cpu_baseline"].update(oracle_rates(w, per_it))
        print(json.dumps(line), flush=True)
    lat.close()


def main():
    args = parse()
    w = WORKLOADS[args.workload]
    inner = args.inner or w["inner"]
    if args.impl == "reference":
        run_reference(args, w)
        return
    import torch

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1111_5059_gb300 import dwf, inputs

    if not os.path.exists(dwf.LIB_PATH):
        from paper_1111_5059_gb300 import build

        build.build()
    hbm_peak, peak_src = measured_peak()
    if w.get("ladder"):
        run_ladder(args, w, inner, world, rank, local, dev, hbm_peak, peak_src)
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], w["eps"])).to(dev)
    b_host = torch.from_numpy(inputs.gaussian_spinor(w["seed"], w["dims"], w["Ls"])).pin_memory()
    b = b_host.to(dev)
    x_host = torch.empty_like(b_host).pin_memory()
    stream = torch.cuda.current_stream(dev)
    lat = dwf.Lattice(w["dims"], w["Ls"], w["M5"], 1.0, 0.0, 1, stream=stream, device=dev)
    lat.set_gauge(U)
    lats = [lat]
    if w["madwf"]:
        mob = dwf.Lattice(w["dims"], w["inner_Ls"], w["M5"], w["b"], w["c"], 1, stream=stream, device=dev)
        mob.set_gauge(U)
        lats.append(mob)
    del U
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def solve(bb):
        if w["madwf"]:
            return dwf.madwf_solve(lat, mob, w["m"], bb, n_dc=w["n_dc"], tol_pv=w["tol_pv"], tol_mob=w["tol_mob"],
                                   tol_final=args.tol, inner_prec=inner, delta=DELTA, check_every=10)
        return lat.cg(w["m"], bb, tol=args.tol, inner=inner, delta=DELTA, check_every=10)

    for _ in range(args.warmup):
        r = solve(b)
    torch.cuda.synchronize()

    # ---- timed region: K solves with inputs resident in HBM
    for L in lats:
        L.set_kernel_timing(True)
    n0 = sum(L.launch_count() for L in lats)
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
    launches = sum(L.launch_count() for L in lats) - n0
    kts = [L.kernel_time(inner) for L in lats]
    for L in lats:
        L.set_kernel_timing(False)
    kt = {k: sum(d[k] for d in kts) for k in ("ms", "launches", "bytes")}
    total_ms = max_over_ranks(world, sum(step_ms), dev)
    ms_step = total_ms / args.steps
    value = ms_step / 1e3 / world  # seconds per solve for the whole job
    st = stats[-1]
    true_res = st["total"]["true_resid"] if w["madwf"] else st["true_resid"]

    # ---- e2e: the same solve through the C ABI from pinned host buffers
    e2e = []
    for _ in range(max(1, min(args.steps, 2))):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bd = b_host.to(dev, non_blocking=True)
        rr = solve(bd)
        x_host.copy_(rr.x, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e.append(e0.elapsed_time(e1))
        del bd, rr
    e2e_ms = max_over_ranks(world, statistics.mean(e2e), dev)

    # ---- comparisons on the same GPU: plain FP64 CG (and mixed CG for MADWF)
    comp = {}
    if not args.no_fp64:
        for name, prec in (("fp64_cg", "f64"),) + ((("mixed_cg", inner),) if w["madwf"] else ()):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rf = lat.cg(w["m"], b, tol=args.tol, inner=prec, delta=DELTA, check_every=10)
            e1.record(stream)
            e1.synchronize()
            secs = e0.elapsed_time(e1) / 1e3
            comp[name] = {"seconds": secs, "iters": rf.stats["iters"], "op_count": rf.stats["op_count"],
                          "true_resid": rf.stats["true_resid"], "speedup_of_headline": secs / (ms_step / 1e3)}
            del rf

    achieved = kt["bytes"] / (kt["ms"] / 1e3) / 1e9 if kt["ms"] > 0 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": (achieved / hbm_peak) if achieved else None,
            "frac_of_nominal_7900_gbs": (achieved / HBM_NOMINAL_GBS) if achieved else None,
            "traffic": hop_traffic(kt["bytes"] / max(1, kt["launches"])) if inner == "f32" else None,
            "traffic_source": "ncu DRAM read+write per algorithmic byte on 24^3x48x16 Ls=16, scaled to this launch size",
            "kernel": f"hop3_kernel<{inner}> (Wilson hop at every s with fused fifth-dimension epilogues)",
            "launches": kt["launches"], "avg_launch_us": kt["ms"] / max(1, kt["launches"]) * 1e3,
            "bytes_per_launch": kt["bytes"] / max(1, kt["launches"]),
            "share_of_step": kt["ms"] / max(1e-9, sum(step_ms)),
            "peak_source": ("of measured hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                            else "of fallback 6.8 TB/s")}
    if w["madwf"]:
        solve_info = {"passes": st["passes"], "pass_resid": st["pass_resid"], "true_resid": true_res,
                      "mobius_iters": st["mobius"]["iters"], "pv_iters": st["pv"]["iters"],
                      "final_iters": st["final_cg"]["iters"],
                      "op_count": {"mobius": st["mobius"]["op_count"], "pv": st["pv"]["op_count"],
                                   "final": st["final_cg"]["op_count"], "total": st["total"]["op_count"]},
                      "step_ms": step_ms}
    else:
        solve_info = {"iters": st["iters"], "reliable_updates": st["reliable_updates"], "op_count": st["op_count"],
                      "true_resid": true_res, "step_ms": step_ms}
    line = {"metric": metric_name(w), "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if inner == "f32" else "f16-storage/f32+f64",
            "data": "synthetic", "config": config_of(w, inner), "roofline": roof,
            "e2e": {"value": e2e_ms / 1e3 / world, "unit": "s", "h2d_bytes_per_step": b_host.numel() * 16,
                    "d2h_bytes_per_step": x_host.numel() * 16},
            "gpu_launches": launches, "solve": solve_info, "clocks": clk.summary()}
    line.update(comp)
    if rank == 0:
        if not args.no_cpu_baseline:
            iters = comp["fp64_cg"]["iters"] if "fp64_cg" in comp else FP64_ITERS[args.workload]
            per_it, cores = oracle_iteration_seconds(w)
            line["cpu_baseline"] = {"value": per_it * iters, "unit": "s", "cores": cores, "kind": "oracle",
                                    "sample": sample_text(w, iters, per_it)}
            line["cpu_baseline"].update(oracle_rates(w, per_it))
        print(json.dumps(line), flush=True)
    for L in lats:
        L.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
