#!/usr/bin/env python3
"""Benchmark of the domain-wall hot path on GB300.

Metric: DWF solve time to a 1e-10 true residual |b - D(m) x| / |b|.  The
headline workload is the Moebius-accelerated solve (MADWF, FP32 inner solves
with FP64 reliable updates and FP64 defect correction) of Shamir DWF on
24^3 x 64 x Ls=32 through a Moebius operator at Ls'=12; plain FP64 and plain
mixed-precision CG on the same GPU and input are measured beside it, and the
Wilson hop (Dslash) kernel's achieved HBM bandwidth is reported against the
measured copy peak.  The headline line also carries the 16^3 x 32 x Ls=16
precision comparison (FP64 / FP32 / FP16-storage CG with each hop's
bandwidth) and the 32^3 x 64 x Ls=16 four-mass ladder (multi-right-hand-side
solve against four sequential solves).

A step is one solve from a zero guess on seeded synthetic inputs already
resident in HBM (timed with CUDA events on the solve's stream).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload madwf|mixed|hopprof|ladder]
                  [--impl native|reference] [--study [--study-ls]] [--md-study] [--hasenbusch-study]
                  [--hmc-study] [--no-fp64] [--no-extras]
                  [--no-cpu-baseline]

--study (with the madwf workload) sweeps the MADWF settings (defect-correction
passes, Pauli-Villars and Moebius tolerances, the Moebius scale b + c, and two
rougher gauge fields) and prints one JSON line per setting; --md-study prints
force-gradient against Omelyan trajectories (dH, force evaluations, time) at
several step sizes on the 16^3 x 8 x Ls=16 force workload.

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

# Reliable-update trigger (the iterated residual is replaced by the FP64 one
# once it has dropped by this factor).  FP32 storage: 1e-4, measured on the
# headline input to give the same iterations and residuals as 1e-2 and 1e-3
# with fewer FP64 residuals per solve (MADWF 3.21 s at 1e-2, 3.02 s at 1e-3
# with polls every 10 iterations; 2.67 s at 1e-3 and 2.61 s at 1e-4 with
# polls every iteration); FP16 storage keeps 1e-2 (its recursion drifts
# faster).
DELTA = 1e-4
DELTA_F16 = 1e-2


# Iterations between the host's convergence polls of a single-right-hand-side
# solve: 1 (each poll is a scalar copy and a stream synchronisation, ~0.5 %
# of a 24^3x64x32 iteration) stops a solve as soon as it converges, against
# 4.5 extra iterations on average at 10 (MADWF 2.92 s against 3.02 s).
CHECK_EVERY = 1


def delta_for(inner):
    return DELTA_F16 if inner == "f16" else DELTA


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic
# byte of the FP32 hop kernel, by slice pairs per 4D site (Lh), from ncu
# captures of the apply workloads (four launches each: M_pc and M_pc^+
# applications); they hold only for the kernel source they were taken on.
HOP_TRAFFIC = {"source_sha256_prefix": "9a3c6a302ef70cb9", "ratio_by_lh": {8: 1.0286, 16: 1.0459, 6: 1.1658},
               "captures": "apply (Lh 8), apply-ls32 (Lh 16), apply-mobius-ls12 (Lh 6)"}

WORKLOADS = {
    # MADWF: Shamir 24^3 x 64 x Ls=32, m_f = 0.002, eps = 0.6, through Moebius Ls' = 12 with
    # b - c = 1 and b + c = Ls / Ls' (b = 11/6, c = 5/6).  Defect-correction passes and the
    # intermediate tolerances are the fastest setting of the --study sweep on this input (one
    # pass, Pauli-Villars 1e-3, Moebius 1e-2; three passes at 1e-6 / 1e-5 took 2.5x longer).
    "madwf": dict(name="madwf-shamir-24^3x64-Ls32-via-mobius-Ls12", dims=(24, 24, 24, 64), Ls=32, M5=1.8,
                  m=0.002, eps=0.6, seed=3, inner="f32", madwf=True, inner_Ls=12, b=11 / 6, c=5 / 6, n_dc=1,
                  tol_pv=1e-3, tol_mob=1e-2, sample=(24, 24, 4, 2)),
    # 16^3 x 32 x Ls=16 Shamir, m_f = 0.01, eps = 0.5: mixed-precision CG
    "mixed": dict(name="shamir-16^3x32-Ls16-mixedCG", dims=(16, 16, 16, 32), Ls=16, M5=1.8, m=0.01, eps=0.5,
                  seed=2, inner="f32", madwf=False, sample=(16, 16, 8, 2)),
    # the kernel-profiling case: every FP32 half-lattice field (509 MB) is larger than L2
    "hopprof": dict(name="shamir-24^3x48-Ls16-mixedCG", dims=(24, 24, 24, 48), Ls=16, M5=1.8, m=0.01, eps=0.5,
                    seed=2, inner="f32", madwf=False, sample=(24, 24, 6, 2)),
    # operator-only case for kernel profiles: FP32 M_pc applications (the solvers' hop launches) on
    # 20^3 x 24 x Ls=16; each FP32 half-lattice field (147 MB) is larger than L2, ~2.5 GB in all
    "apply": dict(name="mpc-f32-shamir-20^3x24-Ls16", dims=(20, 20, 20, 24), Ls=16, M5=1.8, m=0.01, eps=0.5,
                  seed=2, inner="f32", madwf=False, apply=True, sample=(20, 20, 4, 2)),
    # the same at the headline's fifth-dimension shapes (Shamir Ls = 32, Moebius Ls' = 12), for
    # profiling the kernels the headline solve runs; each FP32 half-lattice field exceeds L2
    "apply-ls32": dict(name="mpc-f32-shamir-16^3x32-Ls32", dims=(16, 16, 16, 32), Ls=32, M5=1.8, m=0.002,
                       eps=0.6, seed=3, inner="f32", madwf=False, apply=True, sample=(16, 16, 4, 2)),
    "apply-mobius-ls12": dict(name="mpc-f32-mobius-24^3x32-Ls12", dims=(24, 24, 24, 32), Ls=12, M5=1.8, m=0.002,
                              eps=0.6, seed=3, inner="f32", madwf=False, apply=True, b5=11 / 6, c5=5 / 6,
                              sample=(24, 24, 4, 2)),
    # Hasenbusch ladder: Moebius 32^3 x 64 x Ls=16 (b = 1.5, c = 0.5), four Gaussian sources at the
    # masses {0.001, 0.01, 0.05, 0.2}, solved together by the multi-right-hand-side CG
    "ladder": dict(name="ladder-mobius-32^3x64-Ls16-4rhs", dims=(32, 32, 32, 64), Ls=16, M5=1.8,
                   masses=(0.001, 0.01, 0.05, 0.2), m=0.001, b5=1.5, c5=0.5, eps=0.6, seed=5, inner="f32",
                   madwf=False, ladder=True, sample=(32, 32, 4, 2)),
}
# FP64 CG iterations to 1e-10 on each input (GB300, dwf_cg inner=f64; for the ladder
# the summed iterations of its four mixed-precision solves); they scale the
# per-iteration oracle time of the reference arm when the FP64 solve is not run.
FP64_ITERS = {"madwf": 300, "mixed": 250, "hopprof": 260, "ladder": 1180,
              "apply": 0.5, "apply-ls32": 0.5, "apply-mobius-ls12": 0.5}
# (an apply workload's unit is one M_pc application, half an iteration's work)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="madwf", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--inner", default=None, choices=["f32", "f16"], help="inner precision (default per workload)")
    ap.add_argument("--study", action="store_true", help="sweep the MADWF settings (madwf workload)")
    ap.add_argument("--study-ls", action="store_true", help="with --study: sweep Ls' and b + c in the bench's settings")
    ap.add_argument("--md-study", action="store_true", help="FGI against Omelyan trajectories on the force workload")
    ap.add_argument("--hmc-study", action="store_true",
                    help="HMC chains (heat bath, trajectory, Metropolis) with FGI and Omelyan on the force workload")
    ap.add_argument("--hasenbusch-study", action="store_true",
                    help="geometric and force-balanced Hasenbusch ladders, force solves at 1e-8 and 1e-6")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 CG comparison solve")
    ap.add_argument("--no-extras", action="store_true", help="skip the precision comparison and the ladder")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-10)
    return ap.parse_args()


def host_copy(dwf, arr):
    """A page-locked, huge-page-backed host copy of a numpy array
    (dwf.host_empty): the host side of the end-to-end copies."""
    import torch

    t = dwf.host_empty(arr.shape)
    t.copy_(torch.from_numpy(arr))
    return t


def thp_fraction(t):
    """Fraction of a host tensor's mapping backed by transparent huge pages
    (AnonHugePages over Size in /proc/self/smaps), or None if unknown."""
    try:
        addr = t.data_ptr()
        cur = None
        with open("/proc/self/smaps") as f:
            for line in f:
                head = line.split()
                if head and "-" in head[0] and len(head) >= 5 and ":" not in head[0]:
                    lo, hi = (int(v, 16) for v in head[0].split("-"))
                    cur = {} if lo <= addr < hi else None
                elif cur is not None and line.startswith(("Size:", "AnonHugePages:")):
                    cur[head[0][:-1]] = int(head[1])
                    if len(cur) == 2:
                        return cur["AnonHugePages"] / max(1, cur["Size"])
    except (OSError, ValueError):
        pass
    return None


HOST_BUFFERS = ("page-locked host buffers from dwf_host_alloc (transparent huge pages, cudaHostRegister): "
                "with base pages the first copy after a solve ran at 6-50 GB/s while the host-page "
                "translations were fetched again")


def hop_kernel_name(prec, batch=1):
    """The hop kernel the library launches for this storage precision: the FP32
    single-right-hand-side fast path, else the general slice-pair kernel."""
    if prec == "f32" and batch == 1:
        return ("hopf_kernel (FP32 Wilson hop at every s on slice pairs, bulk-copy staging, fused "
                "fifth-dimension epilogues)")
    return (f"hop3_kernel<{prec}>" + (f" batched over {batch} right-hand sides" if batch > 1 else "")
            + " (Wilson hop at every s on slice pairs, fused fifth-dimension epilogues)")


def hop_traffic(parts, launches):
    """DRAM bytes per launch of the FP32 hop: the algorithmic bytes of each
    lattice's launches (parts: [(Ls, bytes)]) times the measured ratio at its
    Lh, over the launches; None if the kernel source differs from the one
    that was measured or an Lh was not measured."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "paper_1111_5059_gb300", "csrc", "hop2.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    if sha != HOP_TRAFFIC["source_sha256_prefix"] or launches < 1:
        return None
    total = 0.0
    for Ls, nbytes in parts:
        r = HOP_TRAFFIC["ratio_by_lh"].get((Ls + 1) // 2)
        if r is None:
            return None
        total += nbytes * r
    return total / launches


TRAFFIC_SOURCE = ("ncu DRAM read+write per algorithmic byte of the same kernel at the same Lh on a smaller "
                  "lattice (apply workloads), times this run's algorithmic bytes (null: the kernel source "
                  "changed since it was measured)")


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
         "eps": w["eps"], "seed": w["seed"], "tol": 1e-10, "inner": inner, "reliable_update_delta": delta_for(inner), "check_every": CHECK_EVERY,
         "l2": "inputs larger than L2 (each FP32 half-lattice field > 129 MB) plus a 512 MB write between steps"}
    if w["madwf"]:
        c.update({"Ls_inner": w["inner_Ls"], "b_inner": w["b"], "c_inner": w["c"], "n_dc": w["n_dc"],
                  "tol_pv": w["tol_pv"], "tol_mob": w["tol_mob"]})
        if inner == "f32":  # the library's trigger for the FP32 intermediate solves (include/dwf.h)
            c.update({"reliable_update_delta_pv": min(delta_for(inner), max(math.sqrt(w["tol_pv"]), 1e-3)),
                      "reliable_update_delta_mob": min(delta_for(inner), max(math.sqrt(w["tol_mob"]), 1e-3))})
        c["madwf_settings"] = "fastest of the --study sweep on this input"
        c["note"] = ("on these near-identity links plain mixed-precision CG (mixed_cg) is faster than MADWF: the "
                     "direct solve needs only ~300 iterations, so the Pauli-Villars solves of a pass cost more than "
                     "the final solve saves; MADWF gains where direct CG needs many more iterations (rough fields "
                     "at light mass; the paper's direct solve took 11290)")
    if w.get("ladder"):
        c.update({"m_f": list(w["masses"]), "b": w["b5"], "c": w["c5"], "nrhs": len(w["masses"]),
                  "sources": f"Gaussian, seeds {w['seed']}..{w['seed'] + len(w['masses']) - 1}"})
    return c


# --------------------------------------------------------------------------- oracle timing on the host cores

_SAMPLE = None  # (oracle module, EO blocks, vector) of this worker process


def _oracle_init(spec):
    """Worker set-up: the oracle's even-odd blocks on the sample sub-lattice."""
    global _SAMPLE
    sys.path.insert(0, ROOT)
    from oracle import dwf_oracle as O
    from paper_1111_5059_gb300 import inputs

    U = inputs.gauge_field(spec["seed"], spec["sample"], spec["eps"])
    b = inputs.gaussian_spinor(spec["seed"], spec["sample"], spec["Ls"])
    eo = O.EO(U, spec["m"], spec["M5"], spec["Ls"], spec["b5"], spec["c5"])
    _SAMPLE = (O, eo, b * eo.even)


def _oracle_iteration(_):
    """One FP64 oracle CG iteration's operator work (M_pc, then M_pc^+, and a
    norm) on the sample; returns its wall and process CPU seconds."""
    import numpy as np

    O, eo, v = _SAMPLE
    t0, c0 = time.perf_counter(), time.process_time()
    q = eo.Mpc(v)
    v = eo.Mpc(q, True)
    v = v / np.sqrt(O.norm2(v))
    return time.perf_counter() - t0, time.process_time() - c0


class OracleTimer:
    """The FP64 oracle timed on the host's cores: one worker process per core
    (spawned, BLAS threads 1), each running the oracle's CG-iteration work on
    its own copy of a sub-lattice sample of the workload (the oracle's cost
    per 5D site does not depend on the lattice extent).  A step runs one
    iteration on every worker at once; its wall time, scaled by the full
    volume over the volume all workers covered, is the oracle's time per
    full-volume CG iteration on this host."""

    def __init__(self, w, workers=None):
        import multiprocessing as mp

        self.w = w
        self.workers = workers or len(os.sched_getaffinity(0))
        spec = {"seed": w["seed"], "sample": w["sample"], "eps": w["eps"], "Ls": w["Ls"], "m": w["m"],
                "M5": w["M5"], "b5": w.get("b5", 1.0), "c5": w.get("c5", 0.0)}
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        os.environ.update({k: "1" for k in saved})
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_init, initargs=(spec,))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        X, Y, Z, T = w["dims"]
        sx, sy, sz, st = w["sample"]
        self.scale = (X * Y * Z * T) / (self.workers * sx * sy * sz * st)

    def step(self):
        """(wall seconds of one step, seconds per full-volume iteration, busy cores)."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_iteration, range(self.workers), chunksize=1)
        wall = time.perf_counter() - t0
        busy = sum(c for _, c in res) / wall
        return wall, wall * self.scale, max(1, round(busy))

    def sample_text(self, iters, per_it):
        X, Y, Z, T = self.w["dims"]
        sx, sy, sz, st = self.w["sample"]
        what = "the summed iterations of the FP64 CG solves of the ladder's masses" if self.w.get("ladder") \
            else "the iterations of the FP64 CG solve of this input"
        return (f"{self.workers} host cores each run one FP64 oracle CG iteration (M_pc then M_pc^+) on its own "
                f"{sx}x{sy}x{sz}x{st}x{self.w['Ls']} sub-lattice at once; the step's wall time times "
                f"{self.scale:.2f} (the {X}x{Y}x{Z}x{T} volume over the volume covered) gives {per_it:.1f} s per "
                f"full-volume iteration, times {iters}, {what} (extrapolated); numpy on a host with "
                f"{os.cpu_count()} CPUs")

    def close(self):
        self.pool.terminate()
        self.pool.join()


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


def cpu_baseline(w, iters):
    """The oracle's extrapolated solve time on the host's cores (one warm-up step, one timed)."""
    ot = OracleTimer(w)
    try:
        ot.step()
        wall, per_it, cores = ot.step()
    finally:
        ot.close()
    d = {"value": per_it * iters, "unit": "s", "cores": cores, "kind": "oracle",
         "sample": ot.sample_text(iters, per_it), "extrapolated": True, "step_seconds": wall,
         "volume_factor": ot.scale, "iterations": iters}
    d.update(oracle_rates(w, per_it))
    return d


def run_reference(args, w):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    ot = OracleTimer(w)
    try:
        for _ in range(args.warmup):
            ot.step()
        runs = [ot.step() for _ in range(args.steps)]
    finally:
        ot.close()
    wall = statistics.mean(r[0] for r in runs)
    per_it = statistics.mean(r[1] for r in runs)
    cores = max(r[2] for r in runs)
    iters = FP64_ITERS[args.workload]
    value = per_it * iters
    line = {"impl": "reference", "metric": metric_name(w), "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, "f64"),
            "extrapolated": {"value_is": "solve time = measured step wall time x volume_factor x iterations",
                             "step": "one oracle CG iteration on every host core's sub-lattice at once",
                             "step_seconds": wall, "volume_factor": ot.scale, "iterations": iters,
                             "seconds_per_full_iteration": per_it},
            "cpu_baseline": dict({"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                                  "sample": ot.sample_text(iters, per_it)}, **oracle_rates(w, per_it)),
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- native arm helpers


def _events(n):
    import torch

    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def roofline(kt, hbm_peak, peak_src, kernel, extra=None):
    """Achieved algorithmic GB/s of the hop launches of one precision (CUDA
    events around every launch) against the measured copy peak."""
    achieved = kt["bytes"] / (kt["ms"] / 1e3) / 1e9 if kt["ms"] > 0 else None
    r = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
         "frac": (achieved / hbm_peak) if achieved else None,
         "frac_of_nominal_7900_gbs": (achieved / HBM_NOMINAL_GBS) if achieved else None,
         "kernel": kernel, "launches": kt["launches"], "avg_launch_us": kt["ms"] / max(1, kt["launches"]) * 1e3,
         "bytes_per_launch": kt["bytes"] / max(1, kt["launches"]),
         "peak_source": ("of measured hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                         else "of fallback 6.8 TB/s")}
    if extra:
        r.update(extra)
    return r


def precision_comparison(dev, stream, hbm_peak, peak_src, tol):
    """16^3 x 32 x Ls=16 Shamir (m_f = 0.01, eps = 0.5): FP64, FP32 and
    FP16-storage CG to the same true residual, with each precision's hop
    bandwidth (one warm-up solve each, then one event-timed solve)."""
    import torch

    from paper_1111_5059_gb300 import dwf, inputs

    w = WORKLOADS["mixed"]
    U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], w["eps"])).to(dev)
    b = torch.from_numpy(inputs.gaussian_spinor(w["seed"], w["dims"], w["Ls"])).to(dev)
    lat = dwf.Lattice(w["dims"], w["Ls"], w["M5"], 1.0, 0.0, 1, stream=stream, device=dev)
    lat.set_gauge(U)
    x = torch.empty_like(b)
    out = {"workload": w["name"], "lattice": "16x16x16x32", "Ls": 16, "m_f": w["m"], "tol": tol}
    for prec in ("f64", "f32", "f16"):
        lat.cg(w["m"], b, tol=tol, inner=prec, delta=delta_for(prec), check_every=CHECK_EVERY, out=x)
        lat.set_kernel_timing(True)
        e0, e1 = _events(2)
        e0.record(stream)
        r = lat.cg(w["m"], b, tol=tol, inner=prec, delta=delta_for(prec), check_every=CHECK_EVERY, out=x)
        e1.record(stream)
        e1.synchronize()
        kt = lat.kernel_time(prec)
        lat.set_kernel_timing(False)
        kernel = "hop_kernel<f64> (FP64 Wilson hop; bound by the FP64 pipe, not HBM)" if prec == "f64" else \
            hop_kernel_name(prec)
        rf = roofline(kt, hbm_peak, peak_src, kernel,
                      {"traffic": hop_traffic([(w["Ls"], kt["bytes"])], kt["launches"]), "traffic_source": TRAFFIC_SOURCE}
                      if prec == "f32" else None)
        if prec == "f64":
            rf["bound"] = "fp64-alu"
        out[prec] = {"seconds": e0.elapsed_time(e1) / 1e3, "iters": r.stats["iters"],
                     "reliable_updates": r.stats["reliable_updates"], "true_resid": r.stats["true_resid"],
                     "hop": rf}
    lat.close()
    return out


def trajectory_timing(dev, stream):
    """One force-gradient trajectory on the 16^3 x 8 x Ls=16 force workload
    (quotient terms (0.01, 0.1) and (0.1, 1.0), length 0.4 in 4 steps, FP32
    inner solves with FP64 reliable updates to 1e-10), after one warm-up
    trajectory: time, force evaluations, solver iterations and dH."""
    import torch

    from paper_1111_5059_gb300 import dwf, inputs

    dims, Ls = (16, 16, 16, 8), 16
    terms = [(0.01, 0.1), (0.1, 1.0)]
    U0 = torch.from_numpy(inputs.gauge_field(4, dims, 0.5)).to(dev)
    p0 = torch.from_numpy(inputs.gaussian_momenta(4, dims)).to(dev)
    phis = [torch.from_numpy(inputs.gaussian_spinor(50 + k, dims, Ls)).to(dev) for k in range(2)]
    lat = dwf.Lattice(dims, Ls, 1.8, 1.0, 0.0, 1, stream=stream, device=dev)
    out = {"workload": "force-shamir-16^3x8-Ls16-2terms", "integrator": "fgi", "tau": 0.1, "nsteps": 4}
    for rep in range(2):
        U, p = U0.clone(), p0.clone()
        e0, e1 = _events(2)
        e0.record(stream)
        H0, H1, st, nf = dwf.md_trajectory(lat, terms, phis, U, p, 0.1, 4, tol=1e-10, inner="f32", delta=DELTA)
        e1.record(stream)
        e1.synchronize()
        out.update({"seconds": e0.elapsed_time(e1) / 1e3, "force_evaluations": nf, "cg_iters": st["iters"],
                    "dH": H1 - H0})
    lat.close()
    return out


def ladder_comparison(dev, stream, tol):
    """32^3 x 64 x Ls=16 Moebius ladder (masses {0.001, 0.01, 0.05, 0.2},
    four Gaussian sources): the multi-right-hand-side solve (tuned in one
    warm-up call) against the same four solves one after the other."""
    import torch

    from paper_1111_5059_gb300 import dwf, inputs

    w = WORKLOADS["ladder"]
    masses = w["masses"]
    U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], w["eps"])).to(dev)
    lat = dwf.Lattice(w["dims"], w["Ls"], w["M5"], w["b5"], w["c5"], 1, stream=stream, device=dev)
    lat.set_gauge(U)
    del U
    bs = [torch.from_numpy(inputs.gaussian_spinor(w["seed"] + r, w["dims"], w["Ls"])).to(dev)
          for r in range(len(masses))]
    _, _, info, _ = lat.cg_multi(masses, bs, tol=tol, inner="f32", delta=DELTA, check_every=10)
    tune_s = info["tune_seconds"]
    e0, e1, e2 = _events(3)
    e0.record(stream)
    xs, st, info, _ = lat.cg_multi(masses, bs, tol=tol, inner="f32", delta=DELTA, check_every=10)
    e1.record(stream)
    del xs
    seq = [lat.cg(m, bb, tol=tol, inner="f32", delta=DELTA, check_every=10) for m, bb in zip(masses, bs)]
    e2.record(stream)
    e2.synchronize()
    res = {"workload": w["name"], "multi_rhs_seconds": e0.elapsed_time(e1) / 1e3,
           "sequential_seconds": e1.elapsed_time(e2) / 1e3, "batch": info["batch"],
           "ctas_per_sm": info["ctas_per_sm"], "autotune_seconds": tune_s,
           "iters": [s["iters"] for s in st], "true_resid": [s["true_resid"] for s in st],
           "sequential_iters": [r.stats["iters"] for r in seq]}
    del seq, bs
    lat.close()
    return res


# --------------------------------------------------------------------------- native arm


def run_ladder(args, w, inner, world, rank, local, dev, hbm_peak, peak_src):
    """The mass ladder: one step is one dwf_cg_multi call over all masses (CUDA
    graphs on, launch shapes from the autotuner, tuned during warm-up)."""
    import torch

    from paper_1111_5059_gb300 import dwf, inputs

    masses = w["masses"]
    n = len(masses)
    U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], w["eps"])).to(dev)
    b_host = [host_copy(dwf, inputs.gaussian_spinor(w["seed"] + r, w["dims"], w["Ls"])) for r in range(n)]
    bs = [h.to(dev) for h in b_host]
    x_host = [dwf.host_empty(h.shape) for h in b_host]
    stream = torch.cuda.current_stream(dev)
    lat = dwf.Lattice(w["dims"], w["Ls"], w["M5"], w["b5"], w["c5"], 1, stream=stream, device=dev)
    lat.set_gauge(U)
    del U
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def solve(srcs):
        return lat.cg_multi(masses, srcs, tol=args.tol, inner=inner, delta=delta_for(inner), check_every=10)

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
            e0, e1 = _events(2)
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
    bd = [torch.empty_like(b) for b in bs]
    for _ in range(max(1, min(args.steps, 2))):
        flush.fill_(1.0)
        e0, e1 = _events(2)
        e0.record(stream)
        for d, h in zip(bd, b_host):
            d.copy_(h, non_blocking=True)
        xs, _, _, _ = solve(bd)
        for xh, xd in zip(x_host, xs):
            xh.copy_(xd, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e.append(e0.elapsed_time(e1))
        del xs
    e2e_ms = max_over_ranks(world, statistics.mean(e2e), dev)
    del bd

    # ---- the same ladder with every right-hand side in one hop launch (no autotuning)
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    e0.record(stream)
    _, _, info_all, _ = lat.cg_multi(masses, bs, tol=args.tol, inner=inner, delta=delta_for(inner), check_every=10,
                                     autotune=False)
    e1.record(stream)
    e1.synchronize()
    one_launch = {"seconds": e0.elapsed_time(e1) / 1e3, "batch": info_all["batch"]}

    # ---- the same four solves one after the other (single-RHS mixed CG)
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    e0.record(stream)
    seq = [lat.cg(m, bb, tol=args.tol, inner=inner, delta=delta_for(inner), check_every=10) for m, bb in zip(masses, bs)]
    e1.record(stream)
    e1.synchronize()
    seq_s = e0.elapsed_time(e1) / 1e3
    sequential = {"seconds": seq_s, "iters": [r.stats["iters"] for r in seq],
                  "true_resid": [r.stats["true_resid"] for r in seq], "speedup_of_headline": seq_s / (ms_step / 1e3)}
    del seq

    st, info = stats[-1], infos[-1]
    roof = roofline(kt, hbm_peak, peak_src, hop_kernel_name(inner, info["batch"]),
                    {"traffic": hop_traffic([(w["Ls"], kt["bytes"])], kt["launches"])
                     if inner == "f32" and info["batch"] == 1 else None, "traffic_source": TRAFFIC_SOURCE,
                     "timed_launches": "the eager first iteration of each batch (graph replays are not bracketed "
                                       "by events)"})
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
                    "d2h_bytes_per_step": sum(h.numel() * 16 for h in x_host), "host_buffers": HOST_BUFFERS},
            "gpu_launches": launches, "solve": solve_info, "sequential_cg": sequential,
            "all_rhs_one_launch": one_launch, "clocks": clk.summary()}
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, sum(s["iters"] for s in st))
            line["cpu_baseline"]["sample"] += " (the mixed solves' iteration counts stand in for FP64 CG's)"
        print(json.dumps(line), flush=True)
    lat.close()


def run_madwf_study(args, w, dev):
    """MADWF settings on the headline input (Sec. 4-5: Table 1's three
    defect-correction passes of two Pauli-Villars and one Moebius solve each,
    Fig. 1's Moebius accuracy): one JSON line per setting with the time, the
    paper's op counts per solve kind and the pass residuals, each solve from
    a zero guess to the 1e-10 target; the plain mixed-precision CG is the
    n_dc = 0 row."""
    import torch

    from paper_1111_5059_gb300 import dwf, inputs

    stream = torch.cuda.current_stream(dev)
    U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], w["eps"])).to(dev)
    b = torch.from_numpy(inputs.gaussian_spinor(w["seed"], w["dims"], w["Ls"])).to(dev)
    x = torch.empty_like(b)
    lat = dwf.Lattice(w["dims"], w["Ls"], w["M5"], 1.0, 0.0, 1, stream=stream, device=dev)
    lat.set_gauge(U)
    mobs = {}

    def mobius(alpha, Lp=w["inner_Ls"]):
        if (alpha, Lp) not in mobs:
            b5, c5 = (alpha + 1) / 2, (alpha - 1) / 2  # b - c = 1, b + c = alpha
            mobs[(alpha, Lp)] = dwf.Lattice(w["dims"], Lp, w["M5"], b5, c5, 1, stream=stream, device=dev)
            mobs[(alpha, Lp)].set_gauge(U)
        return mobs[(alpha, Lp)]

    if args.study_ls:
        # Ls' and b + c (Sec. 4-5; Fig. 1 uses L' = 16 for L = 32), in the bench's solver settings
        lat.cg(w["m"], b, tol=args.tol, inner="f32", delta=DELTA, check_every=CHECK_EVERY, out=x)  # warm-up
        cases = []
        for Lp in (8, 12, 16):
            a0 = w["Ls"] / Lp
            cases += [(Lp, a0, 1, 1e-3, 1e-2), (Lp, a0, 1, 1e-5, 1e-4), (Lp, a0, 2, 1e-5, 1e-4),
                      (Lp, 0.75 * a0, 1, 1e-5, 1e-4), (Lp, 1.25 * a0, 1, 1e-5, 1e-4)]
        for Lp, alpha, n_dc, tol_pv, tol_mob in cases:
            e0, e1 = _events(2)
            e0.record(stream)
            r = dwf.madwf_solve(lat, mobius(alpha, Lp), w["m"], b, n_dc=n_dc, tol_pv=tol_pv, tol_mob=tol_mob,
                                tol_final=args.tol, inner_prec="f32", delta=DELTA, check_every=CHECK_EVERY, out=x,
                                max_iter=30000, raise_on_fail=False)
            e1.record(stream)
            e1.synchronize()
            st = r.stats
            print(json.dumps({"study": "madwf-Ls'", "Ls_inner": Lp, "b_plus_c": alpha, "n_dc": n_dc,
                              "tol_pv": tol_pv, "tol_mob": tol_mob, "seconds": e0.elapsed_time(e1) / 1e3,
                              "status": r.status,
                              "op_count": {"pv": st["pv"]["op_count"], "mobius": st["mobius"]["op_count"],
                                           "final": st["final_cg"]["op_count"], "total": st["total"]["op_count"]},
                              "iters": {"pv": st["pv"]["iters"], "mobius": st["mobius"]["iters"],
                                        "final": st["final_cg"]["iters"]},
                              "pass_resid": st["pass_resid"], "true_resid": st["total"]["true_resid"]}), flush=True)
            if len(mobs) > 2:  # keep device memory bounded: drop lattices not needed next
                for key in [k for k in mobs if k[1] != Lp]:
                    mobs.pop(key).close()
        for mb in mobs.values():
            mb.close()
        lat.close()
        return
    Lp = w["inner_Ls"]

    base_alpha = w["Ls"] / Lp
    grid = [(w["eps"], 0, None, None, base_alpha)]
    for n_dc in (1, 2, 3):
        for tol_pv in (1e-4, 1e-5, 1e-6):
            for tol_mob in (1e-3, 1e-4, 1e-5):
                grid.append((w["eps"], n_dc, tol_pv, tol_mob, base_alpha))
    for tol_pv, tol_mob in ((1e-3, 1e-3), (1e-3, 1e-2), (1e-4, 1e-2), (3e-4, 3e-3)):
        grid.append((w["eps"], 1, tol_pv, tol_mob, base_alpha))
    for alpha in (2.0, 3.2):
        grid.append((w["eps"], 3, 1e-6, 1e-5, alpha))
        grid.append((w["eps"], 1, 1e-5, 1e-4, alpha))
    # the regime where the direct solve gets expensive: rougher links, same lattice and mass
    for eps in (0.9, 1.2):
        grid += [(eps, 0, None, None, base_alpha), (eps, 1, 1e-4, 1e-3, base_alpha),
                 (eps, 2, 1e-4, 1e-3, base_alpha), (eps, 2, 1e-5, 1e-4, base_alpha)]
    lat.cg(w["m"], b, tol=args.tol, inner="f32", delta=DELTA, check_every=10, out=x)  # warm-up
    cur_eps = w["eps"]
    for eps, n_dc, tol_pv, tol_mob, alpha in grid:
        if eps != cur_eps:
            U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], eps)).to(dev)
            lat.set_gauge(U)
            for mb in mobs.values():
                mb.set_gauge(U)
            cur_eps = eps
        e0, e1 = _events(2)
        e0.record(stream)
        if n_dc == 0:
            r = lat.cg(w["m"], b, tol=args.tol, inner="f32", delta=DELTA, check_every=10, out=x, max_iter=30000,
                       raise_on_fail=False)
        else:
            r = dwf.madwf_solve(lat, mobius(alpha), w["m"], b, n_dc=n_dc, tol_pv=tol_pv, tol_mob=tol_mob,
                                tol_final=args.tol, inner_prec="f32", delta=DELTA, check_every=10, out=x,
                                max_iter=30000, raise_on_fail=False)
        e1.record(stream)
        e1.synchronize()
        row = {"study": "madwf", "eps": eps, "n_dc": n_dc, "tol_pv": tol_pv, "tol_mob": tol_mob, "b_plus_c": alpha,
               "seconds": e0.elapsed_time(e1) / 1e3, "status": r.status}
        if n_dc == 0:
            row.update({"op_count": {"final": r.stats["op_count"], "total": r.stats["op_count"]},
                        "iters": {"final": r.stats["iters"]}, "true_resid": r.stats["true_resid"]})
        else:
            st = r.stats
            row.update({"op_count": {"pv": st["pv"]["op_count"], "mobius": st["mobius"]["op_count"],
                                     "final": st["final_cg"]["op_count"], "total": st["total"]["op_count"]},
                        "iters": {"pv": st["pv"]["iters"], "mobius": st["mobius"]["iters"],
                                  "final": st["final_cg"]["iters"]},
                        "pass_resid": st["pass_resid"], "true_resid": st["total"]["true_resid"]})
        print(json.dumps(row), flush=True)
    for m in mobs.values():
        m.close()
    lat.close()


def run_apply(args, w, world, rank, local, dev, hbm_peak, peak_src):
    """Operator-only workload: one step is 10 applications of M_pc (and 10 of
    M_pc^+) with FP32-stored fields through dwf_apply_Mpc_prec, the solvers'
    own hop launches; the line's value is the time per M_pc application and its
    roofline the FP32 hop's."""
    import torch

    from paper_1111_5059_gb300 import dwf, inputs

    U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], w["eps"])).to(dev)
    x = torch.from_numpy(inputs.gaussian_spinor(w["seed"], w["dims"], w["Ls"])).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    lat = dwf.Lattice(w["dims"], w["Ls"], w["M5"], w.get("b5", 1.0), w.get("c5", 0.0), 1, stream=stream, device=dev)
    lat.set_gauge(U)
    del U
    reps = 10

    def step():
        for _ in range(reps):
            lat.apply_Mpc_prec(w["m"], x, prec="f32", out=y)
            lat.apply_Mpc_prec(w["m"], x, prec="f32", dag=True, out=y)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    lat.set_kernel_timing(True)
    n0 = lat.launch_count()
    step_ms = []
    barrier(world)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            e0, e1 = _events(2)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    barrier(world)
    launches = lat.launch_count() - n0
    kt = lat.kernel_time("f32")
    lat.set_kernel_timing(False)
    ms_step = max_over_ranks(world, sum(step_ms), dev) / args.steps
    value = ms_step / 1e3 / (2 * reps) / world
    roof = roofline(kt, hbm_peak, peak_src, hop_kernel_name("f32") + f" at Lh = {(w['Ls'] + 1) // 2}",
                    {"traffic": hop_traffic([(w["Ls"], kt["bytes"])], kt["launches"]),
                     "traffic_source": TRAFFIC_SOURCE, "share_of_step": kt["ms"] / max(1e-9, sum(step_ms))})
    line = {"metric": "FP32 M_pc application time (two Wilson hops with fused fifth-dimension operators)",
            "value": value, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "lattice": "x".join(map(str, w["dims"])), "Ls": w["Ls"],
                       "b": w.get("b5", 1.0), "c": w.get("c5", 0.0), "m": w["m"], "eps": w["eps"],
                       "applications_per_step": 2 * reps,
                       "l2": "each FP32 half-lattice field is larger than L2 (129 MB)"},
            "roofline": roof, "gpu_launches": launches, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    lat.close()


def run_md_study(args, dev):
    """Force-gradient against Omelyan trajectories (Sec. 2) on the force workload:
    Shamir 16^3 x 8 x Ls=16, quotient terms (0.01, 0.1) and (0.1, 1.0), eps = 0.5,
    Gaussian momenta and pseudofermion sources (seed 4), trajectory length 0.4 at
    several step sizes: one JSON line each with dH, the force evaluations, the
    solver iterations and the time.  Force solves: FP32 inner CG with FP64
    reliable updates to 1e-10."""
    import torch

    from paper_1111_5059_gb300 import dwf, inputs

    dims, Ls, M5 = (16, 16, 16, 8), 16, 1.8
    terms = [(0.01, 0.1), (0.1, 1.0)]
    U0 = torch.from_numpy(inputs.gauge_field(4, dims, 0.5)).to(dev)
    p0 = torch.from_numpy(inputs.gaussian_momenta(4, dims)).to(dev)
    phis = [torch.from_numpy(inputs.gaussian_spinor(50 + k, dims, Ls)).to(dev) for k in range(2)]
    stream = torch.cuda.current_stream(dev)
    lat = dwf.Lattice(dims, Ls, M5, 1.0, 0.0, 1, stream=stream, device=dev)
    length = 0.4
    for integ in ("fgi", "omelyan"):
        for n in (1, 2, 4, 8):
            U, p = U0.clone(), p0.clone()
            e0, e1 = _events(2)
            e0.record(stream)
            H0, H1, st, nf = dwf.md_trajectory(lat, terms, phis, U, p, length / n, n, integrator=integ, tol=1e-10,
                                               inner="f32", delta=1e-2)
            e1.record(stream)
            e1.synchronize()
            print(json.dumps({"study": "md", "workload": "force-shamir-16^3x8-Ls16-2terms", "integrator": integ,
                              "tau": length / n, "nsteps": n, "length": length, "dH": H1 - H0, "H0": H0,
                              "force_evaluations": nf, "cg_iters": st["iters"],
                              "seconds": e0.elapsed_time(e1) / 1e3}), flush=True)
    lat.close()


def run_hasenbusch_study(args, dev):
    """Hasenbusch ladder tuning (Sec. 3) on the force workload (Shamir
    16^3 x 8 x Ls=16, m = 0.01, Pauli-Villars mass 1, eps = 0.5, seed 4): for
    k = 0..3 intermediate masses, the geometric ladder and the ladder tuned to
    equal per-term force norms (paper_1111_5059_gb300.hasenbusch.tune_ladder);
    each term's pseudofermion from the heat bath (Gaussian eta, seed 60 + i).
    Per ladder: the terms' force norms (RMS and max over links of |F_mu(n)|)
    and CG iterations at force-solve tolerances 1e-8 and 1e-6, then one FGI
    trajectory (tau = 0.1, 4 steps) at each tolerance from the same momenta
    (seed 4): dH, the reversibility error max |U - U0| after the trajectory
    and its reverse, CG iterations and time.  One JSON line per ladder."""
    import torch

    from paper_1111_5059_gb300 import dwf, hasenbusch, inputs

    dims, Ls, M5, m = (16, 16, 16, 8), 16, 1.8, 0.01
    stream = torch.cuda.current_stream(dev)
    U0 = torch.from_numpy(inputs.gauge_field(4, dims, 0.5)).to(dev)
    p0 = torch.from_numpy(inputs.gaussian_momenta(4, dims)).to(dev)
    etas = [torch.from_numpy(inputs.gaussian_spinor(60 + i, dims, Ls)).to(dev) for i in range(4)]
    lat = dwf.Lattice(dims, Ls, M5, 1.0, 0.0, 1, stream=stream, device=dev)
    lat.set_gauge(U0)

    def phis_of(ts):
        return [dwf.heatbath(lat, t, etas[i], tol=1e-10, inner="f32", delta=DELTA)[0] for i, t in enumerate(ts)]

    def term_data(ts, tol):
        phis = phis_of(ts)
        out = []
        for t, ph in zip(ts, phis):
            _, F, _, st = dwf.force(lat, [t], [ph], tol=tol, inner="f32", delta=DELTA)
            n2 = (F * F).sum(dim=-1)  # |F_mu(n)|^2
            out.append({"rms": float(n2.mean().sqrt()), "max": float(n2.max().sqrt()), "iters": st["iters"]})
        return out

    cases = [("geometric", 0), ("geometric", 1)] + [("tuned", k) for k in (1, 2, 3)]
    for kind, k in cases:
        ladder = hasenbusch.geometric_ladder(m, k)
        tune_iters = 0
        if kind == "tuned":
            ladder, hist = hasenbusch.tune_ladder(
                ladder, lambda ts: [d["rms"] for d in term_data(ts, 1e-8)], iters=8, rtol=0.05)
            tune_iters = len(hist)
        ts = hasenbusch.terms(ladder)
        d8, d6 = term_data(ts, 1e-8), term_data(ts, 1e-6)
        phis = phis_of(ts)
        traj = {}
        for tol in (1e-8, 1e-6):
            U, p = U0.clone(), p0.clone()
            e0, e1 = _events(2)
            e0.record(stream)
            H0, H1, st, nf = dwf.md_trajectory(lat, ts, phis, U, p, 0.1, 4, integrator="fgi", tol=tol, inner="f32",
                                               delta=DELTA)
            e1.record(stream)
            e1.synchronize()
            secs = e0.elapsed_time(e1) / 1e3
            p.neg_()
            dwf.md_trajectory(lat, ts, phis, U, p, 0.1, 4, integrator="fgi", tol=tol, inner="f32", delta=DELTA)
            traj[f"{tol:.0e}"] = {"dH": H1 - H0, "H0": H0, "reversibility_max_dU": float((U - U0).abs().max()),
                                  "force_evaluations": nf, "cg_iters": st["iters"], "seconds": secs}
            lat.set_gauge(U0)
        print(json.dumps({"study": "hasenbusch", "workload": "force-shamir-16^3x8-Ls16", "m": m, "ladder": kind,
                          "k": k, "masses": ladder, "tune_evaluations": tune_iters,
                          "term_force_rms": [d["rms"] for d in d8], "term_force_max": [d["max"] for d in d8],
                          "term_iters_1e-8": [d["iters"] for d in d8], "term_iters_1e-6": [d["iters"] for d in d6],
                          "trajectory": traj}), flush=True)
    lat.close()


def run_hmc_study(args, dev):
    """HMC chains (Sec. 2: heat bath, one trajectory, Metropolis) on the force
    workload (Shamir 16^3 x 8 x Ls=16, terms (0.01, 0.1) and (0.1, 1),
    eps = 0.5, seed 4): the force-gradient integrator at tau = 0.1 x 4 steps
    against Omelyan 2MN at tau = 0.05 x 8 (about the same dH in the
    trajectory study), 12 updates each from the same start and with the same
    random numbers (update k uses seed 1000 + k).  One JSON line per chain:
    acceptance, <dH>, <exp(-dH)> with its standard error, force evaluations
    and time per update."""
    import torch

    from paper_1111_5059_gb300 import dwf, hmc, inputs

    dims, Ls, M5 = (16, 16, 16, 8), 16, 1.8
    terms = [(0.01, 0.1), (0.1, 1.0)]
    stream = torch.cuda.current_stream(dev)
    U0 = torch.from_numpy(inputs.gauge_field(4, dims, 0.5)).to(dev)
    lat = dwf.Lattice(dims, Ls, M5, 1.0, 0.0, 1, stream=stream, device=dev)
    for integ, tau, n in (("fgi", 0.1, 4), ("omelyan", 0.05, 8)):
        U = U0.clone()
        rows = []
        e0, e1 = _events(2)
        e0.record(stream)
        for k in range(12):
            rows.append(hmc.hmc_update(lat, U, terms, tau, n, 1000 + k, integrator=integ, tol=1e-10, inner="f32",
                                       delta=DELTA))
        e1.record(stream)
        e1.synchronize()
        dHs = [r["dH"] for r in rows]
        w = [math.exp(-d) for d in dHs]
        mean_w = sum(w) / len(w)
        err_w = (sum((v - mean_w) ** 2 for v in w) / (len(w) - 1) / len(w)) ** 0.5
        print(json.dumps({"study": "hmc", "workload": "force-shamir-16^3x8-Ls16-2terms", "integrator": integ,
                          "tau": tau, "nsteps": n, "updates": len(rows),
                          "acceptance": sum(r["accept"] for r in rows) / len(rows), "mean_dH": sum(dHs) / len(dHs),
                          "mean_exp_minus_dH": mean_w, "stderr_exp_minus_dH": err_w, "dH": dHs,
                          "force_evaluations_per_update": rows[0]["force_evaluations"],
                          "cg_iters_per_update": sum(r["cg_iters"] for r in rows) / len(rows),
                          "seconds_per_update": e0.elapsed_time(e1) / 1e3 / len(rows)}), flush=True)
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
    if args.md_study:
        run_md_study(args, dev)
        return
    if args.hasenbusch_study:
        run_hasenbusch_study(args, dev)
        return
    if args.hmc_study:
        run_hmc_study(args, dev)
        return
    if args.study:
        if not w["madwf"]:
            raise SystemExit("--study needs the madwf workload")
        run_madwf_study(args, w, dev)
        return
    if w.get("apply"):
        run_apply(args, w, world, rank, local, dev, hbm_peak, peak_src)
        return
    if w.get("ladder"):
        run_ladder(args, w, inner, world, rank, local, dev, hbm_peak, peak_src)
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    U = torch.from_numpy(inputs.gauge_field(w["seed"], w["dims"], w["eps"])).to(dev)
    b_host = host_copy(dwf, inputs.gaussian_spinor(w["seed"], w["dims"], w["Ls"]))
    b = b_host.to(dev)
    x = torch.empty_like(b)
    x_host = dwf.host_empty(b_host.shape)
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

    def solve(bb, out):
        if w["madwf"]:
            return dwf.madwf_solve(lat, mob, w["m"], bb, n_dc=w["n_dc"], tol_pv=w["tol_pv"], tol_mob=w["tol_mob"],
                                   tol_final=args.tol, inner_prec=inner, delta=delta_for(inner),
                                   check_every=CHECK_EVERY, out=out)
        return lat.cg(w["m"], bb, tol=args.tol, inner=inner, delta=delta_for(inner), check_every=CHECK_EVERY, out=out)

    for _ in range(args.warmup):
        r = solve(b, x)
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
            e0, e1 = _events(2)
            e0.record(stream)
            r = solve(b, x)
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

    # ---- e2e: the same solve through the public API from and to pinned host
    # buffers (device buffers allocated beforehand: nothing is allocated in
    # the timed region); events split it into copy-in, solve and copy-out
    bd = torch.empty_like(b)
    e2e = []
    for _ in range(max(1, min(args.steps, 2))):
        flush.fill_(1.0)
        ev = _events(4)
        ev[0].record(stream)
        bd.copy_(b_host, non_blocking=True)
        ev[1].record(stream)
        solve(bd, x)
        ev[2].record(stream)
        x_host.copy_(x, non_blocking=True)
        ev[3].record(stream)
        ev[3].synchronize()
        e2e.append([ev[0].elapsed_time(ev[3]), ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                    ev[2].elapsed_time(ev[3])])
    del bd
    e2e_ms = max_over_ranks(world, statistics.mean(e[0] for e in e2e), dev)
    h2d_ms = statistics.mean(e[1] for e in e2e)
    d2h_ms = statistics.mean(e[3] for e in e2e)
    nbytes = b_host.numel() * 16

    # ---- comparisons on the same GPU: plain FP64 CG (and mixed CG for MADWF)
    comp = {}
    if not args.no_fp64:
        for name, prec in (("fp64_cg", "f64"),) + ((("mixed_cg", inner),) if w["madwf"] else ()):
            torch.cuda.synchronize()
            e0, e1 = _events(2)
            e0.record(stream)
            rf = lat.cg(w["m"], b, tol=args.tol, inner=prec, delta=delta_for(prec), check_every=CHECK_EVERY, out=x)
            e1.record(stream)
            e1.synchronize()
            secs = e0.elapsed_time(e1) / 1e3
            comp[name] = {"seconds": secs, "iters": rf.stats["iters"], "op_count": rf.stats["op_count"],
                          "true_resid": rf.stats["true_resid"], "speedup_of_headline": secs / (ms_step / 1e3)}
            del rf

    roof = roofline(kt, hbm_peak, peak_src, hop_kernel_name(inner),
                    {"traffic": hop_traffic([(L.Ls, d["bytes"]) for L, d in zip(lats, kts)], kt["launches"])
                     if inner == "f32" else None, "traffic_source": TRAFFIC_SOURCE,
                     "share_of_step": kt["ms"] / max(1e-9, sum(step_ms))})
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
            "e2e": {"value": e2e_ms / 1e3 / world, "unit": "s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "h2d_ms": h2d_ms, "solve_ms": statistics.mean(e[2] for e in e2e),
                    "d2h_ms": d2h_ms, "h2d_gbs": nbytes / (h2d_ms / 1e3) / 1e9 if h2d_ms > 0 else None,
                    "d2h_gbs": nbytes / (d2h_ms / 1e3) / 1e9 if d2h_ms > 0 else None, "host_buffers": HOST_BUFFERS,
                    "huge_page_fraction": [thp_fraction(b_host), thp_fraction(x_host)],
                    "per_step_ms": [[round(v, 2) for v in e[1:]] for e in e2e]},
            "gpu_launches": launches, "solve": solve_info, "clocks": clk.summary()}
    line.update(comp)
    for L in lats:
        L.close()
    del b, x, flush
    if not args.no_extras and world == 1:
        torch.cuda.empty_cache()
        line["precisions_16x32_Ls16"] = precision_comparison(dev, stream, hbm_peak, peak_src, args.tol)
        torch.cuda.empty_cache()
        line["ladder_32x64_Ls16"] = ladder_comparison(dev, stream, args.tol)
        torch.cuda.empty_cache()
        line["trajectory_16x8_Ls16"] = trajectory_timing(dev, stream)
    if rank == 0:
        if not args.no_cpu_baseline:
            iters = comp["fp64_cg"]["iters"] if "fp64_cg" in comp else FP64_ITERS[args.workload]
            line["cpu_baseline"] = cpu_baseline(w, iters)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
