"""bench.py's reference arm (the FP64 oracle timed on the host) prints the
JSON line of the benchmark contract, on the CPU: one line with the metric,
the time-like value, the oracle's cpu_baseline and an e2e block without
host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "mixed",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == "s"
    assert isinstance(cb["cores"], int) and 1 <= cb["cores"] <= (os.cpu_count() or 1)
    assert "sub-lattice" in cb["sample"] and cb["cores"] >= 1
    # the measured step and its extrapolation are reported apart
    ex = d["extrapolated"]
    assert abs(ex["step_seconds"] * 1e3 - d["ms_per_step"]) < 1e-6 * d["ms_per_step"]
    assert ex["volume_factor"] > 0 and ex["iterations"] > 0
    # rates of the oracle: four hops per CG iteration over the 16^3 x 32 x 16 half lattice
    assert cb["hops_per_s"] > 0 and cb["algorithmic_gbs"] > 0
    sites = 16 * 16 * 16 * 32 // 2 * 16
    per_it = 4.0 / cb["hops_per_s"]
    assert abs(cb["algorithmic_gbs"] - 4 * (48 * 8 + 144 * 8 / 16) * sites / per_it / 1e9) < 1e-9 * cb["algorithmic_gbs"]
    assert abs(d["value"] - per_it * 250) < 1e-6 * d["value"]  # 250 FP64 CG iterations on this input
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def _bench():
    sys.path.insert(0, ROOT)
    import bench

    return bench


def test_traffic_figure_follows_the_measured_source_and_lh():
    """roofline.traffic: algorithmic bytes times the ncu ratio at each
    lattice's Lh, only for the kernel source the ratios were measured on."""
    b = _bench()
    ratios = b.HOP_TRAFFIC["ratio_by_lh"]
    got = b.hop_traffic([(32, 1000.0), (12, 500.0)], 3)
    if got is None:  # the kernel source changed since the capture
        return
    assert got == (1000.0 * ratios[16] + 500.0 * ratios[6]) / 3
    assert b.hop_traffic([(10, 100.0)], 1) is None  # Lh = 5 was not measured
    assert b.hop_traffic([(16, 100.0)], 0) is None


def test_solver_settings_by_storage_precision():
    b = _bench()
    assert b.delta_for("f32") == b.DELTA and b.delta_for("f16") == b.DELTA_F16
    assert 0 < b.DELTA < b.DELTA_F16 < 1 and b.CHECK_EVERY >= 1


def test_huge_page_fraction_of_a_plain_buffer():
    import mmap

    import numpy as np
    import torch

    b = _bench()
    m = mmap.mmap(-1, 1 << 22)
    a = np.frombuffer(m, dtype=np.uint8)
    a[:] = 1
    f = b.thp_fraction(torch.from_numpy(a))
    assert f is None or 0.0 <= f <= 1.0
