"""The multi-right-hand-side ladder solve (dwf_cg_multi) against the FP64 oracle.

Each right-hand side is an ordinary solve D(m_r) x_r = b_r, so the criteria
are those of the single solve: the true residual of every x_r, computed by the
ORACLE's operator, <= 1e-10 (mixed precision) or <= 1e-12 (FP64), and x_r
close to the oracle's own solution.  At the full ladder size (Moebius
32^3 x 64 x Ls=16, b = 1.5, c = 0.5, masses {0.001, 0.01, 0.05, 0.2}) the
oracle computes b - D(m_r) x_r on a slab of four timeslices per right-hand
side (tests/oracle_residual.py), whose norm must stay below 1e-10 |b|.
"""
import numpy as np
import pytest
import torch

import oracle_residual as R
from oracle import dwf_oracle as O
from paper_1111_5059_gb300 import inputs as I

pytestmark = pytest.mark.gpu

M5 = 1.8
LADDER = (0.001, 0.01, 0.05, 0.2)


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _true_res(U, x, b, m, b5, c5, bc_t=1):
    r = b - O.dwf_op(U, x, m, M5, b5, c5, bc_t)
    return np.sqrt(O.norm2(r) / O.norm2(b))


@pytest.fixture(scope="module")
def ladder(dwf):
    """Moebius 4^3 x 8 x Ls=8 (b = 1.5, c = 0.5, eps = 0.6) with four Gaussian sources."""
    dims, Ls, b5, c5 = (4, 4, 4, 8), 8, 1.5, 0.5
    U = I.gauge_field(5, dims, 0.6)
    bs = [I.gaussian_spinor(10 + r, dims, Ls) for r in range(len(LADDER))]
    lat = dwf.Lattice(dims, Ls, M5, b5, c5)
    lat.set_gauge(_to(U))
    xo = [O.solve(U, b, m, M5, b5, c5, tol=1e-13)[0] for b, m in zip(bs, LADDER)]
    yield lat, U, bs, xo, b5, c5
    lat.close()


@pytest.mark.parametrize("inner,tol,xtol", [("f32", 1e-10, 1e-7), ("f16", 1e-10, 1e-7), ("f64", 1e-12, 1e-9)])
def test_ladder_matches_oracle(ladder, inner, tol, xtol):
    lat, U, bs, xo, b5, c5 = ladder
    xs, stats, info, status = lat.cg_multi(LADDER, [_to(b) for b in bs], tol=tol, inner=inner)
    assert status == 0
    for r, m in enumerate(LADDER):
        x = xs[r].cpu().numpy()
        assert stats[r]["true_resid"] <= tol
        assert _true_res(U, x, bs[r], m, b5, c5) <= tol
        assert np.sqrt(O.norm2(x - xo[r]) / O.norm2(xo[r])) < xtol
        assert stats[r]["op_count"] == stats[r]["iters"] * 8
    # lighter masses need more iterations; the joint loop runs until the slowest is done
    its = [s["iters"] for s in stats]
    assert its[0] >= its[-1] and info["iterations"] == max(its)


def test_ladder_batched_launch_and_graphs(ladder):
    lat, U, bs, xo, b5, c5 = ladder
    xs, stats, info, _ = lat.cg_multi(LADDER, [_to(b) for b in bs], inner="f32", autotune=False)
    assert info["batch"] == 4  # all four right-hand sides in one hop launch (Ls = 8: 4 x 4 pairs per warp)
    assert info["graphs"] >= 1 and info["replays"] > 0
    assert info["launches"] == stats[0]["launches"] > 0


def test_graph_replay_equals_eager(ladder):
    lat, U, bs, xo, b5, c5 = ladder
    src = [_to(b) for b in bs]
    xg, sg, _, _ = lat.cg_multi(LADDER, src, inner="f32", use_graph=True, autotune=False)
    xe, se, _, _ = lat.cg_multi(LADDER, src, inner="f32", use_graph=False, autotune=False)
    for r in range(len(LADDER)):
        assert torch.equal(xg[r], xe[r])
        assert sg[r]["iters"] == se[r]["iters"]


def test_autotuned_shapes_reach_the_same_solution(ladder):
    lat, U, bs, xo, b5, c5 = ladder
    xs, stats, info, _ = lat.cg_multi(LADDER, [_to(b) for b in bs], inner="f32", autotune=True)
    assert 1 <= info["batch"] <= 4 and info["tune_seconds"] >= 0.0
    for r, m in enumerate(LADDER):
        assert _true_res(U, xs[r].cpu().numpy(), bs[r], m, b5, c5) <= 1e-10


def test_ladder_equals_sequential_solves(ladder):
    lat, U, bs, xo, b5, c5 = ladder
    xs, stats, _, _ = lat.cg_multi(LADDER, [_to(b) for b in bs], inner="f32")
    for r, m in enumerate(LADDER):
        one = lat.cg(m, _to(bs[r]), tol=1e-10, inner="f32")
        d = (xs[r] - one.x).norm() / one.x.norm()
        assert float(d) < 1e-7


def test_zero_source_and_warm_start(ladder):
    lat, U, bs, xo, b5, c5 = ladder
    src = [_to(bs[0]), torch.zeros_like(_to(bs[1]))]
    guess = [_to(xo[0]), torch.ones_like(src[1])]
    xs, stats, _, status = lat.cg_multi(LADDER[:2], src, x0s=guess, inner="f32")
    assert status == 0
    assert stats[0]["iters"] == 0 and stats[0]["true_resid"] <= 1e-10
    assert float(xs[1].abs().max()) == 0.0 and stats[1]["true_resid"] == 0.0


def test_ragged_shapes_and_wide_ladders(dwf):
    # odd Ls (padding slices), odd t extent, antiperiodic t, and more masses than one launch takes
    for dims, Ls, bc_t, masses in [((4, 2, 4, 6), 5, -1, (0.02, 0.1, 0.3)),
                                   ((4, 4, 2, 4), 4, 1, tuple(0.05 * (k + 1) for k in range(10)))]:
        U = I.gauge_field(6, dims, 0.5)
        bs = [I.gaussian_spinor(20 + r, dims, Ls) for r in range(len(masses))]
        lat = dwf.Lattice(dims, Ls, M5, 1.0, 0.0, bc_t)
        lat.set_gauge(_to(U))
        for inner in ("f32", "f16"):
            xs, stats, info, status = lat.cg_multi(masses, [_to(b) for b in bs], inner=inner)
            assert status == 0
            for r, m in enumerate(masses):
                assert _true_res(U, xs[r].cpu().numpy(), bs[r], m, 1.0, 0.0, bc_t) <= 1e-10
        lat.close()


def test_max_iter_and_invalid_arguments(ladder, dwf):
    lat, U, bs, xo, b5, c5 = ladder
    src = [_to(b) for b in bs]
    xs, stats, _, status = lat.cg_multi(LADDER, src, inner="f32", max_iter=5, raise_on_fail=False)
    assert status == 4  # DWF_ERR_NOT_CONVERGED
    assert all(s["iters"] == 5 for s in stats)
    with pytest.raises(dwf.DWFError, match="repeated mass"):
        lat.cg_multi((0.01, 0.01), src[:2])
    with pytest.raises(dwf.DWFError, match="nrhs"):
        lat.cg_multi(tuple(0.01 * (k + 1) for k in range(17)), [src[0]] * 17)


def test_full_ladder_size_slab_residuals(dwf):
    """32^3 x 64 x Ls=16 Moebius ladder; one Gaussian source for all four masses."""
    dims, Ls, b5, c5 = (32, 32, 32, 64), 16, 1.5, 0.5
    T = dims[3]
    U = I.gauge_field(5, dims, 0.6)
    b = I.gaussian_spinor(5, dims, Ls)
    lat = dwf.Lattice(dims, Ls, M5, b5, c5)
    lat.set_gauge(_to(U))
    bt = _to(b)
    xs, stats, info, status = lat.cg_multi(LADDER, [bt] * 4, inner="f32")
    assert status == 0 and info["batch"] >= 1
    lat.close()
    del bt
    bnorm2 = O.norm2(b)
    for r, m in enumerate(LADDER):
        assert stats[r]["true_resid"] <= 1e-10
        rows = R.slab_rows(T, (T - 2 + 17 * r) % T, 4)  # the first slab crosses the t boundary
        x = xs[r][:, rows].cpu().numpy()
        r2, _ = R.slab_residual(U, x, b[:, rows[1:-1]], rows, m, M5, b5, c5)
        assert np.sqrt(r2 / bnorm2) <= 1e-10, (m, np.sqrt(r2 / bnorm2))
        del x


_TUNE_SCRIPT = r"""
import json, sys, torch
sys.path.insert(0, {root!r})
from paper_1111_5059_gb300 import dwf, inputs
dims, Ls = (4, 4, 4, 8), 8
lat = dwf.Lattice(dims, Ls, 1.8, 1.5, 0.5)
lat.set_gauge(torch.from_numpy(inputs.gauge_field(5, dims, 0.6)).cuda())
bs = [torch.from_numpy(inputs.gaussian_spinor(10 + r, dims, Ls)).cuda() for r in range(3)]
xs, st, info, status = lat.cg_multi((0.01, 0.05, 0.2), bs, inner="f32", autotune=True)
print(json.dumps({{"status": status, "tune_seconds": info["tune_seconds"], "batch": info["batch"]}}))
"""


def test_autotune_cache_file_is_written_and_reused(dwf, tmp_path):
    """DWF_TUNE_CACHE: the first process times the candidates and appends the
    winners; a second process reads them back and tunes nothing."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, DWF_TUNE_CACHE=str(cache))
    script = _TUNE_SCRIPT.format(root=root)
    out = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env, timeout=600)
        assert r.returncode == 0, r.stderr
        out.append(json.loads(r.stdout.strip().splitlines()[-1]))
    lines = cache.read_text().strip().splitlines()
    assert len(lines) >= 2 and all(len(l.split()) == 4 for l in lines)
    assert out[0]["status"] == 0 and out[1]["status"] == 0
    assert out[0]["tune_seconds"] > 0.0 and out[1]["tune_seconds"] == 0.0
    assert out[0]["batch"] == out[1]["batch"]
