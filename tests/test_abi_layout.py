"""Host-side checks of the C ABI (CPU only, no compute calls).

* The ctypes structures of the binding have the sizes and field offsets that
  a C compiler gives the structs of include/dwf.h (a C program built with gcc
  prints them), and the binding's constants equal the header's.
* Argument validation happens before any CUDA work: bad lattice parameters
  and null handles come back as DWF_ERR_INVALID_ARG with the reason in
  dwf_last_error(NULL), and dwf_destroy_lattice(NULL) is a no-op.
"""
import ctypes
import json
import math
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct name -> (binding class name, fields)
_STRUCTS = {
    "dwf_params": ("Params", ["dims", "Ls", "M5", "b", "c", "bc_t"]),
    "dwf_cg_params": ("CGParams", ["tol", "max_iter", "inner", "delta", "check_every"]),
    "dwf_stats": ("Stats", ["iters", "reliable_updates", "hop_calls", "op_count", "true_resid", "seconds",
                            "launches"]),
    "dwf_multi_options": ("MultiOptions", ["use_graph", "autotune"]),
    "dwf_multi_info": ("MultiInfo", ["batch", "ctas_per_sm", "tune_seconds", "graphs", "replays", "iterations",
                                     "seconds", "launches"]),
    "madwf_params": ("MadwfParams", ["n_dc", "tol_pv", "tol_mob", "tol_final", "inner", "max_iter", "delta",
                                     "check_every"]),
    "madwf_stats": ("MadwfStats", ["total", "pv", "mobius", "final_cg", "passes", "pass_resid"]),
    "dwf_quotient": ("Quotient", ["m1", "m2"]),
}


def _c_program():
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dwf.h"', "int main(void) {", 'printf("{");']
    for cname, (_, fields) in _STRUCTS.items():
        lines.append(f'printf("\\"{cname}\\": {{\\"size\\": %zu", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf(", \\"{f}\\": %zu", offsetof({cname}, {f}));')
        lines.append('printf("}, ");')
    lines.append('printf("\\"DWF_MAX_RHS\\": %d, \\"MADWF_MAX_PASSES\\": %d, ", DWF_MAX_RHS, MADWF_MAX_PASSES);')
    lines.append('printf("\\"prec\\": [%d, %d, %d], ", (int)DWF_F64, (int)DWF_F32, (int)DWF_F16);')
    lines.append('printf("\\"status\\": [%d, %d, %d, %d, %d, %d, %d]", (int)DWF_OK, (int)DWF_ERR_INVALID_ARG, '
                 "(int)DWF_ERR_CUDA, (int)DWF_ERR_OOM, (int)DWF_ERR_NOT_CONVERGED, (int)DWF_ERR_NAN, "
                 "(int)DWF_ERR_TIMEOUT);")
    lines += ['printf("}\\n");', "return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text(_c_program())
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


def test_binding_structs_match_the_header(c_layout):
    from paper_1111_5059_gb300 import dwf

    for cname, (pyname, fields) in _STRUCTS.items():
        cls = getattr(dwf, pyname)
        assert ctypes.sizeof(cls) == c_layout[cname]["size"], cname
        assert [f for f, _ in cls._fields_] == fields, cname
        for f in fields:
            assert getattr(cls, f).offset == c_layout[cname][f], (cname, f)


def test_binding_constants_match_the_header(c_layout):
    from paper_1111_5059_gb300 import dwf

    assert dwf.DWF_MAX_RHS == c_layout["DWF_MAX_RHS"]
    assert dwf.MADWF_MAX_PASSES == c_layout["MADWF_MAX_PASSES"]
    assert [dwf.DWF_F64, dwf.DWF_F32, dwf.DWF_F16] == c_layout["prec"]
    assert sorted(dwf.STATUS) == c_layout["status"]


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)

    from paper_1111_5059_gb300 import build
    from paper_1111_5059_gb300 import dwf

    build.build()
    return dwf.lib(), dwf


_GOOD = dict(dims=(4, 4, 4, 8), Ls=8, M5=1.8, b=1.0, c=0.0, bc_t=1)


@pytest.mark.parametrize("bad,reason", [
    (dict(dims=(4, 4, 3, 8)), "even"),
    (dict(dims=(4, 0, 4, 8)), "even"),
    (dict(Ls=0), "Ls"),
    (dict(Ls=65), "Ls"),
    (dict(bc_t=0), "bc_t"),
    (dict(M5=math.nan), "non-finite"),
    (dict(c=math.inf), "non-finite"),
    (dict(dims=(1024, 1024, 1024, 1024)), "too large"),
])
def test_create_lattice_rejects_bad_parameters(lib, bad, reason):
    L, dwf = lib
    kw = dict(_GOOD, **bad)
    p = dwf.Params((ctypes.c_int * 4)(*kw["dims"]), kw["Ls"], kw["M5"], kw["b"], kw["c"], kw["bc_t"])
    h = ctypes.c_void_p(12345)
    assert L.dwf_create_lattice(ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert h.value is None
    assert reason in L.dwf_last_error(None).decode()


def test_null_handle_is_rejected_by_every_entry_point(lib):
    L, dwf = lib
    assert L.dwf_destroy_lattice(None) == 0
    dp = ctypes.byref(ctypes.c_double())
    # (entry point, call, start of the message it leaves in dwf_last_error(NULL))
    calls = [
        ("dwf_create_lattice", lambda: L.dwf_create_lattice(None, None, None), "dwf_create_lattice:"),
        ("dwf_set_gauge", lambda: L.dwf_set_gauge(None, None), "dwf_set_gauge:"),
        ("dwf_apply_M", lambda: L.dwf_apply_M(None, 0.1, None, None), "apply:"),
        ("dwf_apply_Mdag", lambda: L.dwf_apply_Mdag(None, 0.1, None, None), "apply:"),
        ("dwf_apply_MdagM", lambda: L.dwf_apply_MdagM(None, 0.1, None, None), "apply:"),
        ("dwf_apply_Mpc", lambda: L.dwf_apply_Mpc(None, 0.1, 0, None, None), "dwf_apply_Mpc:"),
        ("dwf_apply_Mpc_noalloc", lambda: L.dwf_apply_Mpc_noalloc(None, 0.1, 0, None, None),
         "dwf_apply_Mpc_noalloc:"),
        ("dwf_cg", lambda: L.dwf_cg(None, 0.1, None, None, None, None), "dwf_cg:"),
        ("dwf_cg_multi", lambda: L.dwf_cg_multi(None, 1, None, None, None, None, None, None, None), "dwf_cg_multi:"),
        ("madwf_solve", lambda: L.madwf_solve(None, None, 0.1, None, None, None, None), "madwf_solve:"),
        ("dwf_force", lambda: L.dwf_force(None, 1, None, None, None, None, None, None, None, None), "dwf_force:"),
        # dwf_action is dwf_force asked for S only
        ("dwf_action", lambda: L.dwf_action(None, 1, None, None, None, dp), "dwf_force:"),
        ("fgi_link_update", lambda: L.fgi_link_update(None, None, -0.01, None, None), "fgi_link_update:"),
        ("dwf_momentum_update", lambda: L.dwf_momentum_update(None, None, 0.1, None), "dwf_momentum_update:"),
        ("dwf_kinetic", lambda: L.dwf_kinetic(None, None, None), "dwf_kinetic:"),
        ("fgi_step", lambda: L.fgi_step(None, 1, None, None, None, None, 0.1, 1, None, None, None), "fgi_step:"),
        ("dwf_set_kernel_timing", lambda: L.dwf_set_kernel_timing(None, 1), "dwf_set_kernel_timing:"),
        ("dwf_get_kernel_time", lambda: L.dwf_get_kernel_time(None, 0, None, None, None), "dwf_get_kernel_time:"),
        ("dwf_get_launch_count", lambda: L.dwf_get_launch_count(None, None), "dwf_get_launch_count:"),
        ("dwf_apply_Mpc_prec", lambda: L.dwf_apply_Mpc_prec(None, 0.1, 0, 1, None, None), "dwf_apply_Mpc_prec:"),
        ("dwf_set_wait_limit", lambda: L.dwf_set_wait_limit(None, 0), "dwf_set_wait_limit:"),
        ("dwf_heatbath", lambda: L.dwf_heatbath(None, dwf.Quotient(0.1, 1.0), None, None, None, None),
         "dwf_heatbath:"),
        ("dwf_set_fp64_arithmetic", lambda: L.dwf_set_fp64_arithmetic(None, 1), "dwf_set_fp64_arithmetic:"),
        ("dwf_md_trajectory", lambda: L.dwf_md_trajectory(None, 1, None, None, None, None, 0.1, 1, 0, 1, None, None,
                                                          None, None, None), "dwf_md_trajectory:"),
        # not a handle, but the same rule for the host allocator's pointer argument
        ("dwf_host_alloc", lambda: L.dwf_host_alloc(64, None), "dwf_host_alloc:"),
    ]
    for name, call, prefix in calls:
        assert call() == 1, name
        assert L.dwf_last_error(None).decode().startswith(prefix), name
    # every entry point of the header is covered
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "dwf.h")).read(), flags=re.S)
    declared = set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*((?:dwf|madwf|fgi)_\w+)\s*\(", hdr, flags=re.M))
    assert declared == {n for n, _, _ in calls} | {"dwf_destroy_lattice", "dwf_last_error", "dwf_host_free"}


def test_host_allocator_rejects_bad_arguments(lib):
    L, dwf = lib
    p = ctypes.c_void_p(12345)
    assert L.dwf_host_alloc(0, ctypes.byref(p)) == 1
    assert p.value is None
    assert "zero bytes" in L.dwf_last_error(None).decode()
    assert L.dwf_host_free(None) == 0
    buf = ctypes.create_string_buffer(64)
    assert L.dwf_host_free(ctypes.cast(buf, ctypes.c_void_p)) == 1
    assert "not a dwf_host_alloc pointer" in L.dwf_last_error(None).decode()
