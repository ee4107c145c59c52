"""The C-ABI library builds, loads and exports every entry point that
include/dwf.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(dwf_\w+|madwf_\w+|fgi_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1111_5059_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dwf_create_lattice", "dwf_destroy_lattice", "dwf_set_gauge", "dwf_apply_M",
                     "dwf_apply_Mdag", "dwf_apply_MdagM", "dwf_cg"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)

    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1111_5059_gb300 import dwf

    monkeypatch.setattr(dwf, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(dwf, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        dwf.lib()


def test_cpu_tensors_are_rejected(libpath):
    import torch

    from paper_1111_5059_gb300 import dwf

    with pytest.raises(TypeError):
        dwf._ptr(torch.zeros(3, dtype=torch.complex128))
