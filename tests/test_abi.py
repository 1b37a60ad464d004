"""The C-ABI library builds, loads and exports every entry point include/ctrecon.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ctrecon.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:ctr_status|void|char|size_t|unsigned long long|int|ctr_plan)\s*\*?\s*"
                       r"(\w+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import shutil
    from paper_1810_03275_gb300 import build, ctrecon
    if not os.path.exists(ctrecon.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        build.build()
    return ctypes.CDLL(ctrecon.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["rh_forward", "rh_adjoint", "precond_apply", "tv_pd_solve", "tv_pd_run",
                     "ctr_plan_create", "ctr_plan_destroy", "ctr_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1810_03275_gb300 import ctrecon
    names = declared_functions()
    missing = [nm for nm in names if not hasattr(lib, nm)]
    assert not missing, missing
    assert set(names) == set(ctrecon.EXPORTS)


def test_default_params_without_gpu(lib):
    """ctr_default_params and ctr_last_error are pure host functions."""
    from paper_1810_03275_gb300 import ctrecon
    p = ctrecon.default_params()
    assert p.sigma == 1.0 and abs(p.tau - 8 ** -0.5) < 1e-15 and p.power_iters == 50
    assert p.c_margin == 1.05 and p.trace_ratio == 0.8
    lib.ctr_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.ctr_last_error(), bytes)


def test_plan_create_rejects_bad_geometry_before_touching_the_device(lib):
    from paper_1810_03275_gb300 import ctrecon
    ctrecon.load()
    out = ctypes.c_void_p()
    angles = (ctypes.c_double * 4)(0, 0.5, 1.0, 1.5)
    for bad in [ctrecon.Geometry(0, 4, 5, 1.0, 1.0, angles), ctrecon.Geometry(8, 4, 5, -1.0, 1.0, angles),
                ctrecon.Geometry(8, 4, 5, 1.0, 1.0, None)]:
        assert ctrecon.load().ctr_plan_create(ctypes.byref(bad), 0, ctypes.byref(out)) == -1
        assert out.value is None


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: with the library absent the binding raises instead of computing."""
    from paper_1810_03275_gb300 import ctrecon
    monkeypatch.setattr(ctrecon, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        ctrecon.load(str(tmp_path / "missing" / "libctrecon.so"))


def test_binding_declares_every_exported_symbol():
    """The Python binding lists every entry point the header declares (argument
    marshalling only; nothing is computed in Python)."""
    from paper_1810_03275_gb300 import ctrecon
    assert set(declared_functions()) <= set(ctrecon.EXPORTS)
