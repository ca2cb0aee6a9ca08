"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/octmc.h; the binding declares the same set.  No GPU
compute is called here."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "octmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(octmc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_2010_06931_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(lib_path):
    names = header_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_header(lib_path):
    from paper_2010_06931_gb300 import _native
    assert _native.exported_names() == header_functions()


def test_host_only_calls(lib_path):
    from paper_2010_06931_gb300 import _native as N
    L = N.lib()
    d = N.Desc()
    L.octmc_desc_defaults(ctypes.byref(d))
    assert d.lbfgs_m == 8 and d.levels == 1 and abs(d.eps_h - 1e-3) < 1e-18 and abs(d.delta0 - 0.5) < 1e-18
    assert L.octmc_status_string(0) == b"ok"
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert L.octmc_create_problem(None, ctypes.byref(h)) == -1
    assert L.octmc_create_problem(ctypes.byref(d), ctypes.byref(h)) == -1  # w = h = d = 0
    assert L.octmc_level_shape(None, 0, None, None, None) == -1
    assert L.octmc_eval_objective_grad_async(None, 0, None, None, None, None) == -1
    assert L.octmc_barrier_selftest(-1) == -1 and L.octmc_barrier_selftest(2) == -1
    # a negative persistent-level size is rejected before any device work
    buf = (ctypes.c_float * 8)()
    tbuf = (ctypes.c_double * 4)()
    d2 = N.Desc()
    L.octmc_desc_defaults(ctypes.byref(d2))
    d2.w = d2.h = 2
    d2.d = 2
    d2.sx = d2.sy = ctypes.cast(buf, ctypes.c_void_p)
    d2.tx = d2.ty = ctypes.cast(tbuf, ctypes.c_void_p)
    d2.persistent_ascans = -1
    assert L.octmc_create_problem(ctypes.byref(d2), ctypes.byref(h)) == -1
    assert L.octmc_lbfgs_create(0, 8, None, ctypes.byref(h)) == -1
    # history length 1..32: the dot-product kernel holds 2 (m + 1) <= 66 history vectors
    assert L.octmc_lbfgs_create(100, 0, None, ctypes.byref(h)) == -1
    assert L.octmc_lbfgs_create(100, 33, None, ctypes.byref(h)) == -1
    # the adjacent steps validate their arguments before touching the device
    assert L.octmc_merge(None, None, 2.0, 0.05, None, None, None, None, None) == -1
    assert L.octmc_prealign_full(None, None, None, None) == -1
    assert L.octmc_prealign_eval(None, 0, None, None, None) == -1
    assert L.octmc_saccade_validity(None, 4, 4, 4, 0, None, None, None) == -1
    assert L.octmc_saccade_validity(None, 4, 4, 4, 2, None, None, None) == -1
    assert L.octmc_enface(None, None, 4, 4, 4, 0, None, 0.05, 0.95, 0.1, 0.0, None, None, None, None) == -1


def test_product_path_has_no_fallback(monkeypatch, tmp_path):
    from paper_2010_06931_gb300 import _native as N
    monkeypatch.setattr(N, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(N, "_lib", None)
    with pytest.raises(ImportError):
        N.lib()
