"""The C-ABI library loads and exports every entry point include/hji.h declares
(no compute calls: this runs without a GPU), and argument checks that fail
before any device work return the documented status."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "hji.h")).read()
    return sorted(set(re.findall(r"^\s*(?:hji_status|const char\*)\s+(hji_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("hji_grid_create", "hji_dynamics_set", "hji_solve", "hji_value_get",
                 "hji_batch_solve", "hji_grid_destroy", "hji_status_string", "hji_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(hji_lib):
    path = hji_lib.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert getattr(lib, n) is not None


def test_checked_build_exports_every_declared_symbol():
    """The bounds-checked debug build has the same boundary."""
    from paper_1903_07715_gb300 import build as B
    path = B.build(checked=True)  # no-op when up to date
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    assert not [n for n in _declared() if n not in exported]


def test_library_path_selects_the_checked_build(monkeypatch):
    """HJI_CHECKED_BUILD=1 makes the binding load the bounds-checked build;
    anything else, the product library."""
    import paper_1903_07715_gb300 as hji
    monkeypatch.setenv("HJI_CHECKED_BUILD", "1")
    assert hji.library_path().endswith("_hji_checked.so")
    monkeypatch.setenv("HJI_CHECKED_BUILD", "0")
    assert hji.library_path().endswith("_hji.so")
    monkeypatch.delenv("HJI_CHECKED_BUILD")
    assert hji.library_path().endswith("_hji.so")


def test_binding_names_match_header(hji_lib):
    assert sorted(hji_lib.EXPORTS) == sorted(n for n in _declared())
    for n in _declared():
        assert callable(getattr(hji_lib, n))


def test_status_strings(hji_lib):
    assert hji_lib.hji_status_string(0) == "ok"
    assert hji_lib.hji_status_string(4) == "not converged"
    assert hji_lib.hji_status_string(8) == "index check failed"
    assert hji_lib.hji_status_string(99) == "unknown status"


def test_create_rejects_bad_arguments_before_device_work(hji_lib):
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 2)(101, 2)  # an axis with 2 nodes
    lo = (ctypes.c_double * 2)(-1, -1)
    hi = (ctypes.c_double * 2)(1, 1)
    assert hji_lib.hji_grid_create(2, n, lo, hi, None, 0, None, ctypes.byref(h)) == 1
    assert "3 nodes" in hji_lib.hji_last_error(None)
    n = (ctypes.c_int64 * 2)(11, 11)
    assert hji_lib.hji_grid_create(5, n, lo, hi, None, 0, None, ctypes.byref(h)) == 1
    bad_hi = (ctypes.c_double * 2)(1, -2)
    assert hji_lib.hji_grid_create(2, n, lo, bad_hi, None, 0, None, ctypes.byref(h)) == 1
    assert hji_lib.hji_grid_create(2, n, lo, hi, None, 7, None, ctypes.byref(h)) == 1
    assert hji_lib.hji_solve(None, None, None, 0, None, None, None) == 1
    assert hji_lib.hji_value_get(None, None, 0, None) == 1
    assert hji_lib.hji_grid_destroy(None) == 0


def test_product_has_no_oracle_dependency():
    """The CUDA library and its binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1903_07715_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "hji_oracle" not in text, f


def test_selftest_limit_is_validated_before_device_work(hji_lib):
    assert hji_lib.hji_selftest_bounded_wait(10, None) == hji_lib.HJI_E_INVALID
    assert hji_lib.hji_selftest_bounded_wait(10 ** 10, None) == hji_lib.HJI_E_INVALID


def test_stage_times_rejects_null_arguments_before_device_work(hji_lib):
    ms = (ctypes.c_double * 3)()
    assert hji_lib.hji_stage_times(None, None, 0, None, 10, None, ms) == hji_lib.HJI_E_INVALID
    assert "NULL" in hji_lib.hji_last_error(None)
    assert hji_lib.hji_autotune(None, None, 0, None, 10, None, None, None) == hji_lib.HJI_E_INVALID


def test_peak_fma_validates_before_device_work(hji_lib):
    tf = ctypes.c_double()
    assert hji_lib.hji_peak_fma(7, 20.0, None, ctypes.byref(tf), None) == hji_lib.HJI_E_INVALID
    assert hji_lib.hji_peak_fma(0, 0.0, None, ctypes.byref(tf), None) == hji_lib.HJI_E_INVALID
    assert hji_lib.hji_peak_fma(1, 20.0, None, None, None) == hji_lib.HJI_E_INVALID
    assert "target_ms" in hji_lib.hji_peak_last_error()
