"""The bounds-checked debug build (_hji_checked.so: the library's sources
compiled with HJI_CHECKED, every index of the stage kernels' tile and halo
code tested against its array's extent before the access; a failed check is
recorded and makes the solve return HJI_E_CHECK).  It stands in for a
memory-checking tool: tests/checked_build_cases.py runs it, in a child
process that loads that library, on the grids where the tile and halo code
has the most edge logic, and compares every result with the oracle.  The
product library's checks compile to nothing: its recorder self-test records
no failure."""
import ctypes
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _selftest(hji):
    checked, count, site = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    index, extent = ctypes.c_int64(), ctypes.c_int64()
    rc = hji.hji_selftest_index_check(None, ctypes.byref(checked), ctypes.byref(count),
                                      ctypes.byref(site), ctypes.byref(index),
                                      ctypes.byref(extent))
    return rc, checked.value, count.value, site.value, index.value, extent.value


def test_product_build_has_no_checks(hji_lib):
    import torch
    assert torch.cuda.is_available()
    assert not hji_lib.library_path().endswith("_hji_checked.so")
    assert _selftest(hji_lib) == (hji_lib.HJI_OK, 0, 0, 0, 0, 0)


def test_checked_build_passes_every_case():
    from paper_1903_07715_gb300 import build as B
    B.build(checked=True)  # no-op when up to date
    env = dict(os.environ, HJI_CHECKED_BUILD="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_build_cases.py")], env=env,
                       capture_output=True, text=True, timeout=1500)
    rows = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    failed = [x for x in rows if not x.get("ok", True)]
    assert r.returncode == 0, (r.stderr[-3000:], failed)
    assert rows and rows[0]["case"] == "selftest"
    # the recorder: 3 failures, the first one site CK_PLANE (12), index 8, extent 10
    st = rows[0]
    assert (st["checked"], st["count"], st["site"], st["index"], st["extent"]) == (1, 3, 12, 8, 10)
    summary = rows[-1]
    assert summary.get("summary") and summary["failed"] == 0, failed
    assert summary["cases"] >= 150, summary
