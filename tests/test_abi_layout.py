"""The Python binding's view of include/hji.h, checked on CPU: a small C
program compiled against the header prints sizeof / offsetof of every struct
member the ctypes structures declare, and the value of every constant the
binding mirrors; both must agree with the binding exactly."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1903_07715_gb300 as hji

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"hji_allocator": hji.hji_allocator, "hji_dynamics": hji.hji_dynamics,
           "hji_solve_opts": hji.hji_solve_opts, "hji_solve_stats": hji.hji_solve_stats}
CONSTANTS = ["HJI_MAX_DIM", "HJI_MAX_INPUTS", "HJI_MAX_TERMS", "HJI_TILE_VARIANTS", "HJI_OK",
             "HJI_E_INVALID", "HJI_E_NOMEM", "HJI_E_CUDA", "HJI_E_NOT_CONVERGED",
             "HJI_E_TIMEOUT", "HJI_E_STATE", "HJI_E_NONFINITE", "HJI_E_CHECK", "HJI_F64",
             "HJI_F32", "HJI_ENO1", "HJI_ENO2", "HJI_WENO5", "HJI_INIT_STANDARD",
             "HJI_INIT_USER_K", "HJI_INIT_RESIDENT"]


@pytest.fixture(scope="module")
def header_layout():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    out_dir = os.path.join(ROOT, "_build", "abi_layout")
    os.makedirs(out_dir, exist_ok=True)
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hji.h"',
             "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s*)0)->%s));'
                         % (name, field, name, field, name, field))
    for c in CONSTANTS:
        lines.append('  printf("%s %%d\\n", (int)(%s));' % (c, c))
    for fn in ("TAN", "SIN", "COS"):
        lines.append('  printf("HJI_FN_%s %%d\\n", (int)HJI_FN_%s);' % (fn, fn))
    for m in ("AUTO", "PER_STAGE", "MULTI_STEP"):
        lines.append('  printf("HJI_MARCH_%s %%d\\n", (int)HJI_MARCH_%s);' % (m, m))
    lines += ["  return 0;", "}"]
    src = os.path.join(out_dir, "probe.c")
    exe = os.path.join(out_dir, "probe")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", exe, src], check=True)
    res = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    table = {}
    for ln in res.splitlines():
        parts = ln.split()
        table[parts[0] + ("" if parts[1] != "sizeof" else " sizeof")] = \
            [int(p) for p in parts[1:] if p != "sizeof"]
    return table


@pytest.mark.parametrize("name", list(STRUCTS))
def test_struct_layout_matches_header(header_layout, name):
    cls = STRUCTS[name]
    assert header_layout[name + " sizeof"] == [ctypes.sizeof(cls)], name
    for field, ctype in cls._fields_:
        off, size = header_layout["%s.%s" % (name, field)]
        assert getattr(cls, field).offset == off, (name, field)
        assert ctypes.sizeof(ctype) == size, (name, field)


def test_constants_match_header(header_layout):
    for c in CONSTANTS:
        assert header_layout[c] == [getattr(hji, c)], c
    for fn, v in hji.HJI_FN.items():
        assert header_layout["HJI_FN_" + fn.upper()] == [v]
    for m, v in hji.MARCH.items():
        assert header_layout["HJI_MARCH_" + m.upper()] == [v]
