"""The Python binding's view of include/hji.h, checked on CPU: a small C
program compiled against the header prints sizeof / offsetof of every struct
member the ctypes structures declare, and the value of every constant the
binding mirrors; both must agree with the binding exactly.  Every exported
call's ctypes prototype is compared with the header's declaration."""
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


# ---------------------------------------------------------------- prototypes

def _header_prototypes():
    import re
    with open(os.path.join(ROOT, "include", "hji.h")) as f:
        s = f.read()
    s = re.sub(r"/\*.*?\*/", " ", s, flags=re.S)
    s = "\n".join(ln for ln in s.splitlines() if not ln.lstrip().startswith("#"))
    enums = set(re.findall(r"typedef\s+enum\s*\{[^}]*\}\s*(\w+)\s*;", s))
    handles = set(re.findall(r"typedef\s+struct\s+\w+\s*\*\s*(\w+)\s*;", s))
    protos = {}
    for ret, name, args in re.findall(r"([A-Za-z_][\w\s\*]*?)\b(hji_\w+)\s*\(([^;{]*?)\)\s*;", s):
        params = [] if args.strip() in ("", "void") else [a.strip() for a in args.split(",")]
        protos[name] = (" ".join(ret.split()), params)
    return protos, enums, handles


def _c_kind(decl, enums, handles, has_name=True):
    """(base, pointer depth) of a C parameter declaration or return type."""
    toks = decl.replace("*", " * ").split()
    toks = [t for t in toks if t != "const"]
    if has_name and toks and toks[-1] != "*":
        toks = toks[:-1]
    depth = toks.count("*")
    base = [t for t in toks if t != "*"][0]
    if base in enums:
        base = "int"
    if base in handles:
        base, depth = "void", depth + 1
    return {"int": "int", "int64_t": "i64", "size_t": "size", "double": "double",
            "void": "void", "char": "char"}.get(base, base), depth


def _py_kind(t):
    depth = 0
    while hasattr(t, "_type_") and isinstance(getattr(t, "_type_"), type) and \
            t.__name__.startswith("LP_"):
        depth, t = depth + 1, t._type_
    simple = {ctypes.c_int: ("int", 0), ctypes.c_int64: ("i64", 0), ctypes.c_size_t: ("size", 0),
              ctypes.c_double: ("double", 0), ctypes.c_void_p: ("void", 1),
              ctypes.c_char_p: ("char", 1)}
    if t in simple:
        b, d = simple[t]
        return b, depth + d
    return t.__name__, depth


def test_prototypes_match_header(hji_lib):
    """Every exported call's ctypes argtypes / restype against its prototype in
    the header (enums as int, the opaque handles as pointers)."""
    protos, enums, handles = _header_prototypes()
    lib = hji_lib.load()
    assert set(hji.EXPORTS) <= set(protos), set(hji.EXPORTS) - set(protos)
    for name in hji.EXPORTS:
        ret, params = protos[name]
        fn = getattr(lib, name)
        assert _py_kind(fn.restype) == _c_kind(ret, enums, handles, has_name=False), name
        got = [_py_kind(t) for t in fn.argtypes]
        want = [_c_kind(p, enums, handles) for p in params]
        assert got == want, (name, got, want)
