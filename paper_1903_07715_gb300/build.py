"""Build the CUDA library (sm_103a) in-tree: paper_1903_07715_gb300/_hji.so,
and its bounds-checked debug build _hji_checked.so (the same sources with
HJI_CHECKED defined: every index of the stage kernels' tile and halo code is
checked before the access).

Each translation unit compiles in its own nvcc process (all of both builds in
parallel), then one link step per build makes the shared library.  Only
`-gencode arch=compute_103a,code=sm_103a` is emitted: the library targets
GB300 alone.
"""
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "_hji.so")
CHECKED_LIB = os.path.join(HERE, "_hji_checked.so")
SOURCES = ["hji_stage_f64.cu", "hji_stage_f32.cu", "hji_march_f64.cu", "hji_march_f32.cu",
           "hji_llf_f64.cu", "hji_llf_f32.cu",
           "hji_setup.cu", "hji_capi.cu", "hji_noalloc.cu", "hji_peak.cu", "hji_control.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-O3",
              "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "hji.h"))
    files.append(os.path.abspath(__file__))
    return files


def _lib_path(checked):
    return CHECKED_LIB if checked else LIB


def up_to_date(checked=False):
    lib = _lib_path(checked)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force=False, verbose=False, extra_flags=(), checked=False):
    """Build one library: the product build, or (checked=True) the
    bounds-checked debug build.  Returns its path."""
    return build_variants((checked,), force=force, verbose=verbose, extra_flags=extra_flags)[0]


def build_all(force=False, verbose=False):
    """Both builds, every translation unit of both compiled in parallel."""
    return build_variants((False, True), force=force, verbose=verbose)


def build_variants(variants, force=False, verbose=False, extra_flags=()):
    todo = [c for c in variants if force or not up_to_date(c)]
    if not todo:
        return [_lib_path(c) for c in variants]
    nvcc = _nvcc()
    tmp = tempfile.mkdtemp(prefix="hji_build_")
    try:
        procs, objs = [], {c: [] for c in todo}
        for checked in todo:
            defs = ["-DHJI_CHECKED=1"] if checked else []
            for src in SOURCES:
                obj = os.path.join(tmp, ("chk_" if checked else "") + src.replace(".cu", ".o"))
                cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, *extra_flags, "-c", os.path.join(CSRC, src),
                       "-o", obj]
                if verbose:
                    print(" ".join(cmd), flush=True)
                procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                    stderr=subprocess.STDOUT)))
                objs[checked].append(obj)
        failed = []
        for src, p in procs:
            out, _ = p.communicate()
            text = out.decode(errors="replace")
            if p.returncode != 0:
                failed.append((src, text))
            elif verbose and text.strip():
                print(text, flush=True)
        if failed:
            msg = "\n".join("%s:\n%s" % f for f in failed)
            raise RuntimeError("nvcc failed\n" + msg)
        for checked in todo:
            lib = _lib_path(checked)
            out_tmp = lib + ".tmp%d" % os.getpid()
            cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", out_tmp, *objs[checked],
                   "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
            subprocess.run(cmd, check=True)
            os.replace(out_tmp, lib)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return [_lib_path(c) for c in variants]


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(force=True, verbose=v, checked="--checked" in sys.argv,
                extra_flags=("-Xptxas", "-v") if "--ptxas-v" in sys.argv else ()))
