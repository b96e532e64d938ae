"""Build the CUDA library (sm_103a) in-tree: paper_1903_07715_gb300/_hji.so.

Each translation unit compiles in its own nvcc process (in parallel), then one
link step makes the shared library.  Only `-gencode arch=compute_103a,
code=sm_103a` is emitted: the library targets GB300 alone.
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


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force=False, verbose=False, extra_flags=()):
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    tmp = tempfile.mkdtemp(prefix="hji_build_")
    try:
        procs, objs = [], []
        for src in SOURCES:
            obj = os.path.join(tmp, src.replace(".cu", ".o"))
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
            objs.append(obj)
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
        out_tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", out_tmp, *objs,
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        subprocess.run(cmd, check=True)
        os.replace(out_tmp, LIB)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(force=True, verbose=v,
                extra_flags=("-Xptxas", "-v") if "--ptxas-v" in sys.argv else ()))
