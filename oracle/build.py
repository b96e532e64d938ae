"""Compile the FP64 CPU oracle (test infrastructure) into a shared library.

Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark load the result.  The flags keep every floating-point operation
separately rounded (no contraction into FMA) and use OpenMP over cells.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hji_oracle.c")
LIB = os.path.join(HERE, "_hji_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
