"""Builds the oracle's shared library (oracle/_build/liboracle.so) with gcc.

Test infrastructure: the oracle is only loaded by the tests, the smoke check and
the CPU-baseline leg of the benchmark.  Plain C11, -O2, no fast-math and no FMA
contraction so that the x86 and Arm builds round identically; OpenMP only
splits independent amplitude groups across threads.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")
SRC = os.path.join(HERE, "qf_oracle.c")


def build(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
