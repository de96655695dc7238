"""Compile the CPU oracle (test infrastructure) into ``oracle/liboracle_suco.so``.

Plain gcc, no GPU, no shared code with the CUDA library.  ``-ffp-contract=off``
keeps the compiler from fusing any multiply-add other than the explicit
``fmaf`` calls that restate the GPU kernel's FP32 ranking arithmetic.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "suco_oracle.c")
LIB = os.path.join(HERE, "liboracle_suco.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fvisibility=hidden", "-Wall", "-Wextra", "-Wno-unused-parameter",
           "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
