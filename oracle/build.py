"""Compile the C oracle (gcc, plain C99, -O2) into oracle/liboracle.so.

Test infrastructure only.  Host-portable flags (the GPU machine is aarch64).  With
OpenMP available the independent per-cell loops of the 3D oracle may run on
several host threads (oracle_threads); without it the library builds serial.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("wec_oracle.c", "poisson3d.c", "levelset3d.c", "tank3d.c")]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    deps = SRCS + [os.path.join(HERE, "wec_oracle.h"), os.path.abspath(__file__)]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, *SRCS, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
