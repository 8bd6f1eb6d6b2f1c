"""Compile the oracle's C state-vector simulator (test infrastructure).

Plain gcc, no architecture-specific flags, so the same source builds on
x86_64 and aarch64 hosts.  OpenMP splits index ranges only.
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sv.c")
LIB = os.path.join(HERE, "_oracle_sv.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", SRC, "-o", LIB + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
