"""Compile the C part of the oracle (test infrastructure only).

The shared object lands in ``oracle/_build/`` and is rebuilt when the source (or this
file) is newer.  ``gcc -O3`` with OpenMP over chains.  No architecture-specific flags
(no ``-march=native``): the same source and flags build on the x86_64 development host
and on the aarch64 GPU host and give the same results there; the C part is integer
arithmetic only, so the optimisation level changes no result.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "muca_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmuca_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Build ``libmuca_oracle.so`` if missing or stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(__file__))):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
