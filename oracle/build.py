"""Compile the FP64 CPU oracle (test infrastructure) into ``oracle/_oracle.so``.

Plain gcc, ``-O2`` without fast-math (IEEE double semantics are part of the
oracle's definition), OpenMP when the compiler supports it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fno-fast-math",
            "-ffp-contract=off", SRC, "-o", LIB + ".tmp", "-lm"]
    last = None
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
        last = r
    raise RuntimeError("oracle build failed:\n" + (last.stderr if last else ""))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
