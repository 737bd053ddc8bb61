"""Builds the oracle's C sweep (test infrastructure; see oracle/__init__.py)."""
from __future__ import annotations

import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sweep.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_sweep.so")
LIB_OMP = os.path.join(OUT_DIR, "liboracle_sweep_omp.so")


def build(force: bool = False, threads: bool = False) -> str:
    """Compile sweep.c with gcc (plain -O2, no FMA contraction) if stale.
    threads: the -fopenmp build (ordinates on all host cores, the same sums
    in the same order), used only to time the oracle."""
    lib = LIB_OMP if threads else LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(SRC)):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=OUT_DIR)
    os.close(fd)
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99"]
    if threads:
        cmd.append("-fopenmp")
    cmd += [SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
    print(build(force=True, threads=True))
