"""Compile the oracle's C part (plain gcc, no CUDA).  Test infrastructure only."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")


def lib_path(mutant: bool = False) -> str:
    return os.path.join(BUILD, "liboracle_sweeps_mutant.so" if mutant else "liboracle_sweeps.so")


def build(mutant: bool = False, force: bool = False) -> str:
    """Build oracle/_build/liboracle_sweeps.so (or the planted-mistake variant used by
    the pin-sensitivity tests) and return its path."""
    os.makedirs(BUILD, exist_ok=True)
    out = lib_path(mutant)
    src = os.path.join(HERE, "sweeps.c")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", out + ".tmp", src, "-lm"]
    if mutant:
        cmd.insert(1, "-DORACLE_MUTANT_PRINTED_CURVATURE")
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build())
