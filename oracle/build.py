"""Compile the C oracle into oracle/_build/liboracle.so (gcc, OpenMP).

Flags: -O2 -ffp-contract=off and no fast-math, so every double operation in
the oracle is one correctly rounded IEEE-754 operation in source order.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tauleap_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


FLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
         "-Wall", "-Wextra"]


def compile_source(src: str, out: str, extra=()) -> None:
    """Compile one oracle source file into a shared library with the oracle's
    flags (plus `extra`, e.g. sanitizer flags for a checking build)."""
    subprocess.run(["gcc", *FLAGS, *extra, "-o", out, src], check=True)


def build(force: bool = False) -> str:
    """Compile liboracle.so unless it is newer than the source; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    compile_source(SRC, tmp)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
