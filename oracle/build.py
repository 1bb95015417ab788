"""Compile the oracle's C sources into ``oracle/_build/liboracle.so`` (test
infrastructure; gcc, FP64, ``-ffp-contract=off`` so no multiply-add is fused)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ("exact.c", "tree.c")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")
COUNT_OUT = os.path.join(OUT_DIR, "liboracle_count.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    if not force and os.path.exists(OUT):
        t = os.path.getmtime(OUT)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return OUT
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           "-Wall", "-Wno-unused-function", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


def build_count(force: bool = False) -> str:
    """The work-counting build of the closed form (count.cpp, which includes
    exact.c with a counting number type)."""
    srcs = [os.path.join(HERE, s) for s in ("count.cpp", "exact.c")]
    if not force and os.path.exists(COUNT_OUT):
        t = os.path.getmtime(COUNT_OUT)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return COUNT_OUT
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = COUNT_OUT + f".{os.getpid()}.tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           "-fvisibility=hidden", "-o", tmp, srcs[0], "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, COUNT_OUT)
    return COUNT_OUT


if __name__ == "__main__":
    print(build(force=True))
    print(build_count(force=True))
