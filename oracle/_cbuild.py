"""Compiles the oracle's plain-C band routines into a shared library.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "band_ref.c")
LIB = os.path.join(HERE, "_band_ref.so")


def build(force: bool = False) -> str:
    """Build ``_band_ref.so`` next to the source if it is missing or stale."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"],
                   check=True)
    os.replace(tmp, LIB)
    return LIB
