"""Compile the C oracle into ``oracle/libpir_oracle.so`` (gcc, no GPU, any arch).

Test infrastructure: building the checker is not using it.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pir_oracle.c")
LIB = os.path.join(HERE, "libpir_oracle.so")


def command() -> list:
    return ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared", "-pthread", SRC, "-o", LIB]


def build(force: bool = False) -> str:
    stale = (not os.path.exists(LIB)) or os.path.getmtime(LIB) < os.path.getmtime(SRC)
    if force or stale:
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = command()
        cmd[-1] = tmp
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
