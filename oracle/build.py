"""Compiles the CPU oracle (test infrastructure) into oracle/liblcl_oracle.so with gcc.

Flags: -O2 -std=c11 -ffp-contract=off, so that no multiply-add is fused and every
floating-point operation is one IEEE rounding in source order on x86-64 and on Arm.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lcl_oracle.c")


def library_path() -> str:
    return os.path.join(HERE, "liblcl_oracle.so")


def build_oracle(force: bool = False) -> str:
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-Wno-unused-parameter", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force=True))
