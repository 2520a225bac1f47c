"""Build libptrig_cpu.so in-tree with gcc.

    python -m cpu_simd.build

Portable C: no intrinsics and no -march flags, so the same source builds on
x86-64 (SSE2 vectors) and on aarch64 (NEON vectors) and gives the same
results on both (-ffp-contract=off keeps every rounding explicit).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "ptrig_cpu.c")
HDRS = [os.path.join(ROOT, "include", "ptrig_cpu.h"),
        os.path.join(ROOT, "paper_2502_10831_gb300", "csrc", "ptrig_constants.h")]
LIB = os.path.join(HERE, "_build", "libptrig_cpu.so")
FLAGS = ["-O3", "-std=gnu11", "-ffp-contract=off", "-fno-math-errno", "-fno-trapping-math", "-fPIC", "-shared",
         "-pthread", "-Wall", "-Wextra"]


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    deps = [SRC] + HDRS
    if not force and os.path.exists(LIB) and all(os.path.getmtime(d) <= os.path.getmtime(LIB) for d in deps):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *FLAGS, "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2502_10831_gb300", "csrc"), SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 or r.stderr.strip():
        sys.stderr.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError("gcc failed: " + " ".join(cmd))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
