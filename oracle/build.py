"""Compiles the FP64 oracle (test infrastructure) into oracle/_build/libkq_oracle.so,
and the same source with OpenMP (assignment split over the host cores; used only
to time the oracle) into oracle/_build/libkq_oracle_omp.so."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kq_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libkq_oracle.so")
LIB_OMP = os.path.join(OUT_DIR, "libkq_oracle_omp.so")


def _build_one(out: str, extra, force: bool) -> str:
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + ".%d.tmp" % os.getpid()
    # -ffp-contract=off keeps every FP64 operation a separately rounded IEEE operation
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fvisibility=hidden",
           "-Wall", "-Wextra"] + list(extra) + ["-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Builds the serial library (and the OpenMP one) if missing or stale."""
    _build_one(LIB_OMP, ["-fopenmp"], force)
    return _build_one(LIB, [], force)


if __name__ == "__main__":
    print(build(force=True))
