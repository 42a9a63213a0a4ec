"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain C11 + OpenMP, no FMA contraction (so x86 and Arm hosts evaluate the same
IEEE operations).  Called by ``__graft_entry__.build()`` and lazily by
``oracle.load()``.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dgpe_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "dgpe_oracle.h"))
    ):
        return LIB
    cmd = [
        "gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
        "-ffp-contract=off", "-o", LIB + ".tmp", SRC, "-lm",
    ]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
