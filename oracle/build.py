"""Compile the CPU oracle into oracle/liboracle.so (test infrastructure only).

The oracle is built with -ffp-contract=off so that every float energy
operation is one IEEE add or subtract, and without -ffast-math.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ecoevo_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    deps = [SRC, os.path.join(HERE, "ecoevo_oracle.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-Wall", "-ffp-contract=off", "-fPIC",
           "-shared", SRC, "-lm", "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
