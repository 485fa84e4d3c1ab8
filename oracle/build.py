"""Compile the FP64 CPU oracle (``liboracle.so``) with gcc.

Test infrastructure: the oracle checks the CUDA path and is never part of it.
"""
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
STAMP = LIB + ".arch"


def build(force: bool = False) -> str:
    arch_ok = False
    try:
        with open(STAMP) as f:
            arch_ok = f.read().strip() == platform.machine()
    except OSError:
        pass
    if (not force and arch_ok and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    # -ffp-contract=off: binary32 ray set-up must round every operation.
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    with open(STAMP, "w") as f:
        f.write(platform.machine())
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
