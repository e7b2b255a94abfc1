"""Compile the CPU oracle (oracle_vegas.c) into oracle/liboracle_vegas.so.

Test infrastructure only (see oracle_vegas.h).  -ffp-contract=off keeps every
float/double operation a separate IEEE operation on both x86-64 and Arm, where
gcc would otherwise fuse multiply-adds.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle_vegas.c")
LIB = os.path.join(HERE, "liboracle_vegas.so")


def build(force: bool = False) -> str:
    hdr = os.path.join(HERE, "oracle_vegas.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
