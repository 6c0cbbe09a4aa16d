"""Compile the FP64 CPU oracle (``mgr_oracle.c``) into ``liboracle.so``.

Test infrastructure only: the oracle is the independent checker of the CUDA
path and is never linked into the library.  ``-ffp-contract=off`` keeps every
multiply and add separately rounded on both x86_64 and aarch64 hosts, so the
oracle gives bit-identical results on either machine.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mgr_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-o", LIB + ".tmp", SRC]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
