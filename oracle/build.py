"""Compile the FP64 CPU oracle (oracle.c) into liboracle.so.

Test infrastructure only: the library is loaded by tests/, by
__graft_entry__.smoke() and by bench.py's CPU-baseline leg, never by the
product path.  gcc, -O2, OpenMP, and -ffp-contract=off so that no
multiply-add is fused and the result is the same on x86 and Arm.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
