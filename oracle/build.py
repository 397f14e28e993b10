"""Compile the CPU oracle (plain C) into oracle/libdvc_oracle.so.

Test infrastructure: the oracle is built so the test suite, the smoke check
and the benchmark's CPU-baseline leg can load it.  Floating point is compiled
with contraction off so every double operation rounds exactly as written.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dvc_oracle.c")
LIB = os.path.join(HERE, "libdvc_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
