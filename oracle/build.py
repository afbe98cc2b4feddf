"""Compile the C oracle (test infrastructure) into oracle/liboracle.so.

Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
use the oracle.  ``defines`` lets a test build a variant with a planted
mistake into a separate file (see tests/test_oracle_mutants.py).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sfmm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(out=LIB, defines=(), force=False):
    if (not force and not defines and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
           "-Wno-unused-function", SRC, "-o", out + ".tmp", "-lm"]
    cmd[1:1] = ["-D" + d for d in defines]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build(force=True))
