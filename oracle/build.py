"""Compile the plain C oracle into oracle/liboracle.so with gcc.

TEST INFRASTRUCTURE: the oracle is used by the test suite, the smoke check and the CPU-baseline
leg of the benchmark only.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hdarray_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force=False, verbose=False):
    """Build liboracle.so if it is missing or older than its source. Returns the library path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    # the stencil value loops may run on several threads (OpenMP); a compiler without OpenMP
    # builds the same oracle with single-threaded loops
    for cmd in (base[:1] + ["-fopenmp"] + base[1:], base + ["-Wno-unknown-pragmas"]):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        if subprocess.run(cmd).returncode == 0:
            break
    else:
        raise RuntimeError("building the oracle failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
