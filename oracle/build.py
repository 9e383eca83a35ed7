"""Build the CPU oracle shared library (oracle/liboracle.so).

Test infrastructure: the oracle is what the GPU path is checked against; only
tests/, __graft_entry__ and bench.py's CPU-baseline leg use it.

ISO C11 with -ffp-contract=off so that the compiler fuses no multiply-add the
source does not spell out as fma(); OpenMP is used when the compiler has it
(the spatial loops are independent per point, so results do not depend on the
thread count).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "swept_oracle.c")
SRC2D = os.path.join(HERE, "heat2d.c")
INC = os.path.join(HERE, "scheme_body.inc")
LIB = os.path.join(HERE, "liboracle.so")


def _compile(extra):
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", LIB + ".tmp", SRC, SRC2D] + extra + ["-lm"]
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force=False):
    """Compile liboracle.so if it is missing or older than its sources; return its path."""
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(SRC), os.path.getmtime(SRC2D), os.path.getmtime(INC))
        if os.path.getmtime(LIB) >= newest:
            return LIB
    r = _compile(["-fopenmp"])
    if r.returncode != 0:
        r = _compile([])
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
