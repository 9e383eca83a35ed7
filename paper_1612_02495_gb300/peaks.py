"""Measure the unit throughputs the stencil kernels are bound by (probe/peaks_probe.cu).

  python -m paper_1612_02495_gb300.peaks [--out peaks.json]

Compiles the probe for sm_103a with nvcc, runs it on the current GPU and
prints (and optionally writes) its JSON: FP64 FMA rate with constant-bank and
with register operands, the KS update's FP64 instruction mix, FP32 FMA, shared
memory load bandwidth, __syncthreads cost and launch latencies.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "probe", "peaks_probe.cu")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "peaks_probe")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe, SRC],
                       check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        print(r.stdout + r.stderr, file=sys.stderr)
        return r.returncode
    res = json.loads(r.stdout.strip().splitlines()[-1])
    print(json.dumps(res, indent=1))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
