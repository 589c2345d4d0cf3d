"""Count the algorithmic FP32 FLOPs of the chain code (the roofline
numerator of bench.py).

Makes host copies of csrc/sg_chain.cuh and csrc/sg_adjoint.cuh with `float`
replaced by the counting scalar of flops/count.cpp, compiles that driver
with the host C++ compiler and returns its counts:
    {pattern: {"substep", "tip", "substep_adjoint", "tip_vjp", "substep_replay"}}.

    python -m paper_2310_04676_gb300.flops.count
"""
import os
import re
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "csrc")
INCLUDE = os.path.join(os.path.dirname(os.path.dirname(HERE)), "include")


def _host_copy(src, dst, drop_includes):
    text = open(src).read()
    for inc in drop_includes:
        text = text.replace(inc, "")
    text = re.sub(r"\bfloat\b", "CF", text)
    with open(dst, "w") as f:
        f.write(text)


def count():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        raise RuntimeError("a host C++ compiler is required")
    with tempfile.TemporaryDirectory() as tmp:
        _host_copy(os.path.join(CSRC, "sg_chain.cuh"), os.path.join(tmp, "chain_host.h"),
                   ["#include <cuda_runtime.h>"])
        _host_copy(os.path.join(CSRC, "sg_adjoint.cuh"), os.path.join(tmp, "adjoint_host.h"),
                   ['#include "sg_chain.cuh"'])
        exe = os.path.join(tmp, "count")
        cmd = [cxx, "-std=c++17", "-O1", "-I" + tmp, "-I" + CSRC, "-I" + INCLUDE,
               os.path.join(HERE, "count.cpp"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("flop counter build failed:\n" + r.stderr[-3000:])
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    res = {}
    for line in out.strip().splitlines():
        f = line.split()
        res[f[0]] = {f[i]: int(f[i + 1]) for i in range(1, len(f), 2)}
    return res


if __name__ == "__main__":
    for k, v in count().items():
        print(k, v)
    sys.exit(0)
