"""Build the CPU oracle shared libraries (test infrastructure only).

Compiles ``mporacle.c`` twice with gcc: ``liboracle.so`` (plain) and
``liboracle_count.so`` (every binary64 operation counted).  IEEE semantics are
forced: no contraction of a*b+c into FMA and no fast-math, on x86-64 and on
aarch64 alike (gcc's default on aarch64 would otherwise contract).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mporacle.c")
FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def _stale(out):
    return (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(SRC)


def build(force=False):
    outs = []
    procs = []
    for name, extra in (("liboracle.so", []), ("liboracle_count.so", ["-DORACLE_COUNT"])):
        out = os.path.join(HERE, name)
        outs.append(out)
        if force or _stale(out):
            procs.append(subprocess.Popen(["gcc", *FLAGS, *extra, "-o", out, SRC, "-lm"]))
    for p in procs:
        if p.wait() != 0:
            raise RuntimeError("oracle build failed")
    print("oracle: %s" % ("compiled %d shared libraries with gcc" % len(procs) if procs else "up to date"),
          file=sys.stderr)
    return outs


if __name__ == "__main__":
    print(build(force=True))
