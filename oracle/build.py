"""Compile the FP64 REWL oracle (plain C) into ``oracle/librewl_oracle.so``.

Test infrastructure: the oracle is built by ``__graft_entry__.build()`` so that the test suite,
``smoke()`` and the benchmark's CPU-baseline leg can load it.  Flags keep IEEE FP64 semantics:
no contraction into fused multiply-add, no fast-math reassociation.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rewl_oracle.c")
OUT = os.path.join(HERE, "librewl_oracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wno-unused-function"]


def build(force: bool = False) -> str:
    if (not force and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= os.path.getmtime(SRC)
            and os.path.getmtime(OUT) >= os.path.getmtime(os.path.join(HERE, "rewl_oracle.h"))):
        return OUT
    cmd = ["gcc", *CFLAGS, "-o", OUT, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
