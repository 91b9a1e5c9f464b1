"""Compile the test-only cuRAND Philox probe (tests/cuda/libcurand_probe.so)."""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "curand_philox_probe.cu")
OUT = os.path.join(HERE, "libcurand_probe.so")


def build(force=False):
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    "-cudart", "shared", "-o", OUT, SRC], check=True)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
