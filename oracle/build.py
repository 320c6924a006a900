"""Compile the C oracle with gcc (test infrastructure only).

``-ffp-contract=off`` matters: the FP32 candidate-set definition spells out
its fused multiply-adds with fmaf(), and on aarch64 gcc would otherwise fuse
further products on its own.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spin_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")


def library_path():
    return os.path.join(OUT_DIR, "liboracle.so")


def build_oracle(force=False):
    out = library_path()
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


SRC_OMP = os.path.join(HERE, "spin_oracle_omp.c")


def library_path_omp():
    return os.path.join(OUT_DIR, "liboracle_omp.so")


def build_oracle_omp(force=False):
    """The OpenMP image loop (CPU baseline).  Returns None when the host
    compiler has no OpenMP; nothing else depends on it."""
    out = library_path_omp()
    if (not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC_OMP)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-fopenmp",
           "-shared", "-o", tmp, SRC, SRC_OMP, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return None
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force=True))
    print(build_oracle_omp(force=True))
