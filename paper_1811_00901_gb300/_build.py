"""Build libspin_gb300.so in-tree with nvcc for sm_103a.

Every translation unit under csrc/ is compiled in parallel; the objects are
linked into ``_lib/libspin_gb300.so`` next to this file.  The spin kernel is
compiled a second time with SI_DEBUG_BOUNDS (index checks that flag and skip
a bad access instead of trapping) and linked with the other objects into
``_lib/libspin_gb300_bounds.so``, the bounds-checking build the tests run
small cases through.  Rebuilds only when a source or header is newer than the
libraries.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libspin_gb300.so")
LIB_BOUNDS = os.path.join(OUT_DIR, "libspin_gb300_bounds.so")
BOUNDS_SOURCES = ("spin_kernel.cu",)  # compiled again with -DSI_DEBUG_BOUNDS
OBJ_DIR = os.path.join(OUT_DIR, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-I", CSRC,
          "-I", INCLUDE]


def nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date():
    if not os.path.exists(LIB) or not os.path.exists(LIB_BOUNDS):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_BOUNDS))
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(src, verbose_ptxas=False, bounds=False):
    obj = os.path.join(OBJ_DIR, os.path.basename(src) + (".bounds.o" if bounds else ".o"))
    cmd = [nvcc()] + ARCH + COMMON + (["-DSI_DEBUG_BOUNDS"] if bounds else []) + ["-c", src, "-o", obj]
    if src.endswith(".cu"):
        cmd += ["--expt-relaxed-constexpr"]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(force=False, verbose_ptxas=False, quiet=True):
    """Compile and link; returns the library path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)
    srcs = sources()
    jobs = [(s, False) for s in srcs] + [(s, True) for s in srcs if os.path.basename(s) in BOUNDS_SOURCES]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda j: _compile(j[0], verbose_ptxas and not j[1], j[1]), jobs))
    if verbose_ptxas:
        for obj, err in results:
            if err.strip():
                sys.stderr.write(err)
    plain = [o for (o, _), (_, b) in zip(results, jobs) if not b]
    checked = {os.path.basename(s): o for (o, _), (s, b) in zip(results, jobs) if b}
    bounds_objs = [checked.get(os.path.basename(o)[:-2], o) for o in plain]
    for lib, objs in ((LIB, plain), (LIB_BOUNDS, bounds_objs)):
        tmp = lib + ".tmp.%d" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        os.replace(tmp, lib)
    if not quiet:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, quiet=False)
