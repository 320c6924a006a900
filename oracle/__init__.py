"""FP64 CPU oracle for spin-image generation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline and
reference legs may import this package.  The product (the CUDA library under
``paper_1811_00901_gb300``) never imports, links or runs it, and it shares no
code with that library: the two meet only through the seeded input
generators of ``paper_1811_00901_gb300.workloads``, which hold none of the
method's arithmetic.

Contents:
  spin_oracle.c   FP64 brute-force all-pairs spin images (Sec. 2.1,
                  Algorithm 1), boundary flags, FP32 candidate-set definition
  dls.py          chunk sequences of STATIC / SS / GSS / FAC (Sec. 2.2,
                  Algorithm 3's getChunk)
  build.py        compiles spin_oracle.c with gcc into oracle/_build/
"""
import ctypes
import os

import numpy as np

from . import dls  # noqa: F401  (re-exported)
from .build import build_oracle, library_path

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        build_oracle()
    lib = ctypes.CDLL(path)
    f32p = ctypes.POINTER(ctypes.c_float)
    f64p = ctypes.POINTER(ctypes.c_double)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_spin_images.argtypes = [f32p, f32p, ctypes.c_int64, i32p, ctypes.c_int64,
                                       ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                       f64p, i64p, i64p]
    lib.oracle_spin_images.restype = ctypes.c_int
    lib.oracle_pair_coords.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_float, f64p, f64p, i32p]
    lib.oracle_pair_coords.restype = ctypes.c_int
    lib.oracle_candidates_fp32.argtypes = [f32p, ctypes.c_int64, i32p, ctypes.c_int64,
                                           ctypes.c_int32, ctypes.c_float, i64p, u32p]
    lib.oracle_candidates_fp32.restype = ctypes.c_int
    lib.oracle_spin_images_nearest.argtypes = [f32p, f32p, ctypes.c_int64, i32p, ctypes.c_int64, ctypes.c_int32,
                                               ctypes.c_float, ctypes.c_float, i32p,
                                               ctypes.POINTER(ctypes.c_int64), f32p]
    lib.oracle_spin_images_nearest.restype = ctypes.c_int
    lib.oracle_support_radius2.argtypes = [ctypes.c_int32, ctypes.c_float]
    lib.oracle_support_radius2.restype = ctypes.c_double
    lib.oracle_candidate_rc2.argtypes = [ctypes.c_int32, ctypes.c_float]
    lib.oracle_candidate_rc2.restype = ctypes.c_float
    _lib = lib
    return lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f32x3(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("expected an (n, 3) array")
    return a


def _queries(query_idx, m):
    if query_idx is None:
        return None, int(m)
    q = np.ascontiguousarray(query_idx, dtype=np.int32)
    return q, int(q.shape[0])


def spin_images(points, normals, W, bin_size, cos_s, query_idx=None, m=None):
    """FP64 spin images of the queries (all pairs).

    Returns ``(img[m, W, W] float64, support[m] int64, flagged[m] int64)``.
    ``query_idx=None`` means queries 0..m-1 (m defaults to all points).
    """
    p, nr = _f32x3(points), _f32x3(normals)
    n = p.shape[0]
    q, m = _queries(query_idx, n if m is None else m)
    img = np.zeros((m, W, W), dtype=np.float64)
    sup = np.zeros(m, dtype=np.int64)
    flg = np.zeros(m, dtype=np.int64)
    rc = _load().oracle_spin_images(_ptr(p, ctypes.c_float), _ptr(nr, ctypes.c_float), n,
                                    _ptr(q, ctypes.c_int32), m, int(W), float(bin_size),
                                    float(cos_s), _ptr(img, ctypes.c_double),
                                    _ptr(sup, ctypes.c_int64), _ptr(flg, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_spin_images failed with code %d" % rc)
    return img, sup, flg


def pair_coords(points, normals, query, cos_s=-1.0):
    """FP64 (alpha, beta, angle_ok) of every pair (query, X)."""
    p, nr = _f32x3(points), _f32x3(normals)
    n = p.shape[0]
    a = np.zeros(n, dtype=np.float64)
    b = np.zeros(n, dtype=np.float64)
    ok = np.zeros(n, dtype=np.int32)
    rc = _load().oracle_pair_coords(_ptr(p, ctypes.c_float), _ptr(nr, ctypes.c_float), n,
                                    int(query), float(cos_s), _ptr(a, ctypes.c_double),
                                    _ptr(b, ctypes.c_double), _ptr(ok, ctypes.c_int32))
    if rc != 0:
        raise ValueError("oracle_pair_coords failed with code %d" % rc)
    return a, b, ok.astype(bool)


def candidates_fp32(points, W, bin_size, query_idx=None, m=None):
    """FP32 candidate set per query: ``(count[m] int64, hash[m] uint32)``."""
    p = _f32x3(points)
    n = p.shape[0]
    q, m = _queries(query_idx, n if m is None else m)
    cnt = np.zeros(m, dtype=np.int64)
    hs = np.zeros(m, dtype=np.uint32)
    rc = _load().oracle_candidates_fp32(_ptr(p, ctypes.c_float), n, _ptr(q, ctypes.c_int32), m,
                                        int(W), float(bin_size), _ptr(cnt, ctypes.c_int64),
                                        _ptr(hs, ctypes.c_uint32))
    if rc != 0:
        raise ValueError("oracle_candidates_fp32 failed with code %d" % rc)
    return cnt, hs


def spin_images_nearest(points, normals, W, bin_size, cos_s, query_idx=None, m=None):
    """Algorithm 1's own count in IEEE FP32 (see oracle_spin_images_nearest).

    Returns ``(counts[m, W, W] int32, support[m] int64, max_d2[m] float32)``.
    """
    p, nr = _f32x3(points), _f32x3(normals)
    n = p.shape[0]
    q, m = _queries(query_idx, n if m is None else m)
    cnt = np.zeros((m, W, W), dtype=np.int32)
    sup = np.zeros(m, dtype=np.int64)
    dmax = np.zeros(m, dtype=np.float32)
    rc = _load().oracle_spin_images_nearest(_ptr(p, ctypes.c_float), _ptr(nr, ctypes.c_float), n,
                                            _ptr(q, ctypes.c_int32), m, int(W), float(bin_size), float(cos_s),
                                            _ptr(cnt, ctypes.c_int32), _ptr(sup, ctypes.c_int64),
                                            _ptr(dmax, ctypes.c_float))
    if rc != 0:
        raise ValueError("oracle_spin_images_nearest failed with code %d" % rc)
    return cnt, sup, dmax


_lib_omp = None
OMP_RULES = {"static": 0, "dynamic": 1, "guided": 2}


def _load_omp():
    """The OpenMP image loop, or None when the host compiler has no OpenMP."""
    global _lib_omp
    if _lib_omp is not None:
        return _lib_omp or None
    from .build import build_oracle_omp
    path = build_oracle_omp()
    if path is None:
        _lib_omp = False
        return None
    lib = ctypes.CDLL(path)
    f32p = ctypes.POINTER(ctypes.c_float)
    lib.oracle_spin_images_omp.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.c_int32, ctypes.c_int32]
    lib.oracle_spin_images_omp.restype = ctypes.c_int
    lib.oracle_omp_max_threads.restype = ctypes.c_int
    _lib_omp = lib
    return lib


def omp_available():
    return _load_omp() is not None


def omp_max_threads():
    lib = _load_omp()
    return lib.oracle_omp_max_threads() if lib else 0


def spin_images_omp(points, normals, W, bin_size, cos_s, query_idx=None, m=None, rule="static", threads=0):
    """spin_images (without flags) with the image loop under OpenMP
    schedule(static), schedule(dynamic, 1) or schedule(guided)."""
    lib = _load_omp()
    if lib is None:
        raise RuntimeError("the host compiler has no OpenMP")
    p, nr = _f32x3(points), _f32x3(normals)
    n = p.shape[0]
    q, m = _queries(query_idx, n if m is None else m)
    img = np.zeros((m, W, W), dtype=np.float64)
    sup = np.zeros(m, dtype=np.int64)
    rc = lib.oracle_spin_images_omp(_ptr(p, ctypes.c_float), _ptr(nr, ctypes.c_float), n, _ptr(q, ctypes.c_int32),
                                    m, int(W), float(bin_size), float(cos_s), _ptr(img, ctypes.c_double),
                                    _ptr(sup, ctypes.c_int64), OMP_RULES[rule], int(threads))
    if rc != 0:
        raise ValueError("oracle_spin_images_omp failed with code %d" % rc)
    return img, sup


def support_radius2(W, bin_size):
    """R^2 = h^2 + ((W - 1) B)^2, h = W B / 2 (double)."""
    return _load().oracle_support_radius2(int(W), float(bin_size))


def candidate_rc2(W, bin_size):
    """Rc2 = fl32(R^2 (1 + 1e-5))."""
    return _load().oracle_candidate_rc2(int(W), float(bin_size))
