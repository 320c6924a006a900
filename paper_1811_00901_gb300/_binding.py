"""ctypes binding of libspin_gb300.so -- argument marshalling only.

Every entry point keeps the C name (``si_*``).  Tensors are passed as raw
pointers (``tensor.data_ptr()``), streams as the raw ``cudaStream_t`` of a
``torch.cuda.Stream`` (``stream.cuda_stream``); PyTorch supplies device memory
and streams, the library does the work.  A missing library is an error: there
is no fallback path.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libspin_gb300.so")

SI_OK, SI_ERR_INVALID, SI_ERR_CUDA, SI_ERR_OOM, SI_ERR_OVERFLOW, SI_ERR_TIMEOUT, SI_ERR_BUSY = range(7)
STATUS_NAMES = {0: "SI_OK", 1: "SI_ERR_INVALID", 2: "SI_ERR_CUDA", 3: "SI_ERR_OOM", 4: "SI_ERR_OVERFLOW",
                5: "SI_ERR_TIMEOUT", 6: "SI_ERR_BUSY"}
SI_SCHED_STATIC, SI_SCHED_SS, SI_SCHED_GSS, SI_SCHED_FAC, SI_SCHED_FAC_PROB, SI_SCHED_AWF, SI_SCHED_AF = range(7)
SCHED_NAMES = {"STATIC": SI_SCHED_STATIC, "SS": SI_SCHED_SS, "GSS": SI_SCHED_GSS, "FAC": SI_SCHED_FAC,
               "FAC_PROB": SI_SCHED_FAC_PROB, "AWF": SI_SCHED_AWF, "AF": SI_SCHED_AF}
SI_BIN_BILINEAR, SI_BIN_NEAREST = 0, 1
BIN_NAMES = {"BILINEAR": SI_BIN_BILINEAR, "NEAREST": SI_BIN_NEAREST}


class SpinError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class si_schedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("min_chunk", ctypes.c_int32), ("num_workers", ctypes.c_int32),
                ("group", ctypes.c_int32), ("grid_div", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("binning", ctypes.c_int32), ("slow_workers", ctypes.c_int32), ("slowdown", ctypes.c_float),
                ("fac_cov", ctypes.c_float), ("order", ctypes.c_int32)]


class si_probe(ctypes.Structure):
    _fields_ = [("culled", ctypes.c_void_p), ("cand_hash", ctypes.c_void_p), ("support", ctypes.c_void_p),
                ("worker", ctypes.c_void_p), ("step", ctypes.c_void_p), ("examined", ctypes.c_void_p),
                ("angle", ctypes.c_void_p)]


class si_stats(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("images", ctypes.c_int64), ("overflow", ctypes.c_int32),
                ("timeout", ctypes.c_int32), ("bad_query", ctypes.c_int32), ("bad_input", ctypes.c_int32),
                ("grid_cells", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("kernel_ms", ctypes.c_double)]


class si_trace(ctypes.Structure):
    _fields_ = [("claims", ctypes.c_void_p), ("capacity", ctypes.c_int64), ("count", ctypes.c_void_p)]


class si_batch_item(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_void_p), ("query_idx", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("W", ctypes.c_int32), ("bin_size", ctypes.c_float), ("cos_support_angle", ctypes.c_float),
                ("out", ctypes.c_void_p)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "si_mesh_create": ([_P, _P, ctypes.c_int64, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "si_mesh_destroy": ([_P], ctypes.c_int),
    "si_mesh_prepare": ([_P, ctypes.c_int32, ctypes.c_float, ctypes.POINTER(si_schedule), _P], ctypes.c_int),
    "si_default_workers": ([ctypes.c_int32, ctypes.POINTER(si_schedule), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "si_generate": ([_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, si_schedule, _P, _P],
                    ctypes.c_int),
    "si_generate_probe": ([_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, si_schedule,
                           _P, ctypes.POINTER(si_probe), _P], ctypes.c_int),
    "si_generate_traced": ([_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, si_schedule,
                            _P, ctypes.POINTER(si_trace), _P], ctypes.c_int),
    "si_generate_batched": ([ctypes.POINTER(si_batch_item), ctypes.c_int32, ctypes.POINTER(si_schedule), _P],
                            ctypes.c_int),
    "si_generate_host": ([_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float,
                          ctypes.c_float, si_schedule, _P, _P], ctypes.c_int),
    "si_generate_noalloc": ([_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, si_schedule,
                             _P, _P], ctypes.c_int),
    "si_chunk_table":([ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                        ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)],
                       ctypes.c_int),
    "si_schedule_chunks": ([ctypes.POINTER(si_schedule), ctypes.c_int64, ctypes.c_int32,
                            ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)],
                           ctypes.c_int),
    "si_candidate_rc2": ([ctypes.c_int32, ctypes.c_float], ctypes.c_float),
    "si_match": ([_P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P],
                 ctypes.c_int),
    "si_check_bounded_wait": ([ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                               _P], ctypes.c_int),
    "si_candidate_rc2_binned": ([ctypes.c_int32, ctypes.c_float, ctypes.c_int32], ctypes.c_float),
    "si_get_stats": ([_P, ctypes.POINTER(si_stats)], ctypes.c_int),
    "si_reset_stats": ([_P], ctypes.c_int),
    "si_set_timing": ([ctypes.c_int32], None),
    "si_tune_mesh": ([_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _P, ctypes.c_int32,
                      ctypes.POINTER(si_schedule), ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "si_tune_lookup": ([ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(si_schedule)], ctypes.c_int),
    "si_tune_save": ([ctypes.c_char_p], ctypes.c_int),
    "si_tune_load": ([ctypes.c_char_p], ctypes.c_int),
    "si_tune_clear": ([], ctypes.c_int),
    "si_serve_create": ([ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(_P)], ctypes.c_int),
    "si_serve_add_mesh": ([_P, _P, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "si_serve_submit": ([_P, ctypes.POINTER(si_batch_item), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "si_serve_poll": ([_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "si_serve_wait": ([_P, ctypes.c_uint64, ctypes.c_int32], ctypes.c_int),
    "si_serve_result": ([_P, ctypes.c_uint64, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "si_serve_release": ([_P, ctypes.c_uint64], ctypes.c_int),
    "si_serve_destroy": ([_P], ctypes.c_int),
    "si_last_error": ([], ctypes.c_char_p),
    "si_version": ([], ctypes.c_char_p),
    "si_kernel_launches": ([], ctypes.c_int64),
    "si_peak_smem_atomics": ([ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "si_alloc_stats": ([ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "si_debug_fail_allocs": ([ctypes.c_int64, ctypes.c_int64], ctypes.c_int),
}

_lib = None


def load(path=None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libspin_gb300.so not found at %s; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % p)
    lib = ctypes.CDLL(p)
    for name, (args, res) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = lib
    return lib


def exported_names():
    return sorted(_SIGNATURES)


def _check(status):
    if status != SI_OK:
        raise SpinError(status, load().si_last_error().decode(errors="replace"))
    return status


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def make_schedule(kind="GSS", min_chunk=1, num_workers=0, group=0, grid_div=0, slices=0, binning=0,
                  slow_workers=0, slowdown=0.0, fac_cov=0.0, order=0):
    if isinstance(kind, str):
        kind = SCHED_NAMES[kind.upper()]
    if isinstance(binning, str):
        binning = BIN_NAMES[binning.upper()]
    return si_schedule(int(kind), int(min_chunk), int(num_workers), int(group), int(grid_div), int(slices),
                       int(binning), int(slow_workers), float(slowdown), float(fac_cov), int(order))


# ----------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ----------------------------------------------------------------------------

def si_mesh_create(points, normals, n=None, stream=None):
    """points, normals: (n, 3) float32 tensors (CUDA or CPU) or raw pointers."""
    if n is None:
        n = points.shape[0]
    h = ctypes.c_void_p()
    _check(load().si_mesh_create(_ptr(points), _ptr(normals), int(n), _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def si_mesh_destroy(mesh):
    _check(load().si_mesh_destroy(mesh))


def si_mesh_prepare(mesh, W, bin_size, schedule=None, stream=None):
    sp = ctypes.byref(schedule) if schedule is not None else None
    _check(load().si_mesh_prepare(mesh, int(W), float(bin_size), sp, _stream_ptr(stream)))


def si_default_workers(W, schedule=None):
    """Resident workers (SMs x spin-kernel blocks per SM) of a call of width
    W with the schedule's group and binning on the current device."""
    sp = ctypes.byref(schedule) if schedule is not None else None
    v = ctypes.c_int32(0)
    _check(load().si_default_workers(int(W), sp, ctypes.byref(v)))
    return int(v.value)


def si_generate(mesh, query_idx, m, W, bin_size, cos_s, schedule, out, stream=None):
    _check(load().si_generate(mesh, _ptr(query_idx), int(m), int(W), float(bin_size), float(cos_s), schedule,
                              _ptr(out), _stream_ptr(stream)))


def si_generate_probe(mesh, query_idx, m, W, bin_size, cos_s, schedule, out, culled=None, cand_hash=None,
                      support=None, worker=None, step=None, examined=None, angle=None, stream=None):
    pr = si_probe(_ptr(culled), _ptr(cand_hash), _ptr(support), _ptr(worker), _ptr(step), _ptr(examined),
                  _ptr(angle))
    _check(load().si_generate_probe(mesh, _ptr(query_idx), int(m), int(W), float(bin_size), float(cos_s), schedule,
                                    _ptr(out), ctypes.byref(pr), _stream_ptr(stream)))


def si_generate_traced(mesh, query_idx, m, W, bin_size, cos_s, schedule, out, claims, count, stream=None):
    """si_generate with the per-claim trace: claims is a device int64 [capacity, 4] tensor
    (worker, step, start ns, end ns), count a zeroed device uint64/int64 [1] tensor."""
    tr = si_trace(_ptr(claims), int(claims.shape[0]), _ptr(count))
    _check(load().si_generate_traced(mesh, _ptr(query_idx), int(m), int(W), float(bin_size), float(cos_s), schedule,
                                     _ptr(out), ctypes.byref(tr), _stream_ptr(stream)))


def batch_items(items):
    """items: sequence of dicts with mesh, query_idx, m, W, bin_size, cos_s, out."""
    arr = (si_batch_item * len(items))()
    for k, it in enumerate(items):
        arr[k] = si_batch_item(it["mesh"], _ptr(it.get("query_idx")), int(it["m"]), int(it["W"]),
                               float(it["bin_size"]), float(it["cos_s"]), _ptr(it.get("out")))
    return arr


def si_generate_batched(items, schedule=None, stream=None):
    arr = batch_items(items)
    sp = ctypes.byref(schedule) if schedule is not None else None
    _check(load().si_generate_batched(arr, len(items), sp, _stream_ptr(stream)))


def si_generate_host(points, normals, n, query_idx, m, W, bin_size, cos_s, schedule, out, stream=None):
    """All buffers are host pointers / CPU tensors (page-locked output is
    written by the kernel directly)."""
    _check(load().si_generate_host(_ptr(points), _ptr(normals), int(n), _ptr(query_idx), int(m), int(W),
                                   float(bin_size), float(cos_s), schedule, _ptr(out), _stream_ptr(stream)))


def si_generate_noalloc(mesh, query_idx, m, W, bin_size, cos_s, schedule, out, stream=None):
    """si_generate without any device allocation (static scratch; grid prepared beforehand)."""
    _check(load().si_generate_noalloc(mesh, _ptr(query_idx), int(m), int(W), float(bin_size), float(cos_s),
                                      schedule, _ptr(out), _stream_ptr(stream)))


def si_chunk_table(kind, units, workers, min_chunk=1):
    if isinstance(kind, str):
        kind = SCHED_NAMES[kind.upper()]
    nsteps = ctypes.c_int64()
    load().si_chunk_table(int(kind), int(units), int(workers), int(min_chunk), None, 0, ctypes.byref(nsteps))
    cap = nsteps.value + 1
    buf = (ctypes.c_int64 * cap)()
    _check(load().si_chunk_table(int(kind), int(units), int(workers), int(min_chunk), buf, cap,
                                 ctypes.byref(nsteps)))
    return list(buf)


def si_schedule_chunks(schedule, units, workers):
    nsteps = ctypes.c_int64()
    load().si_schedule_chunks(ctypes.byref(schedule), int(units), int(workers), None, 0, ctypes.byref(nsteps))
    cap = nsteps.value + 1
    buf = (ctypes.c_int64 * cap)()
    _check(load().si_schedule_chunks(ctypes.byref(schedule), int(units), int(workers), buf, cap,
                                     ctypes.byref(nsteps)))
    return list(buf)


SI_MATCH_FP32, SI_MATCH_BF16 = 0, 1


def si_match(scene, n_scene, model, n_model, W, k, precision, best_idx, best_corr, stream=None):
    """Each scene image's k best model images by correlation (device buffers)."""
    if isinstance(precision, str):
        precision = {"FP32": SI_MATCH_FP32, "BF16": SI_MATCH_BF16}[precision.upper()]
    _check(load().si_match(_ptr(scene), int(n_scene), _ptr(model), int(n_model), int(W), int(k), int(precision),
                           _ptr(best_idx), _ptr(best_corr), _stream_ptr(stream)))


def si_check_bounded_wait(limit_ms=50, stream=None):
    """Returns (timed_out, waited_ms) of the bounded-wait self-check."""
    t = ctypes.c_int32()
    w = ctypes.c_double()
    _check(load().si_check_bounded_wait(int(limit_ms), ctypes.byref(t), ctypes.byref(w), _stream_ptr(stream)))
    return bool(t.value), w.value


def si_candidate_rc2(W, bin_size):
    return load().si_candidate_rc2(int(W), float(bin_size))


def si_candidate_rc2_binned(W, bin_size, binning):
    if isinstance(binning, str):
        binning = BIN_NAMES[binning.upper()]
    return load().si_candidate_rc2_binned(int(W), float(bin_size), int(binning))


def si_get_stats(mesh, raise_on_flags=True):
    st = si_stats()
    status = load().si_get_stats(mesh, ctypes.byref(st))
    if status not in (SI_OK, SI_ERR_OVERFLOW, SI_ERR_TIMEOUT, SI_ERR_INVALID) or \
            (raise_on_flags and status != SI_OK):
        _check(status)
    return {f: getattr(st, f) for f, _ in si_stats._fields_}, status


def si_reset_stats(mesh):
    _check(load().si_reset_stats(mesh))


def si_set_timing(enabled):
    load().si_set_timing(1 if enabled else 0)


def si_tune_mesh(mesh, query_idx, m, W, bin_size, cos_s, scratch_out, reps=3, stream=None):
    best = si_schedule()
    ms = ctypes.c_double()
    _check(load().si_tune_mesh(mesh, _ptr(query_idx), int(m), int(W), float(bin_size), float(cos_s),
                               _ptr(scratch_out), int(reps), ctypes.byref(best), ctypes.byref(ms),
                               _stream_ptr(stream)))
    return best, ms.value


def si_tune_lookup(W, n, m):
    s = si_schedule()
    status = load().si_tune_lookup(int(W), int(n), int(m), ctypes.byref(s))
    return s if status == SI_OK else None


def si_tune_save(path):
    _check(load().si_tune_save(path.encode()))


def si_tune_load(path):
    _check(load().si_tune_load(path.encode()))


def si_tune_clear():
    _check(load().si_tune_clear())


def si_serve_create(mem_budget_bytes, max_inflight):
    h = ctypes.c_void_p()
    _check(load().si_serve_create(int(mem_budget_bytes), int(max_inflight), ctypes.byref(h)))
    return h.value


def si_serve_add_mesh(server, mesh):
    slot = ctypes.c_int32()
    _check(load().si_serve_add_mesh(server, mesh, ctypes.byref(slot)))
    return slot.value


def si_serve_submit(server, item):
    arr = batch_items([item])
    t = ctypes.c_uint64()
    status = load().si_serve_submit(server, arr, ctypes.byref(t))
    if status == SI_ERR_BUSY:
        return None
    _check(status)
    return t.value


def si_serve_poll(server, ticket):
    d = ctypes.c_int32()
    _check(load().si_serve_poll(server, int(ticket), ctypes.byref(d)))
    return bool(d.value)


def si_serve_wait(server, ticket, timeout_ms=-1):
    status = load().si_serve_wait(server, int(ticket), int(timeout_ms))
    if status == SI_ERR_TIMEOUT:
        return False
    _check(status)
    return True


def si_serve_result(server, ticket):
    p = ctypes.c_void_p()
    lat = ctypes.c_double()
    _check(load().si_serve_result(server, int(ticket), ctypes.byref(p), ctypes.byref(lat)))
    return p.value, lat.value


def si_serve_release(server, ticket):
    _check(load().si_serve_release(server, int(ticket)))


def si_serve_destroy(server):
    _check(load().si_serve_destroy(server))


def si_last_error():
    return load().si_last_error().decode(errors="replace")


def si_version():
    return load().si_version().decode()


def si_kernel_launches():
    return int(load().si_kernel_launches())


def si_alloc_stats():
    """(allocation calls so far, pool bytes in use, pool bytes reserved) of the current device."""
    c, u, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().si_alloc_stats(ctypes.byref(c), ctypes.byref(u), ctypes.byref(r)))
    return c.value, u.value, r.value


def si_debug_fail_allocs(skip, count):
    _check(load().si_debug_fail_allocs(int(skip), int(count)))


def si_peak_smem_atomics(mode=0, stream=None):
    v = ctypes.c_double()
    _check(load().si_peak_smem_atomics(int(mode), ctypes.byref(v), _stream_ptr(stream)))
    return v.value


class device_view:
    """A zero-copy view of library-owned device memory (e.g. a server-allocated
    output) through __cuda_array_interface__: ``torch.as_tensor(device_view(p,
    shape), device="cuda")``.  The memory stays owned by the library."""

    def __init__(self, ptr, shape, typestr="<i4"):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}
