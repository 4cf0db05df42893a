"""GB300-native Pohlig-Hellman exponentiation-cipher PRNG (arXiv:1411.2484).

Thin ctypes binding of libphprng.so: the functions below carry the names of
the C ABI (include/phprng.h) and only marshal arguments.  Every step of the
generator runs in the library's CUDA kernels; there is no Python or CPU
fallback, and every call raises RuntimeError when the compiled library is
absent.  Build it with ``paper_1411_2484_gb300.build.build()``; the
environment variable PHPRNG_LIB selects another build of the same library.

Pointer arguments accept a torch tensor, a numpy array, an int address or
None.  Stream arguments accept a torch.cuda.Stream, an int handle or None
(the legacy default stream).
"""
import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PHPRNG_LIB") or os.path.join(_HERE, "libphprng.so")

PHPRNG_OK = 0
PHPRNG_EINVAL = 1
PHPRNG_ENOTPRIME = 2
PHPRNG_EEXPONENT = 3
PHPRNG_ESKIP = 4
PHPRNG_EDUPLICATE = 5
PHPRNG_ENOMEM = 6
PHPRNG_ECUDA = 7
PHPRNG_ETIMEOUT = 8
PHPRNG_EBUDGET = 9
PHPRNG_REQUIRE_SAFE_PRIME = 0x1
PHPRNG_ALLOW_SHARED_N = 0x2

EXPORTED = [
    "phprng_create", "phprng_create_seeded", "phprng_destroy", "phprng_last_error",
    "phprng_status_string", "phprng_generate", "phprng_skip", "phprng_seek", "phprng_serial_test", "phprng_poker_test", "phprng_runs_test", "phprng_collision_test",
    "phprng_fourier_test", "phprng_interstream_serial_test", "phprng_pattern",
    "phprng_pattern_region", "phprng_pattern_const_region", "phprng_pattern_const",
    "phprng_get_state", "phprng_set_state",
    "phprng_is_prime", "phprng_validate", "phprng_draw_instances", "phprng_microbench",
    "phprng_plan_create", "phprng_plan_launch", "phprng_plan_launch_graph",
    "phprng_plan_autotune", "phprng_plan_tuning", "phprng_plan_destroy", "phprng_generate_batch",
    "phprng_clock_ns", "phprng_server_create", "phprng_server_submit", "phprng_server_poll",
    "phprng_server_release", "phprng_server_stats_get", "phprng_server_destroy",
    "phprng_server_copy", "phprng_generate_stats_noalloc",
]
PHPRNG_CONTINUE = (1 << 64) - 1


class phprng_instance(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("n", "e", "p", "a", "m0", "s0")]


class phprng_request(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("inst", "offset", "len", "c_off", "r_off")]


class phprng_tuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_uint32), ("npt", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("ms", ctypes.c_float)]


class phprng_server_config(ctypes.Structure):
    _fields_ = [("output_budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("inflight", ctypes.c_uint32), ("tile", ctypes.c_uint32),
                ("want_c", ctypes.c_uint32)]


class phprng_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("inst", ctypes.c_uint64),
                ("start", ctypes.c_uint64), ("len", ctypes.c_uint64),
                ("r", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("arrival_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


class phprng_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "submitted", "admitted", "completed", "batches", "tiles", "numbers", "max_waiting",
        "waiting", "outstanding_bytes")]


COMPLETION_DTYPE = np.dtype([("id", "<u8"), ("tag", "<u8"), ("inst", "<u8"), ("start", "<u8"),
                             ("len", "<u8"), ("r", "<u8"), ("c", "<u8"),
                             ("arrival_ns", "<i8"), ("done_ns", "<i8")])
REQUEST_DTYPE = np.dtype([(k, "<u8") for k in ("inst", "offset", "len", "c_off", "r_off")])


class phprng_stats(ctypes.Structure):
    _fields_ = [("x_lo", ctypes.c_uint64), ("x_hi", ctypes.c_uint64),
                ("y_lo", ctypes.c_uint64), ("y_hi", ctypes.c_uint64),
                ("z_lo", ctypes.c_uint64), ("z_hi", ctypes.c_uint64),
                ("count", ctypes.c_uint64),
                ("mean", ctypes.c_double), ("var", ctypes.c_double), ("corr", ctypes.c_double),
                ("hist", ctypes.c_uint32 * 256)]


STATS_DTYPE = np.dtype([("x_lo", "<u8"), ("x_hi", "<u8"), ("y_lo", "<u8"), ("y_hi", "<u8"),
                        ("z_lo", "<u8"), ("z_hi", "<u8"), ("count", "<u8"),
                        ("mean", "<f8"), ("var", "<f8"), ("corr", "<f8"),
                        ("hist", "<u4", (256,))])
assert STATS_DTYPE.itemsize == ctypes.sizeof(phprng_stats)


class PhprngError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (status %d)" % (message, status))
        self.status = status


_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libphprng.so is not built (%s); run "
                               "paper_1411_2484_gb300.build.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        vp, u64, i32, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
        P_inst = ctypes.POINTER(phprng_instance)
        P64 = ctypes.POINTER(ctypes.c_uint64)
        lib.phprng_create.argtypes = [ctypes.POINTER(vp), i32, P_inst, u64, u32, vp]
        lib.phprng_create_seeded.argtypes = [ctypes.POINTER(vp), i32, u64, u64, u32, vp]
        lib.phprng_destroy.argtypes = [vp]
        lib.phprng_last_error.argtypes = [vp]
        lib.phprng_last_error.restype = ctypes.c_char_p
        lib.phprng_status_string.argtypes = [i32]
        lib.phprng_status_string.restype = ctypes.c_char_p
        lib.phprng_generate.argtypes = [vp, u64, u64, u64, vp, vp, vp, vp]
        lib.phprng_generate_stats_noalloc.argtypes = [vp, u64, u64, u64, vp, vp]
        lib.phprng_skip.argtypes = [vp, P64, P64, u64, vp]
        lib.phprng_seek.argtypes = [vp, P64, P64, u64, vp]
        lib.phprng_serial_test.argtypes = [vp, u64, u64, u64, i32, ctypes.c_uint32, vp, vp]
        lib.phprng_poker_test.argtypes = [vp, u64, u64, u64, vp, vp]
        lib.phprng_runs_test.argtypes = [vp, u64, u64, u64, i32, vp, vp]
        u32 = ctypes.c_uint32
        lib.phprng_collision_test.argtypes = [vp, u64, u64, u64, u32, u32, u32, vp, vp]
        lib.phprng_interstream_serial_test.argtypes = [vp, u64, u64, u64, i32, u32, vp, vp]
        lib.phprng_fourier_test.argtypes = [vp, u64, u64, u64, u32, u32, ctypes.c_double, vp, vp, vp]
        lib.phprng_pattern.argtypes = [ctypes.POINTER(phprng_instance), u64, u64, i32,
                                       ctypes.c_uint32, vp, vp]
        lib.phprng_pattern_const.argtypes = [ctypes.POINTER(phprng_instance), u64, u64, u64, i32,
                                             ctypes.c_uint32, vp, vp]
        lib.phprng_pattern_region.argtypes = [ctypes.POINTER(phprng_instance), u64, u64, i32,
                                              ctypes.c_uint32, ctypes.c_uint32, vp, vp]
        lib.phprng_pattern_const_region.argtypes = [ctypes.POINTER(phprng_instance), u64, u64, u64, i32,
                                                    ctypes.c_uint32, ctypes.c_uint32, vp, vp]
        lib.phprng_get_state.argtypes = [vp, u64, P_inst, P64, P64, vp]
        lib.phprng_set_state.argtypes = [vp, u64, u64, u64, u64, u64, vp]
        lib.phprng_is_prime.argtypes = [u64]
        lib.phprng_validate.argtypes = [i32, P_inst, u64, u32, P64]
        lib.phprng_draw_instances.argtypes = [i32, u64, u64, u32, P_inst]
        lib.phprng_microbench.argtypes = [i32, ctypes.POINTER(ctypes.c_double), vp]
        P_req = ctypes.POINTER(phprng_request)
        lib.phprng_plan_create.argtypes = [vp, P_req, u64, u32, ctypes.POINTER(vp), vp]
        lib.phprng_plan_launch.argtypes = [vp, vp, vp, vp]
        lib.phprng_plan_launch_graph.argtypes = [vp, vp, vp, vp]
        lib.phprng_plan_autotune.argtypes = [vp, vp, vp, ctypes.POINTER(phprng_tuning), vp]
        lib.phprng_plan_tuning.argtypes = [vp, ctypes.POINTER(phprng_tuning)]
        lib.phprng_plan_destroy.argtypes = [vp]
        lib.phprng_generate_batch.argtypes = [vp, P_req, u64, vp, vp, vp]
        PI64 = ctypes.POINTER(ctypes.c_int64)
        lib.phprng_clock_ns.argtypes = []
        lib.phprng_clock_ns.restype = ctypes.c_int64
        lib.phprng_server_create.argtypes = [vp, ctypes.POINTER(phprng_server_config),
                                             ctypes.POINTER(vp)]
        lib.phprng_server_submit.argtypes = [vp, P64, P64, P64, PI64, u64, P64]
        lib.phprng_server_poll.argtypes = [vp, vp, u64, P64, ctypes.c_int64]
        lib.phprng_server_release.argtypes = [vp, P64, u64]
        lib.phprng_server_stats_get.argtypes = [vp, ctypes.POINTER(phprng_server_stats)]
        lib.phprng_server_destroy.argtypes = [vp]
        lib.phprng_server_copy.argtypes = [vp, u64, vp, vp]
        _lib = lib
        return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("unsupported pointer argument %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    raise TypeError("unsupported stream argument %r" % type(s))


def _check(rc, ctx=None):
    if rc != PHPRNG_OK:
        msg = _load().phprng_last_error(ctx)
        raise PhprngError(rc, msg.decode() if msg else "error")


def _instances(inst):
    """Accepts a dict of arrays {n, e, p, a, m0, s0}, an (count, 6) array or a
    sequence of 6-tuples; returns a ctypes array of phprng_instance."""
    if isinstance(inst, dict):
        rows = np.stack([np.asarray(inst[k], dtype=np.uint64)
                         for k in ("n", "e", "p", "a", "m0", "s0")], axis=1)
    else:
        rows = np.asarray(inst, dtype=np.uint64).reshape(-1, 6)
    rows = np.ascontiguousarray(rows, dtype=np.uint64)
    arr = (phprng_instance * rows.shape[0])()
    ctypes.memmove(arr, rows.ctypes.data, rows.nbytes)
    return arr, rows.shape[0]


def phprng_create(width, instances, flags=0, stream=None):
    """Returns an opaque context handle (int)."""
    lib = _load()
    arr, count = _instances(instances)
    out = ctypes.c_void_p()
    _check(lib.phprng_create(ctypes.byref(out), int(width), arr, count, int(flags),
                             _stream(stream)))
    return out.value


def phprng_create_seeded(width, count, seed, flags=0, stream=None):
    lib = _load()
    out = ctypes.c_void_p()
    _check(lib.phprng_create_seeded(ctypes.byref(out), int(width), int(count), int(seed),
                                    int(flags), _stream(stream)))
    return out.value


def phprng_destroy(ctx):
    if ctx:
        _load().phprng_destroy(ctx)


def phprng_last_error(ctx=None):
    return _load().phprng_last_error(ctx).decode()


def phprng_status_string(status):
    return _load().phprng_status_string(int(status)).decode()


def phprng_generate(ctx, first, num_inst, per_inst, c_out=None, r_out=None, stats_out=None,
                    stream=None):
    _check(_load().phprng_generate(ctx, int(first), int(num_inst), int(per_inst), _ptr(c_out),
                                   _ptr(r_out), _ptr(stats_out), _stream(stream)), ctx)


def phprng_generate_stats_noalloc(ctx, first, num_inst, per_inst, stats_out, stream=None):
    """Fused statistics without any GPU allocation (fixed 4 MiB scratch);
    for callers that cannot allocate device memory at the call site."""
    _check(_load().phprng_generate_stats_noalloc(ctx, int(first), int(num_inst), int(per_inst),
                                                 _ptr(stats_out), _stream(stream)), ctx)


def phprng_skip(ctx, inst_ids, k, stream=None):
    ids = np.ascontiguousarray(np.asarray(inst_ids, dtype=np.uint64).reshape(-1))
    ks = np.ascontiguousarray(np.asarray(k, dtype=np.uint64).reshape(-1))
    if ids.size != ks.size:
        raise ValueError("inst_ids and k differ in length")
    P64 = ctypes.POINTER(ctypes.c_uint64)
    _check(_load().phprng_skip(ctx, ids.ctypes.data_as(P64), ks.ctypes.data_as(P64), ids.size,
                               _stream(stream)), ctx)


def phprng_serial_test(ctx, first, num_inst, per_inst, D, B, hist, stream=None):
    """Adds the call's D-tuples of floor(B R) bins to the device histogram
    `hist` (B**D uint64 counters) and advances the streams by per_inst."""
    _check(_load().phprng_serial_test(ctx, int(first), int(num_inst), int(per_inst), int(D), int(B),
                                      _ptr(hist), _stream(stream)), ctx)


def phprng_poker_test(ctx, first, num_inst, per_inst, hist, stream=None):
    """Adds the call's five-card hands (categories 0..6) to the device
    counters `hist` (7 uint64) and advances the streams by per_inst."""
    _check(_load().phprng_poker_test(ctx, int(first), int(num_inst), int(per_inst), _ptr(hist),
                                     _stream(stream)), ctx)


def phprng_collision_test(ctx, first, num_inst, per_inst, S, B, H, hist, stream=None):
    """Adds the call's per-segment collision counts (segments of S numbers into
    B bins, counts capped at H-1) to the device counters `hist` (H uint64)."""
    _check(_load().phprng_collision_test(ctx, int(first), int(num_inst), int(per_inst), int(S), int(B),
                                         int(H), _ptr(hist), _stream(stream)), ctx)


def phprng_runs_test(ctx, first, num_inst, per_inst, lmax, hist, stream=None):
    """Adds the call's completed runs (bit-major, lengths capped at lmax) to
    the device counters `hist` (2*lmax uint64); streams advance by per_inst."""
    _check(_load().phprng_runs_test(ctx, int(first), int(num_inst), int(per_inst), int(lmax),
                                    _ptr(hist), _stream(stream)), ctx)


def phprng_interstream_serial_test(ctx, first, num_inst, per_inst, D, B, hist, stream=None):
    """Adds the D-tuples of the call's numbers in interleaved order (number 1
    of every instance, then number 2 of every instance, ...) to the device
    counters `hist` (B**D uint64); streams advance by per_inst."""
    _check(_load().phprng_interstream_serial_test(ctx, int(first), int(num_inst), int(per_inst), int(D),
                                                  int(B), _ptr(hist), _stream(stream)), ctx)


def phprng_fourier_test(ctx, first, num_inst, per_inst, log2M, nbins, w, hist, coef=None,
                        stream=None):
    """Adds the real and imaginary parts of the Fourier coefficients of every
    sequence of 2**log2M numbers to the device counters `hist` (nbins uint64,
    range [-w, w)); `coef` (device float64, optional) receives them as
    (re, im) pairs; streams advance by per_inst."""
    _check(_load().phprng_fourier_test(ctx, int(first), int(num_inst), int(per_inst), int(log2M),
                                       int(nbins), float(w), _ptr(hist),
                                       _ptr(coef) if coef is not None else None, _stream(stream)), ctx)


def phprng_pattern(n, e, p, a, c_lo, L0, D, nb, hist, stream=None):
    """Full-period D-dimensional pattern of the instance (n, e, p, a) for the
    tuples starting at c0 in [c_lo, c_lo+L0), added to the device counters
    `hist` (nb**(D-1) uint64)."""
    inst = phprng_instance(int(n), int(e), int(p), int(a), 0, 1)
    _check(_load().phprng_pattern(ctypes.byref(inst), int(c_lo), int(L0), int(D), int(nb), _ptr(hist),
                                  _stream(stream)), None)


def phprng_pattern_region(n, e, p, a, c_lo, L0, D, nb, L1, hist, stream=None):
    """phprng_pattern over the region [0, nb*L1)^(D-1) of the successors, cells
    of width L1 (tuples outside the region left out)."""
    inst = phprng_instance(int(n), int(e), int(p), int(a), 0, 1)
    _check(_load().phprng_pattern_region(ctypes.byref(inst), int(c_lo), int(L0), int(D), int(nb), int(L1),
                                         _ptr(hist), _stream(stream)), None)


def phprng_pattern_const_region(n, e, b, c_lo, L0, D, nb, L1, hist, stream=None):
    """phprng_pattern_const over the region [0, nb*L1)^(D-1), cells of width L1."""
    inst = phprng_instance(int(n), int(e), 2, 1, 0, 1)
    _check(_load().phprng_pattern_const_region(ctypes.byref(inst), int(b), int(c_lo), int(L0), int(D),
                                               int(nb), int(L1), _ptr(hist), _stream(stream)), None)


def phprng_pattern_const(n, e, b, c_lo, L0, D, nb, hist, stream=None):
    """Full-period D-dimensional pattern of the constant-skip generator
    (skip b; b = 1 is the unit skip) of (n, e) for the tuples starting at c0 in
    [c_lo, c_lo+L0), added to the device counters `hist` (nb**(D-1) uint64)."""
    inst = phprng_instance(int(n), int(e), 2, 1, 0, 1)
    _check(_load().phprng_pattern_const(ctypes.byref(inst), int(b), int(c_lo), int(L0), int(D), int(nb),
                                        _ptr(hist), _stream(stream)), None)


def phprng_seek(ctx, inst_ids, pos, stream=None):
    """Moves the listed streams to absolute positions, forward or backward."""
    ids = np.ascontiguousarray(np.asarray(inst_ids, dtype=np.uint64).reshape(-1))
    ps = np.ascontiguousarray(np.asarray(pos, dtype=np.uint64).reshape(-1))
    if ids.size != ps.size:
        raise ValueError("inst_ids and pos differ in length")
    P64 = ctypes.POINTER(ctypes.c_uint64)
    _check(_load().phprng_seek(ctx, ids.ctypes.data_as(P64), ps.ctypes.data_as(P64), ids.size,
                               _stream(stream)), ctx)


def phprng_set_state(ctx, inst, m, s, c=0, pos=0, stream=None):
    """Sets instance inst to message m, skip s, last ciphertext c at stream
    position pos (the stream is redefined through that state)."""
    _check(_load().phprng_set_state(ctx, int(inst), int(m), int(s), int(c), int(pos), _stream(stream)), ctx)


def phprng_get_state(ctx, inst, stream=None):
    """Returns dict(n, e, p, a, m, s, c, pos) of instance `inst`."""
    st = phprng_instance()
    pos = ctypes.c_uint64()
    c = ctypes.c_uint64()
    _check(_load().phprng_get_state(ctx, int(inst), ctypes.byref(st), ctypes.byref(pos),
                                    ctypes.byref(c), _stream(stream)), ctx)
    return dict(n=st.n, e=st.e, p=st.p, a=st.a, m=st.m0, s=st.s0, c=c.value, pos=pos.value)


def phprng_is_prime(n):
    return bool(_load().phprng_is_prime(int(n)))


def phprng_validate(width, instances, flags=0):
    """Returns (status, first bad index or None, message)."""
    lib = _load()
    arr, count = _instances(instances)
    bad = ctypes.c_uint64(0)
    rc = lib.phprng_validate(int(width), arr, count, int(flags), ctypes.byref(bad))
    if rc == PHPRNG_OK:
        return rc, None, ""
    return rc, bad.value, lib.phprng_last_error(None).decode()


def phprng_draw_instances(width, count, seed, flags=0):
    """Returns the drawn table as a dict of uint64 arrays {n, e, p, a, m0, s0}."""
    lib = _load()
    arr = (phprng_instance * int(count))()
    _check(lib.phprng_draw_instances(int(width), int(count), int(seed), int(flags), arr))
    rows = np.frombuffer(arr, dtype=np.uint64).reshape(-1, 6).copy()
    return {k: rows[:, j] for j, k in enumerate(("n", "e", "p", "a", "m0", "s0"))}


def _requests(reqs):
    """Accepts a REQUEST_DTYPE array, an (n, 5) integer array or a sequence of
    (inst, offset, len, c_off, r_off) tuples."""
    a = np.asarray(reqs)
    if a.dtype != REQUEST_DTYPE:
        a = np.asarray(reqs, dtype=np.uint64).reshape(-1, 5)
        a = np.ascontiguousarray(a).view(REQUEST_DTYPE).reshape(-1)
    a = np.ascontiguousarray(a)
    return a.ctypes.data_as(ctypes.POINTER(phprng_request)), a.size, a


def _tuning_dict(t):
    return dict(tile=t.tile, npt=t.npt, blocks_per_sm=t.blocks_per_sm, ms=t.ms)


def phprng_plan_create(ctx, reqs, tile=0, stream=None):
    ptr, n, _keep = _requests(reqs)
    out = ctypes.c_void_p()
    _check(_load().phprng_plan_create(ctx, ptr, n, int(tile), ctypes.byref(out),
                                      _stream(stream)), ctx)
    return out.value


def phprng_plan_launch(plan, c_base=None, r_base=None, stream=None, ctx=None):
    _check(_load().phprng_plan_launch(plan, _ptr(c_base), _ptr(r_base), _stream(stream)), ctx)


def phprng_plan_launch_graph(plan, c_base=None, r_base=None, stream=None, ctx=None):
    _check(_load().phprng_plan_launch_graph(plan, _ptr(c_base), _ptr(r_base), _stream(stream)),
           ctx)


def phprng_plan_autotune(plan, c_base=None, r_base=None, stream=None, ctx=None):
    t = phprng_tuning()
    _check(_load().phprng_plan_autotune(plan, _ptr(c_base), _ptr(r_base), ctypes.byref(t),
                                        _stream(stream)), ctx)
    return _tuning_dict(t)


def phprng_plan_tuning(plan):
    t = phprng_tuning()
    _check(_load().phprng_plan_tuning(plan, ctypes.byref(t)))
    return _tuning_dict(t)


def phprng_plan_destroy(plan):
    if plan:
        _load().phprng_plan_destroy(plan)


def phprng_generate_batch(ctx, reqs, c_base=None, r_base=None, stream=None):
    ptr, n, _keep = _requests(reqs)
    _check(_load().phprng_generate_batch(ctx, ptr, n, _ptr(c_base), _ptr(r_base),
                                         _stream(stream)), ctx)


def phprng_clock_ns():
    return int(_load().phprng_clock_ns())


def phprng_server_create(ctx, output_budget_bytes, max_batch=0, inflight=0, tile=0, want_c=0):
    cfg = phprng_server_config(int(output_budget_bytes), int(max_batch), int(inflight), int(tile),
                               int(want_c))
    out = ctypes.c_void_p()
    _check(_load().phprng_server_create(ctx, ctypes.byref(cfg), ctypes.byref(out)), ctx)
    return out.value


def _u64arr(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64).reshape(-1))


def phprng_server_submit(srv, inst, length, tag=None, arrival_ns=None):
    """Submits requests (arrays or scalars); returns the id of the first."""
    P64 = ctypes.POINTER(ctypes.c_uint64)
    inst, length = _u64arr(inst), _u64arr(length)
    tag = _u64arr(tag) if tag is not None else None
    arr = (np.ascontiguousarray(np.asarray(arrival_ns, dtype=np.int64).reshape(-1))
           if arrival_ns is not None else None)
    first = ctypes.c_uint64()
    _check(_load().phprng_server_submit(
        srv, inst.ctypes.data_as(P64), length.ctypes.data_as(P64),
        tag.ctypes.data_as(P64) if tag is not None else None,
        arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if arr is not None else None,
        inst.size, ctypes.byref(first)))
    return first.value


def phprng_server_poll(srv, max_items=4096, timeout_ns=0):
    """Returns a COMPLETION_DTYPE array of finished requests."""
    out = np.zeros(int(max_items), dtype=COMPLETION_DTYPE)
    n = ctypes.c_uint64()
    _check(_load().phprng_server_poll(srv, out.ctypes.data, int(max_items), ctypes.byref(n),
                                      int(timeout_ns)))
    return out[:n.value]


def phprng_server_release(srv, ids):
    ids = _u64arr(ids)
    _check(_load().phprng_server_release(srv, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                         ids.size))


def phprng_server_copy(srv, req_id, r_dst=None, c_dst=None):
    _check(_load().phprng_server_copy(srv, int(req_id), _ptr(r_dst), _ptr(c_dst)))


def phprng_server_stats_get(srv):
    st = phprng_server_stats()
    _check(_load().phprng_server_stats_get(srv, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in phprng_server_stats._fields_}


def phprng_server_destroy(srv):
    if srv:
        _check(_load().phprng_server_destroy(srv))


def phprng_microbench(which, stream=None):
    """Operations per second of instruction form `which` on the current device."""
    out = ctypes.c_double()
    _check(_load().phprng_microbench(int(which), ctypes.byref(out), _stream(stream)))
    return out.value


class Generator:
    """Owns one context; thin convenience over the functions above."""

    def __init__(self, width, instances=None, count=None, seed=None, flags=0, stream=None):
        if instances is not None:
            self.ctx = phprng_create(width, instances, flags, stream)
        else:
            self.ctx = phprng_create_seeded(width, count, seed, flags, stream)
        self.width = width

    def generate(self, first, num_inst, per_inst, c_out=None, r_out=None, stats_out=None,
                 stream=None):
        phprng_generate(self.ctx, first, num_inst, per_inst, c_out, r_out, stats_out, stream)

    def skip(self, inst_ids, k, stream=None):
        phprng_skip(self.ctx, inst_ids, k, stream)

    def seek(self, inst_ids, pos, stream=None):
        phprng_seek(self.ctx, inst_ids, pos, stream)

    def state(self, inst, stream=None):
        return phprng_get_state(self.ctx, inst, stream)

    def close(self):
        if self.ctx:
            phprng_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
