"""Thin ctypes binding of the C ABI in include/rfi.h (argument marshalling only).

Every function has the name of the C entry point it calls and raises RfiError when
that entry point returns a status other than RFI_OK.  Buffers may be passed as
torch tensors (their data pointer is used), as integer addresses, or as None where
the C function accepts NULL.  No computation happens here: the flagging runs in the
sm_103a kernels of librfi.so, and importing this module fails loudly when that
library has not been built.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# RFI_LIBRARY selects another build of the library (the debug-bounds build, say)
LIB_PATH = os.environ.get("RFI_LIBRARY") or os.path.join(HERE, "_lib", "librfi.so")

RFI_C64 = 0
RFI_C32H = 1
DTYPES = {"c64": RFI_C64, "f32": RFI_C64, "c32h": RFI_C32H, "f16": RFI_C32H}
STATUS = {0: "RFI_OK", 1: "RFI_EINVAL", 2: "RFI_ENOMEM", 3: "RFI_ECUDA", 4: "RFI_ETIMEOUT",
          5: "RFI_ESTATE", 6: "RFI_EUNSUPPORTED"}

EXPORTED = ["rfi_create", "rfi_create_ex", "rfi_rows", "rfi_outputs_for", "rfi_get_options",
            "rfi_set_thresholds", "rfi_process_block", "rfi_process_block_host",
            "rfi_process_batch", "rfi_batch_graph_create", "rfi_batch_graph_launch",
            "rfi_batch_graph_destroy", "rfi_reset", "rfi_destroy", "rfi_status_str",
            "rfi_last_error", "rfi_process_block_noalloc", "rfi_check", "rfi_state_size",
            "rfi_get_state", "rfi_set_state", "rfi_windows_for", "rfi_set_adaptation",
            "rfi_adaptive_state", "rfi_last_launch"]

# Fixed size of the library's no-allocation scratch (RFI_NOALLOC_SCRATCH_BYTES).
RFI_NOALLOC_SCRATCH_BYTES = 4 << 20


class RfiError(RuntimeError):
    def __init__(self, status, func, detail):
        self.status = status
        super().__init__(f"{func}: {STATUS.get(status, status)}: {detail}")


class rfi_thresholds(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double), ("s_low", ctypes.c_double), ("s_high", ctypes.c_double),
                ("gamma", ctypes.c_double), ("eps", ctypes.c_double)]


class rfi_adaptation(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("k_sigma", ctypes.c_double),
                ("n_warm", ctypes.c_int)]


class rfi_options(ctypes.Structure):
    _fields_ = [("lanes_per_row", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("host_max_T", ctypes.c_int), ("host_chunks", ctypes.c_int),
                ("compensated", ctypes.c_int), ("prefetch_bytes", ctypes.c_int),
                ("prefetch_groups", ctypes.c_int), ("max_registers", ctypes.c_int),
                ("window_F", ctypes.c_int), ("precision", ctypes.c_int),
                ("loader", ctypes.c_int), ("tma_stage_windows", ctypes.c_int),
                ("tma_stages", ctypes.c_int), ("debug_inject_wait_timeout", ctypes.c_int),
                ("buffered_stores", ctypes.c_int), ("partial_windows", ctypes.c_int),
                ("adaptive", ctypes.c_int), ("overlap_bytes", ctypes.c_int),
                ("window_hop", ctypes.c_int), ("lane_split", ctypes.c_int),
                ("independent_launches", ctypes.c_int)]


_lib = None


def load_library(path=None):
    """Load librfi.so (default: the in-tree build) and declare its signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with `python -m paper_2412_14775_b300.build` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(p)
    vp, ip = ctypes.c_void_p, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "rfi_create": ([ctypes.POINTER(vp), ip, ip, ip, ip, ctypes.POINTER(rfi_thresholds), ip], ip),
        "rfi_create_ex": ([ctypes.POINTER(vp), ip, ip, ip, ip, ctypes.POINTER(rfi_thresholds), ip,
                           ctypes.POINTER(rfi_options)], ip),
        "rfi_rows": ([vp, ctypes.POINTER(ctypes.c_longlong)], ip),
        "rfi_outputs_for": ([vp, ip, ctypes.POINTER(ip)], ip),
        "rfi_windows_for": ([vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ctypes.c_longlong)], ip),
        "rfi_get_options": ([vp, ctypes.POINTER(rfi_options)], ip),
        "rfi_last_launch": ([vp, ctypes.POINTER(ip)], ip),
        "rfi_set_thresholds": ([vp, ctypes.POINTER(rfi_thresholds)], ip),
        "rfi_set_adaptation": ([vp, ctypes.POINTER(rfi_adaptation)], ip),
        "rfi_adaptive_state": ([vp, vp, ctypes.c_size_t, ip, vp], ip),
        "rfi_process_block": ([vp, vp, ip, vp, vp, vp, vp, vp], ip),
        "rfi_process_block_host": ([vp, vp, ip, vp, vp, vp, vp, vp], ip),
        "rfi_process_batch": ([pp, ip, pp, ctypes.POINTER(ip), pp, pp, pp, pp, vp], ip),
        "rfi_batch_graph_create": ([ctypes.POINTER(vp), pp, ip, ctypes.POINTER(ip)], ip),
        "rfi_batch_graph_launch": ([vp, pp, pp, pp, pp, pp, vp], ip),
        "rfi_batch_graph_destroy": ([vp], ip),
        "rfi_reset": ([vp], ip),
        "rfi_check": ([vp, vp], ip),
        "rfi_state_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], ip),
        "rfi_get_state": ([vp, vp, ctypes.c_size_t, vp], ip),
        "rfi_set_state": ([vp, vp, ctypes.c_size_t], ip),
        "rfi_destroy": ([vp], ip),
        "rfi_process_block_noalloc": ([ip, ip, ip, ip, ctypes.POINTER(rfi_thresholds), ip,
                                       ctypes.c_longlong, vp, ip, vp, vp, vp, vp, vp], ip),
        "rfi_status_str": ([ip], ctypes.c_char_p),
        "rfi_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = lib
    return lib


def _check(status, func):
    if status != 0:
        detail = load_library().rfi_last_error().decode(errors="replace")
        raise RfiError(status, func, detail)


def _ptr(x):
    """Address of a tensor's data, an int, or None -> c_void_p."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):              # numpy array (host buffers)
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _thr(t):
    if isinstance(t, rfi_thresholds):
        return t
    if isinstance(t, dict):
        return rfi_thresholds(t["d"], t["s_low"], t["s_high"], t["gamma"], t["eps"])
    return rfi_thresholds(*t)


def _dtype(dt):
    return DTYPES[dt] if isinstance(dt, str) else int(dt)


def _ptr_array(xs):
    arr = (ctypes.c_void_p * len(xs))(*[_ptr(x) for x in xs])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


# ---- entry points (same names as the C ABI) ------------------------------------
def rfi_create(stations, channels, window_M, avg_K, thresholds, dtype):
    h = ctypes.c_void_p()
    t = _thr(thresholds)
    _check(load_library().rfi_create(ctypes.byref(h), stations, channels, window_M, avg_K,
                                     ctypes.byref(t), _dtype(dtype)), "rfi_create")
    return h.value


def rfi_create_ex(stations, channels, window_M, avg_K, thresholds, dtype, options=None, **kw):
    h = ctypes.c_void_p()
    t = _thr(thresholds)
    if isinstance(options, rfi_options):
        o = options
    else:
        unknown = set(kw) - {f for f, _ in rfi_options._fields_}
        if unknown:
            raise TypeError(f"unknown options {sorted(unknown)}")
        o = rfi_options(*[int(kw.get(f, 0)) for f, _ in rfi_options._fields_])
    _check(load_library().rfi_create_ex(ctypes.byref(h), stations, channels, window_M, avg_K,
                                        ctypes.byref(t), _dtype(dtype), ctypes.byref(o)),
           "rfi_create_ex")
    return h.value


def rfi_rows(ctx):
    r = ctypes.c_longlong()
    _check(load_library().rfi_rows(ctx, ctypes.byref(r)), "rfi_rows")
    return r.value


def rfi_outputs_for(ctx, T):
    n = ctypes.c_int()
    _check(load_library().rfi_outputs_for(ctx, T, ctypes.byref(n)), "rfi_outputs_for")
    return n.value


def rfi_windows_for(ctx, T):
    """(n_win, first_sample): windows the next block of T samples completes and the
    stream index of the first sample they cover."""
    n = ctypes.c_int()
    first = ctypes.c_longlong()
    _check(load_library().rfi_windows_for(ctx, T, ctypes.byref(n), ctypes.byref(first)),
           "rfi_windows_for")
    return n.value, first.value


def rfi_get_options(ctx):
    o = rfi_options()
    _check(load_library().rfi_get_options(ctx, ctypes.byref(o)), "rfi_get_options")
    return {f: getattr(o, f) for f, _ in rfi_options._fields_}


# How rfi_last_launch reports the order of a context's last flagging launch.
LAUNCH_ORDER = {-1: "none", 0: "plain", 1: "waiting", 2: "independent"}


def rfi_last_launch(ctx):
    """Order of the context's last flagging launch on its stream: 'plain', 'waiting',
    'independent' or 'none' (see rfi_last_launch in rfi.h)."""
    o = ctypes.c_int()
    _check(load_library().rfi_last_launch(ctx, ctypes.byref(o)), "rfi_last_launch")
    return LAUNCH_ORDER[o.value]


def rfi_set_thresholds(ctx, thresholds):
    t = _thr(thresholds)
    _check(load_library().rfi_set_thresholds(ctx, ctypes.byref(t)), "rfi_set_thresholds")


def rfi_set_adaptation(ctx, alpha=1.0 / 64, k_sigma=3.0, n_warm=32):
    p = rfi_adaptation(float(alpha), float(k_sigma), int(n_warm))
    _check(load_library().rfi_set_adaptation(ctx, ctypes.byref(p)), "rfi_set_adaptation")


def rfi_adaptive_state(ctx, state=None, stream=None):
    """Read (state None) or write the per-row online-threshold state, float32 [R/F, 4]
    = (n, mean of tau, mean of tau^2, unused); returns it as a numpy array."""
    import numpy as np
    if state is None:
        R = rfi_rows(ctx)
        F = rfi_get_options(ctx)["window_F"]
        buf = np.zeros((R // F, 4), np.float32)
        write = 0
    else:
        buf = np.ascontiguousarray(state, dtype=np.float32)
        write = 1
    _check(load_library().rfi_adaptive_state(ctx, buf.ctypes.data, buf.size, write,
                                             _stream(stream)), "rfi_adaptive_state")
    return buf


def rfi_process_block(ctx, vis, T, flags, avg, weight, stats, stream=None):
    _check(load_library().rfi_process_block(ctx, _ptr(vis), T, _ptr(flags), _ptr(avg),
                                            _ptr(weight), _ptr(stats), _stream(stream)),
           "rfi_process_block")


def rfi_process_block_host(ctx, vis, T, flags, avg, weight, stats, stream=None):
    _check(load_library().rfi_process_block_host(ctx, _ptr(vis), T, _ptr(flags), _ptr(avg),
                                                 _ptr(weight), _ptr(stats), _stream(stream)),
           "rfi_process_block_host")


def rfi_process_batch(ctxs, vis, T, flags, avg, weight, stats, stream=None):
    n = len(ctxs)
    keep = []
    cp, a = _ptr_array(ctxs); keep.append(a)
    vp_, a = _ptr_array(vis); keep.append(a)
    fp, a = _ptr_array(flags); keep.append(a)
    ap, a = _ptr_array(avg); keep.append(a)
    wp, a = _ptr_array(weight); keep.append(a)
    sp, a = _ptr_array(stats); keep.append(a)
    Ts = (ctypes.c_int * n)(*T)
    _check(load_library().rfi_process_batch(cp, n, vp_, Ts, fp, ap, wp, sp, _stream(stream)),
           "rfi_process_batch")


def rfi_batch_graph_create(ctxs, T):
    n = len(ctxs)
    h = ctypes.c_void_p()
    cp, keep = _ptr_array(ctxs)
    Ts = (ctypes.c_int * n)(*T)
    _check(load_library().rfi_batch_graph_create(ctypes.byref(h), cp, n, Ts),
           "rfi_batch_graph_create")
    return h.value


def rfi_batch_graph_launch(g, vis, flags, avg, weight, stats, stream=None):
    keep = []
    vp_, a = _ptr_array(vis); keep.append(a)
    fp, a = _ptr_array(flags); keep.append(a)
    ap, a = _ptr_array(avg); keep.append(a)
    wp, a = _ptr_array(weight); keep.append(a)
    sp, a = _ptr_array(stats); keep.append(a)
    _check(load_library().rfi_batch_graph_launch(g, vp_, fp, ap, wp, sp, _stream(stream)),
           "rfi_batch_graph_launch")


def rfi_batch_graph_destroy(g):
    _check(load_library().rfi_batch_graph_destroy(g), "rfi_batch_graph_destroy")


def rfi_process_block_noalloc(stations, channels, window_M, avg_K, thresholds, dtype, n_seen,
                              vis, T, flags, avg, weight, stats, stream=None):
    """Context-free block processing that allocates nothing (see include/rfi.h)."""
    t = _thr(thresholds)
    _check(load_library().rfi_process_block_noalloc(
        stations, channels, window_M, avg_K, ctypes.byref(t), _dtype(dtype), n_seen, _ptr(vis),
        T, _ptr(flags), _ptr(avg), _ptr(weight), _ptr(stats), _stream(stream)),
        "rfi_process_block_noalloc")


def rfi_check(ctx, stream=None):
    _check(load_library().rfi_check(ctx, _stream(stream)), "rfi_check")


def rfi_state_size(ctx):
    n = ctypes.c_size_t()
    _check(load_library().rfi_state_size(ctx, ctypes.byref(n)), "rfi_state_size")
    return n.value


def rfi_get_state(ctx, stream=None):
    """The stream's state as bytes (synchronises the stream)."""
    n = rfi_state_size(ctx)
    buf = ctypes.create_string_buffer(n)
    _check(load_library().rfi_get_state(ctx, buf, n, _stream(stream)), "rfi_get_state")
    return buf.raw


def rfi_set_state(ctx, state):
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    _check(load_library().rfi_set_state(ctx, buf, len(state)), "rfi_set_state")


def rfi_reset(ctx):
    _check(load_library().rfi_reset(ctx), "rfi_reset")


def rfi_destroy(ctx):
    _check(load_library().rfi_destroy(ctx), "rfi_destroy")


def rfi_status_str(status):
    return load_library().rfi_status_str(status).decode()


def rfi_last_error():
    return load_library().rfi_last_error().decode(errors="replace")
