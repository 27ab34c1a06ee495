"""B300-native LeaFi search path (learned filters for tree-based series indexes).

A thin ctypes binding of the C ABI in include/leafi.h.  Every function here
only marshals arguments: all computation happens in libleafi.so (CUDA kernels
for sm_103a plus the host-side tree builder).  Arrays may be numpy arrays
(host) or torch tensors (host or CUDA); results are written into caller-owned
arrays of the same kind.  If the shared library is missing the import fails
loudly: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = [
    "LeafiError", "BuildParams", "TrainParams", "SearchStats", "IndexInfo", "lib",
    "leafi_build", "leafi_free", "leafi_set_stream", "leafi_get_info", "leafi_leaf_sizes",
    "leafi_leaf_of", "leafi_leaf_lower_bounds", "leafi_route", "leafi_select_leaves",
    "leafi_set_filters", "leafi_get_filters", "leafi_filter_predict", "leafi_leaf_knn",
    "leafi_train_targets", "leafi_train_filters", "leafi_fit_autotuners",
    "leafi_get_autotuners", "leafi_set_autotuners", "leafi_search", "leafi_search_scanned",
    "leafi_exact_search",
    "leafi_search_mixed", "leafi_launch_count", "leafi_set_profiling", "leafi_get_kernel_times",
    "KERNEL_KINDS", "leafi_leaf_lower_bounds_noalloc", "leafi_get_scan_phases", "SCAN_PHASES",
    "DSTREE", "ISAX", "MAX_K", "EXPORTED_SYMBOLS", "EAGAIN", "ServeParams", "ServeStats",
    "leafi_serve_start", "leafi_serve_submit", "leafi_serve_poll", "leafi_serve_get_stats",
    "leafi_serve_stop", "leafi_select_leaves_auto", "SelectParams", "SelectReport",
    "SgdParams", "TrainReport", "leafi_train_filters_on", "leafi_training_queries",
    "leafi_initial_weights", "leafi_epoch_permutations", "leafi_znormalize",
    "leafi_get_filter_leaves", "leafi_debug_set_lock_tries", "leafi_debug_fail_allocations",
    "leafi_set_calibration_confidence", "leafi_set_query_schedule", "leafi_set_search_lanes",
    "leafi_set_scan_part", "leafi_tune_search", "TuneParams", "TuneReport",
    "leafi_set_search_batch", "leafi_set_calibration_mode", "leafi_calibration_offsets",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libleafi.so")

DSTREE, ISAX = 0, 1
FILTER_MLP, FILTER_CNN = 0, 1
CALIB_STEP, CALIB_STEFFEN = 0, 1
MAX_K = 128
_STATUS = {0: "LEAFI_OK", 1: "LEAFI_EINVAL", 2: "LEAFI_ENOMEM", 3: "LEAFI_ECUDA",
           4: "LEAFI_ETIMEOUT", 5: "LEAFI_ENOTTRAINED", 6: "LEAFI_EINTERNAL",
           7: "LEAFI_EAGAIN"}
EAGAIN = 7

EXPORTED_SYMBOLS = [
    "leafi_build", "leafi_free", "leafi_last_error", "leafi_set_stream", "leafi_get_info",
    "leafi_leaf_sizes", "leafi_leaf_of", "leafi_leaf_lower_bounds", "leafi_route",
    "leafi_select_leaves", "leafi_set_filters", "leafi_get_filters", "leafi_filter_predict",
    "leafi_leaf_knn", "leafi_train_targets", "leafi_train_filters", "leafi_fit_autotuners",
    "leafi_get_autotuners", "leafi_set_autotuners", "leafi_search", "leafi_search_scanned",
    "leafi_exact_search",
    "leafi_search_mixed", "leafi_launch_count", "leafi_set_profiling", "leafi_get_kernel_times",
    "leafi_leaf_lower_bounds_noalloc", "leafi_get_scan_phases",
    "leafi_serve_start", "leafi_serve_submit", "leafi_serve_poll", "leafi_serve_get_stats",
    "leafi_serve_stop", "leafi_select_leaves_auto", "leafi_train_filters_on",
    "leafi_training_queries", "leafi_initial_weights", "leafi_epoch_permutations",
    "leafi_znormalize", "leafi_get_filter_leaves", "leafi_debug_set_lock_tries",
    "leafi_debug_fail_allocations", "leafi_set_calibration_confidence",
    "leafi_set_query_schedule", "leafi_set_search_lanes", "leafi_set_scan_part",
    "leafi_tune_search", "leafi_cnn_params", "leafi_set_cnn_filters", "leafi_get_cnn_filters",
    "leafi_initial_cnn_weights", "leafi_set_search_batch", "leafi_set_calibration_mode",
    "leafi_calibration_offsets",
]

KERNEL_KINDS = ["leaf_scan", "merge", "bounds", "reserved", "filter_forward", "select"]


class LeafiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class BuildParams(C.Structure):
    _fields_ = [("index_type", C.c_int32), ("leaf_capacity", C.c_int32),
                ("dstree_init_segments", C.c_int32), ("isax_segments", C.c_int32),
                ("isax_card_bits", C.c_int32), ("wave", C.c_int32), ("device", C.c_int32),
                ("scan_path", C.c_int32), ("host_build", C.c_int32)]

    def __init__(self, index_type=DSTREE, leaf_capacity=10000, dstree_init_segments=4,
                 isax_segments=16, isax_card_bits=8, wave=64, device=0, scan_path=0,
                 host_build=0):
        super().__init__(index_type, leaf_capacity, dstree_init_segments, isax_segments,
                         isax_card_bits, wave, device, scan_path, host_build)


class IndexInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int32), ("index_type", C.c_int32),
                ("n_leaves", C.c_int32), ("n_nodes", C.c_int32), ("wave", C.c_int32),
                ("n_filters", C.c_int32), ("filters_trained", C.c_int32),
                ("n_calib", C.c_int32), ("n_kclasses", C.c_int32),
                ("kclasses", C.c_int32 * 4), ("device_bytes", C.c_int64),
                ("tensor_scan", C.c_int32), ("scan_row_bytes", C.c_int32),
                ("calib_confidence", C.c_double), ("filter_model", C.c_int32),
                ("filter_width", C.c_int32), ("wave_exact", C.c_int32),
                ("items_per_sm", C.c_int32)]


class TrainParams(C.Structure):
    """Alg. 1 parameters of leafi_train_filters (defaults: the paper's setup)."""
    _fields_ = [("n_filters", C.c_int32), ("a", C.c_double), ("mem_cap", C.c_int64),
                ("hidden", C.c_int32), ("n_train", C.c_int32), ("global_local_ratio", C.c_double),
                ("val_frac", C.c_double), ("noise_lo", C.c_double), ("noise_hi", C.c_double),
                ("batch", C.c_int32), ("max_epochs", C.c_int32), ("patience", C.c_int32),
                ("lr0", C.c_double), ("lr_min", C.c_double), ("n_kclasses", C.c_int32),
                ("kclasses", C.c_int32 * 4), ("seed", C.c_uint64), ("confidence", C.c_double),
                ("tune_search", C.c_int32), ("model", C.c_int32), ("calib_mode", C.c_int32)]

    def __init__(self, n_filters=100, a=2.0, mem_cap=8 << 30, hidden=0, n_train=2000,
                 global_local_ratio=3.0, val_frac=0.2, noise_lo=0.1, noise_hi=0.4, batch=64,
                 max_epochs=1000, patience=10, lr0=0.01, lr_min=1e-5, kclasses=(1,),
                 seed=2502018361, confidence=0.95, tune_search=1, model=0, calib_mode=0):
        kc = (C.c_int32 * 4)(*(list(kclasses) + [0] * (4 - len(kclasses))))
        super().__init__(n_filters, a, mem_cap, hidden, n_train, global_local_ratio, val_frac,
                         noise_lo, noise_hi, batch, max_epochs, patience, lr0, lr_min,
                         len(kclasses), kc, seed, confidence, tune_search, model, calib_mode)


class TuneParams(C.Structure):
    """leafi_tune_search parameters (empty candidate lists take the defaults)."""
    _fields_ = [("n_probe", C.c_int32), ("k", C.c_int32), ("noise_lo", C.c_double),
                ("noise_hi", C.c_double), ("seed", C.c_uint64), ("reps", C.c_int32),
                ("n_waves", C.c_int32), ("waves", C.c_int32 * 8), ("n_items", C.c_int32),
                ("items_per_sm", C.c_int32 * 4), ("target", C.c_double)]

    def __init__(self, n_probe=8192, k=1, noise_lo=0.1, noise_hi=0.4, seed=2502018361, reps=3,
                 waves=(), items_per_sm=(), target=1.0):
        w = (C.c_int32 * 8)(*(list(waves) + [0] * (8 - len(waves))))
        it = (C.c_int32 * 4)(*(list(items_per_sm) + [0] * (4 - len(items_per_sm))))
        super().__init__(n_probe, k, noise_lo, noise_hi, seed, reps, len(waves), w,
                         len(items_per_sm), it, target)


class TuneReport(C.Structure):
    _fields_ = [("wave", C.c_int32), ("items_per_sm", C.c_int32), ("ms_best", C.c_double),
                ("ms_before", C.c_double), ("n_tried", C.c_int32), ("tried_wave", C.c_int32 * 32),
                ("tried_items", C.c_int32 * 32), ("tried_ms", C.c_double * 32)]


class TrainReport(C.Structure):
    _fields_ = [("n_filters", C.c_int32), ("n_gtrain", C.c_int32), ("n_gval", C.c_int32),
                ("n_ltrain", C.c_int32), ("n_lval", C.c_int32), ("select_threshold", C.c_double),
                ("seconds_select", C.c_double), ("seconds_generate", C.c_double),
                ("seconds_train", C.c_double), ("seconds_calibrate", C.c_double)]


class SgdParams(C.Structure):
    """SGD parameters of leafi_train_filters_on (queries supplied by the caller)."""
    _fields_ = [("n_gtrain", C.c_int32), ("n_gval", C.c_int32), ("n_ltrain", C.c_int32),
                ("n_lval", C.c_int32), ("batch", C.c_int32), ("max_epochs", C.c_int32),
                ("patience", C.c_int32), ("lr0", C.c_double), ("lr_min", C.c_double)]

    def __init__(self, n_gtrain=1200, n_gval=300, n_ltrain=400, n_lval=100, batch=64,
                 max_epochs=1000, patience=10, lr0=0.01, lr_min=1e-5):
        super().__init__(n_gtrain, n_gval, n_ltrain, n_lval, batch, max_epochs, patience,
                         lr0, lr_min)


class SearchStats(C.Structure):
    _fields_ = [("leaves_scanned", C.c_int64), ("series_scanned", C.c_int64),
                ("filter_evals", C.c_int64), ("waves", C.c_int64), ("batches", C.c_int64),
                ("distinct_series", C.c_int64), ("rechecks", C.c_int64),
                ("graph_batches", C.c_int64), ("host_wait_ms", C.c_double),
                ("host_ms", C.c_double), ("filter_pruned", C.c_int64), ("lb_pruned", C.c_int64)]


class SelectParams(C.Structure):
    _fields_ = [("a", C.c_double), ("mem_cap", C.c_int64), ("hidden", C.c_int32),
                ("model", C.c_int32)]


class SelectReport(C.Structure):
    _fields_ = [("t_filter_s", C.c_double), ("t_series_s", C.c_double),
                ("threshold", C.c_double), ("filter_bytes", C.c_double),
                ("n_selected", C.c_int32)]


class ServeParams(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("kmax", C.c_int32), ("max_wait_ms", C.c_double),
                ("max_bytes", C.c_int64)]


class ServeStats(C.Structure):
    _fields_ = [("requests", C.c_int64), ("queries", C.c_int64), ("batches", C.c_int64),
                ("graph_batches", C.c_int64), ("search", SearchStats),
                ("admitted_in_flight", C.c_int64), ("device_bytes", C.c_int64)]


_lib = None


def lib():
    """Load libleafi.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libleafi.so is missing: run `python paper_2502_01836_b300/build.py`"
                              " (or __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "leafi_build": [vp, i64, i32, C.POINTER(BuildParams), C.POINTER(vp)],
            "leafi_set_stream": [vp, vp],
            "leafi_get_info": [vp, C.POINTER(IndexInfo)],
            "leafi_leaf_sizes": [vp, vp],
            "leafi_leaf_of": [vp, vp],
            "leafi_leaf_lower_bounds": [vp, vp, i64, vp],
            "leafi_route": [vp, vp, i64, vp],
            "leafi_leaf_lower_bounds_noalloc": [vp, vp, i64, vp],
            "leafi_select_leaves": [vp, i32, vp],
            "leafi_set_filters": [vp, vp, i32, i32, vp, vp, vp, vp],
            "leafi_get_filters": [vp, vp, vp, vp, vp],
            "leafi_set_cnn_filters": [vp, vp, i32, i32, vp],
            "leafi_get_cnn_filters": [vp, vp],
            "leafi_initial_cnn_weights": [vp, i32, i32, C.c_uint64, vp],
            "leafi_filter_predict": [vp, vp, i64, vp],
            "leafi_leaf_knn": [vp, vp, i64, vp, i32, i32, vp, vp],
            "leafi_train_targets": [vp, vp, i64, vp, i64, vp, vp],
            "leafi_train_filters": [vp, C.POINTER(TrainParams), vp, vp, C.POINTER(TrainReport)],
            "leafi_train_filters_on": [vp, C.POINTER(SgdParams), vp, vp, vp, vp, vp],
            "leafi_training_queries": [vp, C.POINTER(TrainParams), vp, i32, vp, vp, vp, vp],
            "leafi_initial_weights": [vp, i32, i32, C.c_uint64, vp, vp, vp, vp],
            "leafi_epoch_permutations": [i32, i32, C.c_uint64, vp],
            "leafi_znormalize": [vp, i64, i32, vp, i32],
            "leafi_get_filter_leaves": [vp, vp],
            "leafi_debug_set_lock_tries": [vp, i32],
            "leafi_debug_fail_allocations": [i64],
            "leafi_set_calibration_confidence": [vp, f64],
            "leafi_set_query_schedule": [vp, i32],
            "leafi_set_search_lanes": [vp, i32],
            "leafi_set_scan_part": [vp, i32, i32, i32, i32],
            "leafi_set_search_batch": [vp, i32],
            "leafi_set_calibration_mode": [vp, i32],
            "leafi_calibration_offsets": [vp, i32, f64, vp, C.POINTER(i32)],
            "leafi_tune_search": [vp, C.POINTER(TuneParams), C.POINTER(TuneReport)],
            "leafi_fit_autotuners": [vp, vp, i64, vp, i32],
            "leafi_get_autotuners": [vp, vp, vp],
            "leafi_set_autotuners": [vp, vp, vp, i64, vp, i32],
            "leafi_search": [vp, vp, i64, i32, f64, vp, vp, C.POINTER(SearchStats)],
            "leafi_exact_search": [vp, vp, i64, i32, vp, vp, C.POINTER(SearchStats)],
            "leafi_search_scanned": [vp, vp, i64, i32, f64, vp, vp, vp],
            "leafi_search_mixed": [vp, vp, i64, vp, vp, i32, vp, vp, C.POINTER(SearchStats)],
            "leafi_set_profiling": [vp, i32],
            "leafi_get_kernel_times": [vp, vp, vp],
            "leafi_get_scan_phases": [vp, vp],
            "leafi_serve_start": [vp, C.POINTER(ServeParams), C.POINTER(vp)],
            "leafi_serve_submit": [vp, vp, i64, vp, vp, C.POINTER(i64)],
            "leafi_serve_poll": [vp, i64, vp, vp, f64, C.POINTER(i32), C.POINTER(f64)],
            "leafi_serve_get_stats": [vp, C.POINTER(ServeStats)],
            "leafi_serve_stop": [vp],
            "leafi_select_leaves_auto": [vp, C.POINTER(SelectParams), vp, C.POINTER(SelectReport)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.leafi_free.argtypes = [vp]
        L.leafi_free.restype = None
        L.leafi_cnn_params.argtypes = [i32]
        L.leafi_cnn_params.restype = C.c_int64
        L.leafi_launch_count.argtypes = []
        L.leafi_launch_count.restype = C.c_int64
        L.leafi_last_error.argtypes = []
        L.leafi_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise LeafiError(st, lib().leafi_last_error().decode())


_NP = {np.float32: "float32", np.float64: "float64", np.int32: "int32", np.int64: "int64",
       np.uint8: "uint8"}


def _ptr(a, dtype, name="array", writable=False):
    """Data pointer of a C-contiguous numpy array or torch tensor of `dtype`."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype) or not a.flags.c_contiguous:
            raise TypeError("%s must be a C-contiguous %s numpy array" % (name, np.dtype(dtype)))
        if writable and not a.flags.writeable:
            raise TypeError("%s must be writable" % name)
        return a.ctypes.data
    mod = type(a).__module__
    if mod.startswith("torch"):
        import torch
        tmap = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
                np.int64: torch.int64, np.uint8: torch.uint8}
        if a.dtype != tmap[dtype] or not a.is_contiguous():
            raise TypeError("%s must be a contiguous torch.%s tensor" % (name, _NP[dtype]))
        return a.data_ptr()
    raise TypeError("%s must be a numpy array or a torch tensor" % name)


def leafi_launch_count() -> int:
    return int(lib().leafi_launch_count())


def leafi_set_profiling(index, level):
    """0 off, 1 (or True) leaf-scan kernel times only, 2 every kernel kind and scan phases."""
    _check(lib().leafi_set_profiling(index, int(level)))


def leafi_get_kernel_times(index):
    """{kind: (total ms, launches)} for the kernels timed since profiling was switched on."""
    ms = np.zeros(6, np.float64)
    n = np.zeros(6, np.int64)
    _check(lib().leafi_get_kernel_times(index, ms.ctypes.data, n.ctypes.data))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


SCAN_PHASES = ["item_setup", "wait_accumulator", "epilogue", "flush_emit", "wait_stage_free",
               "wait_query_tile", "wait_tma", "wait_accumulator_free", "commit", "items", "chunks",
               "tma_issue", "wait_tile_free", "gather", "mma_issue", "epilogue_span",
               "launch_span_ns", "start_skew_ns", "end_skew_ns", "launches"]


def leafi_get_scan_phases(index):
    """Tensor-core scan phase cycle totals recorded while profiling was on."""
    c = np.zeros(20, np.float64)
    _check(lib().leafi_get_scan_phases(index, c.ctypes.data))
    return {k: float(c[i]) for i, k in enumerate(SCAN_PHASES)}


def leafi_build(series, params: BuildParams | None = None):
    """Build an index over `series` [n, m] float32; returns an opaque handle."""
    params = params or BuildParams()
    n, m = series.shape
    h = C.c_void_p()
    _check(lib().leafi_build(_ptr(series, np.float32, "series"), n, m, C.byref(params),
                             C.byref(h)))
    return h


def leafi_free(index):
    lib().leafi_free(index)


def leafi_set_stream(index, stream_handle: int):
    _check(lib().leafi_set_stream(index, C.c_void_p(stream_handle)))


def leafi_get_info(index) -> IndexInfo:
    info = IndexInfo()
    _check(lib().leafi_get_info(index, C.byref(info)))
    return info


def leafi_leaf_sizes(index):
    out = np.empty(leafi_get_info(index).n_leaves, np.int64)
    _check(lib().leafi_leaf_sizes(index, out.ctypes.data))
    return out


def leafi_leaf_of(index):
    out = np.empty(leafi_get_info(index).n, np.int32)
    _check(lib().leafi_leaf_of(index, out.ctypes.data))
    return out


def leafi_leaf_lower_bounds(index, queries, out):
    _check(lib().leafi_leaf_lower_bounds(index, _ptr(queries, np.float32, "queries"),
                                         queries.shape[0], _ptr(out, np.float64, "out", True)))
    return out


def leafi_leaf_lower_bounds_noalloc(index, queries, out):
    """Leaf bounds with no device allocation: `queries` and `out` must be CUDA tensors.

    For callers that cannot allocate device memory (their GPU memory is held by
    another allocator, or their loop cannot take cudaMalloc's device-wide
    synchronisation); the library's static scratch array (16 MiB per GPU)
    bounds nq.  Returns without synchronising.  Shapes are checked here because
    the C side receives bare pointers: queries [nq, m] float32 and out
    [nq, n_leaves] float64, both on the index's device.
    """
    info = leafi_get_info(index)
    for name, a in (("queries", queries), ("out", out)):
        if not type(a).__module__.startswith("torch") or not a.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
    if queries.ndim != 2 or queries.shape[1] != info.m:
        raise ValueError("queries must have shape (nq, %d), got %s" % (info.m, tuple(queries.shape)))
    if tuple(out.shape) != (queries.shape[0], info.n_leaves):
        raise ValueError("out must have shape (%d, %d), got %s"
                         % (queries.shape[0], info.n_leaves, tuple(out.shape)))
    if queries.device != out.device:
        raise ValueError("queries and out must be on the same device")
    _check(lib().leafi_leaf_lower_bounds_noalloc(index, _ptr(queries, np.float32, "queries"),
                                                 queries.shape[0],
                                                 _ptr(out, np.float64, "out", True)))
    return out


def leafi_route(index, queries, out):
    _check(lib().leafi_route(index, _ptr(queries, np.float32, "queries"), queries.shape[0],
                             _ptr(out, np.int32, "out", True)))
    return out


def leafi_select_leaves(index, n_filters):
    out = np.empty(n_filters, np.int32)
    _check(lib().leafi_select_leaves(index, n_filters, out.ctypes.data))
    return out


def leafi_select_leaves_auto(index, a=2.0, mem_cap=8 << 30, hidden=0, model=0):
    """Alg. 3 with this device's measured t^F and t^S: (filter_leaf, report dict)."""
    out = np.zeros(max(1, leafi_get_info(index).n_leaves), np.int32)
    rep = SelectReport()
    _check(lib().leafi_select_leaves_auto(index, C.byref(SelectParams(a, mem_cap, hidden, model)),
                                          out.ctypes.data, C.byref(rep)))
    return out[:rep.n_selected].copy(), {f: getattr(rep, f) for f, _ in SelectReport._fields_}


def leafi_set_filters(index, filter_leaf, W1, b1, w2, b2):
    F, h, _ = W1.shape
    _check(lib().leafi_set_filters(index, _ptr(filter_leaf, np.int32, "filter_leaf"), F, h,
                                   _ptr(W1, np.float32, "W1"), _ptr(b1, np.float32, "b1"),
                                   _ptr(w2, np.float32, "w2"), _ptr(b2, np.float32, "b2")))


def leafi_cnn_params(C_):
    """Parameters of one CNN filter of C_ channels (3 C^2 + 6 C + 1)."""
    return int(lib().leafi_cnn_params(int(C_)))


def leafi_set_cnn_filters(index, filter_leaf, C_, theta):
    """Install CNN filters: theta [F, leafi_cnn_params(C_)] float32 (host or device)."""
    F = theta.shape[0]
    if theta.ndim != 2 or theta.shape[1] != leafi_cnn_params(C_):
        raise ValueError("theta must be [F, leafi_cnn_params(C)]")
    _check(lib().leafi_set_cnn_filters(index, _ptr(filter_leaf, np.int32, "filter_leaf"), F,
                                       int(C_), _ptr(theta, np.float32, "theta")))


def leafi_get_cnn_filters(index):
    info = leafi_get_info(index)
    out = np.zeros((info.n_filters, leafi_cnn_params(info.filter_width)), np.float32)
    _check(lib().leafi_get_cnn_filters(index, out.ctypes.data))
    return out


def leafi_initial_cnn_weights(index, F, C_, seed):
    """Initial CNN parameters [F, leafi_cnn_params(C_)] drawn by the library."""
    out = np.zeros((F, leafi_cnn_params(C_)), np.float32)
    _check(lib().leafi_initial_cnn_weights(index, F, int(C_), seed, out.ctypes.data))
    return out


def leafi_debug_set_lock_tries(index, tries):
    """Failure-detection diagnostic: result-list lock attempts (-1 = default)."""
    _check(lib().leafi_debug_set_lock_tries(index, int(tries)))


def leafi_debug_fail_allocations(after):
    """Failure-detection diagnostic: make the after-th allocation from now fail (-1 disarms)."""
    _check(lib().leafi_debug_fail_allocations(int(after)))


def leafi_set_calibration_confidence(index, confidence):
    """Probability that a certified sorted position meets its recall target (0: point estimate)."""
    _check(lib().leafi_set_calibration_confidence(index, float(confidence)))


def leafi_set_query_schedule(index, on=True):
    """Cut multi-batch calls' batches in route-leaf order (results unchanged)."""
    _check(lib().leafi_set_query_schedule(index, int(bool(on))))


def leafi_set_search_lanes(index, lanes):
    """Batches of one search call in flight (1..8)."""
    _check(lib().leafi_set_search_lanes(index, int(lanes)))


def leafi_set_calibration_mode(index, mode):
    """CALIB_STEP (certified position) or CALIB_STEFFEN (the paper's spline)."""
    _check(lib().leafi_set_calibration_mode(index, int(mode)))


def leafi_calibration_offsets(index, k, recall_target):
    """The offsets [F] a query of this k and target uses, or None if it runs exactly."""
    out = np.zeros(max(1, leafi_get_info(index).n_filters), np.float64)
    use = C.c_int32()
    _check(lib().leafi_calibration_offsets(index, int(k), float(recall_target), out.ctypes.data,
                                           C.byref(use)))
    return out if use.value else None


def leafi_set_search_batch(index, queries=256):
    """Queries per internal batch of a search call (results do not depend on it)."""
    _check(lib().leafi_set_search_batch(index, int(queries)))


def leafi_set_scan_part(index, rows=2048, items_per_sm=4, min_rows=512, blocks=0):
    """Leaf-scan work items: at most `rows` series (multiple of 128); rounds aim at
    items_per_sm items per SM (0: always `rows`) with parts of at least min_rows;
    `blocks` per scan launch (0: one per SM)."""
    _check(lib().leafi_set_scan_part(index, int(rows), int(items_per_sm), int(min_rows),
                                     int(blocks)))


def leafi_tune_search(index, params: TuneParams | None = None):
    """Search-schedule autotuner: returns the report as a dict (the choice is installed)."""
    rep = TuneReport()
    _check(lib().leafi_tune_search(index, C.byref(params or TuneParams()), C.byref(rep)))
    n = rep.n_tried
    return {"wave": rep.wave, "items_per_sm": rep.items_per_sm, "ms_best": rep.ms_best,
            "ms_before": rep.ms_before,
            "tried": [(rep.tried_wave[i], rep.tried_items[i], rep.tried_ms[i]) for i in range(n)]}


def leafi_get_filter_leaves(index):
    out = np.zeros(max(1, leafi_get_info(index).n_filters), np.int32)
    _check(lib().leafi_get_filter_leaves(index, out.ctypes.data))
    return out[:leafi_get_info(index).n_filters].copy()


def leafi_get_filters(index, W1, b1, w2, b2):
    _check(lib().leafi_get_filters(index, _ptr(W1, np.float32, "W1", True),
                                   _ptr(b1, np.float32, "b1", True),
                                   _ptr(w2, np.float32, "w2", True),
                                   _ptr(b2, np.float32, "b2", True)))
    return W1, b1, w2, b2


def leafi_filter_predict(index, queries, out):
    _check(lib().leafi_filter_predict(index, _ptr(queries, np.float32, "queries"),
                                      queries.shape[0], _ptr(out, np.float32, "out", True)))
    return out


def leafi_leaf_knn(index, queries, leaves, k, d2, ids):
    _check(lib().leafi_leaf_knn(index, _ptr(queries, np.float32, "queries"), queries.shape[0],
                                _ptr(leaves, np.int32, "leaves"), leaves.shape[1], k,
                                _ptr(d2, np.float32, "d2", True), _ptr(ids, np.int64, "ids", True)))
    return d2, ids


def leafi_train_targets(index, Qg, Ql, Tg, Tl):
    """Qg [ng, m]; Ql [F, nl, m] -> Tg [ng, F], Tl [F, nl]."""
    nl = Ql.shape[1] if Ql is not None and Ql.ndim == 3 else 0
    _check(lib().leafi_train_targets(index, _ptr(Qg, np.float32, "Qg"), Qg.shape[0],
                                     _ptr(Ql, np.float32, "Ql"), nl,
                                     _ptr(Tg, np.float32, "Tg", True),
                                     _ptr(Tl, np.float32, "Tl", True)))
    return Tg, Tl


def leafi_train_filters(index, params: TrainParams | None = None):
    """Alg. 1 end to end: returns (epochs_run [F], best_val [F], report dict)."""
    params = params or TrainParams()
    L = leafi_get_info(index).n_leaves
    ep = np.zeros(max(L, 1), np.int32)
    bv = np.zeros(max(L, 1), np.float64)
    rep = TrainReport()
    _check(lib().leafi_train_filters(index, C.byref(params), ep.ctypes.data, bv.ctypes.data,
                                     C.byref(rep)))
    F = rep.n_filters
    return ep[:F].copy(), bv[:F].copy(), {f: getattr(rep, f) for f, _ in TrainReport._fields_}


def _alg1_counts(params: TrainParams):
    """(n_global, n_local) as leafi_train_filters derives them."""
    r = params.global_local_ratio
    if np.isinf(r):
        ng = params.n_train
    else:
        ng = int(np.floor(params.n_train * r / (r + 1.0) + 0.5))
    ng = min(max(ng, 2), params.n_train)
    return ng, params.n_train - ng


def leafi_training_queries(index, params: TrainParams, filter_leaf):
    """The training queries Alg. 1 generates for these leaves:
    (Qg [ng, m], Ql [F, nl, m], gpick [ng], lpick [F, nl])."""
    fl = np.ascontiguousarray(filter_leaf, np.int32)
    m = leafi_get_info(index).m
    ng, nl = _alg1_counts(params)
    F = fl.shape[0]
    Qg = np.zeros((ng, m), np.float32)
    Ql = np.zeros((F, nl, m), np.float32)
    gp = np.zeros(ng, np.int64)
    lp = np.zeros((F, nl), np.int64)
    _check(lib().leafi_training_queries(index, C.byref(params), fl.ctypes.data, F,
                                        Qg.ctypes.data, Ql.ctypes.data, gp.ctypes.data,
                                        lp.ctypes.data))
    return Qg, Ql, gp, lp


def leafi_initial_weights(index, F, h, seed):
    """Initial weights (W1 [F,h,m], b1 [F,h], w2 [F,h], b2 [F]) drawn by the library."""
    m = leafi_get_info(index).m
    W = (np.zeros((F, h, m), np.float32), np.zeros((F, h), np.float32),
         np.zeros((F, h), np.float32), np.zeros(F, np.float32))
    _check(lib().leafi_initial_weights(index, F, h, seed, *(w.ctypes.data for w in W)))
    return W


def leafi_epoch_permutations(epochs, n, seed):
    out = np.zeros((epochs, n), np.int32)
    _check(lib().leafi_epoch_permutations(epochs, n, seed, out.ctypes.data))
    return out


def leafi_train_filters_on(index, params: SgdParams, Qg, Ql, perms, epochs_run=None,
                           best_val=None):
    """Alg. 1 target collection and training on caller-supplied queries and shuffles (parity checks)."""
    _check(lib().leafi_train_filters_on(index, C.byref(params), _ptr(Qg, np.float32, "Qg"),
                                        _ptr(Ql, np.float32, "Ql"), _ptr(perms, np.int32, "perms"),
                                        _ptr(epochs_run, np.int32, "epochs_run", True),
                                        _ptr(best_val, np.float64, "best_val", True)))
    return epochs_run, best_val


def leafi_znormalize(x, out=None, device=0):
    """float64 z-normalisation of the rows of x [n, m] on `device` (out may be x)."""
    out = np.empty_like(x) if out is None else out
    n, m = x.shape
    _check(lib().leafi_znormalize(_ptr(x, np.float32, "x"), n, m, _ptr(out, np.float32, "out", True),
                                  device))
    return out


def leafi_fit_autotuners(index, Qc, kclasses):
    kc = np.ascontiguousarray(kclasses, np.int32)
    _check(lib().leafi_fit_autotuners(index, _ptr(Qc, np.float32, "Qc"), Qc.shape[0],
                                      kc.ctypes.data, kc.shape[0]))


def leafi_get_autotuners(index, alpha_sorted, qprime):
    _check(lib().leafi_get_autotuners(index, _ptr(alpha_sorted, np.float64, "alpha", True),
                                      _ptr(qprime, np.float64, "qprime", True)))
    return alpha_sorted, qprime


def leafi_set_autotuners(index, alpha_sorted, qprime, kclasses):
    kc = np.ascontiguousarray(kclasses, np.int32)
    _check(lib().leafi_set_autotuners(index, _ptr(alpha_sorted, np.float64, "alpha"),
                                      _ptr(qprime, np.float64, "qprime"), alpha_sorted.shape[1],
                                      kc.ctypes.data, kc.shape[0]))


def leafi_search(index, queries, k, recall_target, ids, dists, stats: SearchStats | None = None):
    _check(lib().leafi_search(index, _ptr(queries, np.float32, "queries"), queries.shape[0], k,
                              float(recall_target), _ptr(ids, np.int64, "ids", True),
                              _ptr(dists, np.float32, "dists", True),
                              C.byref(stats) if stats is not None else None))
    return ids, dists


def leafi_search_scanned(index, queries, k, recall_target, ids, dists, scanned):
    """leafi_search that also writes scanned [nq, n_leaves] uint8: 1 where the
    search searched the leaf for the query (an inspection export)."""
    _check(lib().leafi_search_scanned(index, _ptr(queries, np.float32, "queries"),
                                      queries.shape[0], k, float(recall_target),
                                      _ptr(ids, np.int64, "ids", True),
                                      _ptr(dists, np.float32, "dists", True),
                                      _ptr(scanned, np.uint8, "scanned", True)))
    return ids, dists, scanned


def leafi_exact_search(index, queries, k, ids, dists, stats: SearchStats | None = None):
    _check(lib().leafi_exact_search(index, _ptr(queries, np.float32, "queries"), queries.shape[0],
                                    k, _ptr(ids, np.int64, "ids", True),
                                    _ptr(dists, np.float32, "dists", True),
                                    C.byref(stats) if stats is not None else None))
    return ids, dists


def leafi_search_mixed(index, queries, k, recall_target, kmax, ids, dists,
                       stats: SearchStats | None = None):
    _check(lib().leafi_search_mixed(index, _ptr(queries, np.float32, "queries"), queries.shape[0],
                                    _ptr(k, np.int32, "k"), _ptr(recall_target, np.float64, "target"),
                                    kmax, _ptr(ids, np.int64, "ids", True),
                                    _ptr(dists, np.float32, "dists", True),
                                    C.byref(stats) if stats is not None else None))
    return ids, dists


# ---------------------------------------------------------------- serving
def leafi_serve_start(index, kmax=1, max_batch=256, max_wait_ms=0.2, max_bytes=0):
    """Start a request loop over `index`; returns the server handle."""
    out = C.c_void_p()
    p = ServeParams(max_batch, kmax, max_wait_ms, max_bytes)
    _check(lib().leafi_serve_start(index, C.byref(p), C.byref(out)))
    return out


def leafi_serve_submit(server, queries, k, recall_target):
    """Queue a request (host arrays); returns its ticket.  LeafiError with status
    EAGAIN when the admission budget is full."""
    t = C.c_int64()
    _check(lib().leafi_serve_submit(server, _ptr(queries, np.float32, "queries"), queries.shape[0],
                                    _ptr(k, np.int32, "k"), _ptr(recall_target, np.float64, "target"),
                                    C.byref(t)))
    return t.value


def leafi_serve_poll(server, ticket, ids, dists, wait_ms=0.0):
    """(done, latency_ms); when done the results are in ids / dists [nq][kmax]."""
    done = C.c_int32()
    lat = C.c_double()
    _check(lib().leafi_serve_poll(server, ticket, _ptr(ids, np.int64, "ids", True),
                                  _ptr(dists, np.float32, "dists", True), wait_ms, C.byref(done),
                                  C.byref(lat)))
    return bool(done.value), lat.value


def leafi_serve_get_stats(server):
    st = ServeStats()
    _check(lib().leafi_serve_get_stats(server, C.byref(st)))
    out = {f: getattr(st, f) for f, _ in ServeStats._fields_ if f != "search"}
    out["search"] = {f: getattr(st.search, f) for f, _ in SearchStats._fields_}
    return out


def leafi_serve_stop(server):
    _check(lib().leafi_serve_stop(server))
