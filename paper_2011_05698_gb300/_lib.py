"""ctypes declarations of the C ABI in include/sfft4.h (argument marshalling only)."""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsfft4.so")

SFFT4_OK = 0
SFFT4_EINVAL = -1
SFFT4_ENOMEM = -2
SFFT4_ECUDA = -3
SFFT4_ESTATE = -4
SFFT4_ETIMEOUT = -5
SFFT4_FP32 = 0
SFFT4_BF16X3 = 1
SFFT4_LOC_MULTISCALE = 0
SFFT4_LOC_TWO_ROUND = 1
SFFT4_FOLD_SIGNAL_MAJOR = 0
SFFT4_FOLD_ITERATION_MAJOR = 1
SFFT4_BATCH_PERSISTENT = 0
SFFT4_BATCH_LEVELS = 1
MAX_ROUNDS = 64


class Opts(ctypes.Structure):
    _fields_ = [("B1", ctypes.c_int32), ("delta", ctypes.c_double), ("precision", ctypes.c_int32),
                ("min_votes", ctypes.c_int32), ("select_factor", ctypes.c_double),
                ("sig_floor", ctypes.c_double), ("mag_tol", ctypes.c_double),
                ("max_iters", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("trace", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("l2_fetch_bytes", ctypes.c_int32), ("graph", ctypes.c_int32), ("location", ctypes.c_int32),
                ("fold_order", ctypes.c_int32), ("trace_signal", ctypes.c_int32),
                ("batch_exec", ctypes.c_int32), ("fold_residues", ctypes.c_int32),
                ("fold_rounds", ctypes.c_int32), ("decode_cluster", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("K", ctypes.c_int64), ("l", ctypes.c_int32),
                ("q_num", ctypes.c_int32), ("B1", ctypes.c_int32), ("n_iters", ctypes.c_int32),
                ("max_R", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("samples_per_transform", ctypes.c_int64), ("found_capacity", ctypes.c_int64),
                ("kernels_per_execute", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("nsig", ctypes.c_int32), ("n_classes", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("kernels_per_execute", ctypes.c_int32), ("Kmax", ctypes.c_int64),
                ("samples_per_execute", ctypes.c_int64), ("precision", ctypes.c_int32)]


class RunStats(ctypes.Structure):
    _fields_ = [("executes", ctypes.c_int64), ("transforms", ctypes.c_int64),
                ("samples_per_execute", ctypes.c_int64), ("iterations", ctypes.c_int32),
                ("kernels_per_execute", ctypes.c_int32), ("last_nsig", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("last_found", ctypes.c_int64),
                ("votes_hist", ctypes.c_int64 * 65)]


class IterInfo(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("S", ctypes.c_int32), ("n_c", ctypes.c_int32),
                ("h", ctypes.c_int32), ("L", ctypes.c_int64),
                ("Lbar", ctypes.c_int64 * MAX_ROUNDS), ("tau", ctypes.c_int64 * MAX_ROUNDS),
                ("H", ctypes.c_uint32 * MAX_ROUNDS), ("unique_samples", ctypes.c_int64)]


class Profile(ctypes.Structure):
    _fields_ = [("fold_launches", ctypes.c_int64), ("fft_launches", ctypes.c_int64),
                ("decode_launches", ctypes.c_int64), ("finalize_launches", ctypes.c_int64),
                ("fold_ms", ctypes.c_double), ("fft_ms", ctypes.c_double),
                ("decode_ms", ctypes.c_double), ("finalize_ms", ctypes.c_double),
                ("fold_samples", ctypes.c_int64)]


class C128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


# (name, restype, argtypes) of every entry point declared in include/sfft4.h
_P = ctypes.c_void_p
SIGNATURES = [
    ("sfft4_opts_default", ctypes.c_int, [ctypes.POINTER(Opts)]),
    ("sfft4_plan", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(Opts)]),
    ("sfft4_destroy", None, [_P]),
    ("sfft4_execute", ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("sfft4_execute_batched", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P, _P, _P]),
    ("sfft4_execute_batched_async", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P, _P, _P]),
    ("sfft4_wait", ctypes.c_int, [_P, _P]),
    ("sfft4_execute_batched_host", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P, _P, _P]),
    ("sfft4_plan_batched", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(Opts)]),
    ("sfft4_execute_batched_v", ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("sfft4_execute_batched_v_async", ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("sfft4_get_batch_info", ctypes.c_int, [_P, ctypes.POINTER(BatchInfo)]),
    ("sfft4_get_plan_info", ctypes.c_int, [_P, ctypes.POINTER(PlanInfo)]),
    ("sfft4_get_iter_info", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(IterInfo)]),
    ("sfft4_get_permutation", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(ctypes.c_uint64)]),
    ("sfft4_get_window", ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    ("sfft4_bucketize", ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    ("sfft4_trace_get", ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P, _P]),
    ("sfft4_profile_get", ctypes.c_int, [_P, ctypes.POINTER(Profile), ctypes.c_int32]),
    ("sfft4_gather_probe", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _P]),
    ("sfft4_gather_probe_ex", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _P]),
    ("sfft4_window_noalloc", ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_double, _P,
                                            ctypes.c_int64, _P, ctypes.c_int64, _P]),
    ("sfft4_sync_status", ctypes.c_int, [_P]),
    ("sfft4_inject_status", ctypes.c_int, [_P, ctypes.c_int32]),
    ("sfft4_stats", ctypes.c_int, [_P, ctypes.POINTER(RunStats)]),
    ("sfft4_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("sfft4_last_cuda_error", ctypes.c_char_p, []),
]

_lib = None


def load(path=LIB_PATH):
    """Load libsfft4.so and declare its signatures.  Raises if the library is missing:
    there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libsfft4.so not built ({path}); run paper_2011_05698_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class Sfft4Error(RuntimeError):
    def __init__(self, code, what):
        lib = load()
        msg = lib.sfft4_strerror(code).decode()
        if code == SFFT4_ECUDA:
            msg += ": " + lib.sfft4_last_cuda_error().decode()
        super().__init__(f"{what}: {msg} ({code})")
        self.code = code


def check(code, what):
    if code != SFFT4_OK:
        raise Sfft4Error(code, what)
