"""ctypes loader and prototypes of libholo.so (the C ABI declared in include/holo.h).

There is no fallback: if the compiled library is missing the import of an operation
fails with an error that says how to build it.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# HOLO_BOUNDS_CHECK=1 selects the build whose device code checks its table-driven indices
# (build.build(bounds_check=True)); results are the same, a failed check is HOLO_ERR_BOUNDS
BOUNDS_CHECK = os.environ.get("HOLO_BOUNDS_CHECK") == "1"
LIB_PATH = os.path.join(HERE, "_build_bc" if BOUNDS_CHECK else "_build", "libholo.so")
MAX_DIST = 8
F2_AMPLITUDE, F1_INTENSITY = 0, 1   # holo_set_functional
ACCUMULATE = 1
ACCUMULATE_Q = 2
DEFER_Q = 4
NOALLOC_MAX_ELEMENTS = 1 << 28   # holo_dot_noalloc: capacity of its static partial-sum array

STATUS = {0: "HOLO_OK", 1: "HOLO_ERR_ARG", 2: "HOLO_ERR_CUDA", 3: "HOLO_ERR_OOM",
          4: "HOLO_ERR_TIMEOUT", 5: "HOLO_ERR_STATE", 6: "HOLO_ERR_NUMERIC",
          7: "HOLO_ERR_UNSUPPORTED", 8: "HOLO_ERR_BOUNDS"}

# Every symbol declared in include/holo.h.
EXPORTS = ("holo_create", "holo_destroy", "holo_set_shifts", "holo_set_probe_shifts",
           "holo_set_data", "holo_set_probe",
           "holo_forward", "holo_gradient", "holo_gradient_host", "holo_propagate", "holo_dot",
           "holo_step", "holo_direction", "holo_dy_dots", "holo_direction_step", "holo_set_functional",
           "holo_initial_probe", "holo_bin_amplitudes", "holo_upsample2", "holo_set_timing",
           "holo_get_timing", "holo_dot_noalloc",
           "holo_set_stream", "holo_read_loss", "holo_set_device_error",
           "holo_workspace_bytes", "holo_launch_count", "holo_status_string", "holo_last_error",
           "holo_set_schedule", "holo_finish_q", "holo_batch_create", "holo_batch_set_problem",
           "holo_batch_prepare", "holo_batch_gradient", "holo_batch_destroy",
           "holo_set_dy_direction", "holo_direction_step_dy", "holo_read_dy")

# Pass ids of holo_get_timing (HOLO_T_* in include/holo.h).
TIMERS = ("probe", "pass_a", "pass_b", "pass_c", "pass_d", "qgrad", "reduce", "vector")


class HoloGeometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("pad", ctypes.c_int), ("n_angles", ctypes.c_int),
                ("n_dist", ctypes.c_int), ("chunk", ctypes.c_int),
                ("wavelength", ctypes.c_double), ("pixel", ctypes.c_double),
                ("Z", ctypes.c_double), ("z", ctypes.c_double * MAX_DIST),
                ("w_ref", ctypes.c_double), ("ext", ctypes.c_double)]


class HoloError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {name}" + (f" ({detail})" if detail else ""))


_lib = None


def _signatures():
    """ctypes parameter types of every status-returning entry point of include/holo.h."""
    P = ctypes.c_void_p
    I, LL, D = ctypes.c_int, ctypes.c_longlong, ctypes.c_double
    U = ctypes.c_uint
    return {
        "holo_create": [ctypes.POINTER(HoloGeometry), P, ctypes.POINTER(P)],
        "holo_destroy": [P],
        "holo_set_shifts": [P, P],
        "holo_set_probe_shifts": [P, P],
        "holo_set_data": [P, P, P],
        "holo_set_probe": [P, P],
        "holo_forward": [P, I, I, P, P, ctypes.POINTER(D)],
        "holo_gradient": [P, I, I, P, ctypes.POINTER(D), P, P, U],
        "holo_gradient_host": [P, I, I, P, P, P, ctypes.POINTER(D), P, P, U],
        "holo_propagate": [P, P, P, D],
        "holo_dot": [P, P, P, LL, ctypes.POINTER(D)],
        "holo_step": [P, P, P, D, LL],
        "holo_direction": [P, P, P, D, LL],
        "holo_dy_dots": [P, P, P, P, LL, ctypes.POINTER(D)],
        "holo_set_functional": [P, ctypes.c_int],
        "holo_initial_probe": [P, P, P],
        "holo_bin_amplitudes": [P, LL, ctypes.c_int, ctypes.c_int, P, P],
        "holo_upsample2": [P, LL, ctypes.c_int, P, P],
        "holo_direction_step": [P, P, P, P, D, D, LL],
        "holo_set_dy_direction": [P, P],
        "holo_direction_step_dy": [P, P, P, P, D, D, LL],
        "holo_read_dy": [P, ctypes.POINTER(D)],
        "holo_dot_noalloc": [P, P, LL, ctypes.POINTER(D), P],
        "holo_set_stream": [P, P],
        "holo_read_loss": [P, ctypes.POINTER(D)],
        "holo_set_device_error": [P, ctypes.c_ulonglong],
        "holo_set_timing": [P, I],
        "holo_get_timing": [P, P, P],
        "holo_workspace_bytes": [P, ctypes.POINTER(LL)],
        "holo_launch_count": [P, ctypes.POINTER(LL)],
        "holo_set_schedule": [P, I, I, I],
        "holo_finish_q": [P, P, U],
        "holo_batch_create": [ctypes.POINTER(P), I, ctypes.POINTER(P)],
        "holo_batch_set_problem": [P, I, P, P, P, P],
        "holo_batch_prepare": [P],
        "holo_batch_gradient": [P, P],
        "holo_batch_destroy": [P],
    }


def load():
    """Load libholo.so once; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        how = ("`python -c 'from paper_2407_20304_gb300 import build; "
               "build.build(bounds_check=True)'`" if BOUNDS_CHECK else
               "`python -c 'import __graft_entry__ as g; g.build()'`")
        raise RuntimeError(f"{LIB_PATH} is missing: build it with {how}")
    lib = ctypes.CDLL(LIB_PATH)
    sigs = _signatures()
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.holo_status_string.argtypes = [ctypes.c_int]
    lib.holo_status_string.restype = ctypes.c_char_p
    lib.holo_last_error.argtypes = [ctypes.c_void_p]
    lib.holo_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib
