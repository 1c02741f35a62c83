"""ctypes declarations of libddh's C ABI (include/ddh.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_float, c_int, c_int64, c_size_t, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libddh.so")

DDH_OK = 0
DDH_EINVAL = -1
DDH_ENOMEM = -2
DDH_ECUDA = -3
DDH_ETIMEOUT = -4
DDH_ENONFINITE = -5
DDH_EBUDGET = -6
DDH_PATH_DEFAULT = 0
DDH_PATH_CLUSTER = 1
DDH_PATH_STAGED = 2


class DdhParams(ctypes.Structure):
    """Mirror of ``ddh_params`` (field order and types must match include/ddh.h)."""
    _fields_ = [
        ("n", c_int),
        ("aperture_diam", c_float),
        ("lam", c_float),
        ("alpha", c_float),
        ("n_k", c_int),
        ("noise_var", c_float),
        ("prior_p", c_float),
        ("prior_q", c_float),
        ("prior_T", c_float),
        ("prior_sigma", c_float),
        ("r_floor", c_float),
        ("tilt_mode", c_int),
        ("phase_block", c_int),
        ("phase_prior", c_float),
        ("phase_sweeps", c_int),
        ("noise_update", c_int),
        ("exec_path", c_int),
    ]


class DdhCompletion(ctypes.Structure):
    """Mirror of ``ddh_completion``."""
    _fields_ = [
        ("tag", ctypes.c_uint64),
        ("sensor", c_int),
        ("frame_index", c_int64),
        ("arrival_s", ctypes.c_double),
        ("done_s", ctypes.c_double),
    ]


class DdhSchedSensor(ctypes.Structure):
    """Mirror of ``ddh_sched_sensor``."""
    _fields_ = [("queued", c_int), ("oldest_arrival_s", ctypes.c_double)]


DDH_SCHED_BACKLOG = 1
DDH_SCHED_AGE = 2


class DdhError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(what)


_SIGS = {
    "ddh_default_params": (c_int, [POINTER(DdhParams), c_int, c_float, c_float]),
    "ddh_static_params": (c_int, [POINTER(DdhParams), c_int, c_float, c_float, c_int]),
    "ddh_tracking_params": (c_int, [POINTER(DdhParams), c_int, c_float, c_float]),
    "ddh_init": (c_int, [POINTER(c_void_p), POINTER(DdhParams), c_void_p]),
    "ddh_step": (c_int, [c_void_p, c_void_p]),
    "ddh_step_trace": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ddh_trace_floats": (c_size_t, [c_int]),
    "ddh_step_host": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ddh_phase": (c_int, [c_void_p, c_void_p]),
    "ddh_reflectance": (c_int, [c_void_p, c_void_p]),
    "ddh_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_int64]),
    "ddh_frame_index": (c_int64, [c_void_p]),
    "ddh_set_params": (c_int, [c_void_p, POINTER(DdhParams)]),
    "ddh_noise_estimate": (c_int, [c_void_p, POINTER(c_float)]),
    "ddh_selftest_wait": (c_int, [c_void_p, ctypes.c_double]),
    "ddh_state_stream": (c_void_p, [c_void_p]),
    "ddh_step_host_async": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ddh_host_wait": (c_int, [c_void_p, c_int64]),
    "ddh_strehl": (c_int, [c_void_p, c_void_p, POINTER(c_float)]),
    "ddh_step_batch": (c_int, [POINTER(c_void_p), POINTER(c_void_p), c_int]),
    "ddh_batch_create": (c_int, [POINTER(c_void_p), POINTER(c_void_p), c_int]),
    "ddh_batch_run": (c_int, [c_void_p, POINTER(c_void_p)]),
    "ddh_batch_free": (c_int, [c_void_p]),
    "ddh_service_create": (c_int, [POINTER(c_void_p), c_void_p, c_size_t, c_int, ctypes.c_uint]),
    "ddh_state_bytes": (c_size_t, [c_int]),
    "ddh_service_admit": (c_int, [c_void_p, c_int, POINTER(DdhParams)]),
    "ddh_service_release": (c_int, [c_void_p, c_int]),
    "ddh_service_state": (c_void_p, [c_void_p, c_int]),
    "ddh_service_submit": (c_int, [c_void_p, c_int, c_void_p, ctypes.c_double, ctypes.c_uint64]),
    "ddh_service_poll": (c_int, [c_void_p, POINTER(DdhCompletion), c_int, POINTER(c_int)]),
    "ddh_service_pending": (c_int64, [c_void_p]),
    "ddh_service_stats": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64), POINTER(c_size_t)]),
    "ddh_service_now": (ctypes.c_double, []),
    "ddh_sched_pick": (c_int, [POINTER(DdhSchedSensor), c_int, c_int, c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_uint, POINTER(ctypes.c_ubyte)]),
    "ddh_service_set_policy": (c_int, [c_void_p, ctypes.c_uint, ctypes.c_double]),
    "ddh_service_start": (c_int, [c_void_p]),
    "ddh_service_stop": (c_int, [c_void_p]),
    "ddh_service_free": (c_int, [c_void_p]),
    "ddh_backward_workspace_bytes": (c_size_t, [c_int]),
    "ddh_unrolled_workspace_bytes": (c_size_t, [c_int]),
    "ddh_unrolled_forward": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ddh_unrolled_backward": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_void_p, c_size_t]),
    "ddh_step_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p, c_size_t]),
    "ddh_step_backward_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_void_p, c_void_p]),
    "ddh_fft_schedule_count": (c_int, [c_int]),
    "ddh_set_fft_schedule": (c_int, [c_int, c_int]),
    "ddh_get_fft_schedule": (c_int, [c_int]),
    "ddh_set_staged_chunk": (c_int, [c_int, c_int]),
    "ddh_get_staged_chunk": (c_int, [c_int]),
    "ddh_set_staged_persistent": (c_int, [c_int]),
    "ddh_get_staged_persistent": (c_int, []),
    "ddh_fft2": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "ddh_sync": (c_int, [c_void_p]),
    "ddh_checkpoint_bytes": (c_size_t, [c_int]),
    "ddh_save": (c_int, [c_void_p, c_void_p, c_size_t]),
    "ddh_load": (c_int, [c_void_p, c_void_p, c_size_t]),
    "ddh_free": (c_int, [c_void_p]),
    "ddh_strerror": (c_char_p, [c_int]),
    "ddh_last_cuda_error": (c_char_p, []),
    "ddh_version": (c_int, []),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libddh.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2305_03284_gb300.build.build()")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def check(code: int) -> int:
    if code != DDH_OK:
        h = lib()
        msg = h.ddh_strerror(code).decode()
        if code == DDH_ECUDA or code == DDH_ENOMEM:
            msg += f" ({h.ddh_last_cuda_error().decode()})"
        raise DdhError(code, f"libddh error {code}: {msg}")
    return code
