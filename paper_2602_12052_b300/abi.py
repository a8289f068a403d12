"""ctypes binding of libtred's C ABI (include/tred.h): argument marshalling only.

Every function here forwards to the entry point of the same name; all work runs in
the library's CUDA kernels.  There is no CPU fallback: loading fails loudly when
libtred.so is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtred.so")

TRED_OK = 0
TRED_ERR_INVALID_ARG = 1
TRED_ERR_CUDA = 2
TRED_ERR_CAPACITY = 3
TRED_ERR_TIMEOUT = 4
TRED_ERR_NOT_READY = 5

TRED_ST_BLOCK_OVERFLOW = 1 << 0
TRED_ST_PAIR_OVERFLOW = 1 << 1
TRED_ST_PIXEL_OVERFLOW = 1 << 2
TRED_ST_HIT_OVERFLOW = 1 << 3
TRED_ST_DRIFT_RANGE = 1 << 4
TRED_ST_TIMEOUT = 1 << 5
TRED_STATUS_WORDS = 8

# every symbol include/tred.h declares
EXPORTS = [
    "tred_create", "tred_destroy", "tred_last_error", "tred_sync_status", "tred_reset_status",
    "tred_set_response", "tred_drift", "tred_blockbin", "tred_effq", "tred_convolve",
    "tred_gather_pixels", "tred_readout", "tred_launch_count", "tred_set_kernel_timing", "tred_kernel_time", "tred_direct_counts",
    "tred_blockbin_noalloc",
    "tred_set_transport", "tred_residual", "tred_adjoint", "tred_param_grads",
    "tred_drift_events", "tred_effq_range", "tred_convolve_range", "tred_drift_lines", "tred_effq_lines",
    "tred_wait_selftest", "tred_gather_readout", "tred_fp32_peak", "tred_effq_convolve",
    "tred_convolve_gather_readout", "tred_convolve_gather_supported", "tred_convolve_spectra_range",
    "tred_wave_gather_readout",
]


class Geometry(ctypes.Structure):
    _fields_ = [("pitch_cm", ctypes.c_float), ("n_sub", ctypes.c_int32), ("tick_us", ctypes.c_float),
                ("npx_x", ctypes.c_int32), ("npx_y", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("bp", ctypes.c_int32), ("bt", ctypes.c_int32), ("kp", ctypes.c_int32),
                ("nr", ctypes.c_int32), ("lt", ctypes.c_int32), ("n_events", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("v_cm_per_us", ctypes.c_float), ("DL_cm2_per_s", ctypes.c_float),
                ("DT_cm2_per_s", ctypes.c_float), ("lifetime_us", ctypes.c_float),
                ("sigma0_cells_xy", ctypes.c_float), ("sigma0_ticks", ctypes.c_float),
                ("nsigma", ctypes.c_float), ("max_drift_cm", ctypes.c_float),
                ("gl_order", ctypes.c_int32), ("effq_mode", ctypes.c_int32),
                ("conv_mode", ctypes.c_int32), ("mpcp", ctypes.c_int32),
                ("compensated_gather", ctypes.c_int32), ("effq_skip_empty", ctypes.c_int32),
                ("conv_rows_cap", ctypes.c_int32), ("conv_keep_spectra", ctypes.c_int32)]


class ReadoutParams(ctypes.Structure):
    _fields_ = [("threshold_e", ctypes.c_float), ("clock_ticks", ctypes.c_int32),
                ("hold_ticks", ctypes.c_int32), ("reset_ticks", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("n_samples", ctypes.c_int32)]


DEPOSIT_FIELDS = ["cell_x", "cell_y", "cell_t", "frac_x", "frac_y", "frac_t", "sigma_x", "sigma_y",
                  "sigma_t", "lo_x", "lo_y", "lo_t", "hi_x", "hi_y", "hi_t", "q"]


class Deposits(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in DEPOSIT_FIELDS]


_P = ctypes.c_void_p
_I = ctypes.c_int32
_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libtred.so (raises OSError if it is missing: no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libtred.so not built at {p}; run paper_2602_12052_b300.build.build()")
    lib = ctypes.CDLL(p)
    lib.tred_create.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(Params), _I, _I, _I,
                                ctypes.POINTER(_P)]
    lib.tred_destroy.argtypes = [_P]
    lib.tred_last_error.argtypes = [_P]
    lib.tred_last_error.restype = ctypes.c_char_p
    lib.tred_sync_status.argtypes = [_P, _P, _P]
    lib.tred_reset_status.argtypes = [_P, _P]
    lib.tred_launch_count.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
    lib.tred_set_kernel_timing.argtypes = [_P, ctypes.c_int32]
    lib.tred_direct_counts.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.tred_kernel_time.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int32)]
    lib.tred_wait_selftest.argtypes = [_P, ctypes.c_int64, _P]
    lib.tred_gather_readout.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(ReadoutParams), _P, _P, _P, _P,
                                        _I, _P]
    lib.tred_convolve_gather_readout.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(ReadoutParams), _P, _P,
                                                 _P, _P, _I, _P]
    lib.tred_convolve_gather_supported.argtypes = [_P]
    lib.tred_convolve_spectra_range.argtypes = [_P, _P, _P, _I, _I, _P, _P]
    lib.tred_wave_gather_readout.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.POINTER(ReadoutParams), _P, _P, _P, _P,
                                             _I, _P]
    lib.tred_set_response.argtypes = [_P, _P, _P]
    lib.tred_drift.argtypes = [_P, _I, _P, _P, _P, _P, _P, ctypes.POINTER(Deposits), _P]
    lib.tred_blockbin.argtypes = [_P, _I, ctypes.POINTER(Deposits), _P, _P, _P, _P, _I, _P, _P]
    lib.tred_effq.argtypes = [_P, _I, ctypes.POINTER(Deposits), _P, _P, _P, _P, _P, _P]
    lib.tred_convolve.argtypes = [_P, _P, _P, _P, _P, _P]
    lib.tred_gather_pixels.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P]
    lib.tred_readout.argtypes = [_P, ctypes.POINTER(ReadoutParams), _P, _P, _P, _P, _P, _P, _P, _I, _P]
    lib.tred_drift_events.argtypes = [_P, _I, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Deposits), _P]
    lib.tred_effq_range.argtypes = [_P, _I, ctypes.POINTER(Deposits), _P, _P, _P, _P, _I, _I, _P, _P]
    lib.tred_convolve_range.argtypes = [_P, _P, _P, _I, _I, _P, _P, _P]
    lib.tred_set_transport.argtypes = [_P, ctypes.POINTER(Params)]
    lib.tred_drift_lines.argtypes = [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Deposits), _P, _P]
    lib.tred_effq_lines.argtypes = [_P, _I, ctypes.POINTER(Deposits), _P, _P, _P, _P, _P, _P, _P]
    lib.tred_residual.argtypes = [_P, _P, _P, _P, _P, _I, _P, _P, _P, _P]
    lib.tred_adjoint.argtypes = [_P, _I, ctypes.POINTER(Deposits), _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
    lib.tred_param_grads.argtypes = [_P, _I, _P, ctypes.POINTER(Deposits), _P, _P, _P, _P]
    lib.tred_effq_convolve.argtypes = [_P, _I, ctypes.POINTER(Deposits), _P, _P, _P, _P, _P, _I, _P, _P]
    lib.tred_fp32_peak.argtypes = [_P, ctypes.c_int64, _I, _P, _P, _P]
    lib.tred_blockbin_noalloc.argtypes = [ctypes.POINTER(Geometry), _I, ctypes.POINTER(Deposits), _P, _P, _P,
                                          _P, _I, _I, _P, _P, _P]
    for name in EXPORTS:
        if name not in ("tred_last_error",):
            getattr(lib, name).restype = ctypes.c_int32
    if path is None:
        _lib = lib
    return lib


class TredError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtred error {code}: {msg}")
        self.code = code
