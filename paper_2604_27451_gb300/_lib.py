"""ctypes binding of libcvsadc (the C ABI declared in include/cvsadc.h).

Argument marshalling only: every computation runs inside the library's
CUDA kernels.  If the shared library is missing this module raises on
import -- there is no fallback of any kind.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcvsadc.so")

CVSADC_OK = 0
CVSADC_EINVAL = -1
CVSADC_ENONHERM = -2
CVSADC_ENOMEM = -3
CVSADC_ECUDA = -4
CVSADC_ETIMEOUT = -5
CVSADC_ESTATE = -6
CVSADC_ENOTCONV = 1

CVSADC_FP64 = 0
CVSADC_MIXED_BF16X3 = 1
CVSADC_MIXED_SLICE4 = 2
CVSADC_FP64_SLICE7 = 3

CVSADC_FLAG_DEVICE_PTRS = 1
CVSADC_FLAG_RETURN_X = 2
CVSADC_FLAG_NO_REFINE = 4
CVSADC_FLAG_DIAG_PRECOND = 8
CVSADC_FLAG_FOLDED = 16


class Params(ctypes.Structure):
    _fields_ = [
        ("ncore", ctypes.c_int32), ("nval", ctypes.c_int32),
        ("nvirt", ctypes.c_int32), ("naux", ctypes.c_int32),
        ("nroots", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("fns_threshold", ctypes.c_double), ("conv_residual", ctypes.c_double),
        ("max_iter", ctypes.c_int32), ("max_subspace", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("refine_sweeps", ctypes.c_int32),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32), ("sigma_vectors", ctypes.c_int32),
        ("nvirt_kept", ctypes.c_int32), ("converged", ctypes.c_int32),
        ("emp2", ctypes.c_double), ("max_residual", ctypes.c_double),
        ("t_prepare_ms", ctypes.c_double), ("t_davidson_ms", ctypes.c_double),
        ("t_refine_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double),
        ("t_sigma_ms", ctypes.c_double), ("t_schur_ms", ctypes.c_double),
        ("schur_theta", ctypes.c_double), ("coupling_vectors", ctypes.c_int32),
        ("schur_builds", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_vp = ctypes.c_void_p
_SIGNATURES = {
    "cvsadc_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "cvsadc_destroy": (None, [_vp]),
    "cvsadc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "cvsadc_last_error": (ctypes.c_char_p, [_vp]),
    "cvsadc_solve": (ctypes.c_int, [_vp, ctypes.POINTER(Params), _vp, _vp, _vp,
                                    _vp, _vp, _vp, ctypes.POINTER(Info)]),
    "cvsadc_grad": (ctypes.c_int, [_vp, ctypes.POINTER(Params), _vp, _vp, _vp, _vp, _vp,
                                   _vp]),
    "cvsadc_solve_batched": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(Params),
                                            _vp, _vp, _vp, _vp, _vp, _vp,
                                            ctypes.POINTER(Info), _vp, ctypes.c_int32]),
    "cvsadc_estimate_bytes": (ctypes.c_int, [ctypes.POINTER(Params),
                                             ctypes.POINTER(ctypes.c_int64)]),
    "cvsadc_device_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "cvsadc_get_schur": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int32, _vp]),
    "cvsadc_prepare": (ctypes.c_int, [_vp, ctypes.POINTER(Params), _vp, _vp, _vp,
                                      ctypes.POINTER(Info)]),
    "cvsadc_prepared_sizes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64)]),
    "cvsadc_get_t2": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.POINTER(ctypes.c_double)]),
    "cvsadc_get_m11": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "cvsadc_get_fns": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp]),
    "cvsadc_get_moments": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "cvsadc_sigma": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                    ctypes.c_int32]),
    "cvsadc_davidson": (ctypes.c_int, [_vp, ctypes.POINTER(Params), _vp, _vp, _vp,
                                       ctypes.POINTER(Info)]),
    "cvsadc_zgemm_small_noalloc": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.c_int32, _vp, ctypes.c_int64,
                                                  _vp, ctypes.c_int64, _vp,
                                                  ctypes.c_int64]),
    "cvsadc_spectrum": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_double, _vp]),
    "cvsadc_block_dot": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int32, _vp,
                                        ctypes.c_int32, ctypes.c_int64, _vp]),
    "cvsadc_launch_count": (ctypes.c_int64, []),
    "cvsadc_kernel_timing": (None, [ctypes.c_int32]),
    "cvsadc_kernel_stats": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]),
    "cvsadc_kernel_stats_reset": (None, []),
    "cvsadc_wait_probe": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "cvsadc_zgemm": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int64,
                                    _vp, ctypes.c_int64, _vp, ctypes.c_int64]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libcvsadc.so and declare every exported entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            "libcvsadc.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_names():
    return list(_SIGNATURES)
