"""ctypes declarations of the C ABI in include/rhseg.h (argument marshalling
only; all computation runs in the CUDA library)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(HERE, "librhseg_b300.so")

RHSEG_OK, RHSEG_EINVAL, RHSEG_ERANGE, RHSEG_ENOMEM = 0, -1, -2, -3
RHSEG_ECUDA, RHSEG_ETIMEOUT, RHSEG_ESTATE, RHSEG_ETRUNC, RHSEG_EDEVICE = -4, -5, -6, -7, -8
RHSEG_NOALLOC_MAX_REGIONS = 65536


class Params(C.Structure):
    _fields_ = [
        ("rnb_levels", C.c_int32), ("conv_nregions", C.c_int32), ("spclust_wght", C.c_double),
        ("connectivity", C.c_int32), ("min_nregions", C.c_int32), ("n_out_levels", C.c_int32),
        ("seam_pass", C.c_int32), ("precision", C.c_int32), ("profile", C.c_int32), ("incremental", C.c_int32),
        ("multi_merge", C.c_int32), ("wait_cycles", C.c_int64), ("screen_group", C.c_int32),
        ("screen_pair", C.c_int32), ("adjacency", C.c_int32), ("reserved", C.c_int32),
    ]


class Merge(C.Structure):
    _fields_ = [
        ("level", C.c_int32), ("section", C.c_int32), ("step", C.c_int32), ("kind", C.c_int32),
        ("survivor_id", C.c_int64), ("absorbed_id", C.c_int64),
        ("key", C.c_double), ("dissim", C.c_double),
        ("nregions_after", C.c_int32), ("pad", C.c_int32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("pairs", C.c_int64), ("iterations", C.c_int64),
        ("merges_adj", C.c_int64), ("merges_spec", C.c_int64), ("seam_splits", C.c_int64),
        ("screened_pairs", C.c_int64), ("candidates", C.c_int64), ("fallbacks", C.c_int64),
        ("stalled_sections", C.c_int32), ("n_levels_out", C.c_int32),
        ("run_ms", C.c_double),
        ("kernel_launches", C.c_int64), ("candidates_below", C.c_int64), ("screen_launches", C.c_int64),
        ("screen_ms", C.c_double), ("adj_ms", C.c_double), ("spec_ms", C.c_double),
        ("screen_impl", C.c_int32), ("pad", C.c_int32),
        ("level_ms", C.c_double * 6), ("level_iters", C.c_int32 * 6),
        ("level_screen_ms", C.c_double * 6), ("level_adj_ms", C.c_double * 6), ("level_spec_ms", C.c_double * 6),
        ("screen_evaluated", C.c_int64), ("device_allocs", C.c_int64),
        ("screen_err_rel_max", C.c_double), ("screen_err_bound_max", C.c_double), ("screen_err_pairs", C.c_int64),
        ("level_screen_evaluated", C.c_int64 * 6), ("adjacency_bytes", C.c_int64),
        ("screen_useful", C.c_int64),
    ]


MERGE_DTYPE = np.dtype([
    ("level", "<i4"), ("section", "<i4"), ("step", "<i4"), ("kind", "<i4"),
    ("survivor_id", "<i8"), ("absorbed_id", "<i8"),
    ("key", "<f8"), ("dissim", "<f8"),
    ("nregions_after", "<i4"), ("pad", "<i4"),
])
assert MERGE_DTYPE.itemsize == C.sizeof(Merge) == 56

# every function declared in include/rhseg.h: name -> (restype, argtypes)
_VP = C.c_void_p
SIGNATURES = {
    "rhseg_create": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, _VP, C.POINTER(Params), _VP, C.POINTER(_VP)]),
    "rhseg_create_device": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, _VP, C.POINTER(Params), _VP,
                                      C.POINTER(_VP)]),
    "rhseg_run": (C.c_int, [_VP, _VP]),
    "rhseg_set_wait_cycles": (C.c_int, [_VP, C.c_int64]),
    "rhseg_set_image": (C.c_int, [_VP, _VP, _VP, _VP]),
    "rhseg_n_levels": (C.c_int, [_VP, C.POINTER(C.c_int32)]),
    "rhseg_get_level": (C.c_int, [_VP, C.c_int32, _VP, _VP, _VP, C.POINTER(C.c_int32)]),
    "rhseg_get_log": (C.c_int, [_VP, _VP, C.c_int64, C.POINTER(C.c_int64)]),
    "rhseg_get_level_noalloc": (C.c_int, [_VP, C.c_int32, _VP, _VP, _VP, C.c_int32, C.POINTER(C.c_int32)]),
    "rhseg_get_stats": (C.c_int, [_VP, C.POINTER(Stats)]),
    "rhseg_destroy": (None, [_VP]),
    "rhseg_strerror": (C.c_char_p, [C.c_int]),
    "rhseg_last_cuda_error": (C.c_char_p, []),
    "rhseg_keys": (C.c_int, [_VP, _VP, C.c_int32, C.c_int32, C.c_int32, _VP, _VP, C.c_int32, _VP, _VP]),
    "rhseg_div_rn": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int32, _VP, _VP]),
    "rhseg_gram_tc": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _VP, _VP]),
}

_lib = None


def load(path: str = SO_PATH):
    """Load the in-tree CUDA library; raise if it is missing (there is no
    fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run python -m paper_2106_12942_b300.build)")
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L
