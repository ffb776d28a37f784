"""ctypes wrapper around the plain C RHSEG/HSEG oracle (rhseg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check of
__graft_entry__ and by the CPU-baseline leg of bench.py.  The library under
paper_2106_12942_b300/ never imports it, and it never imports the library.

Every function here only marshals arguments; the arithmetic (Eq. 1, the
HSEG steps of Section 4.1, RHSEG's recursion and the seam pass) lives in the
C file, which documents the readings it implements.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rhseg_oracle.c")
_SO = os.path.join(_HERE, "_rhseg_oracle.so")

ORC_OK, ORC_EINVAL, ORC_ERANGE, ORC_ENOMEM = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math: IEEE semantics kept)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        compile_source(_SRC, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [
        ("rnb_levels", C.c_int32),
        ("conv_nregions", C.c_int32),
        ("spclust_wght", C.c_double),
        ("connectivity", C.c_int32),
        ("min_nregions", C.c_int32),
        ("n_out_levels", C.c_int32),
        ("seam_pass", C.c_int32),
        ("mode", C.c_int32),
        ("full_adjacency", C.c_int32),
        ("multi_merge", C.c_int32),
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
        ("stalled_sections", C.c_int32), ("n_levels_out", C.c_int32),
    ]


MERGE_DTYPE = np.dtype([
    ("level", "<i4"), ("section", "<i4"), ("step", "<i4"), ("kind", "<i4"),
    ("survivor_id", "<i8"), ("absorbed_id", "<i8"),
    ("key", "<f8"), ("dissim", "<f8"),
    ("nregions_after", "<i4"), ("pad", "<i4"),
])
assert MERGE_DTYPE.itemsize == C.sizeof(Merge)

def compile_source(src: str, so: str) -> str:
    """Compile an oracle source file to a shared object (used by build() and
    by the mutation tests, which compile edited copies)."""
    tmp = so + f".{os.getpid()}.tmp"
    subprocess.check_call(
        ["gcc", "-O2", "-std=gnu11", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC", "-pthread",
         "-o", tmp, src, "-lm"])
    os.replace(tmp, so)
    return so


def load(so_path: str):
    """Bind the C entry points of an oracle shared object."""
    L = C.CDLL(so_path)
    L.orc_div_rn.restype = C.c_double
    L.orc_div_rn.argtypes = [C.c_uint64] * 4
    L.orc_key.restype = C.c_double
    L.orc_key.argtypes = [C.c_int64, C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_int64), C.c_int32]
    L.orc_run.restype = C.c_void_p
    L.orc_run.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                          C.POINTER(Params), C.POINTER(C.c_int32)]
    L.orc_run_threads.restype = C.c_void_p
    L.orc_run_threads.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                  C.POINTER(Params), C.c_int32, C.POINTER(C.c_int32)]
    L.orc_log_len.restype = C.c_int64
    L.orc_log_len.argtypes = [C.c_void_p]
    L.orc_get_log.restype = None
    L.orc_get_log.argtypes = [C.c_void_p, C.c_void_p]
    L.orc_n_levels.restype = C.c_int32
    L.orc_n_levels.argtypes = [C.c_void_p]
    L.orc_level_nregions.restype = C.c_int32
    L.orc_level_nregions.argtypes = [C.c_void_p, C.c_int32]
    L.orc_get_level.restype = C.c_int32
    L.orc_get_level.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    L.orc_get_stats.restype = None
    L.orc_get_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
    L.orc_free.restype = None
    L.orc_free.argtypes = [C.c_void_p]
    L.orc_hseg_leaf.restype = C.c_int32
    L.orc_hseg_leaf.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                C.POINTER(Params), C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                                C.POINTER(C.c_int64), C.POINTER(Stats)]
    return L


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def div_rn(N: int, D: int, L=None) -> float:
    """Correctly rounded binary64 of N / D for 0 <= N, D < 2^128 (reading R1)."""
    m = (1 << 64) - 1
    return (L or lib()).orc_div_rn(N >> 64, N & m, D >> 64, D & m)


def key(ni: int, Si, nj: int, Sj, L=None) -> float:
    """K = d^2 of Eq. 1 from band sums Si, Sj (int64) and pixel counts."""
    a = np.ascontiguousarray(Si, dtype=np.int64)
    b = np.ascontiguousarray(Sj, dtype=np.int64)
    P = C.POINTER(C.c_int64)
    return (L or lib()).orc_key(ni, a.ctypes.data_as(P), nj, b.ctypes.data_as(P), len(a))


@dataclass
class Level:
    labels: np.ndarray   # [rows, cols] int32, 0 = masked, 1..R canonical
    sums: np.ndarray     # [R, bands] int64
    counts: np.ndarray   # [R] int64


@dataclass
class Result:
    log: np.ndarray      # structured MERGE_DTYPE
    levels: list
    stats: dict


def _params(**kw) -> Params:
    p = Params()
    p.rnb_levels = kw.get("rnb_levels", 1)
    p.conv_nregions = kw.get("conv_nregions", 1)
    p.spclust_wght = kw.get("spclust_wght", 0.0)
    p.connectivity = kw.get("connectivity", 8)
    p.min_nregions = kw.get("min_nregions", 0)
    p.n_out_levels = kw.get("n_out_levels", 1)
    p.seam_pass = kw.get("seam_pass", 1)
    p.mode = kw.get("mode", 1)
    p.full_adjacency = kw.get("full_adjacency", 0)
    p.multi_merge = kw.get("multi_merge", 0)
    return p


def _stats_dict(st: Stats) -> dict:
    return {f: getattr(st, f) for f, _ in Stats._fields_}


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}")
        self.code = code


def run(image: np.ndarray, mask: np.ndarray | None = None, L=None, threads: int = 1, **kw) -> Result:
    """Full RHSEG run.  image: uint16 [rows, cols, bands]; mask: [rows, cols]
    nonzero = no data.  Keyword parameters as in Params (mode 1 = cached keys,
    0 = every key recomputed each iteration).  threads > 1 runs the
    independent sections of each level on that many threads; the result is
    the same for every thread count."""
    img = np.ascontiguousarray(image, dtype=np.uint16)
    rows, cols, bands = img.shape
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    p = _params(**kw)
    err = C.c_int32(0)
    L = L or lib()
    if threads == 1:
        h = L.orc_run(img.ctypes.data, rows, cols, bands, None if mk is None else mk.ctypes.data,
                      C.byref(p), C.byref(err))
    else:
        h = L.orc_run_threads(img.ctypes.data, rows, cols, bands, None if mk is None else mk.ctypes.data,
                              C.byref(p), int(threads), C.byref(err))
    if not h:
        raise OracleError(err.value)
    try:
        n = L.orc_log_len(h)
        log = np.zeros(n, dtype=MERGE_DTYPE)
        if n:
            L.orc_get_log(h, log.ctypes.data)
        levels = []
        for k in range(L.orc_n_levels(h)):
            R = L.orc_level_nregions(h, k)
            lab = np.zeros((rows, cols), dtype=np.int32)
            sums = np.zeros((max(R, 0), bands), dtype=np.int64)
            cnt = np.zeros(max(R, 0), dtype=np.int64)
            L.orc_get_level(h, k, lab.ctypes.data, sums.ctypes.data, cnt.ctypes.data)
            levels.append(Level(lab, sums, cnt))
        st = Stats()
        L.orc_get_stats(h, C.byref(st))
        return Result(log, levels, _stats_dict(st))
    finally:
        L.orc_free(h)


def hseg_leaf(image: np.ndarray, mask: np.ndarray | None, section: int, max_iters: int = 0,
              L=None, **kw) -> Result:
    """HSEG of one deepest-level section alone (pixels as regions), at most
    max_iters iterations (0 = to its target)."""
    img = np.ascontiguousarray(image, dtype=np.uint16)
    rows, cols, bands = img.shape
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    p = _params(**kw)
    L = L or lib()
    n = C.c_int64(0)
    st = Stats()
    rc = L.orc_hseg_leaf(img.ctypes.data, rows, cols, bands, None if mk is None else mk.ctypes.data,
                         C.byref(p), section, max_iters, None, 0, C.byref(n), C.byref(st))
    if rc:
        raise OracleError(rc)
    # second call with a buffer of the right size
    log = np.zeros(n.value, dtype=MERGE_DTYPE)
    rc = L.orc_hseg_leaf(img.ctypes.data, rows, cols, bands, None if mk is None else mk.ctypes.data,
                         C.byref(p), section, max_iters, log.ctypes.data, n.value, C.byref(n), C.byref(st))
    if rc:
        raise OracleError(rc)
    return Result(log, [], _stats_dict(st))
