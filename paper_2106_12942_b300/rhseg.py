"""Python binding of the B300 RHSEG library (argument marshalling only).

    seg = RHSEG(image, mask, rnb_levels=3, spclust_wght=0.2, conv_nregions=16)
    seg.run()
    labels, sums, counts = seg.level(seg.n_levels() - 1)
    log = seg.log()

`image` is uint16 [rows, cols, bands]; a numpy array goes through
rhseg_create (host buffers, copied to the device), a CUDA torch tensor
through rhseg_create_device (stays owned by the caller).

Keyword parameters mirror rhseg_params of include/rhseg.h (defaults in
DEFAULTS): rnb_levels, conv_nregions, spclust_wght, connectivity,
min_nregions, n_out_levels, seam_pass; precision (screen arithmetic, same
merges in every form: 1 FP16 tensor cores, 2 BF16 tensor cores, 3 FP32, 0
FP64); incremental (1: exact per-region spectral minima, precision 3 only,
same merges); multi_merge (1: all mutually best pairs per stage merge in one
iteration, a different rule with its own oracle mode); profile (1: per-kernel
CUDA-event times in stats()); wait_cycles (bound of the tensor-core screen's
pipeline waits in clock cycles, 0 = the default of about 2 s; a wait that
runs out makes run() raise RHSEGError with code RHSEG_ETIMEOUT); screen_group
(K slices per tcgen05.commit of the tensor-core screen, 0 = default) and
screen_pair (1: the tensor-core screen as CTA pairs sharing 256x256 tiles),
both chosen by the autotuner, results identical; adjacency (0: a bit matrix per
section, 1: sorted neighbour lists with memory in proportion to the edges;
results identical).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi

DEFAULTS = dict(rnb_levels=1, conv_nregions=1, spclust_wght=0.0, connectivity=8, min_nregions=0,
                n_out_levels=1, seam_pass=1, precision=1, profile=0, incremental=0,
                multi_merge=0, wait_cycles=0, screen_group=0, screen_pair=0,
                adjacency=0)


class RHSEGError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = _abi.load()
        msg = L.rhseg_strerror(code).decode()
        detail = L.rhseg_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({code})" + (f": {detail}" if detail and code == _abi.RHSEG_ECUDA else ""))
        self.code = code


def _check(rc: int, where: str):
    if rc != 0:
        raise RHSEGError(rc, where)


def make_params(**kw) -> _abi.Params:
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise TypeError(f"unknown parameters {sorted(unknown)}")
    d.update(kw)
    p = _abi.Params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class RHSEG:
    def __init__(self, image, mask=None, stream=None, **params):
        self._lib = _abi.load()
        self._h = C.c_void_p()
        self._keep = []
        p = make_params(**params)
        self.params = {f: getattr(p, f) for f, _ in _abi.Params._fields_}
        st = _stream_ptr(stream)
        if hasattr(image, "is_cuda") and image.is_cuda:
            import torch
            img = image.contiguous()
            if img.dtype != torch.uint16:
                raise TypeError("image must be uint16")
            rows, cols, bands = img.shape
            mk = None
            if mask is not None:
                mk = mask.to(device=img.device, dtype=torch.uint8).contiguous()
            self._keep = [img, mk]
            rc = self._lib.rhseg_create_device(C.c_void_p(img.data_ptr()), rows, cols, bands,
                                               None if mk is None else C.c_void_p(mk.data_ptr()),
                                               C.byref(p), st, C.byref(self._h))
            _check(rc, "rhseg_create_device")
        else:
            img = np.ascontiguousarray(image, dtype=np.uint16)
            rows, cols, bands = img.shape
            mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
            rc = self._lib.rhseg_create(img.ctypes.data, rows, cols, bands,
                                        None if mk is None else mk.ctypes.data, C.byref(p), st,
                                        C.byref(self._h))
            _check(rc, "rhseg_create")
        self.shape = (rows, cols, bands)

    def set_image(self, image, mask=None, stream=None):
        """Copy a new host image (same shape) into the handle; `image` may be a
        numpy array or a (pinned) CPU torch tensor."""
        ptr = image.data_ptr() if hasattr(image, "data_ptr") else np.ascontiguousarray(image, np.uint16).ctypes.data
        mptr = None
        if mask is not None:
            mptr = mask.data_ptr() if hasattr(mask, "data_ptr") else np.ascontiguousarray(mask, np.uint8).ctypes.data
        self._keep_host = (image, mask)
        _check(self._lib.rhseg_set_image(self._h, C.c_void_p(ptr), None if mptr is None else C.c_void_p(mptr),
                                         _stream_ptr(stream)), "rhseg_set_image")
        return self

    def set_wait_cycles(self, cycles: int):
        """Bound of the tensor-core screen's pipeline waits for the next runs
        (0 = the default)."""
        _check(self._lib.rhseg_set_wait_cycles(self._h, int(cycles)), "rhseg_set_wait_cycles")
        return self

    def run(self, stream=None):
        _check(self._lib.rhseg_run(self._h, _stream_ptr(stream)), "rhseg_run")
        return self

    def n_levels(self) -> int:
        n = C.c_int32()
        _check(self._lib.rhseg_n_levels(self._h, C.byref(n)), "rhseg_n_levels")
        return n.value

    def level(self, k: int, labels=True, tables=True):
        rows, cols, bands = self.shape
        R = C.c_int32()
        _check(self._lib.rhseg_get_level(self._h, k, None, None, None, C.byref(R)), "rhseg_get_level")
        lab = np.zeros((rows, cols), dtype=np.int32) if labels else None
        sums = np.zeros((R.value, bands), dtype=np.int64) if tables else None
        cnt = np.zeros(R.value, dtype=np.int64) if tables else None
        _check(self._lib.rhseg_get_level(self._h, k, None if lab is None else lab.ctypes.data,
                                         None if sums is None else sums.ctypes.data,
                                         None if cnt is None else cnt.ctypes.data, C.byref(R)),
               "rhseg_get_level")
        return lab, sums, cnt

    def log(self) -> np.ndarray:
        n = C.c_int64()
        _check(self._lib.rhseg_get_log(self._h, None, 0, C.byref(n)), "rhseg_get_log")
        out = np.zeros(n.value, dtype=_abi.MERGE_DTYPE)
        if n.value:
            _check(self._lib.rhseg_get_log(self._h, out.ctypes.data, n.value, C.byref(n)), "rhseg_get_log")
        return out

    def stats(self) -> dict:
        s = _abi.Stats()
        _check(self._lib.rhseg_get_stats(self._h, C.byref(s)), "rhseg_get_stats")
        out = {}
        for f, _ in _abi.Stats._fields_:
            v = getattr(s, f)
            out[f] = list(v) if hasattr(v, "__len__") else v
        return out

    def close(self):
        if self._h:
            self._lib.rhseg_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def keys(S, n, pair_i, pair_j, stream=None):
    """Exact keys K (Eq. 1 squared, correctly rounded) for region pairs, on
    CUDA torch tensors: S int64 [nreg, bands], n int64 [nreg], pair_i/pair_j
    int32 [npairs].  Returns float64 [npairs] on the device."""
    import torch
    L = _abi.load()
    S = S.contiguous()
    out = torch.empty(pair_i.numel(), dtype=torch.float64, device=S.device)
    _check(L.rhseg_keys(C.c_void_p(S.data_ptr()), C.c_void_p(n.data_ptr()), S.shape[0], S.shape[1], S.shape[1],
                        C.c_void_p(pair_i.data_ptr()), C.c_void_p(pair_j.data_ptr()), pair_i.numel(),
                        C.c_void_p(out.data_ptr()), _stream_ptr(stream)), "rhseg_keys")
    return out


def div_rn(n_hi, n_lo, d_hi, d_lo, stream=None):
    """Correctly rounded binary64 of 128-bit N / D (uint64 halves as int64
    CUDA tensors).  Returns float64 on the device."""
    import torch
    L = _abi.load()
    out = torch.empty(n_hi.numel(), dtype=torch.float64, device=n_hi.device)
    _check(L.rhseg_div_rn(C.c_void_p(n_hi.data_ptr()), C.c_void_p(n_lo.data_ptr()), C.c_void_p(d_hi.data_ptr()),
                          C.c_void_p(d_lo.data_ptr()), n_hi.numel(), C.c_void_p(out.data_ptr()),
                          _stream_ptr(stream)), "rhseg_div_rn")
    return out


def gram_tc(X, precision=1, stream=None, cta_pair=0):
    """G = X X^T (FP32) of 16-bit rows on the tensor cores (diagnostic of the
    screen's contraction, in the one-CTA or the CTA-pair form).  X: CUDA
    tensor float16/bfloat16 [rows, Bpad], rows % 128 == 0, Bpad % 32 == 0."""
    import torch
    L = _abi.load()
    X = X.contiguous()
    G = torch.empty(X.shape[0], X.shape[0], dtype=torch.float32, device=X.device)
    _check(L.rhseg_gram_tc(C.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], precision, int(cta_pair), C.c_void_p(G.data_ptr()),
                           _stream_ptr(stream)), "rhseg_gram_tc")
    return G
