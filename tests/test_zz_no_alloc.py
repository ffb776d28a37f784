"""rhseg_get_level_noalloc: hierarchy levels read out without any device
allocation, for callers that must not allocate device memory once running
(a fixed memory budget reserved at start-up, or a host framework whose
allocator owns the whole device).  Its results must equal those of
rhseg_get_level, call after call, since every call shares one fixed working
array inside the library.

This file is collected last on purpose; it also passes when run alone in a
fresh process."""
import ctypes as C
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2106_12942_b300 as P
    return P


def _noalloc(P, seg, level, cap, want=("labels", "sums", "counts")):
    """One call with the requested outputs (the others passed as NULL).  The
    buffers are filled with -7 on torch's stream first; the library runs on
    the handle's own stream, so torch's fill is completed before the call,
    as the header asks of every caller."""
    import torch
    from paper_2106_12942_b300 import _abi
    L = _abi.load()
    rows, cols, bands = seg.shape
    lab = torch.full((rows, cols), -7, dtype=torch.int32, device="cuda")
    sums = torch.full((max(cap, 1), bands), -7, dtype=torch.int64, device="cuda")
    cnt = torch.full((max(cap, 1),), -7, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    R = C.c_int32(-1)

    def ptr(name, t):
        return C.c_void_p(t.data_ptr()) if name in want else None

    rc = L.rhseg_get_level_noalloc(seg._h, level, ptr("labels", lab), ptr("sums", sums), ptr("counts", cnt), cap,
                                   C.byref(R))
    return rc, R.value, lab.cpu().numpy(), sums.cpu().numpy(), cnt.cpu().numpy()


def test_noalloc_levels_equal_get_level_twice(P):
    img, mask = synth.make(4, seed=31, rows=72, cols=60)
    img = np.ascontiguousarray(img[:, :, :20])
    seg = P.RHSEG(img, mask, rnb_levels=3, spclust_wght=0.3, conv_nregions=5, n_out_levels=4, precision=3)
    seg.run()
    n = seg.n_levels()
    assert n >= 2
    want = [seg.level(k) for k in range(n)]      # rhseg_get_level (which allocates), before counting
    allocs0 = seg.stats()["device_allocs"]
    order = list(range(n)) + list(reversed(range(n)))    # every level, then again in the other order
    for _call in range(2):
        for k in order:
            lab, sums, cnt = want[k]
            R = len(cnt)
            rc, Rn, labn, sumsn, cntn = _noalloc(P, seg, k, R + 3)
            assert rc == 0
            assert Rn == R
            assert np.array_equal(labn, lab)
            assert np.array_equal(sumsn[:R], sums)
            assert np.array_equal(cntn[:R], cnt)
            assert np.all(cntn[R:] == -7)          # nothing written past R
            assert np.all(sumsn[R:] == -7)
    # one table only, and labels only (the other outputs NULL)
    k = n // 2
    lab, sums, cnt = want[k]
    R = len(cnt)
    rc, Rn, labn, sumsn, cntn = _noalloc(P, seg, k, R, want=("sums",))
    assert rc == 0 and Rn == R and np.array_equal(sumsn[:R], sums)
    assert np.all(labn == -7) and np.all(cntn == -7)
    rc, Rn, labn, sumsn, cntn = _noalloc(P, seg, k, R, want=("counts",))
    assert rc == 0 and Rn == R and np.array_equal(cntn[:R], cnt)
    assert np.all(labn == -7) and np.all(sumsn == -7)
    rc, Rn, labn, sumsn, cntn = _noalloc(P, seg, k, 0, want=("labels",))
    assert rc == 0 and Rn == R and np.array_equal(labn, lab)
    rc, Rn, labn, sumsn, cntn = _noalloc(P, seg, k, 0, want=())
    assert rc == 0 and Rn == R and np.all(labn == -7)
    # a too-small table buffer: RHSEG_ETRUNC, R still reported, nothing written
    lab, sums, cnt = want[n - 1]
    rc, Rn, labn, sumsn, cntn = _noalloc(P, seg, n - 1, len(cnt) - 1)
    assert rc == -7 and Rn == len(cnt)
    assert np.all(labn == -7) and np.all(sumsn == -7) and np.all(cntn == -7)
    # none of these calls allocated device memory in the library
    assert seg.stats()["device_allocs"] == allocs0
    seg.close()


def test_noalloc_rejects_roots_beyond_its_limit(P):
    from paper_2106_12942_b300 import _abi
    rows, cols = 260, 260                          # 67600 one-pixel regions stay at the root
    assert rows * cols > _abi.RHSEG_NOALLOC_MAX_REGIONS
    img = np.random.default_rng(1).integers(0, 50, (rows, cols, 2)).astype(np.uint16)
    seg = P.RHSEG(img, None, rnb_levels=1, conv_nregions=rows * cols, precision=3)
    seg.run()
    rc, _, _, _, _ = _noalloc(P, seg, 0, 10)
    assert rc == -2                                # RHSEG_ERANGE
    L = _abi.load()
    assert b"at most 65536" in L.rhseg_last_cuda_error()
    seg.close()
