"""Parity of the incremental spectral minima (params incremental=1) with the
CPU oracle.

The mode keeps every region's exact best non-adjacent partner and recomputes
only the rows a merge touches, so its merge log, labels, sums and counts
must be those of the all-pairs method (the oracle) bit for bit.  Cases: the
worked example, the brute-force tie cases, the piecewise scenes (several
64-position tiles, ragged tails, masks, 4- and 8-connectivity), the
32x32x16 and 145x145x200 workloads in full, and sampled sections of the
1024x1024x224 workload, whose whole log must also equal the all-pairs
tensor-core run's."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import synth  # noqa: E402
from test_gpu_parity import SCENES, _assert_same  # noqa: E402
from test_oracle_pins import BRUTE_CASES  # noqa: E402

pytestmark = pytest.mark.gpu

INC_PRECISIONS = [3]          # the mode evaluates binary32 rows


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2106_12942_b300 as P
    return P


def _run(P, img, mask, **kw):
    seg = P.RHSEG(img, mask, incremental=1, **kw)
    seg.run()
    return seg


@pytest.mark.parametrize("precision", INC_PRECISIONS)
def test_inc_worked_example(P, orc, precision):
    img = np.array([0, 100, 200, 1], dtype=np.uint16).reshape(1, 4, 1)
    for w in (1.0, 0.5, 0.0):
        kw = dict(rnb_levels=1, conv_nregions=1, spclust_wght=w, connectivity=4)
        _assert_same(_run(P, img, None, precision=precision, **kw), orc.run(img, None, **kw), f"w={w}")


@pytest.mark.parametrize("precision", INC_PRECISIONS)
def test_inc_tiny_cases_with_ties(P, orc, precision):
    for ci, case in enumerate(BRUTE_CASES):
        rows, cols, B, maxval, mask_p, L, w, conv, conn, min_nr, n_out, seam = case
        for seed in (1, 2, 3):
            img, mask = synth.random_cube(seed * 101 + rows * 7 + cols, rows, cols, B, maxval, mask_p)
            kw = dict(rnb_levels=L, spclust_wght=w, conv_nregions=conv, connectivity=conn,
                      min_nregions=min_nr, n_out_levels=n_out, seam_pass=seam)
            _assert_same(_run(P, img, mask, precision=precision, **kw), orc.run(img, mask, **kw), f"case {ci} s{seed}")


@pytest.mark.parametrize("precision", INC_PRECISIONS)
@pytest.mark.parametrize("si", range(len(SCENES)))
def test_inc_piecewise_scenes(P, orc, precision, si):
    rows, cols, B, L, w, conv, conn, min_nr, n_out, seam, masked = SCENES[si]
    img, mask = synth.make(4 if masked else 2, seed=400 + si, rows=rows, cols=cols)
    img = np.ascontiguousarray(img[:, :, :B])
    kw = dict(rnb_levels=L, spclust_wght=w, conv_nregions=conv, connectivity=conn, min_nregions=min_nr,
              n_out_levels=n_out, seam_pass=seam)
    _assert_same(_run(P, img, mask, precision=precision, **kw), orc.run(img, mask, **kw), f"scene {si}")


def test_inc_workload_hseg_32x32x16(P, orc):
    w = synth.WORKLOADS[1]
    img, mask = synth.make(1)
    kw = {k: v for k, v in w.params.items() if k != "precision"}
    for precision in INC_PRECISIONS:
        _assert_same(_run(P, img, mask, precision=precision, **kw), orc.run(img, mask, **kw), f"32x32x16 p{precision}")


def test_inc_edge_cases(P, orc):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 100, (5, 7, 3)).astype(np.uint16)
    m = np.zeros((5, 7), np.uint8)
    m[:, 3] = 1
    m[2, :] = 1
    cases = [
        (img, np.ones((5, 7), np.uint8), dict(rnb_levels=2, conv_nregions=2, spclust_wght=0.5)),   # all masked
        (img[:1, :1], None, dict(rnb_levels=1, conv_nregions=1, spclust_wght=0.5)),                # one pixel
        (img, None, dict(rnb_levels=6, conv_nregions=3, spclust_wght=0.5)),                        # empty sections
        (img[:1], None, dict(rnb_levels=3, conv_nregions=1, spclust_wght=1.0)),                    # 1-row image
        (img, m, dict(rnb_levels=1, conv_nregions=1, spclust_wght=0.7)),                           # isolated parts
        (np.full((6, 6, 2), 65535, np.uint16), None, dict(rnb_levels=2, conv_nregions=1, spclust_wght=1.0)),
    ]
    for i, (im, mk, kw) in enumerate(cases):
        for precision in INC_PRECISIONS:
            _assert_same(_run(P, im, mk, precision=precision, **kw), orc.run(im, mk, **kw), f"edge {i} p{precision}")


def test_inc_rejects_other_row_forms(P):
    from paper_2106_12942_b300.rhseg import RHSEGError
    img = np.zeros((4, 4, 2), np.uint16)
    for precision in (0, 1, 2):
        with pytest.raises(RHSEGError):
            P.RHSEG(img, None, precision=precision, incremental=1, spclust_wght=0.5)


def test_inc_rhseg_145x145x200(P, orc):
    img, mask = synth.make(2)
    kw = {k: v for k, v in synth.WORKLOADS[2].params.items() if k != "precision"}
    ref = orc.run(img, mask, **kw)
    _assert_same(_run(P, img, mask, precision=3, **kw), ref, "145x145x200 incremental")


def test_inc_rhseg_1024x1024x224(P, orc):
    img, mask = synth.make(4)
    kw = dict(synth.WORKLOADS[4].params)
    seg = _run(P, img, mask, **dict(kw, precision=3))
    full = P.RHSEG(img, mask, **kw)
    full.run()
    a, b = seg.log(), full.log()
    assert len(a) == len(b)
    for f in ["level", "section", "step", "kind", "survivor_id", "absorbed_id", "nregions_after"]:
        assert np.array_equal(a[f], b[f]), f
    assert np.array_equal(a["key"].view(np.uint64), b["key"].view(np.uint64))
    for k in range(seg.n_levels()):
        la, sa, ca = seg.level(k)
        lb, sb, cb = full.level(k)
        assert np.array_equal(la, lb) and np.array_equal(sa, sb) and np.array_equal(ca, cb)
    assert seg.stats()["pairs"] == full.stats()["pairs"]
    L = kw["rnb_levels"]
    okw = {k: v for k, v in kw.items() if k != "precision"}
    for s in (0, 255):
        ref = orc.hseg_leaf(img, mask, s, max_iters=150, **okw)
        part = a[(a["level"] == L) & (a["section"] == s)][:len(ref.log)]
        assert len(ref.log) > 0
        for f in ["step", "kind", "survivor_id", "absorbed_id", "nregions_after"]:
            assert np.array_equal(part[f], ref.log[f]), (s, f)
        assert np.array_equal(part["key"].view(np.uint64), ref.log["key"].view(np.uint64)), s
