"""Parity of the several-merges-per-iteration mode (params multi_merge = 1,
the reading of Section 6.2's idea) with the oracle's multi-merge mode.

The rule differs from the single-merge one, so the reference is the oracle
run with multi_merge = 1, which is pinned on CPU against an independent
brute force and a hand-derived example.  The bar is the same as for the
single-merge path: merge logs, labels, sums and counts identical.  Cases:
the hand-derived 1x6 example, the brute-force tie cases, the piecewise
scenes in every screen precision, edge cases, the 145x145x200 workload in
full and a sampled deepest-level section of the 1024x1024x224 workload."""
import json
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import synth  # noqa: E402
from test_gpu_parity import PRECISIONS, SCENES, _assert_same  # noqa: E402
from test_oracle_pins import BRUTE_CASES  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2106_12942_b300 as P
    return P


def _run(P, img, mask, **kw):
    seg = P.RHSEG(img, mask, multi_merge=1, **kw)
    seg.run()
    return seg


def test_multi_worked_example(P, orc):
    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_1x6_multi_merge.json")))
    im = d["image"]
    img = np.array(im["values"], dtype=np.uint16).reshape(im["rows"], im["cols"], im["bands"])
    for case in d["cases"]:
        kw = {k: v for k, v in d["params"].items() if k != "multi_merge"}
        kw["spclust_wght"] = case["spclust_wght"]
        if "conv_nregions" in case:
            kw["conv_nregions"] = case["conv_nregions"]
        ref = orc.run(img, None, multi_merge=1, **kw)
        assert len(ref.log) == len(case["log"])
        for precision in PRECISIONS:
            _assert_same(_run(P, img, None, precision=precision, **kw), ref, f"{case} p{precision}")


def test_multi_tiny_cases_with_ties(P, orc):
    for ci, case in enumerate(BRUTE_CASES):
        rows, cols, B, maxval, mask_p, L, w, conv, conn, min_nr, n_out, seam = case
        for seed in (1, 2, 3):
            img, mask = synth.random_cube(seed * 101 + rows * 7 + cols, rows, cols, B, maxval, mask_p)
            kw = dict(rnb_levels=L, spclust_wght=w, conv_nregions=conv, connectivity=conn,
                      min_nregions=min_nr, n_out_levels=n_out, seam_pass=seam)
            ref = orc.run(img, mask, multi_merge=1, **kw)
            for precision in (0, 1):
                _assert_same(_run(P, img, mask, precision=precision, **kw), ref, f"case {ci} s{seed} p{precision}")


@pytest.mark.parametrize("si", range(len(SCENES)))
def test_multi_piecewise_scenes(P, orc, si):
    rows, cols, B, L, w, conv, conn, min_nr, n_out, seam, masked = SCENES[si]
    img, mask = synth.make(4 if masked else 2, seed=400 + si, rows=rows, cols=cols)
    img = np.ascontiguousarray(img[:, :, :B])
    kw = dict(rnb_levels=L, spclust_wght=w, conv_nregions=conv, connectivity=conn, min_nregions=min_nr,
              n_out_levels=n_out, seam_pass=seam)
    ref = orc.run(img, mask, multi_merge=1, **kw)
    for precision in PRECISIONS:
        _assert_same(_run(P, img, mask, precision=precision, **kw), ref, f"scene {si} p{precision}")


def test_multi_edge_cases(P, orc):
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
        ref = orc.run(im, mk, multi_merge=1, **kw)
        for precision in PRECISIONS:
            _assert_same(_run(P, im, mk, precision=precision, **kw), ref, f"edge {i} p{precision}")


def test_multi_rejects_bad_combinations(P):
    from paper_2106_12942_b300.rhseg import RHSEGError
    img = np.zeros((4, 4, 2), np.uint16)
    with pytest.raises(RHSEGError):
        P.RHSEG(img, None, precision=3, incremental=1, multi_merge=1, spclust_wght=0.5)
    with pytest.raises(RHSEGError):
        P.RHSEG(img, None, multi_merge=2, spclust_wght=0.5)


def test_multi_rhseg_145x145x200(P, orc):
    img, mask = synth.make(3)
    kw = {k: v for k, v in synth.WORKLOADS[3].params.items() if k != "precision"}
    ref = orc.run(img, mask, multi_merge=1, **kw)
    _assert_same(_run(P, img, mask, precision=1, **kw), ref, "145x145x200 multi-merge")


def test_multi_rhseg_1024x1024x224_section(P, orc):
    img, mask = synth.make(4)
    kw = dict(synth.WORKLOADS[4].params)
    seg = _run(P, img, mask, **kw)
    log = seg.log()
    L = kw["rnb_levels"]
    okw = {k: v for k, v in kw.items() if k != "precision"}
    ref = orc.hseg_leaf(img, mask, 0, multi_merge=1, **okw)
    part = log[(log["level"] == L) & (log["section"] == 0)]
    assert len(ref.log) > 0 and len(part) == len(ref.log)
    for f in ["step", "kind", "survivor_id", "absorbed_id", "nregions_after"]:
        assert np.array_equal(part[f], ref.log[f]), f
    assert np.array_equal(part["key"].view(np.uint64), ref.log["key"].view(np.uint64))
    lab, sums, cnt = seg.level(seg.n_levels() - 1)
    unm = mask == 0
    assert np.all((lab == 0) == ~unm)
    assert np.array_equal(sums.sum(0), img[unm].astype(np.int64).sum(0))
    assert seg.stats()["iterations"] < 100 * 4 ** (L - 1)          # a few tens of iterations per section
