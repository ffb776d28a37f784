"""Measurement studies of the path (GPU; results as JSON lines on stdout).

    python -m paper_2106_12942_b300.studies bands      # band-count sweep
    python -m paper_2106_12942_b300.studies recursion  # RHSEG vs full-image HSEG

bands: the thesis times its kernels for band counts 3 to 220 (Table 5.6);
here the same counts run through the whole path on a 256x256 crop of the
synthetic 224-band cube (bands cropped), with 64x64 sections (3 levels)
and 32x32 sections (4 levels), FP16 tensor-core screen: run time, screen
time, and the screen's algorithmic rate (2 B flops per screened pair).
At small B the K extent of each tensor-core unit is short (Bpad = 32 for
B = 3), so the rate per pair is bounded by the fixed per-unit costs.

recursion: RHSEG with L = 2, 3 against full-image HSEG (L = 1, the
recursion's reference result, Section 4.1) on the same cube and final
region count: adjusted Rand index of the final label maps and run times.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _peak_tflops() -> float | None:
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d.get("bf16_tflops"))
    except Exception:
        return None


def _cube(rows: int, cols: int, bands: int | None, seed: int = 7):
    sys.path.insert(0, ROOT)
    import synth
    img, mask = synth.make(4, seed=seed, rows=rows, cols=cols)
    if bands is not None:
        img = np.ascontiguousarray(img[:, :, :bands])
    return img, mask


def _timed_run(P, img, mask, **kw):
    import torch
    seg = P.RHSEG(img, mask, profile=1, **kw)
    seg.run()                                   # warm-up (first-use costs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seg.run()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return seg, wall


def bands(band_list=(3, 10, 50, 100, 150, 220), size=256, levels=(3, 4), precision=1):
    import paper_2106_12942_b300 as P
    peak = _peak_tflops()
    full, mask = _cube(size, size, None)
    for L in levels:
        sec = size >> (L - 1)
        for B in band_list:
            img = np.ascontiguousarray(full[:, :, :B])
            seg, wall = _timed_run(P, img, mask, rnb_levels=L, spclust_wght=0.1, conv_nregions=64,
                                   connectivity=8, precision=precision)
            st = seg.stats()
            tf = 2.0 * B * st["screened_pairs"] / (st["screen_ms"] * 1e-3) / 1e12 if st["screen_ms"] > 0 else 0.0
            print(json.dumps({"study": "bands", "bands": B, "section": f"{sec}x{sec}", "levels": L,
                              "run_ms": round(st["run_ms"], 2), "screen_ms": round(st["screen_ms"], 2),
                              "screened_pairs": st["screened_pairs"],
                              "screen_pairs_per_s": st["screened_pairs"] / (st["screen_ms"] * 1e-3) if st["screen_ms"] else None,
                              "screen_tflops": round(tf, 2), "frac_of_measured_peak": round(tf / peak, 4) if peak else None,
                              "iterations": st["iterations"]}), flush=True)
            seg.close()


def adjusted_rand_index(a: np.ndarray, b: np.ndarray) -> float:
    """ARI of two label maps over the pixels labelled in both (> 0)."""
    m = (a > 0) & (b > 0)
    a = a[m].astype(np.int64)
    b = b[m].astype(np.int64)
    n = a.size
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    cont = np.bincount(ai * (bi.max() + 1) + bi).astype(np.float64)
    comb = lambda x: x * (x - 1) / 2.0
    sum_ij = comb(cont).sum()
    sum_a = comb(np.bincount(ai).astype(np.float64)).sum()
    sum_b = comb(np.bincount(bi).astype(np.float64)).sum()
    expected = sum_a * sum_b / comb(float(n))
    maxv = 0.5 * (sum_a + sum_b)
    return float((sum_ij - expected) / (maxv - expected)) if maxv != expected else 1.0


def recursion(sizes=(128, 256), levels=(1, 2, 3), conv=64, w=0.1, precision=1):
    import paper_2106_12942_b300 as P
    for size in sizes:
        img, mask = _cube(size, size, 224)
        ref = None
        for L in levels:
            seg, wall = _timed_run(P, img, mask, rnb_levels=L, spclust_wght=w, conv_nregions=conv,
                                   connectivity=8, precision=precision)
            lab, _, cnt = seg.level(seg.n_levels() - 1)
            st = seg.stats()
            if ref is None:
                ref = lab
            print(json.dumps({"study": "recursion", "size": f"{size}x{size}x224", "levels": L,
                              "regions": int(len(cnt)), "run_ms": round(st["run_ms"], 2),
                              "pairs": st["pairs"], "ari_vs_L1": round(adjusted_rand_index(lab, ref), 5),
                              "same_labels_as_L1": bool(np.array_equal(lab, ref))}), flush=True)
            seg.close()


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "bands"
    {"bands": bands, "recursion": recursion}[what]()
