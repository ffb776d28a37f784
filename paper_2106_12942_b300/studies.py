"""Measurement studies of the path (GPU; results as JSON lines on stdout).

    python -m paper_2106_12942_b300.studies bands      # band-count sweep
    python -m paper_2106_12942_b300.studies recursion  # RHSEG vs full-image HSEG
    python -m paper_2106_12942_b300.studies screen_error

bands: the thesis times its kernels for band counts 3 to 220 (Table 5.6);
here the same counts run through the whole path on a 256x256 crop of the
synthetic 224-band cube (bands cropped), with 64x64 sections (3 levels)
and 32x32 sections (4 levels), FP16 tensor-core screen: run time, screen
time, and the screen's algorithmic rate (2 B flops per pair its kept units
cover).
At small B the K extent of each tensor-core unit is short (Bpad = 32 for
B = 3), so the rate per pair is bounded by the fixed per-unit costs.

screen_error: the error of the tensor-core screen's arithmetic on real
operands, against the bound its reject test relies on.  Rows of the screen's
form (centred means, binary32, rounded to FP16 or BF16) go through the
tensor-core Gram; from it K~ = c 4^s (q_i + q_j - 2 g_ij), c = n_i n_j /
(n_i + n_j), against the exact key K (Eq. 1 squared, from integer sums).
Samples: all pairs of the regions at the start of the root level of the
145x145x200 run (precision 1), and all pairs of 2048 random pixels of that
cube.  Reported: max |K~ - K| / K, max |K~ - K| / bound (must be <= 1),
and the run's candidate fraction.

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
            covered = st["screen_evaluated"] or st["screened_pairs"]      # pairs the MMAs covered
            tf = 2.0 * B * covered / (st["screen_ms"] * 1e-3) / 1e12 if st["screen_ms"] > 0 else 0.0
            print(json.dumps({"study": "bands", "bands": B, "section": f"{sec}x{sec}", "levels": L,
                              "run_ms": round(st["run_ms"], 2), "screen_ms": round(st["screen_ms"], 2),
                              "screened_pairs": st["screened_pairs"], "covered_pairs": covered,
                              "screen_pairs_per_s": st["screened_pairs"] / (st["screen_ms"] * 1e-3) if st["screen_ms"] else None,
                              "screen_tflops": round(tf, 2), "frac_of_measured_peak": round(tf / peak, 4) if peak else None,
                              "iterations": st["iterations"]}), flush=True)
            seg.close()


# unit roundoff and subnormal half-spacing of the 16-bit operand formats
_ROW_FORMATS = {1: (2.0 ** -11, 2.0 ** -25), 2: (2.0 ** -8, 2.0 ** -134)}


def screen_rows(S: np.ndarray, n: np.ndarray, Bpad: int):
    """Operand rows in the screen's form, before the 16-bit rounding:
    x_i = (S_i / n_i - r) 2^-s in binary32, r an integer reference spectrum,
    s chosen so that |x| < 2^15.  Returns (x32 [R, Bpad], s, xs) with xs the
    exact x_i in float64 for the error bound."""
    S = np.asarray(S, np.int64)
    n = np.asarray(n, np.int64)
    R, B = S.shape
    r = np.rint((S / n[:, None]).mean(axis=0)).astype(np.int64)
    v = S - n[:, None] * r[None, :]                                 # exact
    x = v.astype(np.float32) * (np.float32(1.0) / n.astype(np.float32))[:, None]
    amax = float(np.abs(x).max()) if x.size else 1.0
    s = max(0, int(np.ceil(np.log2(max(amax, 1.0)))) - 14)
    x32 = np.zeros((R, Bpad), np.float32)
    x32[:, :B] = x * np.float32(2.0 ** -s)
    xs = (v.astype(np.float64) / n[:, None]) * 2.0 ** -s
    return x32, s, xs


def exact_keys(S: np.ndarray, n: np.ndarray) -> np.ndarray:
    """K_ij = sum_b (n_j S_ib - n_i S_jb)^2 / (n_i n_j (n_i + n_j)) for all
    pairs (Eq. 1 squared, times the size factor).  The differences are exact
    int64, the squares non-negative, so float64 holds K to ~B 2^-53."""
    S = np.asarray(S, np.int64)
    n = np.asarray(n, np.int64)
    R = len(n)
    K = np.zeros((R, R))
    for i0 in range(0, R, 32):
        i1 = min(R, i0 + 32)
        d = n[None, :, None] * S[i0:i1, None, :] - n[i0:i1, None, None] * S[None, :, :]
        df = d.astype(np.float64)
        N = np.einsum("ijb,ijb->ij", df, df)
        D = (n[i0:i1, None] * n[None, :]).astype(np.float64) * (n[i0:i1, None] + n[None, :]).astype(np.float64)
        K[i0:i1] = N / D
    return K


def screen_error_of(S, n, precision: int, gram) -> dict:
    """Error of K~ against K over all pairs of the regions (S, n), with
    `gram` mapping 16-bit rows [Rpad, Bpad] to their FP32 Gram.  The bound
    per pair is c 4^s [gamma (|x^_i| + |x^_j|)^2 + e (2 |x_i - x_j| + e)],
    e = e_i + e_j, e_i = (u + 3 2^-24)(1 + 2^-20)|x_i| + eta sqrt(B) (the
    binary32 conversion and the 16-bit rounding), gamma = Bpad 2^-22."""
    import torch
    S = np.asarray(S, np.int64)
    n = np.asarray(n, np.int64)
    R, B = S.shape
    Bpad = ((B + 31) // 32) * 32
    u, eta = _ROW_FORMATS[precision]
    x32, s, xs = screen_rows(S, n, Bpad)
    Rpad = ((R + 127) // 128) * 128
    dt = torch.float16 if precision == 1 else torch.bfloat16
    X = torch.zeros(Rpad, Bpad, dtype=torch.float32)
    X[:R] = torch.from_numpy(x32)
    Xh = X.to(dt)
    G = np.asarray(gram(Xh), np.float64)[:R, :R]
    xh = Xh[:R].float().numpy().astype(np.float64)
    q = np.diag(G)
    st = q[:, None] + q[None, :] - 2.0 * G
    c = (n[:, None] * n[None, :]).astype(np.float64) / (n[:, None] + n[None, :]).astype(np.float64)
    Kt = c * 4.0 ** s * st
    K = exact_keys(S, n)
    gamma = Bpad * 2.0 ** -22
    nh = np.sqrt((xh * xh).sum(axis=1))
    nx = np.sqrt((xs * xs).sum(axis=1))
    ei = (u + 3 * 2.0 ** -24) * (1 + 2.0 ** -20) * nx + eta * np.sqrt(B)
    e = ei[:, None] + ei[None, :]
    dx = np.sqrt(K / c) * 2.0 ** -s
    bound = c * 4.0 ** s * (gamma * (nh[:, None] + nh[None, :]) ** 2 + e * (2 * dx + e))
    iu = np.triu_indices(R, 1)
    err = np.abs(Kt - K)[iu]
    Ku, bu = K[iu], bound[iu]
    pos = Ku > 0
    rel = err[pos] / Ku[pos]
    return {"pairs": int(len(err)), "max_rel_err": float(rel.max()) if rel.size else 0.0,
            "median_rel_err": float(np.median(rel)) if rel.size else 0.0,
            "max_err_over_bound": float((err / bu).max()) if err.size else 0.0,
            "median_err_over_bound": float(np.median(err / bu)) if err.size else 0.0, "sigma": s}


def screen_error(precision=1, pixels=2048, seed=11):
    import torch
    import paper_2106_12942_b300 as P
    sys.path.insert(0, ROOT)
    import synth
    w = synth.WORKLOADS[3]
    img, mask = synth.make(3)
    kw = dict(w.params, precision=precision, n_out_levels=8)
    seg = P.RHSEG(img, mask, **kw)
    seg.run()
    st = seg.stats()
    _, sums, cnt = seg.level(0)
    gram = lambda Xh: P.gram_tc(Xh.cuda(), precision=precision).cpu().numpy()
    out = []
    reg = screen_error_of(sums, cnt, precision, gram)
    out.append(dict(reg, study="screen_error", sample=f"all pairs of the {len(cnt)} regions at the root level's start",
                    workload=w.name, precision=precision,
                    candidate_fraction=st["candidates"] / max(1, st["screened_pairs"]),
                    candidates_below_threshold=st["candidates_below"], candidates=st["candidates"]))
    seg.close()
    rng = np.random.default_rng(seed)
    flat = img.reshape(-1, img.shape[2]).astype(np.int64)
    idx = rng.choice(flat.shape[0], size=min(pixels, flat.shape[0]), replace=False)
    pix = screen_error_of(flat[idx], np.ones(len(idx), np.int64), precision, gram)
    out.append(dict(pix, study="screen_error", sample=f"all pairs of {len(idx)} random pixels", workload=w.name,
                    precision=precision))
    torch.cuda.synchronize()
    return out


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
    if what == "screen_error":
        for prec in (1, 2):
            for line in screen_error(precision=prec):
                print(json.dumps(line), flush=True)
    else:
        {"bands": bands, "recursion": recursion}[what]()
