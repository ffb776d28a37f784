"""Seeded synthetic hyperspectral cubes (uint16 [rows, cols, bands]).

This module only draws inputs; it holds none of the segmentation method's
arithmetic.  Both the CUDA-path tests/benchmark and the oracle tests take
their images from here.

The thesis measures on Indian Pines (145x145, 220 bands) and Pavia (102/103
bands) crops (Section 5.1); those scenes are not available, so piecewise-
constant Voronoi scenes with smooth class spectra and Gaussian noise stand in
for them, at the same shapes.

Recipe (all draws from numpy's PCG64 generator seeded with 1000 + workload):
  * seeds uniform over [0, cols) x [0, rows); a pixel (r, c) is assigned to
    the seed nearest to its centre (c + 0.5, r + 0.5); ties go to the lower
    seed index.  Anisotropic cells (workload 5): each seed has an angle
    U(0, pi) and stretch U(1, 4); the distance is measured in the seed's frame
    rotated by the angle with the along-axis coordinate divided by the
    stretch; the nearest seed is chosen among the 16 Euclidean-nearest seeds.
  * seed k has class k mod n_classes.  Workload 1 gives every cell its own
    spectrum, U(500, 4000) per band.  Otherwise a class spectrum is a sum of 6
    Gaussian bumps over the band index (weights U(0.2, 1), centres
    U(0, B-1), widths U(B/30, B/6)) affinely rescaled to min 1000 and max
    U(4000, 8000).
  * pixel = class spectrum + N(0, sigma^2) i.i.d. per pixel and band (drawn in
    float32, row blocks in order), rounded half-to-even, clipped.
  * optional no-data mask: i.i.d. Bernoulli(p) per pixel.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

try:
    from scipy.spatial import cKDTree
except Exception:  # pragma: no cover - scipy is in the image
    cKDTree = None


@dataclass(frozen=True)
class Workload:
    name: str
    rows: int
    cols: int
    bands: int
    n_seeds: int
    n_classes: int          # 0: every cell has its own U(500, 4000) spectrum
    sigma: float
    clip_max: int
    mask_p: float
    anisotropic: bool
    params: dict = field(default_factory=dict)


WORKLOADS = {
    1: Workload("hseg_32x32x16", 32, 32, 16, 12, 0, 40.0, 4095, 0.0, False,
                dict(rnb_levels=1, spclust_wght=0.5, conv_nregions=8, connectivity=8, precision=0)),
    2: Workload("rhseg_145x145x200_fp64", 145, 145, 200, 120, 16, 80.0, 10000, 0.0, False,
                dict(rnb_levels=3, spclust_wght=0.2, conv_nregions=16, connectivity=8, precision=0)),
    3: Workload("rhseg_145x145x200_mixed", 145, 145, 200, 120, 16, 80.0, 10000, 0.0, False,
                dict(rnb_levels=3, spclust_wght=0.2, conv_nregions=16, connectivity=8, precision=2)),
    4: Workload("rhseg_1024x1024x224_mixed", 1024, 1024, 224, 3000, 64, 100.0, 10000, 0.1, False,
                dict(rnb_levels=5, spclust_wght=0.1, conv_nregions=64, connectivity=8, precision=1)),
    5: Workload("rhseg_2048x2048x128_mixed", 2048, 2048, 128, 12000, 128, 60.0, 16383, 0.0, True,
                dict(rnb_levels=6, spclust_wght=0.5, conv_nregions=128, connectivity=8, precision=1,
                     n_out_levels=8)),
}


def _class_spectra(rng: np.random.Generator, n_classes: int, B: int) -> np.ndarray:
    b = np.arange(B, dtype=np.float64)
    out = np.empty((n_classes, B), dtype=np.float64)
    for c in range(n_classes):
        w = rng.uniform(0.2, 1.0, 6)
        mu = rng.uniform(0.0, max(B - 1, 1), 6)
        sd = rng.uniform(B / 30.0, B / 6.0, 6)
        curve = (w[:, None] * np.exp(-0.5 * ((b[None, :] - mu[:, None]) / sd[:, None]) ** 2)).sum(0)
        hi = rng.uniform(4000.0, 8000.0)
        lo_c, hi_c = curve.min(), curve.max()
        span = hi_c - lo_c if hi_c > lo_c else 1.0
        out[c] = 1000.0 + (curve - lo_c) / span * (hi - 1000.0)
    return out


def voronoi(rows: int, cols: int, seeds: np.ndarray, angle=None, stretch=None) -> np.ndarray:
    """Index of the nearest seed per pixel ([rows, cols] int32)."""
    yy, xx = np.meshgrid(np.arange(rows) + 0.5, np.arange(cols) + 0.5, indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel()], 1)
    ns = len(seeds)
    out = np.empty(len(pts), dtype=np.int32)
    k = min(16 if angle is not None else 8, ns)
    tree = cKDTree(seeds) if cKDTree is not None else None
    step = 1 << 18
    for s in range(0, len(pts), step):
        P = pts[s:s + step]
        if tree is not None:
            _, cand = tree.query(P, k=k)
            cand = np.sort(np.asarray(cand).reshape(len(P), k), axis=1)
        else:
            cand = np.broadcast_to(np.arange(ns), (len(P), ns))
        d = P[:, None, :] - seeds[cand]
        if angle is not None:
            ca, sa = np.cos(angle[cand]), np.sin(angle[cand])
            u = (d[..., 0] * ca + d[..., 1] * sa) / stretch[cand]
            v = -d[..., 0] * sa + d[..., 1] * ca
            dist = u * u + v * v
        else:
            dist = d[..., 0] ** 2 + d[..., 1] ** 2
        out[s:s + step] = cand[np.arange(len(P)), np.argmin(dist, axis=1)]
    return out.reshape(rows, cols)


def make(w: Workload | int, seed: int | None = None, rows: int | None = None, cols: int | None = None):
    """Return (image uint16 [rows, cols, bands], mask uint8 [rows, cols] or None).

    rows/cols override the workload's size (same recipe, same density of
    seeds per pixel) for scaled-down parity cases."""
    if isinstance(w, int):
        seed = 1000 + w if seed is None else seed
        w = WORKLOADS[w]
    seed = 1000 if seed is None else seed
    R = rows or w.rows
    Cc = cols or w.cols
    n_seeds = max(2, int(round(w.n_seeds * (R * Cc) / (w.rows * w.cols))))
    rng = np.random.default_rng(seed)
    seeds = np.stack([rng.uniform(0, Cc, n_seeds), rng.uniform(0, R, n_seeds)], 1)
    angle = stretch = None
    if w.anisotropic:
        angle = rng.uniform(0.0, np.pi, n_seeds)
        stretch = rng.uniform(1.0, 4.0, n_seeds)
    if w.n_classes == 0:
        spectra = rng.uniform(500.0, 4000.0, (n_seeds, w.bands))
        cls = np.arange(n_seeds)
    else:
        spectra = _class_spectra(rng, w.n_classes, w.bands)
        cls = np.arange(n_seeds) % w.n_classes
    cell = voronoi(R, Cc, seeds, angle, stretch)
    spectra32 = spectra.astype(np.float32)
    img = np.empty((R, Cc, w.bands), dtype=np.uint16)
    blk = max(1, (1 << 22) // max(1, Cc * w.bands))
    for r0 in range(0, R, blk):
        r1 = min(R, r0 + blk)
        base = spectra32[cls[cell[r0:r1]]]                 # [rows of the block, C, B]
        noise = rng.standard_normal((r1 - r0, Cc, w.bands), dtype=np.float32) * np.float32(w.sigma)
        v = np.rint(base + noise)
        img[r0:r1] = np.clip(v, 0, w.clip_max).astype(np.uint16)
    mask = None
    if w.mask_p > 0:
        mask = (rng.random((R, Cc)) < w.mask_p).astype(np.uint8)
    return img, mask


def random_cube(seed: int, rows: int, cols: int, bands: int, maxval: int = 50, mask_p: float = 0.0):
    """Small i.i.d. uniform integer cube (values 0..maxval) for brute-force
    tests; small maxval makes equal dissimilarities (ties) common."""
    rng = np.random.default_rng(seed)
    img = rng.integers(0, maxval + 1, (rows, cols, bands)).astype(np.uint16)
    mask = None
    if mask_p > 0:
        mask = (rng.random((rows, cols)) < mask_p).astype(np.uint8)
    return img, mask
