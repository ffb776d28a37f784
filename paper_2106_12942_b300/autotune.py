"""Autotuner of the tensor-core screen's schedule (results never change).

The screen streams each unit's K slices through a shared-memory ring and
releases ring slots with tcgen05.commit.  Each commit costs the tensor pipe
about one MMA, so committing once per several K slices saves pipe time,
while committing more often frees slots earlier for the next loads.  The
screen comes in two forms: one CTA per 128x256 unit (an 8-slot ring of
24 KB slices), or CTA pairs sharing 256x256 tiles (a 12-slot ring of 16 KB
slices per CTA).  The grouping is a choice of the pair form only.  The best choice depends on
the band count (K slices per unit) and on the section size (units per step,
which sets how much the ring overlaps).

tune() times whole RHSEG runs of a synthetic cube with the given band count
and deepest-section size once per candidate (form, grouping), and keeps the one with
the fastest screen (CUDA events around every screen launch).  The choice is
stored in a JSON cache keyed by (architecture, bands, section-size bucket);
lookup() returns the parameters for a workload, or {} when it was never
tuned (the library's default then applies).

    python -m paper_2106_12942_b300.autotune --bands 224 --section 64
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "autotune_cache.json")
ARCH = "sm_103a"
CANDIDATES = (1, 2, 4, 7, 8)          # K slices per commit (screen_group)
FORMS = (0, 1)                        # screen_pair: one CTA per unit, CTA pairs


def bucket(section_px: int) -> int:
    """Power-of-two bucket of the deepest sections' pixel count."""
    return 1 << max(0, math.ceil(math.log2(max(1, section_px))))


def cache_key(bands: int, section_px: int, arch: str = ARCH) -> str:
    return f"{arch}/B{bands}/n{bucket(section_px)}"


def load_cache(path: str = CACHE) -> dict:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def lookup(bands: int, section_px: int, path: str = CACHE) -> dict:
    """Parameters the tuner chose for this band count and section size ({}
    when it has not been tuned)."""
    e = load_cache(path).get(cache_key(bands, section_px))
    return {"screen_group": int(e["screen_group"]), "screen_pair": int(e.get("screen_pair", 0))} if e else {}


def deepest_section_px(rows: int, cols: int, levels: int) -> int:
    """Pixels of the largest deepest-level section (floor halving)."""
    h, w = rows, cols
    for _ in range(levels - 1):
        h, w = (h + 1) // 2, (w + 1) // 2
    return h * w


def tune(bands: int = 224, section: int = 64, sections_per_side: int = 8, precision: int = 1, reps: int = 2,
         candidates=CANDIDATES, forms=FORMS, path: str = CACHE, verbose: bool = True) -> dict:
    """Time the candidates on a crop of the seeded 1024x1024x224 cube (its
    bands cut to `bands`): sections_per_side^2 deepest sections of
    section x section pixels, w = 0.1, 64 final regions."""
    import numpy as np
    import torch
    import synth
    from .rhseg import RHSEG
    side = section * sections_per_side
    levels = 1 + int(round(math.log2(sections_per_side)))
    img, mask = synth.make(4, rows=side, cols=side)
    if bands > img.shape[2]:
        raise ValueError(f"at most {img.shape[2]} bands")
    img = np.ascontiguousarray(img[:, :, :bands])
    kw = dict(rnb_levels=levels, spclust_wght=0.1, conv_nregions=64, connectivity=8, precision=precision, profile=1)
    times = {}
    for f in forms:
        for g in (candidates if f else (0,)):        # the one-CTA form groups 4, fixed
            seg = RHSEG(img, mask, screen_group=g, screen_pair=f, **kw)
            best = float("inf")
            for _ in range(reps + 1):                   # the first run warms up
                seg.run()
                torch.cuda.synchronize()
                best = min(best, seg.stats()["screen_ms"])
            seg.close()
            times[(f, g)] = best
            if verbose:
                print(f"  screen_pair={f} screen_group={g}: screen {best:.2f} ms", flush=True)
    f_best, g_best = min(times, key=times.get)
    entry = {"screen_pair": f_best, "screen_group": g_best,
             "screen_ms": {f"pair{f}/g{g}": round(v, 3) for (f, g), v in times.items()},
             "workload": f"{side}x{side}x{bands}, L={levels}, precision {precision}",
             "gpu": torch.cuda.get_device_name(), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    cache = load_cache(path)
    cache[cache_key(bands, deepest_section_px(side, side, levels))] = entry
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return entry


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--bands", type=int, nargs="+", default=[224])
    ap.add_argument("--section", type=int, nargs="+", default=[64])
    ap.add_argument("--precision", type=int, default=1)
    a = ap.parse_args()
    for b in a.bands:
        for s in a.section:
            print(f"B={b}, {s}x{s} sections:", flush=True)
            e = tune(bands=b, section=s, precision=a.precision)
            print(f"  -> screen_pair={e['screen_pair']} screen_group={e['screen_group']}", flush=True)


if __name__ == "__main__":
    main()
