#!/usr/bin/env python
"""Benchmark of the RHSEG hot path on one B300 per rank.

One step = one whole RHSEG run (deepest level to root) on the synthetic
1024x1024x224 workload (L=5, w=0.1, 64 regions, 10% no-data mask, FP16
tensor-core screen), image already resident in HBM.  The metric is region-pair
dissimilarities per second: the pairs the method defines (adjacent pairs of
each adjacent step + non-adjacent pairs of each spectral step) divided by the
device time of the run; the end-to-end seconds per run are ms_per_step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: replicas (each rank runs the whole workload; no collective on the
data path), value = pairs of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "region-pair dissimilarities/s and RHSEG end-to-end s at 1024²×224, mixed vs FP64, label-exact"
UNIT = "pairs/s"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, ncu, cold L2) per
# pair covered by the tcgen05 screen's MMAs, summed over every screen launch of
# the deepest level of the 512x512x224 crop (64 sections of 64x64 pixels,
# the size of the 1024x1024x224 run's deepest sections) and divided by that
# level's covered pairs (stats level_screen_evaluated); keyed by (bands,
# screen_pair).  The screen reads the operand rows of the units it keeps, so
# its traffic follows the covered pairs.
SCREEN_DRAM_BYTES_PER_COVERED_PAIR = {
    # one-CTA form, 16-bit operands: 210.50 GB over the 3,657 deepest-level launches of the crop,
    # whose covered pairs were 2.1223e11
    (224, 0): 0.9918,
}
PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.path.join("/tmp", f"rhseg_clocks_{os.getpid()}.csv"), "w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.strip().split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(x: float, dist, device) -> float:
    """Max of a per-rank scalar over all ranks (x itself when dist is None)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, pairs_per_step: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas, each running `steps` steps of
    `pairs_per_step` pairs: pairs of all ranks / the slowest rank's time."""
    return world * pairs_per_step * steps / seconds


def workload(k, rows=None, cols=None):
    import synth
    w = synth.WORKLOADS[k]
    img, mask = synth.make(k, rows=rows, cols=cols)
    if rows or cols:
        import dataclasses
        w = dataclasses.replace(w, name=f"{w.name}_crop{img.shape[0]}x{img.shape[1]}", rows=img.shape[0],
                                cols=img.shape[1])
    return w, img, mask


def oracle_golden(w):
    """The oracle's stored digests of a whole run of this workload (written by
    tests/golden/make_full_run_goldens.py), or None for workloads without one
    (crops)."""
    p = os.path.join(ROOT, "tests", "golden", f"full_run_{w.name}.json")
    return json.load(open(p)) if os.path.exists(p) else None


def label_exact(seg, golden):
    """The run's whole output (log, every level, counters) against the
    oracle's digests: (True, "") or (False, where they first differ)."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import _digest
    levels = [seg.level(k) for k in range(seg.n_levels())]
    got = _digest.result_digest(seg.log(), levels, seg.stats())
    diff = _digest.first_difference(golden, got)
    return diff == "", diff


def cpu_baseline(img, mask, params, target_s=15.0):
    """The oracle as it stands (plain mode: every pair recomputed each
    iteration, single thread), on a bounded sample: the first iterations of
    deepest-level section 0.  Returns pairs/s."""
    import oracle
    kw = {k: v for k, v in params.items() if k != "precision"}
    t0 = time.perf_counter()
    r = oracle.hseg_leaf(img, mask, 0, max_iters=1, mode=0, **kw)
    dt = time.perf_counter() - t0
    iters = 1
    pairs = r.stats["pairs"]
    if dt < target_s:
        n = max(1, min(50, int(target_s / max(dt, 1e-3))))
        t0 = time.perf_counter()
        r = oracle.hseg_leaf(img, mask, 0, max_iters=n, mode=0, **kw)
        dt = time.perf_counter() - t0
        iters = n
        pairs = r.stats["pairs"]
    return {"value": pairs / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"plain oracle (all pairs recomputed per iteration), first {iters} HSEG iteration(s) of "
                      f"deepest-level section 0 (64x64 px, {int(r.stats['pairs'])} pairs, {dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, img, mask = workload(args.workload)
    import oracle
    oracle.build()
    kw = {k: v for k, v in w.params.items() if k != "precision"}
    times, pairs = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.hseg_leaf(img, mask, 0, max_iters=1, mode=0, **kw)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            pairs.append(r.stats["pairs"])
    val = sum(pairs) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int128-exact/f64",
        "data": "synthetic", "config": {"workload": w.name, "sample": "HSEG iteration 1 of deepest section 0"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "plain oracle, first HSEG iteration of deepest-level section 0 per step"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=4)
    ap.add_argument("--precision", type=int, default=None)
    ap.add_argument("--incremental", type=int, default=None, choices=[0, 1],
                    help="1: incremental spectral minima (same results, row updates instead of the all-pairs screen)")
    ap.add_argument("--multi-merge", type=int, default=None, choices=[0, 1],
                    help="1: several merges per iteration (a different rule; its own oracle mode)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rows", type=int, default=None, help="scaled-down image (profiling); not a bench line")
    ap.add_argument("--cols", type=int, default=None)
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="1: the screen schedule the autotuner stored for this band count and section size "
                         "(paper_2106_12942_b300/autotune_cache.json), if any")
    ap.add_argument("--screen-pair", type=int, default=None, choices=[0, 1],
                    help="tensor-core screen form (overrides the stored choice): 0 one CTA per 128x256 unit, "
                         "1 CTA pairs sharing 256x256 tiles")
    ap.add_argument("--profile", type=int, default=1, choices=[0, 1],
                    help="1: CUDA events around every step kernel (per-kernel times, the roofline's launch "
                         "times); 0: none, the run as a user makes it")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2106_12942_b300 as P
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w, img, mask = workload(args.workload, args.rows, args.cols)
    params = dict(w.params)
    if args.levels is not None:
        params["rnb_levels"] = args.levels
    if args.precision is not None:
        params["precision"] = args.precision
    if args.incremental is not None:
        params["incremental"] = args.incremental
    if args.multi_merge is not None:
        params["multi_merge"] = args.multi_merge
    params["profile"] = args.profile
    tuned = {}
    if args.autotune and params.get("precision") in (1, 2):
        from paper_2106_12942_b300 import autotune
        sec_px = autotune.deepest_section_px(w.rows, w.cols, params["rnb_levels"])
        tuned = autotune.lookup(w.bands, sec_px)
        params.update(tuned)
    if args.screen_pair is not None:
        params["screen_pair"] = args.screen_pair
    # a stream of our own (the legacy default stream cannot be captured as a
    # CUDA graph, which the library does for runs without per-kernel events)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    img_d = torch.from_numpy(img.view(np.int16)).cuda().view(torch.uint16)
    mask_d = None if mask is None else torch.from_numpy(mask).cuda()
    seg = P.RHSEG(img_d, mask_d, stream=stream, **params)

    for _ in range(args.warmup):
        seg.run(stream=stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = ClockSampler()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        seg.run(stream=stream)
        stats.append(seg.stats())
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    if dist:
        dist.barrier()
    pairs = stats[-1]["pairs"]
    golden = oracle_golden(w) if (args.rows is None and args.cols is None and args.levels is None
                                  and not params.get("multi_merge")) else None
    pairs_source = "library counter (no stored oracle run for this configuration)"
    exact = None
    if golden is not None:
        # the numerator is the oracle's own count for the whole run; the run
        # must reproduce the oracle's output exactly for the number to count
        ok, where = label_exact(seg, golden)
        exact = {"label_exact": ok, "checked": "log, every level's labels/sums/counts, counters vs the oracle's "
                                               "digests", **({} if ok else {"first_difference": where})}
        assert golden["stats"]["pairs"] == pairs or not ok, "pair count differs from the oracle's"
        pairs = golden["stats"]["pairs"]
        pairs_source = "oracle's full run (stored digests)"
    value = job_rate(world, pairs, args.steps, ms / 1000.0)

    # the same runs without the per-kernel events (profile = 0), to state what
    # the events cost; not part of the timed region above
    prof_overhead = None
    if args.profile == 1 and not args.no_e2e:
        seg0 = P.RHSEG(img_d, mask_d, stream=stream, **dict(params, profile=0))
        seg0.run(stream=stream)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            seg0.run(stream=stream)
        f1.record(stream)
        torch.cuda.synchronize()
        seg0.close()
        ms0 = f0.elapsed_time(f1) / args.steps
        prof_overhead = {"ms_per_step_profile0": ms0, "ms_per_step_profile1": ms / args.steps,
                         "overhead_frac": (ms / args.steps - ms0) / ms0}

    # dominant kernel: the spectral screen; algorithmic flops 2*B per screened pair
    peaks = load_peaks()
    scr_ms = sum(s["screen_ms"] for s in stats)
    scr_n = sum(s["screen_launches"] for s in stats)
    scr_pairs = sum(s["screened_pairs"] for s in stats)
    # pairs the screen's MMAs actually covered (units proven empty are skipped)
    scr_eval = sum(s.get("screen_evaluated", 0) for s in stats)
    run_ms = sum(s["run_ms"] for s in stats)
    B = w.bands
    prec = params["precision"]
    flops = 2.0 * B * (scr_eval if scr_eval > 0 else scr_pairs)
    achieved = flops / (scr_ms / 1000.0) / 1e12 if scr_ms > 0 else 0.0
    impl = stats[-1]["screen_impl"]
    if impl == 3:
        bound, peak = "tensor", float(peaks["bf16_tflops"])
        peak_note = f"{peaks['_source']} bf16 dense burst (fp16 has the same nominal rate)"
    elif impl == 1:
        bound, peak = "alu", 148 * 2 * 2.0 * float(peaks.get("sm_max_mhz", 2032.0)) / 1e6
        peak_note = "fp64: 148 SM x 2 DFMA/clk x 2 flop x max SM clock (nominal 1.25 TFLOP/s)"
    else:
        bound, peak = "alu", 148 * 128 * 2.0 * float(peaks.get("sm_max_mhz", 2032.0)) / 1e6
        peak_note = "fp32 FMA: 148 SM x 128 lanes x 2 flop x max SM clock"
    traffic, traffic_basis = None, "no ncu capture of this screen form and band count"
    bpp = SCREEN_DRAM_BYTES_PER_COVERED_PAIR.get((B, int(params.get("screen_pair", 0))))
    if impl == 3 and bpp is not None and scr_n > 0 and scr_eval > 0:
        traffic = bpp * scr_eval / scr_n
        traffic_basis = (f"{bpp:.4g} DRAM bytes per covered pair (ncu, every deepest-level screen launch of the "
                         f"512x512x224 crop, same section size) x this run's covered pairs per launch")
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "traffic": traffic, "traffic_basis": traffic_basis,
                "kernel": {1: "screen_simt<f64>", 2: "screen_simt<f32 accumulate>",
                           3: "screen_tcgen05_cta_pair" if params.get("screen_pair") else "screen_tcgen05"}.get(impl, "none"),
                "launches": scr_n, "avg_launch_ms": scr_ms / max(scr_n, 1),
                "share_of_run": scr_ms / run_ms if run_ms else None, "peak_source": peak_note,
                "achieved_useful": (achieved * sum(s.get("screen_useful", 0) for s in stats) / scr_eval
                                    if scr_eval > 0 else None)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "int64+f64", 1: "int64+f16", 2: "int64+bf16", 3: "int64+f32"}[prec],
        "data": "synthetic",
        "config": {"workload": w.name, "rows": w.rows, "cols": w.cols, "bands": w.bands,
                   "rnb_levels": params["rnb_levels"], "spclust_wght": params["spclust_wght"],
                   "conv_nregions": params["conv_nregions"], "precision": prec,
                   "multi_merge": params.get("multi_merge", 0), "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (cube 470 MB, region tables several GB)",
                   "pairs_per_step": pairs, "seconds_per_rhseg_run": ms / args.steps / 1000.0},
        "roofline": roofline,
        "clocks": clocks,
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "kernel_ms": {"screen": scr_ms / args.steps, "adj_step": sum(s["adj_ms"] for s in stats) / args.steps,
                      "spec_step": sum(s["spec_ms"] for s in stats) / args.steps},
        "screen": {"screened_pairs": stats[-1]["screened_pairs"], "candidates": stats[-1]["candidates"],
                   "candidate_fraction": stats[-1]["candidates"] / max(1, stats[-1]["screened_pairs"]),
                   "candidates_below_threshold": stats[-1]["candidates_below"],
                   "fallbacks": stats[-1]["fallbacks"],
                   "evaluated_pairs": stats[-1].get("screen_evaluated", 0),
                   # the method's pairs per pair the MMAs covered (> 1: skipped units count as screened)
                   "screened_over_covered": stats[-1]["screened_pairs"] / max(1, stats[-1].get("screen_evaluated", 0)),
                   # of the covered pairs, those (i, j), i < j, of positions in use; the rest is the lower
                   # triangle of diagonal units and the rows past the last position
                   "useful_fraction_of_covered": stats[-1].get("screen_useful", 0) / max(1, stats[-1].get("screen_evaluated", 0)),
                   "error_vs_exact": {"max_rel": stats[-1]["screen_err_rel_max"],
                                      "max_over_bound": stats[-1]["screen_err_bound_max"],
                                      "rechecked_pairs": stats[-1]["screen_err_pairs"]}},
        "pairs_source": pairs_source,
        "autotune": tuned or "no stored choice (library defaults)",
        "parity": exact,
        "profile_overhead": prof_overhead,
        "level_ms": [round(x, 2) for x in stats[-1]["level_ms"][:params["rnb_levels"]]],
        "level_iters": stats[-1]["level_iters"][:params["rnb_levels"]],
        "level_kernel_ms": {k: [round(x, 1) for x in stats[-1]["level_" + k + "_ms"][:params["rnb_levels"]]]
                            for k in ("screen", "adj", "spec")},
        "level_screen_evaluated": stats[-1]["level_screen_evaluated"][:params["rnb_levels"]],
        "level_screen_launches": stats[-1]["level_iters"][:params["rnb_levels"]] if params["spclust_wght"] > 0 else None,
    }

    if not args.no_e2e:
        # end to end through the C ABI with host buffers: H2D of the cube and
        # mask from pinned memory, the run, D2H of the final labels and tables
        img_h = torch.from_numpy(img.view(np.int16)).pin_memory()
        mask_h = None if mask is None else torch.from_numpy(mask).pin_memory()
        seg.close()
        # the handle a user makes: no per-kernel events
        segh = P.RHSEG(img, mask, stream=stream, **dict(params, profile=0))
        segh.set_image(img_h, mask_h, stream=stream).run(stream=stream)
        nl = segh.n_levels()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.steps):
            segh.set_image(img_h, mask_h, stream=stream)
            segh.run(stream=stream)
            lab, sums, cnt = segh.level(nl - 1)
            d2h = lab.nbytes + sums.nbytes + cnt.nbytes
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        h2d = img.nbytes + (0 if mask is None else mask.nbytes)
        line["e2e"] = {"value": job_rate(world, pairs, args.steps, te), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h), "seconds_per_step": te / args.steps}
        segh.close()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(img, mask, params)
        if golden is not None:
            # whole-run time of the plain single-core oracle, extrapolated from
            # the sample's rate over the run's pairs (not measured), and the
            # measured whole run of the cached-key oracle on several threads
            cb["extrapolated_full_run_s"] = golden["stats"]["pairs"] / cb["value"]
            cb["extrapolation"] = "oracle pairs of the whole run / the sample's pairs/s (plain mode, 1 core)"
            cb["oracle_cached_full_run"] = {"seconds": golden["wall_s"], "threads": golden["threads"],
                                            "cpu": golden.get("cpu"), "mode": "cached keys (bit-identical results)"}
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
