"""Store the oracle's result digests of whole RHSEG runs at full workload size.

    python tests/golden/make_full_run_goldens.py [workload ...] [--threads N]

For each workload (default: 4 = 1024x1024x224, 5 = 2048x2048x128) this runs
the C oracle (cached-key mode, the sections of each level spread over N host
threads; the thread count changes no result) on the seeded synthetic cube and
writes tests/golden/full_run_<name>.json: SHA-256 digests of the canonical
merge log, of every (level, section) log segment, of every hierarchy level's
labels, band sums and counts, and the run counters.  Only oracle/ computes
anything here; the GPU tests compare the library's output with these
digests.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import synth  # noqa: E402
import _digest  # noqa: E402


def golden_path(name: str) -> str:
    return os.path.join(HERE, f"full_run_{name}.json")


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or "unknown"


def make(k: int, threads: int) -> dict:
    w = synth.WORKLOADS[k]
    img, mask = synth.make(k)
    kw = {a: b for a, b in w.params.items() if a != "precision"}
    t0 = time.time()
    r = oracle.run(img, mask, threads=threads, mode=1, **kw)
    wall = time.time() - t0
    d = _digest.result_digest(r.log, [(lv.labels, lv.sums, lv.counts) for lv in r.levels], r.stats)
    d = {
        "workload": w.name,
        "params": kw,
        "source": "oracle/rhseg_oracle.c, cached-key mode (mode 1), orc_run_threads",
        "threads": threads,
        "wall_s": round(wall, 1),
        "cpu": cpu_model(),
        **d,
    }
    return d


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", type=int, default=[4, 5])
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    oracle.build()
    for k in a.workloads:
        d = make(k, a.threads)
        with open(golden_path(d["workload"]), "w") as f:
            json.dump(d, f, indent=1)
        print(f"{d['workload']}: {d['log_len']} records, {len(d['levels'])} levels, "
              f"{d['stats']['pairs']} pairs, {d['wall_s']} s on {a.threads} threads", flush=True)


if __name__ == "__main__":
    main()
