"""Canonical SHA-256 digests of an RHSEG result: the merge log, every
hierarchy level (labels, band sums, counts) and the run counters.

Test infrastructure: holds none of the method's arithmetic.  Both the script
that stores the oracle's digests (tests/golden/make_full_run_goldens.py) and
the GPU tests that check the library against them build their digests here,
from arrays in the layouts both sides already return, so a stored digest and
a computed one are comparable byte for byte.
"""
from __future__ import annotations

import hashlib

import numpy as np

# one log record without its padding; key and dissim as their binary64 bits
LOG_RECORD = np.dtype([
    ("level", "<i4"), ("section", "<i4"), ("step", "<i4"), ("kind", "<i4"),
    ("survivor_id", "<i8"), ("absorbed_id", "<i8"),
    ("key", "<u8"), ("dissim", "<u8"), ("nregions_after", "<i4"),
])

STAT_KEYS = ("pairs", "iterations", "merges_adj", "merges_spec", "seam_splits", "stalled_sections",
             "n_levels_out")


def _sha(b: bytes) -> str:
    return hashlib.sha256(b).hexdigest()


def log_records(log: np.ndarray) -> np.ndarray:
    """The log as packed LOG_RECORD entries (field by field, bit patterns of
    the two binary64 fields)."""
    out = np.zeros(len(log), dtype=LOG_RECORD)
    for f in LOG_RECORD.names:
        v = log[f]
        out[f] = v.view(np.uint64) if f in ("key", "dissim") else v
    return out


def log_digest(log: np.ndarray) -> str:
    return _sha(log_records(log).tobytes())


def segment_digests(log: np.ndarray) -> dict:
    """'level:section' -> 'records:sha256' for every (level, section) with
    records; the log is canonical (levels deepest first, sections in Z
    order), so each segment is one contiguous run."""
    rec = log_records(log)
    out = {}
    if len(rec) == 0:
        return out
    key = rec["level"].astype(np.int64) * (1 << 32) + rec["section"].astype(np.int64)
    cut = np.flatnonzero(np.diff(key)) + 1
    starts = np.concatenate([[0], cut])
    ends = np.concatenate([cut, [len(rec)]])
    for a, b in zip(starts, ends):
        out[f"{int(rec['level'][a])}:{int(rec['section'][a])}"] = f"{int(b - a)}:{_sha(rec[a:b].tobytes())}"
    return out


def level_digest(labels: np.ndarray, sums: np.ndarray, counts: np.ndarray) -> dict:
    return {
        "R": int(len(counts)),
        "labels": _sha(np.ascontiguousarray(labels, dtype="<i4").tobytes()),
        "sums": _sha(np.ascontiguousarray(sums, dtype="<i8").tobytes()),
        "counts": _sha(np.ascontiguousarray(counts, dtype="<i8").tobytes()),
    }


def stats_subset(stats: dict) -> dict:
    return {k: int(stats[k]) for k in STAT_KEYS}


def first_difference(want: dict, got: dict) -> str:
    """Where two result digests first differ, for an assertion message."""
    if want["log_len"] != got["log_len"] or want["log_sha256"] != got["log_sha256"]:
        for seg, v in want["segments"].items():
            g = got["segments"].get(seg)
            if g != v:
                n = v.split(":")[0]
                return f"log segment level:section {seg}: want {n} records, got {None if g is None else g.split(':')[0]}"
        extra = sorted(set(got["segments"]) - set(want["segments"]))
        return f"log: unexpected segments {extra[:5]}"
    for k, (a, b) in enumerate(zip(want["levels"], got["levels"])):
        for f in ("R", "labels", "sums", "counts"):
            if a[f] != b[f]:
                return f"level {k}: {f} differs"
    if len(want["levels"]) != len(got["levels"]):
        return f"levels: want {len(want['levels'])}, got {len(got['levels'])}"
    if want["stats"] != got["stats"]:
        return f"stats: want {want['stats']}, got {got['stats']}"
    return ""


def result_digest(log: np.ndarray, levels: list, stats: dict) -> dict:
    """levels: list of (labels, sums, counts)."""
    return {
        "log_len": int(len(log)),
        "log_sha256": log_digest(log),
        "segments": segment_digests(log),
        "levels": [level_digest(*lv) for lv in levels],
        "stats": stats_subset(stats),
    }
