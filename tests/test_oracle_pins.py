"""Pins of the oracle's HSEG/RHSEG loop against things other than itself:
an independent brute force over exact rationals on tiny images, textbook
Ward clustering (scipy, scikit-learn) as the special cases w = 0, and
invariants that hold at any size."""
import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import _brute  # noqa: E402
import synth  # noqa: E402


def _log_tuples(log):
    return [(int(m["level"]), int(m["section"]), int(m["step"]), int(m["kind"]), int(m["survivor_id"]),
             int(m["absorbed_id"]), float(m["key"]), int(m["nregions_after"])) for m in log]


BRUTE_CASES = [
    # (rows, cols, bands, maxval, mask_p, L, w, conv, conn, min_nr, n_out, seam)
    (3, 3, 1, 3, 0.0, 1, 0.0, 1, 4, 0, 1, 1),
    (3, 3, 2, 3, 0.0, 1, 0.7, 1, 8, 0, 3, 1),
    (3, 3, 1, 2, 0.2, 1, 1.0, 2, 4, 0, 2, 1),
    (4, 4, 1, 3, 0.0, 1, 0.5, 1, 8, 0, 4, 1),
    (4, 4, 3, 5, 0.0, 1, 1.0, 2, 4, 0, 1, 1),
    (4, 4, 2, 9, 0.1, 2, 0.3, 2, 8, 2, 3, 1),
    (4, 4, 1, 4, 0.0, 2, 0.0, 1, 4, 1, 2, 1),
    (4, 5, 2, 6, 0.0, 2, 1.0, 3, 8, 2, 2, 1),
    (5, 4, 1, 3, 0.15, 2, 0.5, 2, 4, 3, 2, 0),
    (5, 6, 2, 20, 0.0, 2, 0.25, 3, 8, 4, 3, 1),
    (6, 6, 1, 40, 0.0, 3, 0.6, 2, 8, 1, 4, 1),
    (6, 5, 3, 7, 0.1, 3, 0.0, 2, 4, 2, 2, 1),
    (1, 6, 1, 9, 0.0, 2, 1.0, 1, 4, 1, 1, 1),
]


@pytest.mark.parametrize("case", BRUTE_CASES)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_oracle_equals_brute_force(orc, case, seed):
    rows, cols, B, maxval, mask_p, L, w, conv, conn, min_nr, n_out, seam = case
    img, mask = synth.random_cube(seed * 101 + rows * 7 + cols, rows, cols, B, maxval, mask_p)
    kw = dict(rnb_levels=L, spclust_wght=w, conv_nregions=conv, connectivity=conn,
              min_nregions=min_nr, n_out_levels=n_out, seam_pass=seam)
    br = _brute.Brute(img, mask, **kw).run()
    for mode in (0, 1):
        r = orc.run(img, mask, mode=mode, **kw)
        assert _log_tuples(r.log) == br.log
        assert r.stats["pairs"] == br.pairs
        assert len(r.levels) == len(br.levels)
        for lv, (lab, sums, counts) in zip(r.levels, br.levels):
            assert lv.labels.tolist() == lab
            assert lv.counts.tolist() == counts
            assert lv.sums.tolist() == sums


def test_plain_equals_cached_on_piecewise_scenes(orc):
    for seed, (rows, cols, L, w) in enumerate([(20, 20, 2, 0.5), (17, 23, 2, 0.2), (24, 24, 3, 1.0)]):
        img, mask = synth.make(2, seed=50 + seed, rows=rows, cols=cols)
        img = img[:, :, :12].copy()
        kw = dict(rnb_levels=L, spclust_wght=w, conv_nregions=5, connectivity=8, n_out_levels=3)
        a = orc.run(img, mask, mode=0, **kw)
        b = orc.run(img, mask, mode=1, **kw)
        assert np.array_equal(a.log, b.log)
        assert a.stats == b.stats
        for x, y in zip(a.levels, b.levels):
            assert np.array_equal(x.labels, y.labels) and np.array_equal(x.sums, y.sums)


def test_plain_equals_cached_on_workloads(orc):
    # the 32x32x16 workload in full under both merge rules, and the first
    # iterations of a 145x145x200 section (plain mode recomputes every pair)
    img, mask = synth.make(1)
    kw = {k: v for k, v in synth.WORKLOADS[1].params.items() if k != "precision"}
    for multi in (0, 1):
        a = orc.run(img, mask, mode=0, multi_merge=multi, **kw)
        b = orc.run(img, mask, mode=1, multi_merge=multi, **kw)
        assert np.array_equal(a.log, b.log) and a.stats == b.stats
        assert np.array_equal(a.levels[-1].labels, b.levels[-1].labels)
    img, mask = synth.make(2)
    kw = {k: v for k, v in synth.WORKLOADS[2].params.items() if k != "precision"}
    for multi in (0, 1):
        a = orc.hseg_leaf(img, mask, 5, max_iters=10 if multi == 0 else 2, mode=0, multi_merge=multi, **kw)
        b = orc.hseg_leaf(img, mask, 5, max_iters=10 if multi == 0 else 2, mode=1, multi_merge=multi, **kw)
        assert len(a.log) >= 10 and np.array_equal(a.log, b.log)


def test_complete_adjacency_is_unconstrained_ward(orc):
    # Every pair adjacent, w = 0, one level: HSEG is Ward's agglomeration;
    # scipy's Ward heights are sqrt(2 K) (K = increase of the within-cluster
    # sum of squares).
    from scipy.cluster.hierarchy import linkage
    rng = np.random.default_rng(21)
    for trial in range(6):
        n, B = int(rng.integers(5, 40)), int(rng.integers(1, 5))
        X = rng.integers(0, 65536, (n, B)).astype(np.uint16)
        img = X.reshape(1, n, B)
        r = orc.run(img, None, rnb_levels=1, spclust_wght=0.0, conv_nregions=1, full_adjacency=1)
        Z = linkage(X.astype(np.float64), method="ward")
        assert len(r.log) == n - 1
        np.testing.assert_allclose(np.sqrt(2 * r.log["key"]), Z[:, 2], rtol=1e-9)
        # same partition after each merge: compare cluster member sets
        members = {i: {i} for i in range(n)}
        scip = []
        for k, (a, b, _, _) in enumerate(Z):
            s = members.pop(int(a)) | members.pop(int(b))
            members[n + k] = s
            scip.append(frozenset(s))
        groups = {i + 1: {i} for i in range(n)}
        ours = []
        for m in r.log:
            s = groups[int(m["survivor_id"])] | groups.pop(int(m["absorbed_id"]))
            groups[int(m["survivor_id"])] = s
            ours.append(frozenset(s))
        assert ours == scip


@pytest.mark.parametrize("conn", [4, 8])
def test_grid_hswo_matches_sklearn_ward_tree(orc, conn):
    # w = 0, one level: HSWO = Ward clustering constrained to the pixel grid.
    from scipy.sparse import lil_matrix
    from sklearn.cluster import ward_tree
    rng = np.random.default_rng(31 + conn)
    for trial in range(4):
        rows, cols, B = int(rng.integers(3, 8)), int(rng.integers(3, 8)), int(rng.integers(1, 4))
        img = rng.integers(0, 65536, (rows, cols, B)).astype(np.uint16)
        n = rows * cols
        A = lil_matrix((n, n))
        offs = _brute.nb_offsets(conn)
        for y in range(rows):
            for x in range(cols):
                for dy, dx in offs:
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < rows and 0 <= xx < cols:
                        A[y * cols + x, yy * cols + xx] = 1
        X = img.reshape(n, B).astype(np.float64)
        children, _, _, _, dist = ward_tree(X, connectivity=A, return_distance=True)
        r = orc.run(img, None, rnb_levels=1, spclust_wght=0.0, conv_nregions=1, connectivity=conn)
        assert len(r.log) == n - 1
        np.testing.assert_allclose(np.sqrt(2 * r.log["key"]), dist, rtol=1e-9)
        members = {i: {i} for i in range(n)}
        sk = []
        for k, (a, b) in enumerate(children):
            s = members.pop(int(a)) | members.pop(int(b))
            members[n + k] = s
            sk.append(frozenset(s))
        groups = {i + 1: {i} for i in range(n)}
        ours = []
        for m in r.log:
            s = groups[int(m["survivor_id"])] | groups.pop(int(m["absorbed_id"]))
            groups[int(m["survivor_id"])] = s
            ours.append(frozenset(s))
        assert ours == sk


def _check_invariants(img, mask, r, kw):
    rows, cols, B = img.shape
    unm = np.ones((rows, cols), bool) if mask is None else (mask == 0)
    tot_sum = img[unm].astype(np.int64).sum(0)
    log = r.log
    # IDs: survivor smaller than absorbed for merges
    mg = log[log["kind"] != 2]
    assert np.all(mg["survivor_id"] < mg["absorbed_id"])
    assert np.array_equal(log["dissim"], np.sqrt(log["key"]))
    # count strictly decreasing by one within each section's HSEG
    for (lev, sec) in {(int(a), int(b)) for a, b in zip(mg["level"], mg["section"])}:
        s = mg[(mg["level"] == lev) & (mg["section"] == sec)]
        assert np.all(np.diff(s["nregions_after"]) == -1)
        assert np.all(np.diff(s["step"]) >= 0)
    # spectral merges below the threshold of the adjacent merge of the same step
    w = kw["spclust_wght"]
    for i in np.nonzero(log["kind"] == 1)[0]:
        m = log[i]
        prev = log[i - 1] if i > 0 else None
        if prev is not None and prev["kind"] == 0 and prev["step"] == m["step"] and \
                prev["section"] == m["section"] and prev["level"] == m["level"]:
            assert m["key"] < (w * w) * prev["key"]
    # canonical order of the log: levels deepest first, sections ascending
    order = list(zip(-log["level"], log["section"]))
    assert order == sorted(order)
    for lv in r.levels:
        lab = lv.labels
        assert np.all((lab == 0) == ~unm)
        R = len(lv.counts)
        # labels 1..R, first appearance in raster order
        flat = lab.ravel()
        nz = flat[flat > 0]
        _, first = np.unique(nz, return_index=True)
        assert np.array_equal(np.unique(nz), np.arange(1, R + 1))
        assert np.all(np.diff(first) > 0)
        assert np.array_equal(np.bincount(nz, minlength=R + 1)[1:], lv.counts)
        assert lv.counts.sum() == unm.sum()
        assert np.array_equal(lv.sums.sum(0), tot_sum)
        for k in range(1, R + 1):
            assert np.array_equal(img[lab == k].astype(np.int64).sum(0), lv.sums[k - 1])
    assert len(r.levels[-1].counts) >= min(kw["conv_nregions"], int(unm.sum()))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rhseg_invariants_piecewise(orc, seed):
    img, mask = synth.make(4, seed=200 + seed, rows=40, cols=36)
    img = img[:, :, :10].copy()
    kw = dict(rnb_levels=3, spclust_wght=0.3, conv_nregions=6, connectivity=8, n_out_levels=4,
              min_nregions=10)
    r = orc.run(img, mask, mode=1, **kw)
    _check_invariants(img, mask, r, kw)
    assert (r.log["kind"] == 2).sum() == r.stats["seam_splits"]


def test_output_levels_follow_geometric_counts(orc):
    img, mask = synth.make(2, seed=77, rows=24, cols=24)
    img = img[:, :, :8].copy()
    K, conv = 5, 4
    r = orc.run(img, mask, rnb_levels=2, spclust_wght=0.0, conv_nregions=conv, n_out_levels=K, mode=1)
    c0 = int(r.log[(r.log["level"] == 1) & (r.log["kind"] != 2)][0]["nregions_after"]) + 1
    want = [c0] + [int(round(conv * math.pow(c0 / conv, (K - 1 - k) / (K - 1)))) for k in range(1, K - 1)] + [conv]
    got = [len(lv.counts) for lv in r.levels]
    assert got == want
    # a coarser level is a union of regions of a finer one
    for a, b in zip(r.levels[:-1], r.levels[1:]):
        pairs = set(zip(a.labels.ravel().tolist(), b.labels.ravel().tolist()))
        fine_to_coarse = {}
        for f, c in pairs:
            assert fine_to_coarse.setdefault(f, c) == c


def test_leaf_run_equals_full_run_deepest_level(orc):
    img, mask = synth.make(4, seed=300, rows=32, cols=32)
    img = img[:, :, :8].copy()
    kw = dict(rnb_levels=3, spclust_wght=0.1, conv_nregions=6, connectivity=8)
    full = orc.run(img, mask, mode=1, **kw)
    for s in (0, 5, 15):
        leaf = orc.hseg_leaf(img, mask, s, mode=1, **kw)
        part = full.log[(full.log["level"] == 3) & (full.log["section"] == s)]
        assert np.array_equal(leaf.log, part)
    # bounded run is a prefix
    leaf = orc.hseg_leaf(img, mask, 5, max_iters=7, mode=0, **kw)
    part = full.log[(full.log["level"] == 3) & (full.log["section"] == 5)]
    assert np.array_equal(leaf.log, part[:len(leaf.log)]) and leaf.stats["iterations"] == 7


MUTANTS = [
    # (what, original text, planted mistake)
    ("tie-break on larger ID", "if (lo != blo) return lo < blo;", "if (lo != blo) return lo > blo;"),
    ("sign of the band difference", "(i128)nj * Si[b] - (i128)ni * Sj[b]", "(i128)nj * Si[b] + (i128)ni * Sj[b]"),
    ("dropped (n_i + n_j) factor", "(u128)ni * (u128)nj * (u128)(ni + nj)", "(u128)ni * (u128)nj * (u128)(nj)"),
    ("transposed counts", "(i128)nj * Si[b] - (i128)ni * Sj[b]", "(i128)ni * Si[b] - (i128)nj * Sj[b]"),
    ("threshold w instead of w^2", "(w * w) * Kadj", "w * Kadj"),
    ("no stop test after the adjacent merge", "if (count <= target) break;\n        }", "}"),
    ("one-sided adjacency union", "s->adj[(size_t)r * m + a] = 1;", "(void)0;"),
    ("seam test reversed", "if (best < Kr) { split_of[li] = rs;", "if (best > Kr) { split_of[li] = rs;"),
    ("IDs not re-derived after seam splits", "for (int i = 0; i < nold; i++) regs->v[i].id = newid[i];", "(void)newid;"),
    ("ties rounded away from zero", "up = (int)(mant & 1);", "up = 1;"),
    ("Z order of children", "else if (digit == 1) { r.r1 = r.r0 + h2; r.c0 = r.c0 + w2; }\n        else if (digit == 2) { r.r0 = r.r0 + h2; r.c1 = r.c0 + w2; }",
     "else if (digit == 2) { r.r1 = r.r0 + h2; r.c0 = r.c0 + w2; }\n        else if (digit == 1) { r.r0 = r.r0 + h2; r.c1 = r.c0 + w2; }"),
    ("multi-merge: pairs merged without the mutual test", "if (j > i && best[j] == i) {", "if (j > i) {"),
    ("multi-merge: stage merged in slot order, not key order", "qsort(P, (size_t)np, sizeof(mpair_t), cmp_mpair);",
     "(void)cmp_mpair;"),
    ("multi-merge: no stop test inside a stage", "for (int k = 0; k < np && *count > target; k++)",
     "for (int k = 0; k < np; k++)"),
    ("multi-merge: threshold from the last adjacent merge", "if (*nmerged == 0) *kfirst = P[k].K;",
     "*kfirst = P[k].K;"),
]

MULTI_CASES = [1, 3, 4, 5, 7, 9, 10, 12]          # indices into BRUTE_CASES


def _pins_pass(orc, L):
    """Run a compact version of the pin suite against a bound oracle."""
    import random
    from fractions import Fraction
    rng = random.Random(1)
    for _ in range(300):
        N, D = rng.getrandbits(rng.randint(1, 120)), rng.getrandbits(rng.randint(1, 120)) or 1
        if orc.div_rn(N, D, L=L) != N / D:
            return False
    for q in range(1 << 52, (1 << 52) + 40):
        if orc.div_rn(2 * q + 1, 2, L=L) != (2 * q + 1) / 2:
            return False
    nrng = np.random.default_rng(2)
    for _ in range(50):
        B = int(nrng.integers(1, 8))
        ni, nj = int(nrng.integers(1, 50)), int(nrng.integers(1, 50))
        Si, Sj = nrng.integers(0, 5000, B), nrng.integers(0, 5000, B)
        want = Fraction(ni * nj, ni + nj) * sum((Fraction(int(a), ni) - Fraction(int(b), nj)) ** 2
                                                for a, b in zip(Si, Sj))
        if orc.key(ni, Si, nj, Sj, L=L) != float(want):
            return False
    for ci, case in enumerate(BRUTE_CASES):
        rows, cols, B, maxval, mask_p, Lv, w, conv, conn, min_nr, n_out, seam = case
        img, mask = synth.random_cube(101 + rows * 7 + cols, rows, cols, B, maxval, mask_p)
        kw = dict(rnb_levels=Lv, spclust_wght=w, conv_nregions=conv, connectivity=conn,
                  min_nregions=min_nr, n_out_levels=n_out, seam_pass=seam)
        for multi in ((0, 1) if ci in MULTI_CASES else (0,)):
            br = _brute.Brute(img, mask, multi_merge=multi, **kw).run()
            r = orc.run(img, mask, L=L, mode=0, multi_merge=multi, **kw)
            if _log_tuples(r.log) != br.log:
                return False
            for lv, (lab, _, _) in zip(r.levels, br.levels):
                if lv.labels.tolist() != lab:
                    return False
    d, img = _multi_fixture()
    for case in d["cases"]:
        r = orc.run(img, None, L=L, mode=0, **_case_params(d, case))
        if _fixture_log(r.log) != _fixture_want(case) or r.stats["pairs"] != case["pairs"]:
            return False
    return True


def _multi_fixture():
    import json
    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_1x6_multi_merge.json")))
    im = d["image"]
    return d, np.array(im["values"], dtype=np.uint16).reshape(im["rows"], im["cols"], im["bands"])


def _case_params(d, case):
    kw = dict(d["params"], spclust_wght=case["spclust_wght"])
    if "conv_nregions" in case:
        kw["conv_nregions"] = case["conv_nregions"]
    return kw


def _fixture_log(log):
    return [(int(m["step"]), int(m["kind"]), int(m["survivor_id"]), int(m["absorbed_id"]), float(m["key"]))
            for m in log]


def _fixture_want(case):
    from fractions import Fraction
    return [(st, k, a, b, float(Fraction(K))) for st, k, a, b, K in case["log"]]


def test_unmodified_oracle_passes_compact_pins(orc):
    assert _pins_pass(orc, orc.oracle.lib())


@pytest.mark.parametrize("what,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(orc, tmp_path, what, orig, bad):
    # The mistake is planted in a copy of the oracle source, compiled on the
    # CPU; the pins must reject it.
    src = open(os.path.join(os.path.dirname(orc.oracle.__file__), "rhseg_oracle.c")).read()
    assert src.count(orig) >= 1, what
    mut = src.replace(orig, bad, 1)
    path = tmp_path / "mutant.c"
    path.write_text(mut)
    so = orc.compile_source(str(path), str(tmp_path / "mutant.so"))
    L = orc.load(so)
    assert not _pins_pass(orc, L), what


# --- reading R12: several merges per iteration (params multi_merge = 1) ---

def test_multi_merge_worked_example_fixture(orc):
    d, img = _multi_fixture()
    for case in d["cases"]:
        want = _fixture_want(case)
        kw = _case_params(d, case)
        for mode in (0, 1):
            r = orc.run(img, None, mode=mode, **kw)
            assert _fixture_log(r.log) == want, (case["spclust_wght"], mode)
            assert r.stats["pairs"] == case["pairs"]
        br = _brute.Brute(img, None, **kw).run()
        assert [(it, k, a, b, K) for (_, _, it, k, a, b, K, _) in br.log] == want
        assert br.pairs == case["pairs"]


@pytest.mark.parametrize("ci", MULTI_CASES)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_multi_merge_oracle_equals_brute_force(orc, ci, seed):
    rows, cols, B, maxval, mask_p, L, w, conv, conn, min_nr, n_out, seam = BRUTE_CASES[ci]
    img, mask = synth.random_cube(seed * 101 + rows * 7 + cols, rows, cols, B, maxval, mask_p)
    kw = dict(rnb_levels=L, spclust_wght=w, conv_nregions=conv, connectivity=conn,
              min_nregions=min_nr, n_out_levels=n_out, seam_pass=seam, multi_merge=1)
    br = _brute.Brute(img, mask, **kw).run()
    for mode in (0, 1):
        r = orc.run(img, mask, mode=mode, **kw)
        assert _log_tuples(r.log) == br.log
        assert r.stats["pairs"] == br.pairs
        for lv, (lab, sums, counts) in zip(r.levels, br.levels):
            assert lv.labels.tolist() == lab
            assert lv.counts.tolist() == counts
            assert lv.sums.tolist() == sums


def _stage_groups(log):
    """Records grouped by (level, section, step, kind), in log order."""
    groups, key = [], None
    for m in log:
        k = (int(m["level"]), int(m["section"]), int(m["step"]), int(m["kind"]))
        if k != key:
            groups.append([])
            key = k
        groups[-1].append(m)
    return groups


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_multi_merge_invariants_piecewise(orc, seed):
    """Properties of the rule at sizes the brute force cannot reach: within a
    stage the merged pairs are disjoint and come in (K, lo, hi) order; the
    count drops by one per record; the first merge of a section equals the
    single-merge rule's first merge; spectral merges stay below the
    iteration's threshold; sums and counts are conserved; and the rule needs
    no more iterations than the single-merge rule."""
    rows, cols, L, w = [(24, 24, 2, 0.5), (21, 27, 2, 0.2), (32, 32, 3, 1.0)][seed]
    img, mask = synth.make(2, seed=300 + seed, rows=rows, cols=cols)
    img = np.ascontiguousarray(img[:, :, :6])
    kw = dict(rnb_levels=L, spclust_wght=w, conv_nregions=6, connectivity=8, n_out_levels=3)
    multi = orc.run(img, mask, multi_merge=1, **kw)
    single = orc.run(img, mask, multi_merge=0, **kw)
    assert orc.run(img, mask, multi_merge=1, mode=0, **kw).log.tobytes() == multi.log.tobytes()
    groups = _stage_groups(multi.log[multi.log["kind"] != 2])
    assert any(len(g) > 1 for g in groups)
    for g in groups:
        ids = [int(m["survivor_id"]) for m in g] + [int(m["absorbed_id"]) for m in g]
        assert len(set(ids)) == len(ids)
        keys = [(float(m["key"]), int(m["survivor_id"]), int(m["absorbed_id"])) for m in g]
        assert keys == sorted(keys)
        assert all(int(m["survivor_id"]) < int(m["absorbed_id"]) for m in g)
    prev = None
    for m in multi.log:
        if prev is not None and (m["level"], m["section"]) == (prev["level"], prev["section"]) and m["kind"] != 2 \
                and prev["kind"] != 2:
            assert int(m["nregions_after"]) == int(prev["nregions_after"]) - 1
        prev = m
    thr = {}
    for g in groups:
        m0 = g[0]
        k = (int(m0["level"]), int(m0["section"]), int(m0["step"]))
        if int(m0["kind"]) == 0:
            thr[k] = (w * w) * float(m0["key"])
        else:
            assert all(float(m["key"]) < thr.get(k, float("inf")) for m in g)
    deepest = L
    for s in range(4 ** (L - 1)):
        a = multi.log[(multi.log["level"] == deepest) & (multi.log["section"] == s)]
        b = single.log[(single.log["level"] == deepest) & (single.log["section"] == s)]
        if len(b):
            assert a[0].tobytes() == b[0].tobytes()
    assert multi.stats["iterations"] <= single.stats["iterations"]
    tot = img.reshape(-1, img.shape[2]).astype(np.int64)
    keep = (mask == 0).ravel() if mask is not None else np.ones(tot.shape[0], bool)
    for lv in multi.levels:
        assert np.array_equal(lv.sums.sum(axis=0), tot[keep].sum(axis=0))
        assert lv.counts.sum() == keep.sum()


def test_multi_merge_one_merge_equals_single_merge(orc):
    """With a target one below the start count the rule makes exactly the
    single-merge rule's merge."""
    img, mask = synth.random_cube(77, 6, 7, 3, 50, 0.0)
    for w in (0.0, 0.5, 1.0):
        kw = dict(rnb_levels=1, spclust_wght=w, conv_nregions=6 * 7 - 1, connectivity=8)
        a = orc.run(img, mask, multi_merge=1, **kw)
        b = orc.run(img, mask, multi_merge=0, **kw)
        assert a.log.tobytes() == b.log.tobytes() and len(a.log) == 1


def test_multi_merge_complete_adjacency_gives_the_ward_dendrogram(orc):
    """Ward linkage is reducible (Lance-Williams), so merging every pair of
    reciprocal nearest neighbours at once, and repeating, builds the same
    dendrogram as the sequential algorithm (the basis of the
    nearest-neighbour-chain method).  With every pair adjacent and w = 0 the
    several-merges rule is exactly that: its clusters and heights must be
    scipy's Ward linkage, in a different order, in fewer iterations."""
    from scipy.cluster.hierarchy import linkage
    rng = np.random.default_rng(23)
    fewer = 0
    for trial in range(8):
        n, B = int(rng.integers(6, 48)), int(rng.integers(1, 5))
        X = rng.integers(0, 65536, (n, B)).astype(np.uint16)
        img = X.reshape(1, n, B)
        r = orc.run(img, None, rnb_levels=1, spclust_wght=0.0, conv_nregions=1, full_adjacency=1, multi_merge=1)
        Z = linkage(X.astype(np.float64), method="ward")
        assert len(r.log) == n - 1
        members = {i: {i} for i in range(n)}
        scip = {}
        for k, (a, b, h, _) in enumerate(Z):
            s = members.pop(int(a)) | members.pop(int(b))
            members[n + k] = s
            scip[frozenset(s)] = h
        groups = {i + 1: {i} for i in range(n)}
        ours = {}
        for m in r.log:
            s = groups[int(m["survivor_id"])] | groups.pop(int(m["absorbed_id"]))
            groups[int(m["survivor_id"])] = s
            ours[frozenset(s)] = np.sqrt(2 * float(m["key"]))
        assert set(ours) == set(scip)
        for c, h in scip.items():
            assert abs(ours[c] - h) <= 1e-9 * h
        fewer += r.stats["iterations"] < n - 1
    assert fewer > 0


def test_oracle_equals_brute_force_random_sweep(orc):
    """Random configurations beyond the fixed list: sizes up to 7x7, 1-3
    bands, value ranges small enough for ties, L up to 3, every weight class,
    both connectivities, seam pass on and off, masks, both merge rules."""
    rng = np.random.default_rng(2024)
    for k in range(300):
        rows, cols = int(rng.integers(1, 8)), int(rng.integers(2, 8))
        B, maxval = int(rng.integers(1, 4)), int(rng.choice([2, 4, 9, 40]))
        mask_p = float(rng.choice([0.0, 0.0, 0.15]))
        L = int(rng.integers(1, 4 if min(rows, cols) >= 4 else 3)) if min(rows, cols) >= 2 else 1
        kw = dict(rnb_levels=L, spclust_wght=float(rng.choice([0.0, 0.3, 0.5, 1.0])),
                  conv_nregions=int(rng.integers(1, 4)), connectivity=int(rng.choice([4, 8])),
                  min_nregions=int(rng.integers(0, 4)), n_out_levels=int(rng.integers(1, 4)),
                  seam_pass=int(rng.integers(0, 2)), multi_merge=int(rng.integers(0, 2)))
        img, mask = synth.random_cube(5000 + k, rows, cols, B, maxval, mask_p)
        br = _brute.Brute(img, mask, **kw).run()
        r = orc.run(img, mask, mode=int(k % 2), **kw)
        assert _log_tuples(r.log) == br.log, (k, kw)
        assert r.stats["pairs"] == br.pairs, (k, kw)
        for lv, (lab, sums, counts) in zip(r.levels, br.levels):
            assert lv.labels.tolist() == lab and lv.counts.tolist() == counts and lv.sums.tolist() == sums, (k, kw)


# --- the threaded driver over the sections of a level (full-size goldens) ---

def _same_result(a, b):
    if not np.array_equal(a.log, b.log) or a.stats != b.stats or len(a.levels) != len(b.levels):
        return False
    return all(np.array_equal(x.labels, y.labels) and np.array_equal(x.sums, y.sums)
               and np.array_equal(x.counts, y.counts) for x, y in zip(a.levels, b.levels))


@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threaded_run_equals_single_thread_on_tiny_cases(orc, threads):
    # the brute-force cases with several sections per level, both merge rules
    for ci, case in enumerate(BRUTE_CASES):
        rows, cols, B, maxval, mask_p, L, w, conv, conn, min_nr, n_out, seam = case
        if L < 2:
            continue
        img, mask = synth.random_cube(101 + rows * 7 + cols, rows, cols, B, maxval, mask_p)
        kw = dict(rnb_levels=L, spclust_wght=w, conv_nregions=conv, connectivity=conn,
                  min_nregions=min_nr, n_out_levels=n_out, seam_pass=seam)
        for multi in (0, 1):
            a = orc.run(img, mask, multi_merge=multi, **kw)
            b = orc.run(img, mask, threads=threads, multi_merge=multi, **kw)
            assert _same_result(a, b), (ci, multi)


def test_threaded_run_equals_single_thread_on_workloads(orc):
    # the 32x32x16 workload (one section) and the 145x145x200 cube of the
    # next two workloads cropped to 96x96, L=3 (16 sections, seam pass)
    img, mask = synth.make(1)
    kw = {k: v for k, v in synth.WORKLOADS[1].params.items() if k != "precision"}
    assert _same_result(orc.run(img, mask, **kw), orc.run(img, mask, threads=4, **kw))
    img, mask = synth.make(2)
    img = np.ascontiguousarray(img[:96, :96])
    kw = {k: v for k, v in synth.WORKLOADS[2].params.items() if k != "precision"}
    a = orc.run(img, None, **kw)
    for t in (2, 5):
        assert _same_result(a, orc.run(img, None, threads=t, **kw)), t
    # a masked crop of the 1024x1024x224 cube, L=4 (64 sections)
    img, mask = synth.make(4, rows=128, cols=128)
    img = np.ascontiguousarray(img[:, :, :32])
    kw = dict(rnb_levels=4, spclust_wght=0.1, conv_nregions=12, connectivity=8, n_out_levels=3)
    assert _same_result(orc.run(img, mask, **kw), orc.run(img, mask, threads=7, **kw))


def test_threaded_run_rejects_bad_thread_counts(orc):
    import ctypes as C
    img = np.zeros((4, 4, 1), dtype=np.uint16)
    L = orc.oracle.lib()
    p = orc.oracle._params(rnb_levels=2)
    err = C.c_int32(0)
    for t in (0, -1, 1025):
        h = L.orc_run_threads(img.ctypes.data, 4, 4, 1, None, C.byref(p), t, C.byref(err))
        assert not h and err.value == orc.oracle.ORC_EINVAL
