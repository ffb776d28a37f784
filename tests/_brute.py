"""Independent brute-force RHSEG for tiny images (pure Python, exact rationals).

Used only to pin the C oracle.  It is written in a different style on
purpose: regions are sets of pixel indices, every dissimilarity is recomputed
from the raw pixel values of Eq. 1 (means, not band sums) as an exact
Fraction, and adjacency is recomputed from the pixel grid at every iteration.
Ranking follows reading R1 (nearest-even binary64 of the exact value, Python's
int/Fraction -> float conversion is correctly rounded) and R2 (ties on
(K, smaller ID, larger ID)).
"""
from __future__ import annotations

from fractions import Fraction


def nb_offsets(conn):
    if conn == 4:
        return [(-1, 0), (0, -1), (0, 1), (1, 0)]
    return [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]


def exact_K(img, A, B):
    """Eq. 1 squared: n_i n_j / (n_i + n_j) * sum_b (mu_ib - mu_jb)^2 (Fraction)."""
    bands = len(img[next(iter(A))])
    nA, nB = len(A), len(B)
    tot = Fraction(0)
    for b in range(bands):
        mA = Fraction(sum(int(img[p][b]) for p in A), nA)
        mB = Fraction(sum(int(img[p][b]) for p in B), nB)
        tot += (mA - mB) ** 2
    return Fraction(nA * nB, nA + nB) * tot


def rkey(img, A, B):
    return float(exact_K(img, A, B))


def section_rect(rows, cols, lev, s):
    r0, r1, c0, c1 = 0, rows, 0, cols
    digits = []
    for _ in range(lev - 1):
        digits.append(s & 3)
        s >>= 2
    for dgt in reversed(digits):
        h2, w2 = (r1 - r0) // 2, (c1 - c0) // 2
        if dgt in (0, 1):
            r1 = r0 + h2
        else:
            r0 = r0 + h2
        if dgt in (0, 2):
            c1 = c0 + w2
        else:
            c0 = c0 + w2
    return r0, r1, c0, c1


class Brute:
    def __init__(self, img, mask, rnb_levels=1, spclust_wght=0.0, conv_nregions=1, connectivity=8,
                 min_nregions=0, n_out_levels=1, seam_pass=1, multi_merge=0):
        self.rows, self.cols, self.B = img.shape
        self.pix = {}
        for r in range(self.rows):
            for c in range(self.cols):
                p = r * self.cols + c
                if mask is None or not mask[r, c]:
                    self.pix[p] = [int(v) for v in img[r, c]]
        self.L, self.w, self.conv, self.conn = rnb_levels, spclust_wght, conv_nregions, connectivity
        self.min_nr = min_nregions or conv_nregions
        self.n_out = n_out_levels or 1
        self.seam = seam_pass
        self.multi = multi_merge
        self.log = []
        self.pairs = 0
        self.levels = []

    # -- helpers ---------------------------------------------------------
    def neighbours(self, p, rect):
        r0, r1, c0, c1 = rect
        y, x = divmod(p, self.cols)
        for dy, dx in nb_offsets(self.conn):
            yy, xx = y + dy, x + dx
            if r0 <= yy < r1 and c0 <= xx < c1:
                q = yy * self.cols + xx
                if q in self.pix:
                    yield q

    def adjacent(self, regs, rect):
        owner = {}
        for rid, S in regs.items():
            for p in S:
                owner[p] = rid
        adj = set()
        for rid, S in regs.items():
            for p in S:
                for q in self.neighbours(p, rect):
                    o = owner[q]
                    if o != rid:
                        adj.add((min(rid, o), max(rid, o)))
        return adj

    def _mutual_stage(self, regs, cands, target, lev, sec, it, kind, snaps):
        """Reading R12: cands maps each pair (a, b), a < b, to (K, a, b).
        Every region's best candidate; the pairs that are best for both
        ends, merged smallest first while above the target."""
        best = {}
        for (a, b), k in cands.items():
            for r in (a, b):
                if r not in best or k < best[r]:
                    best[r] = k
        mutual = sorted({k for k in best.values() if best[k[1]] == k and best[k[2]] == k})
        done = []
        for K, a, b in mutual:
            if len(regs) <= target:
                break
            regs[a] = regs[a] | regs.pop(b)
            done.append(K)
            self.log.append((lev, sec, it, kind, a, b, K, len(regs)))
            if snaps is not None:
                snaps(regs)
        return done

    def _hseg_multi(self, regs, rect, target, lev, sec, snaps):
        it = 0
        while len(regs) > target:
            it += 1
            adj = self.adjacent(regs, rect)
            self.pairs += len(adj)
            cands = {(a, b): (rkey(self.pix, regs[a], regs[b]), a, b) for (a, b) in adj}
            done_a = self._mutual_stage(regs, cands, target, lev, sec, it, 0, snaps)
            if len(regs) <= target:
                break
            done_s = []
            if self.w > 0:
                t = (self.w * self.w) * min(done_a) if done_a else float("inf")
                adj = self.adjacent(regs, rect)
                ids = sorted(regs)
                cands = {}
                for i, a in enumerate(ids):
                    for b in ids[i + 1:]:
                        if (a, b) in adj:
                            continue
                        self.pairs += 1
                        K = rkey(self.pix, regs[a], regs[b])
                        if K < t:
                            cands[(a, b)] = (K, a, b)
                done_s = self._mutual_stage(regs, cands, target, lev, sec, it, 1, snaps)
            if not done_a and not done_s:
                break
        return regs

    def hseg(self, regs, rect, target, lev, sec, snaps=None):
        it = 0
        if snaps is not None:
            snaps(regs)
        if self.multi:
            return self._hseg_multi(regs, rect, target, lev, sec, snaps)
        while len(regs) > target:
            it += 1
            adj = self.adjacent(regs, rect)
            self.pairs += len(adj)
            best = None
            for (a, b) in adj:
                k = (rkey(self.pix, regs[a], regs[b]), a, b)
                if best is None or k < best:
                    best = k
            merged = False
            Kadj = float("inf")
            if best is not None:
                K, a, b = best
                Kadj = K
                regs[a] = regs[a] | regs.pop(b)
                merged = True
                self.log.append((lev, sec, it, 0, a, b, K, len(regs)))
                if snaps is not None:
                    snaps(regs)
                if len(regs) <= target:
                    break
            if self.w > 0:
                t = (self.w * self.w) * Kadj if best is not None else float("inf")
                adj = self.adjacent(regs, rect)
                ids = sorted(regs)
                cbest = None
                for i, a in enumerate(ids):
                    for b in ids[i + 1:]:
                        if (a, b) in adj:
                            continue
                        self.pairs += 1
                        K = rkey(self.pix, regs[a], regs[b])
                        if K < t and (cbest is None or (K, a, b) < cbest):
                            cbest = (K, a, b)
                if cbest is not None:
                    K, a, b = cbest
                    regs[a] = regs[a] | regs.pop(b)
                    merged = True
                    self.log.append((lev, sec, it, 1, a, b, K, len(regs)))
                    if snaps is not None:
                        snaps(regs)
            if not merged:
                break
        return regs

    def seam_split(self, regs, rect, lev, sec):
        r0, r1, c0, c1 = rect
        h2, w2 = (r1 - r0) // 2, (c1 - c0) // 2
        owner = {p: rid for rid, S in regs.items() for p in S}

        def quad(p):
            y, x = divmod(p, self.cols)
            return ((y - r0) >= h2, (x - c0) >= w2)

        splits = []
        for p in sorted(owner):
            cross = [q for q in self.neighbours(p, rect) if quad(q) != quad(p)]
            if not cross:
                continue
            R = owner[p]
            kr = rkey(self.pix, {p}, regs[R])
            kq = min(rkey(self.pix, {p}, regs[owner[q]]) for q in cross)
            if kq < kr:
                splits.append((p, R, kr))
        for p, R, _ in splits:
            regs[R] = regs[R] - {p}
        new = {}
        for rid, S in regs.items():
            if S:
                new[min(S) + 1] = S
        for p, _, _ in splits:
            new[p + 1] = {p}
        for p, R, kr in splits:
            self.log.append((lev, sec, 0, 2, R, p + 1, kr, len(new)))
        return new

    def run(self):
        L = self.L
        prev = None
        for lev in range(L, 0, -1):
            cur = []
            for s in range(4 ** (lev - 1)):
                rect = section_rect(self.rows, self.cols, lev, s)
                r0, r1, c0, c1 = rect
                if lev == L:
                    regs = {}
                    for y in range(r0, r1):
                        for x in range(c0, c1):
                            p = y * self.cols + x
                            if p in self.pix:
                                regs[p + 1] = {p}
                else:
                    regs = {}
                    for c in range(4):
                        regs.update(prev[4 * s + c])
                    if self.seam:
                        regs = self.seam_split(regs, rect, lev, s)
                if lev == 1:
                    regs = self._root(regs, rect)
                else:
                    regs = self.hseg(regs, rect, self.min_nr, lev, s)
                cur.append(regs)
            prev = cur
        return self

    def _root(self, regs, rect):
        c0 = len(regs)
        K, conv = self.n_out, self.conv
        import math
        if c0 <= conv:
            targets = [c0]
        elif K == 1:
            targets = [conv]
        else:
            targets = [c0] + [int(round(conv * math.pow(c0 / conv, (K - 1 - k) / (K - 1))))
                              for k in range(1, K - 1)] + [conv]
        tt = []
        for t in targets:
            if not tt or tt[-1] != t:
                tt.append(t)
        self.targets = tt
        taken = []

        def snap(rg):
            while len(taken) < len(tt) and len(rg) == tt[len(taken)]:
                taken.append({k: set(v) for k, v in rg.items()})

        regs = self.hseg(regs, rect, conv, 1, 0, snaps=snap)
        while len(taken) < len(tt):
            taken.append({k: set(v) for k, v in regs.items()})
        for rg in taken:
            lab = [[0] * self.cols for _ in range(self.rows)]
            counts, sums = [], []
            for i, rid in enumerate(sorted(rg)):
                S = rg[rid]
                for p in S:
                    y, x = divmod(p, self.cols)
                    lab[y][x] = i + 1
                counts.append(len(S))
                sums.append([sum(self.pix[p][b] for p in S) for b in range(self.B)])
            self.levels.append((lab, sums, counts))
        return regs
