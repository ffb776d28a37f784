/*
 * rhseg_oracle.c -- plain, slow reference of RHSEG/HSEG.
 *
 * Every section's HSEG runs in one thread.  The sections of one recursion
 * level are independent (Section 4.1: a section only meets its siblings when
 * the four are reassembled one level up), so orc_run_threads may run them on
 * several threads and then joins their records in Z order; orc_run uses one.
 * The thread count changes no result (a pin checks it).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, includes or calls
 * this file; only tests/, the smoke check in __graft_entry__ and the CPU
 * baseline leg of bench.py use it (through oracle/oracle.py).  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * What it follows (thesis "High Performance Hyperspectral Image Classification
 * using Graphics Processing Units", 2015):
 *   - Eq. 1 (Section 4.1): square root of band-sum mean squared error between
 *     regions i and j:  sqrt( n_i n_j / (n_i + n_j) * sum_b (mu_ib - mu_jb)^2 ).
 *   - HSEG steps 1-4 (Section 4.1): every pixel starts as a region; merge the
 *     adjacent pair of minimum dissimilarity; then merge the non-adjacent pair
 *     of minimum dissimilarity if it is below the minimum found among adjacent
 *     pairs (scaled by the spectral clustering weight); stop at the target.
 *   - RHSEG (Section 4.1, Fig. 4.3/4.4): 4^(L-1) sections at the deepest
 *     level, HSEG per section, reassembly in groups of four with regions on
 *     the seams linked across in an 8-neighbourhood, HSEG again, up to level 1.
 *   - Boundary-artifact pass: named as future work in Section 6.2; the
 *     reading implemented here is the seam-pixel split test described below.
 *
 * Readings of points the thesis leaves open (each one is a convention that
 * the CUDA path implements independently):
 *   R1  Ranking uses K = d^2 = N / D with N = sum_b (n_j S_ib - n_i S_jb)^2 and
 *       D = n_i n_j (n_i + n_j), both exact integers (S = band sums).  K is
 *       the correctly rounded (nearest-even) binary64 value of the exact
 *       rational; dissim = sqrt(K).
 *   R2  Ties are broken lexicographically on (K, smaller ID, larger ID).
 *   R3  The spectral step runs on the state after the adjacent merge of the
 *       same iteration, over non-adjacent pairs only, and merges iff
 *       K < t with t = (w*w) * K_adj in binary64 (t = +inf when no adjacent
 *       pair exists; w = 0 disables the step).
 *   R4  The stop test "count <= target" is made before each iteration and
 *       after every merge.  An iteration that merges nothing stalls the
 *       section.
 *   R5  Region ID = 1 + smallest raster index (whole image) of its pixels; the
 *       survivor of a merge is the region with the smaller ID.
 *   R6  Sections split at floor(h/2), floor(w/2); children in Z order
 *       (top-left, top-right, bottom-left, bottom-right).
 *   R7  Seam pass at each reassembly: a seam pixel p has a neighbour (under
 *       the configured connectivity) inside the parent but in another child.
 *       p leaves its region R and becomes a one-pixel region iff
 *       min_Q K({p}, Q) < K({p}, R) over the regions Q of those neighbours
 *       (R still containing p).  All tests use the state before the pass;
 *       then all splits are applied, IDs re-derived (R5), empty regions
 *       dropped.
 *   R8  Per-section target below the root = min_nregions (0 -> conv_nregions).
 *   R9  Output levels: c_0 = count at the start of the root HSEG,
 *       c_{K-1} = conv_nregions, c_k = nearest-even rounding of
 *       conv * (c_0/conv)^((K-1-k)/(K-1)) in between, duplicates removed.  A
 *       snapshot is taken when the count first equals c_k (final state if
 *       the root stalls first).  Labels are renumbered 1..R in raster order
 *       of first appearance.
 *   R10 Pairs evaluated per iteration = number of adjacent pairs in the
 *       adjacent step + (if the spectral step runs) number of non-adjacent
 *       pairs in the spectral step.
 *   R12 Multiple merges per iteration (Section 6.2 names the idea only;
 *       params.multi_merge = 1).  In each stage every region takes its best
 *       partner among the stage's pairs (R2 order): adjacent pairs in the
 *       adjacent stage; non-adjacent pairs with K < t in the spectral stage.
 *       The mutually best pairs are disjoint, so each keeps its key while the
 *       others merge.  They merge in (K, lo ID, hi ID) order with the R4 stop
 *       test after each.  t = (w*w) * K_adj, with K_adj the smallest key
 *       merged in the adjacent stage (the global minimum, which is always
 *       mutually best), on the state after that stage.  The first merge of
 *       every iteration is therefore the single-merge rule's.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

/* ------------------------------------------------------------------------- */
/* Exact key: correctly rounded binary64 of N / D (reading R1).              */
/* ------------------------------------------------------------------------- */

static int bitlen128(u128 x)
{
    int n = 0;
    while (x) { x >>= 1; n++; }
    return n;
}

/* Round-to-nearest-even binary64 of the exact quotient N / D, D > 0.
 * Plain restoring long division producing 55 quotient bits and a sticky bit. */
double orc_div_rn(uint64_t n_hi, uint64_t n_lo, uint64_t d_hi, uint64_t d_lo)
{
    u128 N = ((u128)n_hi << 64) | n_lo;
    u128 D = ((u128)d_hi << 64) | d_lo;
    if (D == 0) return NAN;
    if (N == 0) return 0.0;
    const u128 two53 = (u128)1 << 53;
    if (N < two53 && D < two53)          /* both exact in binary64; IEEE  */
        return (double)(uint64_t)N / (double)(uint64_t)D;  /* division is RN */

    /* e = floor(log2(N/D)) */
    int e = bitlen128(N) - bitlen128(D);
    /* bring R and Dsh to the same scale: Dsh <= R < 2 Dsh after fixing e */
    u128 R, Dsh;
    if (e >= 0) { R = N; Dsh = D << e; } else { R = N << (-e); Dsh = D; }
    if (R < Dsh) {
        e -= 1;
        if (e >= 0) { R = N; Dsh = D << e; } else { R = N << (-e); Dsh = D; }
    }
    /* 55 quotient bits: q = floor(N / D * 2^(54-e)) */
    uint64_t q = 0;
    for (int i = 0; i < 55; i++) {
        q <<= 1;
        if (R >= Dsh) { q |= 1; R -= Dsh; }
        R <<= 1;
    }
    int sticky = (R != 0);
    uint64_t mant = q >> 2;          /* 53 bits, top bit set */
    unsigned low = (unsigned)(q & 3);
    int up = 0;
    if (low > 2 || (low == 2 && sticky)) up = 1;
    else if (low == 2 && !sticky) up = (int)(mant & 1);  /* tie: to even */
    mant += (uint64_t)up;
    int ex = e - 52;
    if (mant == ((uint64_t)1 << 53)) { mant >>= 1; ex += 1; }
    return ldexp((double)mant, ex);
}

static double div_rn128(u128 N, u128 D)
{
    return orc_div_rn((uint64_t)(N >> 64), (uint64_t)N, (uint64_t)(D >> 64), (uint64_t)D);
}

/* K(i, j) of Eq. 1 squared, from exact band sums and pixel counts. */
double orc_key(int64_t ni, const int64_t *Si, int64_t nj, const int64_t *Sj, int32_t B)
{
    u128 N = 0;
    for (int b = 0; b < B; b++) {
        i128 d = (i128)nj * Si[b] - (i128)ni * Sj[b];
        u128 a = (u128)(d < 0 ? -d : d);
        N += a * a;
    }
    u128 D = (u128)ni * (u128)nj * (u128)(ni + nj);
    return div_rn128(N, D);
}

/* ------------------------------------------------------------------------- */
/* Public structures (ctypes mirrors these in oracle.py).                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t rnb_levels;
    int32_t conv_nregions;
    double  spclust_wght;
    int32_t connectivity;
    int32_t min_nregions;
    int32_t n_out_levels;
    int32_t seam_pass;
    int32_t mode;            /* 0 plain: every key recomputed each iteration;
                                1 cached: key matrix, touched row recomputed */
    int32_t full_adjacency;  /* test hook: every pair counts as adjacent */
    int32_t multi_merge;     /* reading R12: all mutually best pairs per stage */
} orc_params;

typedef struct {
    int32_t level, section, step, kind;   /* kind 0 adjacent, 1 spectral, 2 seam split */
    int64_t survivor_id, absorbed_id;
    double  key, dissim;
    int32_t nregions_after, pad;
} orc_merge;

typedef struct {
    int64_t pairs;           /* reading R10, summed over all sections */
    int64_t iterations;
    int64_t merges_adj, merges_spec, seam_splits;
    int32_t stalled_sections, n_levels_out;
} orc_stats;

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ERANGE = -2, ORC_ENOMEM = -3 };

/* growable log */
typedef struct { orc_merge *v; int64_t n, cap; } mlog_t;

static int log_push(mlog_t *L, orc_merge m)
{
    if (L->n == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 1024;
        orc_merge *nv = (orc_merge *)realloc(L->v, (size_t)nc * sizeof(orc_merge));
        if (!nv) return ORC_ENOMEM;
        L->v = nv; L->cap = nc;
    }
    L->v[L->n++] = m;
    return ORC_OK;
}

/* region table of one section */
typedef struct {
    int m, B;
    int64_t *id, *n, *S;     /* [m], [m], [m*B] */
    uint8_t *alive;
    uint8_t *adj;            /* dense m x m, symmetric */
    int *parent;             /* absorbed slot -> survivor slot */
    double *kmat;            /* cached mode only: m x m keys */
} sect_t;

static void sect_free(sect_t *s)
{
    free(s->id); free(s->n); free(s->S); free(s->alive); free(s->adj);
    free(s->parent); free(s->kmat);
    memset(s, 0, sizeof(*s));
}

static int sect_alloc(sect_t *s, int m, int B, int cached)
{
    memset(s, 0, sizeof(*s));
    s->m = m; s->B = B;
    size_t mm = (size_t)(m ? m : 1);
    s->id = (int64_t *)calloc(mm, sizeof(int64_t));
    s->n = (int64_t *)calloc(mm, sizeof(int64_t));
    s->S = (int64_t *)calloc(mm * (size_t)B, sizeof(int64_t));
    s->alive = (uint8_t *)calloc(mm, 1);
    s->adj = (uint8_t *)calloc(mm * mm, 1);
    s->parent = (int *)calloc(mm, sizeof(int));
    if (cached) s->kmat = (double *)calloc(mm * mm, sizeof(double));
    if (!s->id || !s->n || !s->S || !s->alive || !s->adj || !s->parent || (cached && !s->kmat)) {
        sect_free(s);
        return ORC_ENOMEM;
    }
    for (int i = 0; i < m; i++) { s->alive[i] = 1; s->parent[i] = i; }
    return ORC_OK;
}

static double sect_key(const sect_t *s, int i, int j)
{
    return orc_key(s->n[i], s->S + (size_t)i * s->B, s->n[j], s->S + (size_t)j * s->B, s->B);
}

/* (K, id_i, id_j) lexicographic comparison; ids of the pair given as
 * (lo, hi) with lo < hi (reading R2). */
static int pair_less(double K, int64_t lo, int64_t hi, double bK, int64_t blo, int64_t bhi)
{
    if (K < bK) return 1;
    if (K > bK) return 0;
    if (lo != blo) return lo < blo;
    return hi < bhi;
}

static int find_root(int *parent, int x)
{
    while (parent[x] != x) x = parent[x];
    return x;
}

/* merge slot b into slot a (id[a] < id[b]) */
static void sect_merge(sect_t *s, int a, int b)
{
    int m = s->m, B = s->B;
    for (int k = 0; k < B; k++) s->S[(size_t)a * B + k] += s->S[(size_t)b * B + k];
    s->n[a] += s->n[b];
    s->alive[b] = 0;
    s->parent[b] = a;
    for (int r = 0; r < m; r++) {
        if (s->adj[(size_t)b * m + r]) {
            s->adj[(size_t)a * m + r] = 1;
            s->adj[(size_t)r * m + a] = 1;
        }
    }
    for (int r = 0; r < m; r++) {
        s->adj[(size_t)b * m + r] = 0;
        s->adj[(size_t)r * m + b] = 0;
    }
    s->adj[(size_t)a * m + a] = 0;
    if (s->kmat) {
        for (int r = 0; r < m; r++) {
            if (r == a || !s->alive[r]) continue;
            double K = sect_key(s, a, r);
            s->kmat[(size_t)a * m + r] = K;
            s->kmat[(size_t)r * m + a] = K;
        }
    }
}

/* snapshot hook used at the root */
typedef struct snapctl snapctl_t;
static int take_snapshot(snapctl_t *c, const sect_t *s);

typedef struct { int i, j; double K; int64_t lo, hi; } mpair_t;

static int cmp_mpair(const void *a, const void *b)
{
    const mpair_t *x = (const mpair_t *)a, *y = (const mpair_t *)b;
    if (pair_less(x->K, x->lo, x->hi, y->K, y->lo, y->hi)) return -1;
    if (pair_less(y->K, y->lo, y->hi, x->K, x->lo, x->hi)) return 1;
    return 0;
}

/*
 * One stage of reading R12: spectral = 0 takes the adjacent pairs, 1 the
 * non-adjacent pairs with K < t.  Each region's best partner, then the
 * mutually best pairs merged in (K, lo, hi) order until the count reaches
 * the target.  *nmerged = merges done, *kfirst = key of the first merge.
 */
static int stage_multi(sect_t *s, int spectral, double t, int mode, int *count, int target, int level,
                       int section, int32_t iter, mlog_t *log, orc_stats *st, snapctl_t *snap,
                       int *nmerged, double *kfirst)
{
    int m = s->m;
    *nmerged = 0;
    *kfirst = INFINITY;
    if (m == 0) return ORC_OK;
    int *best = (int *)malloc((size_t)m * sizeof(int));
    double *bK = (double *)malloc((size_t)m * sizeof(double));
    mpair_t *P = (mpair_t *)malloc((size_t)(m / 2 + 1) * sizeof(mpair_t));
    if (!best || !bK || !P) { free(best); free(bK); free(P); return ORC_ENOMEM; }
    for (int i = 0; i < m; i++) { best[i] = -1; bK[i] = INFINITY; }
    int64_t npairs = 0;
    for (int i = 0; i < m; i++) {
        if (!s->alive[i]) continue;
        for (int j = i + 1; j < m; j++) {
            if (!s->alive[j]) continue;
            int a = s->adj[(size_t)i * m + j] != 0;
            if (a == spectral) continue;
            npairs++;
            double K = (mode == 1) ? s->kmat[(size_t)i * m + j] : sect_key(s, i, j);
            if (spectral && !(K < t)) continue;
            /* slots are in ID order: the pair is (id[i], id[j]) */
            if (best[i] < 0 || pair_less(K, s->id[i], s->id[j], bK[i],
                                         s->id[i] < s->id[best[i]] ? s->id[i] : s->id[best[i]],
                                         s->id[i] < s->id[best[i]] ? s->id[best[i]] : s->id[i])) {
                best[i] = j; bK[i] = K;
            }
            if (best[j] < 0 || pair_less(K, s->id[i], s->id[j], bK[j],
                                         s->id[j] < s->id[best[j]] ? s->id[j] : s->id[best[j]],
                                         s->id[j] < s->id[best[j]] ? s->id[best[j]] : s->id[j])) {
                best[j] = i; bK[j] = K;
            }
        }
    }
    st->pairs += npairs;
    int np = 0;
    for (int i = 0; i < m; i++) {
        int j = best[i];
        if (j > i && best[j] == i) {
            mpair_t q = { i, j, bK[i], s->id[i], s->id[j] };
            P[np++] = q;
        }
    }
    qsort(P, (size_t)np, sizeof(mpair_t), cmp_mpair);
    int rc = ORC_OK;
    for (int k = 0; k < np && *count > target; k++) {
        sect_merge(s, P[k].i, P[k].j);
        (*count)--;
        if (*nmerged == 0) *kfirst = P[k].K;
        (*nmerged)++;
        if (spectral) st->merges_spec++; else st->merges_adj++;
        orc_merge rec = { level, section, iter, spectral, P[k].lo, P[k].hi, P[k].K, sqrt(P[k].K), *count, 0 };
        if ((rc = log_push(log, rec))) break;
        if (snap && (rc = take_snapshot(snap, s))) break;
    }
    free(best); free(bK); free(P);
    return rc;
}

/*
 * HSEG on one section (steps 2-4 of Section 4.1 with readings R2-R4, R10).
 * Returns ORC_OK; *stalled set when an iteration merged nothing.
 */
static int hseg(sect_t *s, int target, double w, int mode, int multi, int level, int section,
                mlog_t *log, orc_stats *st, int64_t max_iters, snapctl_t *snap, int *stalled)
{
    int m = s->m;
    int count = 0;
    for (int i = 0; i < m; i++) count += s->alive[i];
    *stalled = 0;
    if (mode == 1) {
        for (int i = 0; i < m; i++)
            for (int j = i + 1; j < m; j++) {
                double K = sect_key(s, i, j);
                s->kmat[(size_t)i * m + j] = K;
                s->kmat[(size_t)j * m + i] = K;
            }
    }
    if (snap) { int rc = take_snapshot(snap, s); if (rc) return rc; }
    int32_t iter = 0;
    while (count > target) {
        if (max_iters > 0 && st->iterations >= max_iters) break;
        iter++;
        st->iterations++;
        if (multi) {
            /* reading R12: both stages merge every mutually best pair */
            int na = 0, ns = 0;
            double ka = INFINITY, ks = INFINITY;
            int rc = stage_multi(s, 0, INFINITY, mode, &count, target, level, section, iter, log, st, snap, &na, &ka);
            if (rc) return rc;
            if (count <= target) break;
            if (w > 0.0) {
                double t = na ? (w * w) * ka : INFINITY;
                rc = stage_multi(s, 1, t, mode, &count, target, level, section, iter, log, st, snap, &ns, &ks);
                if (rc) return rc;
            }
            if (na + ns == 0) { *stalled = 1; break; }
            continue;
        }
        /* --- step 2: adjacent pairs --- */
        int bi = -1, bj = -1;
        double bK = INFINITY;
        int64_t nadj = 0;
        for (int i = 0; i < m; i++) {
            if (!s->alive[i]) continue;
            for (int j = i + 1; j < m; j++) {
                if (!s->alive[j] || !s->adj[(size_t)i * m + j]) continue;
                nadj++;
                double K = (mode == 1) ? s->kmat[(size_t)i * m + j] : sect_key(s, i, j);
                if (bi < 0 || pair_less(K, s->id[i], s->id[j], bK, s->id[bi], s->id[bj])) {
                    bi = i; bj = j; bK = K;
                }
            }
        }
        st->pairs += nadj;
        int merged = 0;
        double Kadj = INFINITY;
        if (bi >= 0) {
            Kadj = bK;
            sect_merge(s, bi, bj);
            count--;
            merged = 1;
            st->merges_adj++;
            orc_merge rec = { level, section, iter, 0, s->id[bi], s->id[bj], bK, sqrt(bK), count, 0 };
            int rc = log_push(log, rec); if (rc) return rc;
            if (snap) { rc = take_snapshot(snap, s); if (rc) return rc; }
            if (count <= target) break;
        }
        /* --- step 3: non-adjacent pairs, threshold from step 2 --- */
        if (w > 0.0) {
            double t = (bi >= 0) ? (w * w) * Kadj : INFINITY;
            int ci = -1, cj = -1;
            double cK = INFINITY;
            int64_t nnon = 0;
            for (int i = 0; i < m; i++) {
                if (!s->alive[i]) continue;
                for (int j = i + 1; j < m; j++) {
                    if (!s->alive[j] || s->adj[(size_t)i * m + j]) continue;
                    nnon++;
                    double K = (mode == 1) ? s->kmat[(size_t)i * m + j] : sect_key(s, i, j);
                    if (!(K < t)) continue;
                    if (ci < 0 || pair_less(K, s->id[i], s->id[j], cK, s->id[ci], s->id[cj])) {
                        ci = i; cj = j; cK = K;
                    }
                }
            }
            st->pairs += nnon;
            if (ci >= 0) {
                sect_merge(s, ci, cj);
                count--;
                merged = 1;
                st->merges_spec++;
                orc_merge rec = { level, section, iter, 1, s->id[ci], s->id[cj], cK, sqrt(cK), count, 0 };
                int rc = log_push(log, rec); if (rc) return rc;
                if (snap) { rc = take_snapshot(snap, s); if (rc) return rc; }
            }
        }
        if (!merged) { *stalled = 1; break; }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Image geometry                                                            */
/* ------------------------------------------------------------------------- */

typedef struct { int r0, r1, c0, c1; } rect_t;

/* rectangle of Z-order section `s` at recursion level `lev` (level 1 = whole
 * image; reading R6) */
static rect_t section_rect(int rows, int cols, int lev, int64_t s)
{
    rect_t r = { 0, rows, 0, cols };
    for (int d = 1; d < lev; d++) {
        int digit = (int)((s >> (2 * (lev - 1 - d))) & 3);
        int h2 = (r.r1 - r.r0) / 2, w2 = (r.c1 - r.c0) / 2;
        if (digit == 0)      { r.r1 = r.r0 + h2; r.c1 = r.c0 + w2; }
        else if (digit == 1) { r.r1 = r.r0 + h2; r.c0 = r.c0 + w2; }
        else if (digit == 2) { r.r0 = r.r0 + h2; r.c1 = r.c0 + w2; }
        else                 { r.r0 = r.r0 + h2; r.c0 = r.c0 + w2; }
    }
    return r;
}

static int in_rect(const rect_t *r, int y, int x)
{
    return y >= r->r0 && y < r->r1 && x >= r->c0 && x < r->c1;
}

static const int NB8[8][2] = { {-1,-1},{-1,0},{-1,1},{0,-1},{0,1},{1,-1},{1,0},{1,1} };
static const int NB4[4][2] = { {-1,0},{0,-1},{0,1},{1,0} };

/* ------------------------------------------------------------------------- */
/* Whole-run state                                                           */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t id, n;
    int64_t *S;              /* [B] owned */
} oreg_t;

typedef struct { oreg_t *v; int n; } rlist_t;

typedef struct {
    int rows, cols, B;
    const uint16_t *img;
    const uint8_t *mask;
    orc_params p;
    int32_t *label;          /* [rows*cols] current region ID, 0 = masked */
    int32_t *slot_of_id;     /* scratch [rows*cols + 1] */
    mlog_t log;
    orc_stats st;
    /* snapshots */
    int nlev;
    int64_t *targets;        /* [nlev] region counts c_k */
    int32_t **snap_labels;   /* [nlev][rows*cols] */
    int64_t **snap_sums;     /* [nlev][R*B] */
    int64_t **snap_counts;   /* [nlev][R] */
    int32_t *snap_R;
} orc_run_t;

struct snapctl {
    orc_run_t *run;
    rect_t rect;
    int32_t *pix_slot;       /* [rows*cols]: slot at root start, -1 masked/outside */
    int next;                /* next snapshot index to take */
};

static int take_snapshot(snapctl_t *c, const sect_t *s)
{
    orc_run_t *R = c->run;
    int count = 0;
    for (int i = 0; i < s->m; i++) count += s->alive[i];
    while (c->next < R->nlev && count == R->targets[c->next]) {
        int k = c->next++;
        int P = R->rows * R->cols, B = R->B;
        int32_t *lab = (int32_t *)calloc((size_t)P, sizeof(int32_t));
        int32_t *canon = (int32_t *)malloc((size_t)(s->m ? s->m : 1) * sizeof(int32_t));
        if (!lab || !canon) { free(lab); free(canon); return ORC_ENOMEM; }
        /* live slots in ID order get canonical labels 1..R: first raster
         * appearance of a region is its smallest pixel index, i.e. its ID */
        int nr = 0;
        for (int i = 0; i < s->m; i++) canon[i] = s->alive[i] ? ++nr : 0;
        int64_t *sums = (int64_t *)calloc((size_t)(nr ? nr : 1) * B, sizeof(int64_t));
        int64_t *cnts = (int64_t *)calloc((size_t)(nr ? nr : 1), sizeof(int64_t));
        if (!sums || !cnts) { free(lab); free(canon); free(sums); free(cnts); return ORC_ENOMEM; }
        for (int i = 0; i < s->m; i++) {
            if (!s->alive[i]) continue;
            int cl = canon[i] - 1;
            cnts[cl] = s->n[i];
            memcpy(sums + (size_t)cl * B, s->S + (size_t)i * B, (size_t)B * sizeof(int64_t));
        }
        int *par = s->parent;
        for (int p = 0; p < P; p++) {
            int sl = c->pix_slot[p];
            if (sl < 0) continue;
            lab[p] = canon[find_root(par, sl)];
        }
        free(canon);
        R->snap_labels[k] = lab; R->snap_sums[k] = sums; R->snap_counts[k] = cnts; R->snap_R[k] = nr;
    }
    return ORC_OK;
}

static int pix_unmasked(const orc_run_t *R, int p)
{
    return R->mask ? (R->mask[p] == 0) : 1;
}

/* Build the section table from a region list (sorted by ID) and the label map. */
static int build_section(orc_run_t *R, const rect_t *rc, rlist_t *regs, sect_t *s)
{
    int B = R->B, cols = R->cols;
    int rcode = sect_alloc(s, regs->n, B, R->p.mode == 1);
    if (rcode) return rcode;
    for (int i = 0; i < regs->n; i++) {
        s->id[i] = regs->v[i].id;
        s->n[i] = regs->v[i].n;
        memcpy(s->S + (size_t)i * B, regs->v[i].S, (size_t)B * sizeof(int64_t));
        R->slot_of_id[regs->v[i].id] = i;
    }
    int m = regs->n;
    if (R->p.full_adjacency) {
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++)
                s->adj[(size_t)i * m + j] = (i != j);
        return ORC_OK;
    }
    int nn = R->p.connectivity == 4 ? 4 : 8;
    const int (*nb)[2] = R->p.connectivity == 4 ? NB4 : NB8;
    for (int y = rc->r0; y < rc->r1; y++)
        for (int x = rc->c0; x < rc->c1; x++) {
            int p = y * cols + x;
            if (!pix_unmasked(R, p)) continue;
            for (int k = 0; k < nn; k++) {
                int yy = y + nb[k][0], xx = x + nb[k][1];
                if (!in_rect(rc, yy, xx)) continue;
                int q = yy * cols + xx;
                if (!pix_unmasked(R, q)) continue;
                if (R->label[p] == R->label[q]) continue;
                int a = R->slot_of_id[R->label[p]], b = R->slot_of_id[R->label[q]];
                s->adj[(size_t)a * m + b] = 1;
                s->adj[(size_t)b * m + a] = 1;
            }
        }
    return ORC_OK;
}

static int cmp_oreg(const void *a, const void *b)
{
    int64_t x = ((const oreg_t *)a)->id, y = ((const oreg_t *)b)->id;
    return (x > y) - (x < y);
}

static void rlist_free(rlist_t *l)
{
    for (int i = 0; i < l->n; i++) free(l->v[i].S);
    free(l->v);
    l->v = NULL; l->n = 0;
}

/* After HSEG: survivors into a list, pixel labels to survivor IDs. */
static int collect_survivors(orc_run_t *R, const rect_t *rc, sect_t *s, rlist_t *out)
{
    int B = R->B, cols = R->cols;
    int nr = 0;
    for (int i = 0; i < s->m; i++) nr += s->alive[i];
    out->v = (oreg_t *)calloc((size_t)(nr ? nr : 1), sizeof(oreg_t));
    out->n = 0;
    if (!out->v) return ORC_ENOMEM;
    for (int i = 0; i < s->m; i++) {
        if (!s->alive[i]) continue;
        oreg_t r;
        r.id = s->id[i]; r.n = s->n[i];
        r.S = (int64_t *)malloc((size_t)B * sizeof(int64_t));
        if (!r.S) return ORC_ENOMEM;
        memcpy(r.S, s->S + (size_t)i * B, (size_t)B * sizeof(int64_t));
        out->v[out->n++] = r;
    }
    for (int y = rc->r0; y < rc->r1; y++)
        for (int x = rc->c0; x < rc->c1; x++) {
            int p = y * cols + x;
            if (!pix_unmasked(R, p)) continue;
            int sl = R->slot_of_id[R->label[p]];
            R->label[p] = (int32_t)s->id[find_root(s->parent, sl)];
        }
    return ORC_OK;
}

/* Seam pass (reading R7) on parent rectangle `pr` whose regions are `regs`
 * (sorted by ID, labels current).  Modifies regs and labels in place. */
static int seam_pass(orc_run_t *R, const rect_t *pr, int lev, int64_t sec, rlist_t *regs, mlog_t *log,
                     orc_stats *st)
{
    int B = R->B, cols = R->cols;
    int h2 = (pr->r1 - pr->r0) / 2, w2 = (pr->c1 - pr->c0) / 2;
    int nn = R->p.connectivity == 4 ? 4 : 8;
    const int (*nb)[2] = R->p.connectivity == 4 ? NB4 : NB8;
    for (int i = 0; i < regs->n; i++) R->slot_of_id[regs->v[i].id] = i;
    int area = (pr->r1 - pr->r0) * (pr->c1 - pr->c0);
    int32_t *split_of = (int32_t *)malloc((size_t)(area ? area : 1) * sizeof(int32_t)); /* region slot or -1 */
    double *split_key = (double *)malloc((size_t)(area ? area : 1) * sizeof(double));
    int64_t *xp = (int64_t *)malloc((size_t)B * sizeof(int64_t));
    if (!split_of || !split_key || !xp) { free(split_of); free(split_key); free(xp); return ORC_ENOMEM; }
    int nsplit = 0;
    /* decisions against the pre-pass state */
    for (int y = pr->r0; y < pr->r1; y++)
        for (int x = pr->c0; x < pr->c1; x++) {
            int li = (y - pr->r0) * (pr->c1 - pr->c0) + (x - pr->c0);
            split_of[li] = -1;
            int p = y * cols + x;
            if (!pix_unmasked(R, p)) continue;
            int qy = (y - pr->r0) >= h2, qx = (x - pr->c0) >= w2;
            int rs = R->slot_of_id[R->label[p]];
            const oreg_t *Rg = &regs->v[rs];
            for (int b = 0; b < B; b++) xp[b] = R->img[(size_t)p * B + b];
            int seam = 0;
            double best = INFINITY;
            for (int k = 0; k < nn; k++) {
                int yy = y + nb[k][0], xx = x + nb[k][1];
                if (!in_rect(pr, yy, xx)) continue;
                int q = yy * cols + xx;
                if (!pix_unmasked(R, q)) continue;
                int qqy = (yy - pr->r0) >= h2, qqx = (xx - pr->c0) >= w2;
                if (qqy == qy && qqx == qx) continue;
                seam = 1;
                const oreg_t *Qg = &regs->v[R->slot_of_id[R->label[q]]];
                double K = orc_key(1, xp, Qg->n, Qg->S, B);
                if (K < best) best = K;
            }
            if (!seam) continue;
            double Kr = orc_key(1, xp, Rg->n, Rg->S, B);
            if (best < Kr) { split_of[li] = rs; split_key[li] = Kr; nsplit++; }
        }
    /* apply all splits together */
    oreg_t *nv = (oreg_t *)realloc(regs->v, (size_t)(regs->n + nsplit + 1) * sizeof(oreg_t));
    if (!nv) { free(split_of); free(split_key); free(xp); return ORC_ENOMEM; }
    regs->v = nv;
    int nold = regs->n;
    int64_t *old_id = (int64_t *)malloc((size_t)(nold ? nold : 1) * sizeof(int64_t));
    if (!old_id) { free(split_of); free(split_key); free(xp); return ORC_ENOMEM; }
    for (int i = 0; i < nold; i++) old_id[i] = regs->v[i].id;
    /* records are emitted after the count is known; remember them */
    for (int y = pr->r0; y < pr->r1; y++)
        for (int x = pr->c0; x < pr->c1; x++) {
            int li = (y - pr->r0) * (pr->c1 - pr->c0) + (x - pr->c0);
            int rs = split_of[li];
            if (rs < 0) continue;
            int p = y * cols + x;
            oreg_t *Rg = &regs->v[rs];
            oreg_t sg;
            sg.id = (int64_t)p + 1; sg.n = 1;
            sg.S = (int64_t *)malloc((size_t)B * sizeof(int64_t));
            if (!sg.S) { free(split_of); free(split_key); free(xp); free(old_id); return ORC_ENOMEM; }
            for (int b = 0; b < B; b++) {
                sg.S[b] = R->img[(size_t)p * B + b];
                Rg->S[b] -= sg.S[b];
            }
            Rg->n -= 1;
            regs->v[regs->n++] = sg;
            R->label[p] = -(rs + 1);          /* mark: singleton, parent slot rs */
        }
    /* re-derive IDs: 1 + smallest raster index of remaining pixels */
    int64_t *newid = (int64_t *)malloc((size_t)(nold ? nold : 1) * sizeof(int64_t));
    if (!newid) { free(split_of); free(split_key); free(xp); free(old_id); return ORC_ENOMEM; }
    for (int i = 0; i < nold; i++) newid[i] = INT64_MAX;
    for (int y = pr->r0; y < pr->r1; y++)
        for (int x = pr->c0; x < pr->c1; x++) {
            int p = y * cols + x;
            if (!pix_unmasked(R, p) || R->label[p] < 0) continue;
            int sl = R->slot_of_id[R->label[p]];
            if ((int64_t)p + 1 < newid[sl]) newid[sl] = (int64_t)p + 1;
        }
    for (int y = pr->r0; y < pr->r1; y++)
        for (int x = pr->c0; x < pr->c1; x++) {
            int p = y * cols + x;
            if (!pix_unmasked(R, p)) continue;
            if (R->label[p] < 0) R->label[p] = p + 1;
            else R->label[p] = (int32_t)newid[R->slot_of_id[R->label[p]]];
        }
    for (int i = 0; i < nold; i++) regs->v[i].id = newid[i];
    /* drop empty regions, sort by ID */
    int k = 0;
    for (int i = 0; i < regs->n; i++) {
        if (regs->v[i].n == 0) { free(regs->v[i].S); continue; }
        regs->v[k++] = regs->v[i];
    }
    regs->n = k;
    qsort(regs->v, (size_t)regs->n, sizeof(oreg_t), cmp_oreg);
    /* log records in raster order of the split pixels */
    int rc = ORC_OK;
    for (int y = pr->r0; y < pr->r1 && rc == ORC_OK; y++)
        for (int x = pr->c0; x < pr->c1; x++) {
            int li = (y - pr->r0) * (pr->c1 - pr->c0) + (x - pr->c0);
            int rs = split_of[li];
            if (rs < 0) continue;
            int p = y * cols + x;
            orc_merge m = { lev, (int32_t)sec, 0, 2, old_id[rs], (int64_t)p + 1,
                            split_key[li], sqrt(split_key[li]), regs->n, 0 };
            rc = log_push(log, m);
            if (rc) break;
            st->seam_splits++;
        }
    free(split_of); free(split_key); free(xp); free(old_id); free(newid);
    return rc;
}

/* output level targets (reading R9) */
static int make_targets(orc_run_t *R, int64_t c0)
{
    int K = R->p.n_out_levels > 0 ? R->p.n_out_levels : 1;
    int64_t conv = R->p.conv_nregions;
    int64_t *t = (int64_t *)malloc((size_t)K * sizeof(int64_t));
    if (!t) return ORC_ENOMEM;
    if (c0 <= conv) {
        t[0] = c0; K = 1;
    } else if (K == 1) {
        t[0] = conv;
    } else {
        for (int k = 0; k < K; k++) {
            if (k == 0) t[k] = c0;
            else if (k == K - 1) t[k] = conv;
            else {
                double v = (double)conv * pow((double)c0 / (double)conv, (double)(K - 1 - k) / (double)(K - 1));
                t[k] = (int64_t)nearbyint(v);   /* default rounding mode: nearest-even */
            }
        }
    }
    int n = 0;
    for (int k = 0; k < K; k++)
        if (n == 0 || t[k] != t[n - 1]) t[n++] = t[k];
    R->nlev = n;
    R->targets = t;
    R->snap_labels = (int32_t **)calloc((size_t)n, sizeof(int32_t *));
    R->snap_sums = (int64_t **)calloc((size_t)n, sizeof(int64_t *));
    R->snap_counts = (int64_t **)calloc((size_t)n, sizeof(int64_t *));
    R->snap_R = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!R->snap_labels || !R->snap_sums || !R->snap_counts || !R->snap_R) return ORC_ENOMEM;
    return ORC_OK;
}

void orc_free(void *h);

/* exact-key range check: B * (P^2/4 * maxval)^2 < 2^127 and P^2/4*maxval < 2^62 */
static int range_ok(int64_t P, int64_t maxval, int B)
{
    long double a = (long double)P * (long double)P / 4.0L * (long double)maxval;
    if (a >= ldexpl(1.0L, 62)) return 0;
    return (long double)B * a * a < ldexpl(1.0L, 127);
}

/*
 * One section of one level (Section 4.1): its regions (the pixels at the
 * deepest level; else the survivors of its four children, then the seam
 * pass), HSEG to the section's target, the survivors into cur[s].  The
 * section writes only the label-map pixels of its own rectangle and the
 * slot_of_id entries of its own region IDs (an ID is a raster index of one
 * of its pixels), and its records and counters go to its own log and stats;
 * so the sections of one level are independent, as the recursion makes them.
 */
static int run_section(orc_run_t *R, int lev, int64_t s, rlist_t *prev, rlist_t *cur, mlog_t *log, orc_stats *st)
{
    const orc_params *p = &R->p;
    int rows = R->rows, cols = R->cols, bands = R->B;
    int64_t P = (int64_t)rows * cols;
    int L = p->rnb_levels;
    int min_nr = p->min_nregions > 0 ? p->min_nregions : p->conv_nregions;
    rect_t rc_ = section_rect(rows, cols, lev, s);
    rlist_t regs = { NULL, 0 };
    int rc = ORC_OK;
    if (lev == L) {
        int area = (rc_.r1 - rc_.r0) * (rc_.c1 - rc_.c0);
        regs.v = (oreg_t *)calloc((size_t)(area ? area : 1), sizeof(oreg_t));
        if (!regs.v) return ORC_ENOMEM;
        for (int y = rc_.r0; y < rc_.r1 && rc == ORC_OK; y++)
            for (int x = rc_.c0; x < rc_.c1; x++) {
                int q = y * cols + x;
                if (!pix_unmasked(R, q)) continue;
                oreg_t r;
                r.id = (int64_t)q + 1; r.n = 1;
                r.S = (int64_t *)malloc((size_t)bands * sizeof(int64_t));
                if (!r.S) { rc = ORC_ENOMEM; break; }
                for (int b = 0; b < bands; b++) r.S[b] = R->img[(size_t)q * bands + b];
                regs.v[regs.n++] = r;
            }
        if (rc) { rlist_free(&regs); return rc; }
    } else {
        int tot = 0;
        for (int c = 0; c < 4; c++) tot += prev[4 * s + c].n;
        regs.v = (oreg_t *)calloc((size_t)(tot ? tot : 1), sizeof(oreg_t));
        if (!regs.v) return ORC_ENOMEM;
        for (int c = 0; c < 4; c++) {
            rlist_t *ch = &prev[4 * s + c];
            for (int i = 0; i < ch->n; i++) regs.v[regs.n++] = ch->v[i];
            free(ch->v); ch->v = NULL; ch->n = 0;   /* ownership moved */
        }
        qsort(regs.v, (size_t)regs.n, sizeof(oreg_t), cmp_oreg);
        if (p->seam_pass) {
            rc = seam_pass(R, &rc_, lev, s, &regs, log, st);
            if (rc) { rlist_free(&regs); return rc; }
        }
    }
    sect_t sec;
    rc = build_section(R, &rc_, &regs, &sec);
    if (rc) { rlist_free(&regs); return rc; }
    snapctl_t sc, *scp = NULL;
    int32_t *pix_slot = NULL;
    if (lev == 1) {
        rc = make_targets(R, (int64_t)regs.n);
        if (rc) { sect_free(&sec); rlist_free(&regs); return rc; }
        pix_slot = (int32_t *)malloc((size_t)P * sizeof(int32_t));
        if (!pix_slot) { sect_free(&sec); rlist_free(&regs); return ORC_ENOMEM; }
        for (int64_t q = 0; q < P; q++)
            pix_slot[q] = R->label[q] ? R->slot_of_id[R->label[q]] : -1;
        sc.run = R; sc.rect = rc_; sc.pix_slot = pix_slot; sc.next = 0;
        scp = &sc;
    }
    rlist_free(&regs);
    int target = (lev == 1) ? p->conv_nregions : min_nr;
    int stalled = 0;
    rc = hseg(&sec, target, p->spclust_wght, p->mode, p->multi_merge, lev, (int32_t)s, log, st, 0, scp, &stalled);
    if (stalled) st->stalled_sections++;
    if (rc == ORC_OK && scp) {
        /* levels never reached (stall) take the final state */
        while (sc.next < R->nlev) {
            R->targets[sc.next] = 0;
            for (int i = 0; i < sec.m; i++) R->targets[sc.next] += sec.alive[i];
            rc = take_snapshot(&sc, &sec);
            if (rc) break;
        }
    }
    free(pix_slot);
    if (rc == ORC_OK) rc = collect_survivors(R, &rc_, &sec, &cur[s]);
    sect_free(&sec);
    return rc;
}

/* The sections of one level, shared out to worker threads one at a time. */
typedef struct {
    orc_run_t *R;
    int lev;
    int64_t nsec;
    rlist_t *prev, *cur;
    mlog_t *logs;            /* [nsec] */
    orc_stats *sts;          /* [nsec] */
    int *rcs;                /* [nsec] */
    int64_t next;            /* next section to take (atomic) */
} level_job_t;

static void *level_worker(void *arg)
{
    level_job_t *J = (level_job_t *)arg;
    for (;;) {
        int64_t s = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (s >= J->nsec) break;
        J->rcs[s] = run_section(J->R, J->lev, s, J->prev, J->cur, &J->logs[s], &J->sts[s]);
    }
    return NULL;
}

/*
 * Full RHSEG run.  img is [rows][cols][bands] uint16, mask [rows][cols]
 * (nonzero = no data) or NULL.  The sections of a level run on `nthreads`
 * threads (1 = all in the calling thread); their records are then joined in
 * Z order, so the log, the levels and the counters do not depend on
 * nthreads.  Returns a handle or NULL with *err set.
 */
void *orc_run_threads(const uint16_t *img, int32_t rows, int32_t cols, int32_t bands,
                      const uint8_t *mask, const orc_params *p, int32_t nthreads, int32_t *err)
{
    *err = ORC_OK;
    if (!img || rows <= 0 || cols <= 0 || bands <= 0 || !p || p->rnb_levels < 1 ||
        p->rnb_levels > 12 || !(p->spclust_wght >= 0.0 && p->spclust_wght <= 1.0) ||
        p->conv_nregions < 1 || (p->connectivity != 4 && p->connectivity != 8) ||
        p->min_nregions < 0 || p->n_out_levels < 0 || (p->mode != 0 && p->mode != 1) ||
        (p->multi_merge != 0 && p->multi_merge != 1) || nthreads < 1 || nthreads > 1024 ||
        (int64_t)rows * cols >= ((int64_t)1 << 31) - 1) {
        *err = ORC_EINVAL;
        return NULL;
    }
    int64_t P = (int64_t)rows * cols;
    int64_t unmasked = 0, maxval = 0;
    for (int64_t q = 0; q < P; q++) {
        if (mask && mask[q]) continue;
        unmasked++;
        for (int b = 0; b < bands; b++)
            if (img[q * bands + b] > maxval) maxval = img[q * bands + b];
    }
    if (!range_ok(unmasked, maxval, bands)) { *err = ORC_ERANGE; return NULL; }

    orc_run_t *R = (orc_run_t *)calloc(1, sizeof(orc_run_t));
    if (!R) { *err = ORC_ENOMEM; return NULL; }
    R->rows = rows; R->cols = cols; R->B = bands; R->img = img; R->mask = mask; R->p = *p;
    R->label = (int32_t *)calloc((size_t)P, sizeof(int32_t));
    R->slot_of_id = (int32_t *)calloc((size_t)P + 1, sizeof(int32_t));
    if (!R->label || !R->slot_of_id) { orc_free(R); *err = ORC_ENOMEM; return NULL; }
    for (int64_t q = 0; q < P; q++) R->label[q] = (mask && mask[q]) ? 0 : (int32_t)(q + 1);

    int L = p->rnb_levels;
    rlist_t *prev = NULL;    /* survivors of the level below, by section */
    int rc = ORC_OK;
    for (int lev = L; lev >= 1 && rc == ORC_OK; lev--) {
        int64_t nsec = (int64_t)1 << (2 * (lev - 1));
        rlist_t *cur = (rlist_t *)calloc((size_t)nsec, sizeof(rlist_t));
        mlog_t *logs = (mlog_t *)calloc((size_t)nsec, sizeof(mlog_t));
        orc_stats *sts = (orc_stats *)calloc((size_t)nsec, sizeof(orc_stats));
        int *rcs = (int *)calloc((size_t)nsec, sizeof(int));
        if (!cur || !logs || !sts || !rcs) {
            free(cur); free(logs); free(sts); free(rcs);
            rc = ORC_ENOMEM;
            break;
        }
        level_job_t J = { R, lev, nsec, prev, cur, logs, sts, rcs, 0 };
        int nt = nthreads < nsec ? nthreads : (int)nsec;
        if (nt <= 1) {
            level_worker(&J);
        } else {
            pthread_t *tid = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
            int started = 0;
            if (tid)
                for (; started < nt; started++)
                    if (pthread_create(&tid[started], NULL, level_worker, &J) != 0) break;
            if (started == 0) level_worker(&J);      /* no thread could start: run here */
            for (int t = 0; t < started; t++) pthread_join(tid[t], NULL);
            free(tid);
        }
        /* records and counters joined in Z order of the sections */
        for (int64_t s = 0; s < nsec; s++) {
            if (rcs[s] && rc == ORC_OK) rc = rcs[s];
            for (int64_t k = 0; k < logs[s].n && rc == ORC_OK; k++) rc = log_push(&R->log, logs[s].v[k]);
            R->st.pairs += sts[s].pairs;
            R->st.iterations += sts[s].iterations;
            R->st.merges_adj += sts[s].merges_adj;
            R->st.merges_spec += sts[s].merges_spec;
            R->st.seam_splits += sts[s].seam_splits;
            R->st.stalled_sections += sts[s].stalled_sections;
            free(logs[s].v);
        }
        free(logs); free(sts); free(rcs);
        if (prev) {
            int64_t pn = nsec * 4;
            for (int64_t s = 0; s < pn; s++) rlist_free(&prev[s]);
            free(prev);
        }
        prev = cur;
    }
    if (prev) { rlist_free(&prev[0]); free(prev); }
    R->st.n_levels_out = R->nlev;
    if (rc) { orc_free(R); *err = rc; return NULL; }
    return R;
}

/* Full RHSEG run in the calling thread (see orc_run_threads). */
void *orc_run(const uint16_t *img, int32_t rows, int32_t cols, int32_t bands,
              const uint8_t *mask, const orc_params *p, int32_t *err)
{
    return orc_run_threads(img, rows, cols, bands, mask, p, 1, err);
}

int64_t orc_log_len(void *h) { return ((orc_run_t *)h)->log.n; }

void orc_get_log(void *h, orc_merge *out)
{
    orc_run_t *R = (orc_run_t *)h;
    memcpy(out, R->log.v, (size_t)R->log.n * sizeof(orc_merge));
}

int32_t orc_n_levels(void *h) { return ((orc_run_t *)h)->nlev; }

int32_t orc_level_nregions(void *h, int32_t k)
{
    orc_run_t *R = (orc_run_t *)h;
    if (k < 0 || k >= R->nlev) return -1;
    return R->snap_R[k];
}

int32_t orc_get_level(void *h, int32_t k, int32_t *labels, int64_t *sums, int64_t *counts)
{
    orc_run_t *R = (orc_run_t *)h;
    if (k < 0 || k >= R->nlev) return ORC_EINVAL;
    int64_t P = (int64_t)R->rows * R->cols;
    int nr = R->snap_R[k];
    if (labels) memcpy(labels, R->snap_labels[k], (size_t)P * sizeof(int32_t));
    if (sums) memcpy(sums, R->snap_sums[k], (size_t)nr * R->B * sizeof(int64_t));
    if (counts) memcpy(counts, R->snap_counts[k], (size_t)nr * sizeof(int64_t));
    return ORC_OK;
}

void orc_get_stats(void *h, orc_stats *s) { *s = ((orc_run_t *)h)->st; }

void orc_free(void *h)
{
    orc_run_t *R = (orc_run_t *)h;
    if (!R) return;
    free(R->label); free(R->slot_of_id); free(R->log.v); free(R->targets);
    for (int k = 0; k < R->nlev; k++) {
        if (R->snap_labels) free(R->snap_labels[k]);
        if (R->snap_sums) free(R->snap_sums[k]);
        if (R->snap_counts) free(R->snap_counts[k]);
    }
    free(R->snap_labels); free(R->snap_sums); free(R->snap_counts); free(R->snap_R);
    free(R);
}

/*
 * HSEG of one deepest-level section in isolation (pixels as regions), for at
 * most max_iters iterations (0 = to the target).  The deepest sections are
 * independent, so this reproduces exactly the part of a full run that
 * belongs to that section; used for sampled checks at full image size and
 * for the bounded CPU baseline.  Writes up to log_cap records.
 */
int32_t orc_hseg_leaf(const uint16_t *img, int32_t rows, int32_t cols, int32_t bands,
                      const uint8_t *mask, const orc_params *p, int64_t section,
                      int64_t max_iters, orc_merge *log_out, int64_t log_cap,
                      int64_t *log_len, orc_stats *st_out)
{
    if (!img || rows <= 0 || cols <= 0 || bands <= 0 || !p || p->rnb_levels < 1 ||
        (p->connectivity != 4 && p->connectivity != 8) || (p->mode != 0 && p->mode != 1) ||
        (p->multi_merge != 0 && p->multi_merge != 1) ||
        section < 0 || section >= ((int64_t)1 << (2 * (p->rnb_levels - 1))))
        return ORC_EINVAL;
    orc_run_t *R = (orc_run_t *)calloc(1, sizeof(orc_run_t));
    if (!R) return ORC_ENOMEM;
    int64_t P = (int64_t)rows * cols;
    R->rows = rows; R->cols = cols; R->B = bands; R->img = img; R->mask = mask; R->p = *p;
    R->label = (int32_t *)calloc((size_t)P, sizeof(int32_t));
    R->slot_of_id = (int32_t *)calloc((size_t)P + 1, sizeof(int32_t));
    if (!R->label || !R->slot_of_id) { orc_free(R); return ORC_ENOMEM; }
    for (int64_t q = 0; q < P; q++) R->label[q] = (mask && mask[q]) ? 0 : (int32_t)(q + 1);
    int L = p->rnb_levels;
    rect_t rc_ = section_rect(rows, cols, L, section);
    rlist_t regs = { NULL, 0 };
    int area = (rc_.r1 - rc_.r0) * (rc_.c1 - rc_.c0);
    regs.v = (oreg_t *)calloc((size_t)(area ? area : 1), sizeof(oreg_t));
    if (!regs.v) { orc_free(R); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (int y = rc_.r0; y < rc_.r1 && rc == ORC_OK; y++)
        for (int x = rc_.c0; x < rc_.c1; x++) {
            int q = y * cols + x;
            if (!pix_unmasked(R, q)) continue;
            oreg_t r;
            r.id = (int64_t)q + 1; r.n = 1;
            r.S = (int64_t *)malloc((size_t)bands * sizeof(int64_t));
            if (!r.S) { rc = ORC_ENOMEM; break; }
            for (int b = 0; b < bands; b++) r.S[b] = img[(size_t)q * bands + b];
            regs.v[regs.n++] = r;
        }
    sect_t sec;
    if (rc == ORC_OK) rc = build_section(R, &rc_, &regs, &sec);
    rlist_free(&regs);
    if (rc == ORC_OK) {
        int target = (L == 1) ? p->conv_nregions : (p->min_nregions > 0 ? p->min_nregions : p->conv_nregions);
        int stalled = 0;
        rc = hseg(&sec, target, p->spclust_wght, p->mode, p->multi_merge, L, (int32_t)section, &R->log, &R->st,
                  max_iters, NULL, &stalled);
        if (stalled) R->st.stalled_sections++;
        sect_free(&sec);
    }
    if (rc == ORC_OK) {
        if (log_len) *log_len = R->log.n;
        if (log_out) {
            int64_t n = R->log.n < log_cap ? R->log.n : log_cap;
            memcpy(log_out, R->log.v, (size_t)n * sizeof(orc_merge));
        }
        if (st_out) *st_out = R->st;
    }
    orc_free(R);
    return rc;
}
