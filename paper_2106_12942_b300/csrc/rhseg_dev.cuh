// rhseg_dev.cuh -- device-side data structures and exact arithmetic shared by
// the RHSEG kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define RHSEG_KEY_NONE 0xFFFFFFFFFFFFFFFFull   // larger than the bits of any K (incl. +inf)
#define RHSEG_INF_BITS 0x7FF0000000000000ull

namespace rhseg {

// ---------------------------------------------------------------------------
// Per-section device state (one record per section of the current level).
// ---------------------------------------------------------------------------
struct SecState {
    int32_t m0;            // slots (regions at level start)
    int32_t count;         // live regions
    int32_t target;
    int32_t done;          // finished: target reached or stalled
    int32_t stalled;
    int32_t iter;          // HSEG iterations done
    int32_t spec_pending;  // the spectral step of this iteration is still to run
    int32_t merged_adj;    // the adjacent step of this iteration merged
    int32_t mc;            // compact positions in use by the screen
    int32_t nmerge;        // merges done at this level (ordinal of the last one)
    double  Kadj;          // key of this iteration's adjacent merge (+inf if none)
    double  tthr;          // (w*w) * Kadj
    int64_t nadj;          // adjacent pairs (undirected) currently
    int64_t pairs;         // dissimilarities the method defines, accumulated
    int64_t screened;      // pairs evaluated by the screen
    int64_t cands;         // candidates passed to the exact re-check
    int64_t cands_true;    // of those, non-adjacent pairs with exact K below the threshold
    int64_t fallbacks;     // spectral steps resolved exhaustively
    int64_t log_n;         // records written in this section's log segment
    uint32_t ncand;        // candidates emitted in the current step
    int32_t madj, mspec;   // merges by kind
    int32_t nsplit;        // seam splits applied at the start of this level
    int32_t rows_from;     // > 0: the position list was rebuilt this iteration (old extent)
    int32_t pm_a[2], pm_b[2];   // incremental mode: merges (survivor, absorbed) whose rows are pending
    int32_t npm;
    int32_t nunits;        // tensor-core screen: units kept for this step (the rest are proven empty)
    int64_t evaluated;     // pairs covered by the kept units, accumulated
    // screening error of the tensor-core screen over the re-checked pairs:
    // max |K~ - K| / K and max |K~ - K| / bound (binary32 bits, non-negative)
    uint32_t err_rel_bits, err_bnd_bits;
    int64_t err_pairs;     // re-checked pairs the two maxima cover
    int32_t ranges_stale;  // the kept norm ranges of the position blocks need a full recompute
    int32_t ptop;          // CSR adjacency: words in use in the current half of the section's pool
    int32_t phalf;         // CSR adjacency: the half of the pool in use (0 or 1)
    int32_t pad3;
    int64_t useful;        // of the pairs the kept units cover, those (i, j), i < j, of positions below mc
};

// Geometry and buffers of the level in flight (device pointers).  Arrays
// indexed by "slot" are section-local: slot s of section k lives at global
// index roff[k] + s.  Positions (screen rows) likewise at poff[k] + pos.
struct LevelDev {
    int32_t level, nsec, B, Bs, Bpad;
    int32_t precision;
    double  w, ww;
    int32_t sigma_shift;       // fp16 operand scaling 2^-sigma
    // per section
    SecState *st;
    const int64_t *roff;       // slot offsets
    const int64_t *poff;       // position offsets (multiple of 128)
    const int64_t *aoff;       // adjacency word offsets
    const int32_t *W;          // words per adjacency row
    const int64_t *loff;       // log segment offsets
    const int32_t *ref;        // [nsec][Bs] reference spectrum
    const int32_t *rect;       // [nsec][4] r0, r1, c0, c1
    // per slot
    int64_t *S;                // [nslots][Bs]
    int64_t *n;
    uint32_t *rid;
    uint8_t *alive;
    int32_t *parent;
    int32_t *absorbed_at;      // merge ordinal at which the slot was absorbed (INT_MAX alive)
    uint64_t *bestK;           // K bits of the best adjacent pair of the slot
    int32_t *bestP;            // partner slot of that pair
    int32_t *pos_of_slot;
    // per position
    int32_t *slot_of_pos;
    void    *X;                // [npos][Bpad] half/bf16 (precision 1/2) or double (0)
    float   *Af;  float  *kf;  // screen row terms (precision 1/2)
    float   *H;                // h_i = (A_i - T k_i) / 2 of the current step (tensor-core screen)
    double  *Ad;  double *kd;  // screen row terms (precision 0)
    // adjacency bitmaps
    uint32_t *adj;
    // CSR adjacency (csr = 1; the bitmap fields are then unused): slot r's
    // neighbour slots, sorted ascending, at nbr[pbase[k] + phalf * hcap[k] +
    // nofs[r]], ndeg[r] of them; each section's pool has two halves of
    // hcap[k] words, used in turn by the compaction
    int32_t csr;
    int32_t *nbr;
    const int64_t *pbase;
    const int64_t *hcap;
    int32_t *nofs, *ndeg;
    // candidates
    uint32_t *cand;            // [nsec][cand_cap][2] positions
    int64_t cand_cap;
    float *candg;              // [nsec][cand_cap] the screen's tested value g - h_j of each
                               // candidate (tensor-core forms; null otherwise)
    float *qf;                 // per position: binary32 ||x^||^2 of the operand row (with candg)
    double err_gamma, err_u, err_etaB;   // the screen's gamma, u and eta sqrt(B) (error report)
    // log
    void *log;                 // rhseg_merge records
    int32_t *err;              // device error word
    long long wait_cycles;     // bound of the screen's pipeline waits (0: the default)
    int32_t tc_group;          // K slices per tcgen05.commit of the screen (0: the default)
    int32_t tc_pair;           // 1: the screen runs as CTA pairs; ulist then lists unit pairs
    int32_t count_useful;      // 1 (with per-kernel timing): count the useful pairs of the kept units
    int32_t *wlist;            // [nsec] sections whose positions were rebuilt this iteration
    int32_t *wcount;           // their number
    // incremental spectral minima (null unless that mode is on)
    int32_t incremental;
    uint64_t *sbK;             // per slot: K bits of the best non-adjacent pair
    int32_t *sbP;              // per slot: partner slot of that pair
    unsigned long long *stie;  // per slot: scratch (lowest slot pair among equal keys)
    uint8_t *inR;              // per slot: scratch (row listed for recomputation)
    int32_t *srow;             // per slot: scratch (rows to recompute)
    unsigned long long *sinit; // per position: approximate argmin, then the row's bound
    float *sT;                 // per position: the row's binary32 threshold
    float *sE, *sk;            // per position: operand error norm, 4^-sigma / n (both rounded up)
    float *nlo, *nhi;          // per position: bounds of the true norm ||x|| of the row (tensor-core screen)
    float *brng;               // per 128-position block x 4: kept (min nlo, max nhi, max sk), exact at a
                               // rebuild and widened by every merge since (tensor-core screen)
    int32_t *ulist;            // [nsec][ucap] kept units of the step, (I << 16) | Jp; with tc_pair
                               // pairs of kept units of one column block Jp: (I0 << 16) | Jp, I1 (-1: none)
    int32_t ucap;
    unsigned long long *sortk; // per slot x 2: scratch of the norm-order sort of the positions
    float inc_onepg;           // 1 + gamma_B for a binary32 sum of Bpad non-negative terms (rounded up)
    float *sbuf;               // per position x 8: scratch (sums of squared differences of a row update)
    float *srowx;              // per section: staged row vectors of a row update [Bpad][8]
    struct IncInfo *sinfo;     // per section: state of a row update between its kernels
    unsigned long long *ckey;  // [nsec][cand_cap] exact keys of candidates
    // several merges per iteration (reading R12; null unless that mode is on)
    int32_t multi;
    unsigned long long *mlist; // per slot x 2: the stage's mutually best pairs (K bits, (i << 32) | j)
    uint64_t *mK;              // per slot: K bits of the best below-threshold non-adjacent pair
    uint32_t *mP;              // per slot: partner slot of that pair (~0u: none)
};

// ---------------------------------------------------------------------------
// Exact 128-bit helpers
// ---------------------------------------------------------------------------
struct u128 { uint64_t lo, hi; };

__device__ __forceinline__ u128 u128_add(u128 a, u128 b)
{
    u128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}

__device__ __forceinline__ u128 u128_sq(uint64_t a)
{
    u128 r;
    r.lo = a * a;
    r.hi = __umul64hi(a, a);
    return r;
}

__device__ __forceinline__ u128 u128_mul64(uint64_t a, uint64_t b)
{
    u128 r;
    r.lo = a * b;
    r.hi = __umul64hi(a, b);
    return r;
}

__device__ __forceinline__ u128 warp_sum_u128(u128 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        u128 t;
        t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        v = u128_add(v, t);
    }
    return v;
}

// 192-bit unsigned (three limbs, little endian)
struct u192 { uint64_t w0, w1, w2; };

__device__ __forceinline__ u192 mul128x64(u128 a, uint64_t b)
{
    u192 r;
    uint64_t p0lo = a.lo * b, p0hi = __umul64hi(a.lo, b);
    uint64_t p1lo = a.hi * b, p1hi = __umul64hi(a.hi, b);
    r.w0 = p0lo;
    r.w1 = p0hi + p1lo;
    r.w2 = p1hi + (r.w1 < p0hi ? 1ull : 0ull);
    return r;
}

__device__ __forceinline__ u192 shl192(u192 a, int s)   // 0 <= s < 192
{
    u192 r = {0, 0, 0};
    if (s == 0) return a;
    if (s >= 128) { r.w2 = a.w0 << (s - 128); return r; }
    if (s >= 64) {
        int t = s - 64;
        r.w2 = t ? ((a.w1 << t) | (a.w0 >> (64 - t))) : a.w1;
        r.w1 = a.w0 << t;
        r.w0 = 0;
        return r;
    }
    r.w2 = (a.w2 << s) | (a.w1 >> (64 - s));
    r.w1 = (a.w1 << s) | (a.w0 >> (64 - s));
    r.w0 = a.w0 << s;
    return r;
}

__device__ __forceinline__ int cmp192(u192 a, u192 b)
{
    if (a.w2 != b.w2) return a.w2 < b.w2 ? -1 : 1;
    if (a.w1 != b.w1) return a.w1 < b.w1 ? -1 : 1;
    if (a.w0 != b.w0) return a.w0 < b.w0 ? -1 : 1;
    return 0;
}

// sign of N/D - M * 2^E  (M < 2^55, N < 2^127, D < 2^127, the two within a
// few binary64 ulps of each other so every shifted operand fits in 192 bits)
__device__ __forceinline__ int cmp_quot(u128 N, u128 D, uint64_t M, int E)
{
    u192 lhs = {N.lo, N.hi, 0};
    u192 rhs = mul128x64(D, M);
    if (E >= 0) rhs = shl192(rhs, E);
    else lhs = shl192(lhs, -E);
    return cmp192(lhs, rhs);
}

__device__ __forceinline__ double u128_to_double_approx(u128 a)
{
    return (double)a.hi * 18446744073709551616.0 + (double)a.lo;
}

// Correctly rounded (nearest-even) binary64 of N / D, N < 2^127, 0 < D < 2^127.
// Estimate with binary64 arithmetic, then settle the rounding exactly by
// comparing N/D with the midpoints next to the estimate (integer compare).
__device__ __noinline__ double div_rn_u128(u128 N, u128 D, int32_t *err)
{
    if ((N.lo | N.hi) == 0) return 0.0;
    const uint64_t two53 = 1ull << 53;
    if (N.hi == 0 && D.hi == 0 && N.lo < two53 && D.lo < two53)
        return __ddiv_rn((double)N.lo, (double)D.lo);
    double q = __ddiv_rn(u128_to_double_approx(N), u128_to_double_approx(D));
    for (int it = 0; it < 16; it++) {
        uint64_t bits = (uint64_t)__double_as_longlong(q);
        int ex = (int)((bits >> 52) & 0x7ff);
        uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
        int e = ex - 1075;                  // q = mant * 2^e
        int chi = cmp_quot(N, D, 2 * mant + 1, e - 1);
        if (chi > 0) { q = __longlong_as_double((long long)(bits + 1)); continue; }
        int clo;
        if (mant == (1ull << 52)) clo = cmp_quot(N, D, 4 * mant - 1, e - 2);
        else clo = cmp_quot(N, D, 2 * mant - 1, e - 1);
        if (clo < 0) { q = __longlong_as_double((long long)(bits - 1)); continue; }
        if (chi == 0 && (mant & 1)) return __longlong_as_double((long long)(bits + 1));
        if (clo == 0 && (mant & 1)) return __longlong_as_double((long long)(bits - 1));
        return q;
    }
    if (err) atomicExch(err, 0x44495600);   // "DIV": estimate did not settle
    return q;
}

// Exact key of regions (Si, ni) and (Sj, nj) over B bands, computed by one
// full warp (lanes over bands).  Every lane returns the key.
__device__ __forceinline__ double warp_key(const int64_t *__restrict__ Si, int64_t ni,
                                           const int64_t *__restrict__ Sj, int64_t nj, int B,
                                           int32_t *err)
{
    int lane = threadIdx.x & 31;
    u128 acc = {0, 0};
    // four bands per lane loaded together, then accumulated in band order
    for (int b0 = lane; b0 < B; b0 += 128) {
        int64_t si[4], sj[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int b = b0 + 32 * u;
            si[u] = (b < B) ? Si[b] : 0;
            sj[u] = (b < B) ? Sj[b] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            int64_t d = nj * si[u] - ni * sj[u];
            uint64_t a = (uint64_t)(d < 0 ? -d : d);
            acc = u128_add(acc, u128_sq(a));
        }
    }
    acc = warp_sum_u128(acc);
    double K = 0.0;
    if (lane == 0) {
        u128 D = u128_mul64((uint64_t)ni * (uint64_t)nj, (uint64_t)(ni + nj));
        K = div_rn_u128(acc, D, err);
    }
    return __shfl_sync(0xffffffffu, K, 0);
}

__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }


// Packed (K bits, lo slot, hi slot) comparisons.
// Decode a local upper-triangle tile index into (I, J), I <= J < nb
// (binary32 estimate, exact integer correction; no FP64 instruction).
__device__ __forceinline__ void tri_decode(long long local, long long nb, int &I, int &J)
{
    float a = 2.0f * (float)(int)nb + 1.0f;                 // 32-bit conversions only
    float disc = fmaxf(a * a - 8.0f * (float)(int)local, 0.0f);
    long long i = (long long)((a - sqrtf(disc)) * 0.5f);
    if (i < 0) i = 0;
    if (i > nb - 1) i = nb - 1;
    while (i > 0 && i * nb - i * (i - 1) / 2 > local) i--;
    while (i + 1 < nb && (i + 1) * nb - (i + 1) * i / 2 <= local) i++;
    long long off = i * nb - i * (i - 1) / 2;
    I = (int)i;
    J = (int)(i + (local - off));
}

struct PairKey { uint64_t k; uint32_t lo, hi; };

__device__ __forceinline__ bool pk_less(const PairKey &a, const PairKey &b)
{
    if (a.k != b.k) return a.k < b.k;
    if (a.lo != b.lo) return a.lo < b.lo;
    return a.hi < b.hi;
}

__device__ __forceinline__ PairKey pk_make(uint64_t k, int i, int j)
{
    PairKey p;
    p.k = k;
    p.lo = (uint32_t)min(i, j);
    p.hi = (uint32_t)max(i, j);
    return p;
}

__device__ __forceinline__ PairKey pk_none()
{
    PairKey p; p.k = RHSEG_KEY_NONE; p.lo = 0xffffffffu; p.hi = 0xffffffffu; return p;
}

__device__ __forceinline__ PairKey warp_min_pk(PairKey v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        PairKey t;
        t.k = __shfl_xor_sync(0xffffffffu, v.k, o);
        t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        if (pk_less(t, v)) v = t;
    }
    return v;
}

// Block-wide min of PairKey; `sh` needs blockDim.x/32 entries.  All threads
// get the result.
__device__ __forceinline__ PairKey block_min_pk(PairKey v, PairKey *sh)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_min_pk(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    PairKey r = (lane < nw) ? sh[lane] : pk_none();
    r = warp_min_pk(r);
    return r;
}

__device__ __forceinline__ long long block_sum_ll(long long v, long long *sh)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    long long r = (lane < nw) ? sh[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

}  // namespace rhseg
