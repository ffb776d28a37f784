// rhseg_kernels.cuh -- level set-up, HSEG step and level-transition kernels.
//
// Data layout of a level (all sections of the level at once):
//   slots      regions present at the level start, section-local index sorted
//              by region ID (so slot order = ID order, reading R5);
//   positions  compact list of live slots used by the spectral screen
//              (tensor-core forms: in certified-norm order), rebuilt with
//              the order kept whenever the live count drops below a
//              128-position block boundary;
//   adjacency  one dense bitmap per section, m0 x W words (W = ceil(m0/32)
//              rounded to 4), symmetric, no self bits; or (L.csr) sorted
//              neighbour lists per slot in a per-section pool
//              (rhseg_csr.cuh);
//   bestK/P    per slot: the smallest (K, pair) over its adjacent partners
//              (kept exact and current after every merge);
//   log        one segment per (level, section);
//   mlist      (multi_merge only) per slot x 2 words: a stage's mutually best
//              pairs, sorted, before they merge.
#pragma once
#include "rhseg_dev.cuh"
#include "../../include/rhseg.h"

namespace rhseg {

constexpr int STEP_THREADS = 256;     // two step blocks per SM: every section of a level in one wave
constexpr int NB_CHUNK_WORDS = 64;      // adjacency words gathered per chunk
constexpr int RESCAN_CAP = 512;

struct PixGeom {
    int32_t rows, cols, B, Bs;
    const uint16_t *img;       // [P][B]
    const uint8_t *mask;       // [P] or null
};

__device__ __forceinline__ bool unmasked(const PixGeom &g, int64_t p)
{
    return g.mask == nullptr || g.mask[p] == 0;
}

// section index (Z order) of pixel (y, x) at a level with `nbits` split
// levels below the root: interleave row band and column band bits.
__device__ __forceinline__ int32_t morton2(int32_t rb, int32_t cb, int nbits)
{
    int32_t s = 0;
    for (int i = nbits - 1; i >= 0; i--) {
        s = (s << 2) | (((rb >> i) & 1) << 1) | ((cb >> i) & 1);
    }
    return s;
}

}  // namespace rhseg
#include "rhseg_csr.cuh"
namespace rhseg {

// ---------------------------------------------------------------------------
// Level set-up
// ---------------------------------------------------------------------------

// Deepest level: every unmasked pixel is a region with ID p+1 (reading R5).
__global__ void k_init_labels(PixGeom g, uint32_t *label, uint8_t *isid, int32_t *srcslot)
{
    int64_t P = (int64_t)g.rows * g.cols;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        bool u = unmasked(g, p);
        label[p] = u ? (uint32_t)(p + 1) : 0u;
        isid[p] = u ? 1 : 0;
        srcslot[p] = -1;
    }
}

// One block per section: raster scan of the section rectangle; every pixel
// that carries a region ID (isid) gets the next slot.  Seam splits (kind 2
// records) are written in the same raster order.
__global__ void k_section_scan(PixGeom g, int32_t nsec, const int32_t *rect, const uint8_t *isid,
                               const uint8_t *split, const double *split_key, const uint32_t *split_from,
                               const int64_t *roff, int32_t *slot_of_id, SecState *st,
                               rhseg_merge *log, const int64_t *loff, int32_t level)
{
    int sec = blockIdx.x;
    if (sec >= nsec) return;
    __shared__ int32_t wsum[32];
    __shared__ int32_t wsplit[32];
    __shared__ int32_t base, sbase;
    int r0 = rect[4 * sec], r1 = rect[4 * sec + 1], c0 = rect[4 * sec + 2], c1 = rect[4 * sec + 3];
    int64_t w = c1 - c0;
    int64_t area = (int64_t)(r1 - r0) * w;
    if (threadIdx.x == 0) { base = 0; sbase = 0; }
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t c = 0; c < area; c += blockDim.x) {
        int64_t li = c + threadIdx.x;
        int flag = 0, sp = 0;
        int64_t p = 0;
        if (li < area) {
            p = (int64_t)(r0 + li / w) * g.cols + (c0 + li % w);
            flag = isid[p];
            sp = split ? split[p] : 0;
        }
        unsigned bal = __ballot_sync(0xffffffffu, flag);
        unsigned bsp = __ballot_sync(0xffffffffu, sp);
        int pre = __popc(bal & ((1u << lane) - 1));
        int spre = __popc(bsp & ((1u << lane) - 1));
        if (lane == 0) { wsum[wid] = __popc(bal); wsplit[wid] = __popc(bsp); }
        __syncthreads();
        int off = 0, soff = 0, tot = 0, stot = 0;
        for (int i = 0; i < nw; i++) {
            if (i < wid) { off += wsum[i]; soff += wsplit[i]; }
            tot += wsum[i]; stot += wsplit[i];
        }
        if (flag) slot_of_id[p] = (int32_t)(roff[sec] + base + off + pre);
        if (sp) {
            int64_t k = sbase + soff + spre;
            rhseg_merge m;
            m.level = level; m.section = sec; m.step = 0; m.kind = 2;
            m.survivor_id = split_from[p]; m.absorbed_id = p + 1;
            m.key = split_key[p]; m.dissim = sqrt(split_key[p]);
            m.nregions_after = 0; m.pad = 0;      // patched once m0 is known
            log[loff[sec] + k] = m;
        }
        __syncthreads();
        if (threadIdx.x == 0) { base += tot; sbase += stot; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        SecState s = {};
        s.m0 = base;
        s.count = base;
        s.log_n = sbase;
        s.nsplit = sbase;
        st[sec] = s;
    }
}

// Fill the slot tables from the region sources (warp per region).
// srcslot[id-1] = previous-level slot of the region with that ID, or -1 for
// a one-pixel region taken from the image.
__global__ void k_fill_tables(PixGeom g, int64_t P, const uint8_t *isid, const int32_t *srcslot,
                              const int32_t *slot_of_id, const int64_t *S_prev, const int64_t *n_prev,
                              int64_t *S, int64_t *n, uint32_t *rid, uint8_t *alive, int32_t *parent,
                              int32_t *absorbed_at, uint64_t *bestK, int32_t *bestP)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < P; p += nwarps) {
        if (!isid[p]) continue;
        int64_t gsl = slot_of_id[p];
        int32_t src = srcslot[p];
        int64_t *dst = S + gsl * g.Bs;
        if (src < 0) {
            const uint16_t *x = g.img + p * g.B;
            for (int b = lane; b < g.Bs; b += 32) dst[b] = (b < g.B) ? (int64_t)x[b] : 0;
        } else {
            const int64_t *s = S_prev + (int64_t)src * g.Bs;
            for (int b = lane; b < g.Bs; b += 32) dst[b] = s[b];
        }
        if (lane == 0) {
            n[gsl] = (src < 0) ? 1 : n_prev[src];
            rid[gsl] = (uint32_t)(p + 1);
            alive[gsl] = 1;
            absorbed_at[gsl] = 0x7fffffff;
            bestK[gsl] = RHSEG_KEY_NONE;
            bestP[gsl] = -1;
        }
    }
}

// parent[g] = g for all slots of the level (global slot indices)
__global__ void k_init_parent(int32_t *parent, const int64_t *roff, const SecState *st, int32_t nsec)
{
    int sec = blockIdx.y;
    if (sec >= nsec) return;
    int m0 = st[sec].m0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m0; i += gridDim.x * blockDim.x)
        parent[roff[sec] + i] = (int32_t)(roff[sec] + i);
}

// Adjacency bitmap from the label map: pixels p, q neighbours (4 or 8
// connectivity) inside the same section, both unmasked, different labels.
__global__ void k_build_adj(PixGeom g, const uint32_t *label, const int32_t *slot_of_id,
                            const int32_t *rowband, const int32_t *colband, int nbits, int conn,
                            const int64_t *roff, const int64_t *aoff, const int32_t *Wrow, uint32_t *adj)
{
    int64_t P = (int64_t)g.rows * g.cols;
    // forward half of the neighbourhood: each undirected pixel pair once
    const int dy8[4] = {0, 1, 1, 1}, dx8[4] = {1, -1, 0, 1};
    const int dy4[2] = {0, 1}, dx4[2] = {1, 0};
    int nn = conn == 8 ? 4 : 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t lp = label[p];
        if (lp == 0) continue;
        int y = (int)(p / g.cols), x = (int)(p % g.cols);
        int sp = morton2(rowband[y], colband[x], nbits);
        for (int k = 0; k < nn; k++) {
            int yy = y + (conn == 8 ? dy8[k] : dy4[k]);
            int xx = x + (conn == 8 ? dx8[k] : dx4[k]);
            if (yy < 0 || yy >= g.rows || xx < 0 || xx >= g.cols) continue;
            int64_t q = (int64_t)yy * g.cols + xx;
            uint32_t lq = label[q];
            if (lq == 0 || lq == lp) continue;
            if (morton2(rowband[yy], colband[xx], nbits) != sp) continue;
            int64_t a = slot_of_id[lp - 1] - roff[sp];
            int64_t b = slot_of_id[lq - 1] - roff[sp];
            int W = Wrow[sp];
            uint32_t *ra = adj + aoff[sp] + a * W;
            uint32_t *rb = adj + aoff[sp] + b * W;
            uint32_t ma = 1u << (b & 31), mb = 1u << (a & 31);
            if (!(ra[b >> 5] & ma)) atomicOr(&ra[b >> 5], ma);
            if (!(rb[a >> 5] & mb)) atomicOr(&rb[a >> 5], mb);
        }
    }
}

// Exact best adjacent partner of every slot (warp per slot).
__global__ void k_init_best(LevelDev L)
{
    int sec = blockIdx.y;
    const SecState &s = L.st[sec];
    int m0 = s.m0;
    int W = L.W[sec];
    int64_t ro = L.roff[sec];
    const uint32_t *A = L.adj + L.aoff[sec];
    int lane = threadIdx.x & 31;
    int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < m0; i += gridDim.x * wpb) {
        const uint32_t *row = A + (int64_t)i * W;
        PairKey best = pk_none();
        const int64_t *Si = L.S + (ro + i) * L.Bs;
        int64_t ni = L.n[ro + i];
        if (L.csr) {
            int d;
            const int32_t *lst = csr_row(L, sec, 0, ro, i, d);
            for (int e = 0; e < d; e++) {
                const int r = lst[e];
                double K = warp_key(Si, ni, L.S + (ro + r) * L.Bs, L.n[ro + r], L.B, L.err);
                PairKey c = pk_make(dbits(K), i, r);
                if (pk_less(c, best)) best = c;
            }
        }
        for (int w = 0; w < (L.csr ? 0 : W); w++) {
            uint32_t bits = row[w];
            while (bits) {
                int r = w * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                double K = warp_key(Si, ni, L.S + (ro + r) * L.Bs, L.n[ro + r], L.B, L.err);
                PairKey c = pk_make(dbits(K), i, r);
                if (pk_less(c, best)) best = c;
            }
        }
        if (lane == 0) {
            L.bestK[ro + i] = best.k;
            L.bestP[ro + i] = (best.k == RHSEG_KEY_NONE) ? -1 : (int32_t)(best.lo == (uint32_t)i ? best.hi : best.lo);
        }
    }
}

// ---------------------------------------------------------------------------
// Screen operand rows (region means relative to a per-section reference).
// ---------------------------------------------------------------------------

struct ScreenConst {
    double u, eta;        // componentwise rounding of the operand: |e| <= u|x| + eta
    double two_one_inv_delta;   // 2 (1 + 1/delta)
    double gamma;         // accumulation + evaluation slack, relative to q
    double kscale;        // (1 + delta) * 4^-sigma
    double xscale;        // 2^-sigma
    // single-precision row terms (precision 1, 2, 3):
    //   A = q * Fq - E0 (rounded down),  k = kscale_f / n (rounded up), with
    //   Fq = 1 - gamma - 4 (1 + 1/delta) u^2 and E0 = 4 (1 + 1/delta) eta^2 B,
    //   from eps^2 <= 2 u^2 q + 2 eta^2 B
    float Fq, E0, kscale_f, xscale_f;
    // incremental minima (binary32 rows): eps = u_f * sqrt(q * onepg_f) + etaB_f
    // bounds ||x^ - x|| (rounded up); k1_f / n = 4^-sigma / n (rounded up)
    float u_f, etaB_f, onepg_f, k1_f;
};

template <typename T>
__device__ __forceinline__ T to_op(double v);
template <> __device__ __forceinline__ double to_op<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_op<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __half to_op<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_op<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

template <typename T>
__device__ __forceinline__ T to_op_f(float v);
template <> __device__ __forceinline__ float to_op_f<float>(float v) { return v; }
template <> __device__ __forceinline__ double to_op_f<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ __half to_op_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_op_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T>
__device__ __forceinline__ float op_to_f(T v);
template <> __device__ __forceinline__ float op_to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float op_to_f<double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float op_to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float op_to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ double op_to_d(T v);
template <> __device__ __forceinline__ double op_to_d<double>(double v) { return v; }
template <> __device__ __forceinline__ double op_to_d<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double op_to_d<__half>(__half v) { return (double)__half2float(v); }
template <> __device__ __forceinline__ double op_to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// Write operand row `pos` from slot `slot` (warp-cooperative).  The FP64
// form computes in binary64; the other forms compute the row in binary32
// (no FP64 instruction: B300's FP64 rate is low) with the extra roundings
// counted in ScreenConst.
template <typename T>
__device__ void warp_write_row(const LevelDev &L, int sec, int slot, int pos, const ScreenConst &sc)
{
    int lane = threadIdx.x & 31;
    int64_t ro = L.roff[sec];
    const int64_t *S = L.S + (ro + slot) * L.Bs;
    int64_t n = L.n[ro + slot];
    const int32_t *ref = L.ref + (int64_t)sec * L.Bs;
    T *X = (T *)L.X + (L.poff[sec] + pos) * (int64_t)L.Bpad;
    if (sizeof(T) == 8) {
        double rinv = 1.0 / (double)n;
        double q = 0.0;
        for (int b = lane; b < L.Bpad; b += 32) {
            T v;
            if (b < L.B) v = to_op<T>((double)(S[b] - n * (int64_t)ref[b]) * rinv * sc.xscale);
            else v = to_op<T>(0.0);
            X[b] = v;
            double xd = op_to_d<T>(v);
            q = fma(xd, xd, q);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (lane == 0) {
            double qq = q * (1.0 + 0x1p-40);
            double eps = (sc.u * sqrt(qq) + sc.eta * sqrt((double)L.B)) * (1.0 + 0x1p-30);
            double A = qq - sc.two_one_inv_delta * eps * eps - sc.gamma * qq;
            double k = sc.kscale / (double)n * (1.0 + 0x1p-40);
            L.Ad[L.poff[sec] + pos] = A;
            L.kd[L.poff[sec] + pos] = k;
        }
        return;
    }
    const float nf = __int2float_rn((int)n);                 // n < 2^31 (pixels of the image)
    const float rinv = 1.0f / nf;
    float q = 0.0f;
    for (int b0 = lane; b0 < L.Bpad; b0 += 256) {
        // eight bands per lane loaded together (the stores below could alias them)
        int64_t sv[8];
        int32_t rv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int b = b0 + 32 * u;
            sv[u] = (b < L.B) ? S[b] : 0;
            rv[u] = (b < L.B) ? ref[b] : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int b = b0 + 32 * u;
            if (b >= L.Bpad) break;
            float x = 0.0f;
            if (b < L.B) {
                // |S - n ref| < 2^55: two exact 32-bit halves, one rounding in the fma
                int64_t v = sv[u] - n * (int64_t)rv[u];
                float xv = fmaf(__int2float_rn((int)(v >> 24)), 16777216.0f, __int2float_rn((int)(v & 0xFFFFFF)));
                x = xv * rinv * sc.xscale_f;
            }
            T v = to_op_f<T>(x);
            X[b] = v;
            float xd = op_to_f<T>(v);
            q = fmaf(xd, xd, q);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) {
        L.Af[L.poff[sec] + pos] = __fmaf_rd(q, sc.Fq, -sc.E0);
        if (L.qf != nullptr) L.qf[L.poff[sec] + pos] = q;
        L.kf[L.poff[sec] + pos] = __fdiv_ru(sc.kscale_f, __int2float_rd((int)n));
        if (L.sE != nullptr || L.nlo != nullptr) {
            // operand error norm e >= ||x^ - x|| and 4^-sigma/n (rounded up)
            const float e = __fmul_ru(__fadd_ru(__fmul_ru(sc.u_f, __fsqrt_ru(__fmul_ru(q, sc.onepg_f))), sc.etaB_f),
                                      1.0f + 0x1p-20f);
            const float kp = __fdiv_ru(sc.k1_f, __int2float_rd((int)n));
            if (L.sE != nullptr) L.sE[L.poff[sec] + pos] = e;
            L.sk[L.poff[sec] + pos] = kp;
            if (L.nlo != nullptr) {
                // bounds of the true norm: ||x^|| within sqrt(q (1 +- gamma_B)), then +- e
                L.nlo[L.poff[sec] + pos] = fmaxf(0.0f, __fsub_rd(__fsqrt_rd(__fdiv_rd(q, sc.onepg_f)), e));
                L.nhi[L.poff[sec] + pos] = __fadd_ru(__fsqrt_ru(__fmul_ru(q, sc.onepg_f)), e);
            }
        }
    }
}

__device__ __forceinline__ void mark_pos_dead(const LevelDev &L, int sec, int pos)
{
    if (L.precision == 0) L.Ad[L.poff[sec] + pos] = __longlong_as_double(0x7FF0000000000000ll);
    else L.Af[L.poff[sec] + pos] = __int_as_float(0x7f800000);
}

__device__ __forceinline__ void write_row_any(const LevelDev &L, int sec, int slot, int pos, const ScreenConst &sc)
{
    switch (L.precision) {
    case 0: warp_write_row<double>(L, sec, slot, pos, sc); break;
    case 1: warp_write_row<__half>(L, sec, slot, pos, sc); break;
    case 2: warp_write_row<__nv_bfloat16>(L, sec, slot, pos, sc); break;
    default: warp_write_row<float>(L, sec, slot, pos, sc); break;
    }
}


// Per section: reference spectrum, positions, screen rows, counters.
__global__ void __launch_bounds__(STEP_THREADS) k_init_section(LevelDev L, ScreenConst sc, int32_t target)
{
    int sec = blockIdx.x;
    if (sec >= L.nsec) return;
    __shared__ long long red[32];
    SecState *st = &L.st[sec];
    int m0 = st->m0;
    int64_t ro = L.roff[sec];
    // reference spectrum: floor of the section's mean pixel spectrum
    long long ntot = 0;
    for (int i = threadIdx.x; i < m0; i += blockDim.x) ntot += L.n[ro + i];
    ntot = block_sum_ll(ntot, red);
    int32_t *ref = (int32_t *)(L.ref + (int64_t)sec * L.Bs);
    for (int b = threadIdx.x; b < L.Bs; b += blockDim.x) {
        long long v = 0;
        if (b < L.B)
            for (int i = 0; i < m0; i++) v += L.S[(ro + i) * L.Bs + b];
        ref[b] = (b < L.B && ntot > 0) ? (int32_t)(v / ntot) : 0;
    }
    __syncthreads();
    __threadfence_block();
    for (int i = threadIdx.x; i < m0; i += blockDim.x) {
        L.pos_of_slot[ro + i] = i;
        L.slot_of_pos[L.poff[sec] + i] = i;
    }
    // adjacent pairs
    const uint32_t *A = L.adj + L.aoff[sec];
    int W = L.W[sec];
    long long pc = 0;
    if (L.csr) {
        for (int i = threadIdx.x; i < m0; i += blockDim.x) pc += L.ndeg[L.roff[sec] + i];
    } else {
        for (int64_t w = threadIdx.x; w < (int64_t)m0 * W; w += blockDim.x) pc += __popc(A[w]);
    }
    pc = block_sum_ll(pc, red);
    __syncthreads();
    (void)sc;    // operand rows are written by k_write_rows (rows_from = m0)
    if (threadIdx.x == 0) {
        st->target = target;
        st->nadj = pc / 2;
        st->mc = m0;
        st->rows_from = m0;
        st->ranges_stale = 1;
        st->npm = 0;
        st->ncand = 0;
        st->nunits = 0;
        st->done = (m0 <= target) ? 1 : 0;
        st->Kadj = __longlong_as_double(0x7FF0000000000000ll);
        st->tthr = st->Kadj;
        // seam records carry the count after the pass
        rhseg_merge *lg = (rhseg_merge *)L.log + L.loff[sec];
        for (int64_t k = 0; k < st->log_n; k++) lg[k].nregions_after = m0;
    }
}

// ---------------------------------------------------------------------------
// HSEG step kernels
// ---------------------------------------------------------------------------

constexpr int PAIR_CAP = 1408;   // pair entries of one batched key phase (static shared memory stays below 48 KB)
constexpr int ROW_CAP = 256;     // rows whose best partner one merge recomputes (incl. the merged row)

struct StepSmem {
    PairKey pk[32];
    long long ll[32];
    SecState st;                               // section state for the kernel's lifetime
    int32_t pi[PAIR_CAP], pj[PAIR_CAP];        // pair (row slot, partner slot)
    int16_t prow[PAIR_CAP];                    // row index of the entry in rows[]
    unsigned long long pkey[PAIR_CAP];         // K bits
    int32_t npair;
    int32_t rows[ROW_CAP];                     // rows[0] = the merged row
    unsigned long long rowK[ROW_CAP], rowT[ROW_CAP];
    int32_t nrows;
    int32_t overflow;
    int32_t nb[NB_CHUNK_WORDS * 32];
    int32_t nnb;
};

// Exact keys of the pairs wid, wid + nw, wid + 2 nw, ... (at most 32 of them)
// of a shared-memory list, computed by warp `wid` of `nw`: the lanes run
// over the bands of four pairs at a time (independent loads in flight) and
// lane e keeps the sum of the warp's pair e; then every lane rounds its own
// pair's quotient, so the divisions run side by side.
__device__ void warp_keys_batch(const LevelDev &L, int64_t ro, const int32_t *pi, const int32_t *pj,
                                unsigned long long *pkey, int first, int stride, int cnt)
{
    const int lane = threadIdx.x & 31;
    const int m = (cnt > first) ? min(32, (cnt - first + stride - 1) / stride) : 0;
    u128 mine = {0, 0};
    int64_t ni_m = 0, nj_m = 0;
    for (int e0 = 0; e0 < m; e0 += 4) {
        const int g = min(4, m - e0);
        int ii[4], jj[4];
        int64_t ni[4], nj[4];
        const int64_t *Si[4], *Sj[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int idx = first + (e0 + min(u, g - 1)) * stride;
            ii[u] = pi[idx];
            jj[u] = pj[idx];
            Si[u] = L.S + (ro + ii[u]) * L.Bs;
            Sj[u] = L.S + (ro + jj[u]) * L.Bs;
            ni[u] = L.n[ro + ii[u]];
            nj[u] = L.n[ro + jj[u]];
        }
        u128 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        // two band steps of the four pairs per round: 16 independent loads in
        // flight per lane (the region rows mostly come from DRAM)
        for (int b0 = lane; b0 < L.B; b0 += 64) {
            const bool two = b0 + 32 < L.B;
            int64_t si[4][2], sj[4][2];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                si[u][0] = Si[u][b0];
                sj[u][0] = Sj[u][b0];
                si[u][1] = two ? Si[u][b0 + 32] : 0;
                sj[u][1] = two ? Sj[u][b0 + 32] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int t = 0; t < 2; t++) {
                    const int64_t d = nj[u] * si[u][t] - ni[u] * sj[u][t];
                    acc[u] = u128_add(acc[u], u128_sq((uint64_t)(d < 0 ? -d : d)));
                }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const u128 t = warp_sum_u128(acc[u]);
            if (u < g && lane == e0 + u) { mine = t; ni_m = ni[u]; nj_m = nj[u]; }
        }
    }
    if (lane < m) {
        u128 D = u128_mul64((uint64_t)ni_m * (uint64_t)nj_m, (uint64_t)(ni_m + nj_m));
        pkey[first + lane * stride] = dbits(div_rn_u128(mine, D, L.err));
    }
}

// All keys of a list of cnt pairs by the whole block (warps round-robin).
__device__ __forceinline__ void block_keys(const LevelDev &L, int64_t ro, const int32_t *pi, const int32_t *pj,
                                           unsigned long long *pkey, int cnt)
{
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < cnt; base += 32 * nw) warp_keys_batch(L, ro, pi, pj, pkey, base + wid, nw, cnt);
}

__device__ __forceinline__ void set_best(const LevelDev &L, int64_t ro, int r, unsigned long long K,
                                         unsigned long long T)
{
    if (K == RHSEG_KEY_NONE) {
        L.bestK[ro + r] = RHSEG_KEY_NONE;
        L.bestP[ro + r] = -1;
    } else {
        uint32_t lo = (uint32_t)(T >> 32), hi = (uint32_t)T;
        L.bestK[ro + r] = K;
        L.bestP[ro + r] = (int32_t)(lo == (uint32_t)r ? hi : lo);
    }
}

// Exact best adjacent partner of slot r recomputed by one warp (the row's
// words are read by the lanes, set bits visited in order, one key per bit).
template <bool CSR>
__device__ void warp_rescan_row(const LevelDev &L, int sec, int r, int phalf)
{
    const int lane = threadIdx.x & 31;
    const int64_t ro = L.roff[sec];
    const int W = CSR ? 0 : L.W[sec];
    const uint32_t *row = L.adj + (CSR ? 0 : L.aoff[sec]) + (int64_t)r * W;
    const int64_t *Sr = L.S + (ro + r) * L.Bs;
    const int64_t nr = L.n[ro + r];
    PairKey best = pk_none();
    if (CSR) {                                     // lists: one key per entry
        int d;
        const int32_t *lst = csr_row(L, sec, phalf, ro, r, d);
        for (int e = 0; e < d; e++) {
            const int q = lst[e];
            double K = warp_key(Sr, nr, L.S + (ro + q) * L.Bs, L.n[ro + q], L.B, L.err);
            PairKey c = pk_make(dbits(K), r, q);
            if (pk_less(c, best)) best = c;
        }
    }
    for (int w0 = 0; w0 < W; w0 += 32) {
        uint32_t word = (w0 + lane < W) ? row[w0 + lane] : 0u;
        unsigned nz = __ballot_sync(0xffffffffu, word != 0);
        while (nz) {
            int src = __ffs(nz) - 1;
            nz &= nz - 1;
            uint32_t bits = __shfl_sync(0xffffffffu, word, src);
            while (bits) {
                int q = (w0 + src) * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                double K = warp_key(Sr, nr, L.S + (ro + q) * L.Bs, L.n[ro + q], L.B, L.err);
                PairKey c = pk_make(dbits(K), r, q);
                if (pk_less(c, best)) best = c;
            }
        }
    }
    if (lane == 0) {
        L.bestK[ro + r] = best.k;
        L.bestP[ro + r] = (best.k == RHSEG_KEY_NONE) ? -1 : (int32_t)(best.lo == (uint32_t)r ? best.hi : best.lo);
    }
}

// Best adjacent partners after merging b into a, when the batched lists do
// not fit: the merged row by warps over its neighbours, re-scans one warp
// per row.
template <bool CSR>
__device__ void block_best_update_slow(const LevelDev &L, int sec, int a, int b, StepSmem &sm)
{
    const int64_t ro = L.roff[sec];
    const int W = CSR ? 0 : L.W[sec];
    const uint32_t *rowA = L.adj + (CSR ? 0 : L.aoff[sec]) + (int64_t)a * W;
    int dA = 0;
    const int32_t *lstA = CSR ? csr_row(L, sec, sm.st.phalf, ro, a, dA) : nullptr;
    const int tid = threadIdx.x, nt = blockDim.x, wid = tid >> 5, nw = nt >> 5, lane = tid & 31;
    const int64_t *Sa = L.S + (ro + a) * L.Bs;
    const int64_t na = L.n[ro + a];
    PairKey best = pk_none();
    // neighbours of a: their key with a; rows whose best partner was a or b
    // are re-scanned afterwards (listed in sm.nb, processed per chunk of
    // bitmap words, or of list entries)
    const int nunit = CSR ? dA : W, ustep = CSR ? NB_CHUNK_WORDS * 32 : NB_CHUNK_WORDS;
    for (int w0 = 0; w0 < nunit; w0 += ustep) {
        __syncthreads();
        if (tid == 0) sm.nnb = 0;
        __syncthreads();
        if (CSR) {
            for (int e = w0 + tid; e < min(dA, w0 + ustep); e += nt) sm.nb[atomicAdd(&sm.nnb, 1)] = lstA[e];
        } else {
            for (int w = w0 + tid; w < min(W, w0 + NB_CHUNK_WORDS); w += nt) {
                uint32_t bits = rowA[w];
                while (bits) {
                    int q = w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    sm.nb[atomicAdd(&sm.nnb, 1)] = q;
                }
            }
        }
        __syncthreads();
        const int cnt = sm.nnb;
        for (int t = wid; t < cnt; t += nw) {
            const int r = sm.nb[t];
            const double Kr = warp_key(Sa, na, L.S + (ro + r) * L.Bs, L.n[ro + r], L.B, L.err);
            const PairKey c = pk_make(dbits(Kr), a, r);
            if (pk_less(c, best)) best = c;
            int bp = L.bestP[ro + r];
            bool rescan = (bp == a || bp == b || bp < 0);
            if (!rescan && lane == 0) {
                PairKey old = pk_make(L.bestK[ro + r], r, bp);
                PairKey nc = pk_make(dbits(Kr), r, a);
                if (pk_less(nc, old)) { L.bestK[ro + r] = nc.k; L.bestP[ro + r] = a; }
            }
            __syncwarp();
            if (rescan) warp_rescan_row<CSR>(L, sec, r, sm.st.phalf);
        }
    }
    best = block_min_pk(best, sm.pk);
    if (tid == 0) {
        L.bestK[ro + a] = best.k;
        L.bestP[ro + a] = (best.k == RHSEG_KEY_NONE) ? -1 : (int32_t)(best.lo == (uint32_t)a ? best.hi : best.lo);
    }
    __syncthreads();
}

// Merge slot b into slot a (a < b, so a keeps the smaller ID).  Whole block;
// st is the block's shared copy of the section state.
template <bool CSR>
__device__ void block_merge(const LevelDev &L, int sec, SecState &st, int a, int b, double K, int kind,
                            const ScreenConst &sc, StepSmem &sm)
{
    const int64_t ro = L.roff[sec];
    constexpr bool csr = CSR;
    const int W = csr ? 0 : L.W[sec];
    uint32_t *A = L.adj + (csr ? 0 : L.aoff[sec]);
    uint32_t *rowA = A + (int64_t)a * W;
    uint32_t *rowB = A + (int64_t)b * W;
    const int tid = threadIdx.x, nt = blockDim.x, wid = tid >> 5;
    int ab = csr ? 0 : (int)((rowA[b >> 5] >> (b & 31)) & 1);
    long long pa = 0, pb = 0;
    for (int w = tid; w < W; w += nt) { pa += __popc(rowA[w]); pb += __popc(rowB[w]); }
    pa = block_sum_ll(pa, sm.ll);
    pb = block_sum_ll(pb, sm.ll);
    __syncthreads();
    // features (exact integers) and bookkeeping
    for (int k = tid; k < L.Bs; k += nt) L.S[(ro + a) * L.Bs + k] += L.S[(ro + b) * L.Bs + k];
    if (tid == 0) {
        const int64_t na = L.n[ro + a], nb = L.n[ro + b];
        const uint32_t ida = L.rid[ro + a], idb = L.rid[ro + b];
        L.n[ro + a] = na + nb;
        L.alive[ro + b] = 0;
        L.parent[ro + b] = (int32_t)(ro + a);
        const int ord = ++st.nmerge;
        if (kind == 0) st.madj += 1; else st.mspec += 1;
        L.absorbed_at[ro + b] = ord;
        L.bestK[ro + b] = RHSEG_KEY_NONE;
        L.bestP[ro + b] = -1;
        if (L.sbK) { L.sbK[ro + b] = RHSEG_KEY_NONE; L.sbP[ro + b] = -1; }
        st.count -= 1;
        rhseg_merge m;
        m.level = L.level; m.section = sec; m.step = st.iter; m.kind = kind;
        m.survivor_id = ida; m.absorbed_id = idb;
        m.key = K; m.dissim = sqrt(K);
        m.nregions_after = st.count; m.pad = 0;
        ((rhseg_merge *)L.log)[L.loff[sec] + st.log_n] = m;
        st.log_n += 1;
    }
    long long pn = 0;
    int dA = 0;
    const int32_t *lstA = nullptr;
    if (csr) {
        // lists: a's union at the top of the pool, b replaced by a elsewhere
        int ipa, ipb, iab, ipn;
        csr_merge(L, sec, st, a, b, ipa, ipb, iab, ipn);
        pa = ipa; pb = ipb; ab = iab; pn = ipn;
        lstA = csr_row(L, sec, st.phalf, ro, a, dA);
    } else {
        // adjacency: row a |= row b, neighbours of b now point to a
        for (int w = tid; w < W; w += nt) rowA[w] |= rowB[w];
        __syncthreads();
        if (tid == 0) {
            rowA[a >> 5] &= ~(1u << (a & 31));
            rowA[b >> 5] &= ~(1u << (b & 31));
        }
        for (int w = tid; w < W; w += nt) {
            uint32_t bits = rowB[w];
            while (bits) {
                int r = w * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                if (r == a) continue;
                uint32_t *rowR = A + (int64_t)r * W;
                atomicOr(&rowR[a >> 5], 1u << (a & 31));
                atomicAnd(&rowR[b >> 5], ~(1u << (b & 31)));
            }
        }
        __syncthreads();
        for (int w = tid; w < W; w += nt) rowB[w] = 0;
        __syncthreads();
        for (int w = tid; w < W; w += nt) pn += __popc(rowA[w]);
        pn = block_sum_ll(pn, sm.ll);
    }
    if (tid == 0) {
        st.nadj = st.nadj - pa - pb + ab + pn;
        sm.npair = 0;
        sm.nrows = 1;
        sm.rows[0] = a;
        sm.overflow = 0;
    }
    __syncthreads();
    // ---- exact best partners: one batched key phase ----
    // entries of row 0: (a, r) for every neighbour r of a
    for (int e = tid; e < dA; e += nt) {
        int idx = atomicAdd(&sm.npair, 1);
        if (idx < PAIR_CAP) { sm.pi[idx] = a; sm.pj[idx] = lstA[e]; sm.prow[idx] = 0; }
        else sm.overflow = 1;
    }
    for (int w = tid; w < W; w += nt) {
        uint32_t bits = rowA[w];
        while (bits) {
            int r = w * 32 + __ffs(bits) - 1;
            bits &= bits - 1;
            int idx = atomicAdd(&sm.npair, 1);
            if (idx < PAIR_CAP) { sm.pi[idx] = a; sm.pj[idx] = r; sm.prow[idx] = 0; }
            else sm.overflow = 1;
        }
    }
    __syncthreads();
    if (!sm.overflow) {
        // rows whose best partner was a or b are recomputed in full
        const int n0 = sm.npair;
        for (int e = tid; e < n0; e += nt) {
            const int r = sm.pj[e];
            const int bp = L.bestP[ro + r];
            if (bp == a || bp == b || bp < 0) {
                int k = atomicAdd(&sm.nrows, 1);
                if (k < ROW_CAP) sm.rows[k] = r; else sm.overflow = 1;
            }
        }
        __syncthreads();
        const int nr = min(sm.nrows, ROW_CAP);
        if (!sm.overflow && csr) {
            const int lane = tid & 31, nw = nt >> 5;
            for (int k = 1 + wid; k < nr; k += nw) {
                const int r = sm.rows[k];
                int dr;
                const int32_t *lr = csr_row(L, sec, st.phalf, ro, r, dr);
                for (int e = lane; e < dr; e += 32) {
                    int idx = atomicAdd(&sm.npair, 1);
                    if (idx < PAIR_CAP) { sm.pi[idx] = r; sm.pj[idx] = lr[e]; sm.prow[idx] = (int16_t)k; }
                    else sm.overflow = 1;
                }
            }
        }
        if (!sm.overflow && !csr) {
            for (int64_t f = tid; f < (int64_t)(nr - 1) * W; f += nt) {
                const int k = 1 + (int)(f / W), w = (int)(f % W);
                const int r = sm.rows[k];
                uint32_t bits = A[(int64_t)r * W + w];
                while (bits) {
                    int q = w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    int idx = atomicAdd(&sm.npair, 1);
                    if (idx < PAIR_CAP) { sm.pi[idx] = r; sm.pj[idx] = q; sm.prow[idx] = (int16_t)k; }
                    else sm.overflow = 1;
                }
            }
        }
        __syncthreads();
    }
    if (sm.overflow) {
        block_best_update_slow<CSR>(L, sec, a, b, sm);
    } else {
        const int np = sm.npair, nr = sm.nrows;
        for (int k = tid; k < nr; k += nt) { sm.rowK[k] = RHSEG_KEY_NONE; sm.rowT[k] = ~0ull; }
        block_keys(L, ro, sm.pi, sm.pj, sm.pkey, np);
        __syncthreads();
        for (int e = tid; e < np; e += nt) atomicMin(&sm.rowK[sm.prow[e]], sm.pkey[e]);
        __syncthreads();
        for (int e = tid; e < np; e += nt) {
            const int k = sm.prow[e];
            if (sm.pkey[e] == sm.rowK[k]) {
                const uint32_t i = (uint32_t)sm.pi[e], j = (uint32_t)sm.pj[e];
                const unsigned long long t = ((unsigned long long)min(i, j) << 32) | max(i, j);
                atomicMin(&sm.rowT[k], t);
            }
            if (k == 0) {
                // neighbour r of a whose best partner is neither a nor b: compare with K(r, a)
                const int r = sm.pj[e];
                const int bp = L.bestP[ro + r];
                if (!(bp == a || bp == b || bp < 0)) {
                    PairKey old = pk_make(L.bestK[ro + r], r, bp);
                    PairKey nc = pk_make(sm.pkey[e], r, a);
                    if (pk_less(nc, old)) { L.bestK[ro + r] = nc.k; L.bestP[ro + r] = a; }
                }
            }
        }
        __syncthreads();
        for (int k = tid; k < nr; k += nt) set_best(L, ro, sm.rows[k], sm.rowK[k], sm.rowT[k]);
        __syncthreads();
    }
    // screen rows of a (new features) and b (dead)
    const int pa_pos = L.pos_of_slot[ro + a], pb_pos = L.pos_of_slot[ro + b];
    if (wid == 0) write_row_any(L, sec, a, pa_pos, sc);
    if (tid == 32) mark_pos_dead(L, sec, pb_pos);
    __syncthreads();
    if (L.brng != nullptr && tid == 0) {
        // the norm range of a's position block takes in a's new row (b's stays
        // in its block's range: a wider range only keeps more units)
        const int64_t gp = L.poff[sec] + pa_pos;
        float4 *r = (float4 *)L.brng + (gp >> 7);
        float4 v = *r;
        v.x = fminf(v.x, L.nlo[gp]);
        v.y = fmaxf(v.y, L.nhi[gp]);
        v.z = fmaxf(v.z, L.sk[gp]);
        *r = v;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Several merges per iteration (reading R12; Section 6.2 names the idea).
// ---------------------------------------------------------------------------

// Every live slot i whose best partner j > i has i as its own best partner
// gives one pair; such pairs are disjoint.  They are listed in the
// section's scratch as (K bits, (i << 32) | j) and sorted ascending: slots are
// in ID order, so this is the (K, lo ID, hi ID) order.  Then they merge one
// by one in that order while the count is above the target; each keeps its
// listed key, since the other listed pairs do not touch its two regions.
// bK / bP: the stage's per-slot best (bP < 0 or bK = RHSEG_KEY_NONE: none).
// Returns the merges done (uniform over the block); *kfirst = the first
// one's key, the stage's smallest.
template <bool CSR>
__device__ int block_merge_mutual(const LevelDev &L, int sec, SecState &st, const uint64_t *bK,
                                  const int32_t *bP, int kind, const ScreenConst &sc, StepSmem &sm,
                                  double *kfirst)
{
    const int64_t ro = L.roff[sec];
    const int m0 = st.m0;
    unsigned long long *list = L.mlist + 2 * ro;       // 2 m0 words: n <= m0 / 2 pairs, padded n2 <= m0
    __shared__ int32_t nmut;
    if (threadIdx.x == 0) nmut = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < m0; i += blockDim.x) {
        const unsigned long long k = __ldcg((const unsigned long long *)bK + ro + i);
        const int32_t j = __ldcg(bP + ro + i);
        if (k == RHSEG_KEY_NONE || j <= i || j >= m0) continue;
        if (__ldcg(bP + ro + j) != i) continue;
        const int e = atomicAdd(&nmut, 1);
        list[2 * e] = k;
        list[2 * e + 1] = ((unsigned long long)(uint32_t)i << 32) | (uint32_t)j;
    }
    __syncthreads();
    const int n = nmut;
    int n2 = n > 0 ? 1 : 0;
    while (n2 < n) n2 <<= 1;
    for (int e = n + threadIdx.x; e < n2; e += blockDim.x) { list[2 * e] = ~0ull; list[2 * e + 1] = ~0ull; }
    __syncthreads();
    // bitonic sort of the n2 entries on (K bits, slot pair)
    for (int k = 2; k <= n2; k <<= 1)
        for (int d = k >> 1; d > 0; d >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int l = i ^ d;
                if (l <= i) continue;
                const unsigned long long ak = list[2 * i], at = list[2 * i + 1];
                const unsigned long long bk = list[2 * l], bt = list[2 * l + 1];
                const bool gt = ak > bk || (ak == bk && at > bt);
                if (gt == ((i & k) == 0)) {
                    list[2 * i] = bk; list[2 * i + 1] = bt;
                    list[2 * l] = ak; list[2 * l + 1] = at;
                }
            }
            __syncthreads();
        }
    int done = 0;
    *kfirst = __longlong_as_double(0x7FF0000000000000ll);
    for (int e = 0; e < n; e++) {
        if (st.count <= st.target) break;              // st.count is updated inside block_merge
        const unsigned long long kb = list[2 * e], t = list[2 * e + 1];
        const double K = __longlong_as_double((long long)kb);
        if (e == 0) *kfirst = K;
        block_merge<CSR>(L, sec, st, (int)(t >> 32), (int)(t & 0xffffffffu), K, kind, sc, sm);
        done++;
    }
    __syncthreads();
    return done;
}

// New position list of the live slots in order of their rows' certified
// norms (the tensor-core screen then finds whole units of pairs far apart in
// norm, which its norm bound proves to be above the threshold).  Bitonic
// sort of (norm bits, slot) in the section's scratch (whole block); the
// operand rows are then rewritten by k_write_rows.
__device__ void block_sort_positions(const LevelDev &L, int sec, SecState &st)
{
    const int m0 = st.m0;
    const int64_t ro = L.roff[sec], pb = L.poff[sec];
    unsigned long long *a = L.sortk + 2 * ro;
    int n2 = 1;
    while (n2 < m0) n2 <<= 1;
    __shared__ int32_t nlive;
    if (threadIdx.x == 0) nlive = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        unsigned long long v = ~0ull;
        if (i < m0 && L.alive[ro + i]) {
            const float nr = L.nhi[pb + L.pos_of_slot[ro + i]];             // >= 0: bits order as floats
            v = ((unsigned long long)(uint32_t)__float_as_int(nr) << 32) | (uint32_t)i;
            atomicAdd(&nlive, 1);
        }
        a[i] = v;
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long x = a[i], y = a[ixj];
                    if ((x > y) == ((i & k) == 0)) { a[i] = y; a[ixj] = x; }
                }
            }
            __syncthreads();
        }
    }
    const int n = nlive;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int slot = (int)(uint32_t)a[i];
        L.pos_of_slot[ro + slot] = i;
        L.slot_of_pos[pb + i] = slot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st.rows_from = max(st.mc, 1);   // old extent: positions past the new end are marked dead
        st.mc = n;
        st.ranges_stale = 1;
    }
    __syncthreads();
}

// Compaction that keeps the live positions in their current order (the norm
// order set at level start; a merged region keeps its position, its new
// norm close to its parts'), in place (new positions never exceed old ones).
// Exclusive prefix over the block of one count per thread (whole block);
// *total gets the sum.  Its first barrier also orders every read before it
// against the writes after it.
__device__ __forceinline__ int block_excl_scan(int v, int *total)
{
    __shared__ int32_t ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    int off = 0, tot = 0;
    for (int k = 0; k < nw; k++) {
        const int w = ws[k];
        if (k < wid) off += w;
        tot += w;
    }
    *total = tot;
    return off + incl - v;
}

constexpr int CP_PER = 16;     // positions per thread per round of a compaction

// Compaction that keeps the live positions in their current order (the norm
// order set at level start; a merged region keeps its position, its new
// norm close to its parts'), in place.  Each round gives every thread
// CP_PER consecutive positions: their slots and liveness are loaded
// together, one block scan places them, and the writes follow the scan's
// barrier (a new position never exceeds its old one, and every position of
// the round was read before any is written).
__device__ void block_compact_in_order(const LevelDev &L, int sec, SecState &st)
{
    const int mc = st.mc;
    const int64_t ro = L.roff[sec], pb = L.poff[sec];
    int base = 0;
    for (int c = 0; c < mc; c += blockDim.x * CP_PER) {
        const int p0 = c + threadIdx.x * CP_PER;
        int sl[CP_PER];
        uint8_t f[CP_PER];
#pragma unroll
        for (int u = 0; u < CP_PER; u++) sl[u] = (p0 + u < mc) ? L.slot_of_pos[pb + p0 + u] : -1;
#pragma unroll
        for (int u = 0; u < CP_PER; u++) f[u] = (sl[u] >= 0) ? L.alive[ro + sl[u]] : 0;
        int cnt = 0;
#pragma unroll
        for (int u = 0; u < CP_PER; u++) cnt += f[u] ? 1 : 0;
        int tot;
        int np = base + block_excl_scan(cnt, &tot);
#pragma unroll
        for (int u = 0; u < CP_PER; u++)
            if (f[u]) {
                L.pos_of_slot[ro + sl[u]] = np;
                L.slot_of_pos[pb + np] = sl[u];
                np++;
            }
        base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st.rows_from = st.mc;       // old extent: positions past the new end are marked dead
        st.mc = base;
    }
    __syncthreads();
}

// New stable position list of the live slots (the screen's operand rows are
// then rewritten by k_write_rows).
__device__ void block_compact_stable(const LevelDev &L, int sec, SecState &st);

__device__ void block_compact_positions(const LevelDev &L, int sec, SecState &st)
{
    if (L.sortk != nullptr) block_compact_in_order(L, sec, st);
    else block_compact_stable(L, sec, st);
    // the section's operand rows are rewritten by the next k_write_rows, and
    // the norm ranges of its position blocks recomputed by the next unit list
    if (threadIdx.x == 0) {
        if (L.wcount != nullptr) L.wlist[atomicAdd(L.wcount, 1)] = sec;
        st.ranges_stale = 1;
    }
    __syncthreads();
}

__device__ void block_compact_stable(const LevelDev &L, int sec, SecState &st)
{
    // the live slots in slot (= ID) order, rounds as in block_compact_in_order
    const int m0 = st.m0;
    const int64_t ro = L.roff[sec];
    int base = 0;
    for (int c = 0; c < m0; c += blockDim.x * CP_PER) {
        const int i0 = c + threadIdx.x * CP_PER;
        uint8_t f[CP_PER];
#pragma unroll
        for (int u = 0; u < CP_PER; u++) f[u] = (i0 + u < m0) ? L.alive[ro + i0 + u] : 0;
        int cnt = 0;
#pragma unroll
        for (int u = 0; u < CP_PER; u++) cnt += f[u] ? 1 : 0;
        int tot;
        int np = base + block_excl_scan(cnt, &tot);
#pragma unroll
        for (int u = 0; u < CP_PER; u++)
            if (f[u]) {
                L.pos_of_slot[ro + i0 + u] = np;
                L.slot_of_pos[L.poff[sec] + np] = i0 + u;
                np++;
            }
        base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st.rows_from = st.mc;       // old extent: positions past the new end are marked dead
        st.mc = base;
    }
    __syncthreads();
}

// Operand rows of every position of the sections whose position list was
// (re)built this iteration.  A single wave of blocks: every block takes the
// list of those sections (from_list: the list the compactions appended to;
// otherwise a scan of every section, at level start), then the blocks share
// out (section, chunk) items, one warp per row.  With few sections rebuilt,
// each gets more chunks, so every warp writes a few rows; with none, every
// block leaves after one read.
constexpr int WR_MAX_SECTIONS = 1024;    // 4^5 sections at the deepest of 6 levels
constexpr int WR_CHUNKS = 64;            // chunks per section at least
constexpr int WR_CHUNKS_MAX = 1024;

__global__ void __launch_bounds__(256) k_write_rows(LevelDev L, ScreenConst sc, int from_list)
{
    __shared__ int32_t list[WR_MAX_SECTIONS];
    __shared__ int32_t wcnt[32];
    __shared__ int32_t nlist;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) nlist = from_list ? min(*(volatile const int32_t *)L.wcount, WR_MAX_SECTIONS) : 0;
    __syncthreads();
    if (from_list) {
        const int n = nlist;
        if (n == 0) return;                                  // uniform
        for (int i = threadIdx.x; i < n; i += blockDim.x) list[i] = L.wlist[i];
        __syncthreads();
    } else {
        for (int c = 0; c < L.nsec; c += blockDim.x) {
            const int sec = c + threadIdx.x;
            bool f = false;
            if (sec < L.nsec) {
                const SecState &st = L.st[sec];
                f = st.rows_from > 0 && !st.done;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (lane == 0) wcnt[wid] = __popc(bal);
            __syncthreads();
            int off = 0, tot = 0;
            for (int k = 0; k < nw; k++) { if (k < wid) off += wcnt[k]; tot += wcnt[k]; }
            if (f) list[nlist + off + __popc(bal & ((1u << lane) - 1))] = sec;
            __syncthreads();
            if (threadIdx.x == 0) nlist += tot;
            __syncthreads();
        }
    }
    const int nl = nlist;
    if (nl == 0) return;
    const int chunks = min(WR_CHUNKS_MAX, max(WR_CHUNKS, (int)gridDim.x / nl));
    const int items = nl * chunks;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int sec = list[it / chunks], chunk = it % chunks;
        const SecState &st = L.st[sec];
        const int old = st.rows_from, mc = st.mc;
        const int pend = ((max(old, mc) + 127) / 128) * 128;
        const int gw = chunk * nw + wid, ngw = chunks * nw;
        for (int pos = gw; pos < mc; pos += ngw) write_row_any(L, sec, L.slot_of_pos[L.poff[sec] + pos], pos, sc);
        for (int pos = mc + chunk * blockDim.x + threadIdx.x; pos < pend; pos += chunks * blockDim.x)
            mark_pos_dead(L, sec, pos);
    }
}

// Units of this step's tensor-core screen that may hold a pair with K < t
// (whole block).  For rows i, j: ||x_i - x_j|| >= | ||x_i|| - ||x_j|| |, so
// every pair of 128-position blocks b, c has K >= gap(b, c)^2 / (kmax_b +
// kmax_c), gap being the distance between the blocks' certified norm
// ranges; a unit (I, Jp) is dropped when that bound is >= t for both of its
// column blocks 2 Jp, 2 Jp + 1 (all in binary32, rounded to the safe side).
// The kept units are listed in order; their count and covered pairs go to st.
constexpr int UL_MAX_BLOCKS = 512;     // sections of up to 65536 positions skip units; larger keep all

// Pairs (r, c), r < c, with r in [r0, r1) and c in [c0, c1) (closed form).
__device__ __forceinline__ long long pairs_upper(long long r0, long long r1, long long c0, long long c1)
{
    if (r1 <= r0 || c1 <= c0) return 0;
    const long long n1 = max(0ll, min(r1, c0) - r0);            // rows below every column: all pairs
    long long s = n1 * (c1 - c0);
    const long long a = max(r0, c0), e = min(r1, c1 - 1);     // rows inside the column range
    if (e > a) s += (2 * c1 - 1 - a - e) * (e - a) / 2;         // sum of (c1 - 1 - r), r in [a, e)
    return s;
}

__device__ void block_unit_list(const LevelDev &L, int sec, SecState &st, float Tf)
{
    const int mc = st.mc;
    const int64_t pb = L.poff[sec];
    const int nb = (mc + 127) / 128, nbp = (nb + 1) / 2;
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    const float inf = __int_as_float(0x7f800000);
    __shared__ float blo[UL_MAX_BLOCKS], bhi[UL_MAX_BLOCKS], bkm[UL_MAX_BLOCKS];
    __shared__ int32_t wsum[32];
    __shared__ int32_t base;
    __shared__ unsigned long long s_useful;
    const bool ranges = nb <= UL_MAX_BLOCKS;
    float4 *brng = (L.brng != nullptr) ? (float4 *)L.brng + (pb >> 7) : nullptr;
    if (ranges && brng != nullptr && !st.ranges_stale) {
        // the kept ranges (exact at the last rebuild, widened by every merge since)
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const float4 r = brng[b];
            blo[b] = r.x; bhi[b] = r.y; bkm[b] = r.z;
        }
    } else if (ranges) {
        for (int b = wid; b < nb; b += nw) {
            float lo = inf, hi = -inf, km = 0.0f;
            float af[4], nl[4], nh[4], kk[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int pos = b * 128 + lane + 32 * u;
                const bool in = pos < mc;
                af[u] = in ? L.Af[pb + pos] : inf;
                nl[u] = in ? L.nlo[pb + pos] : inf;
                nh[u] = in ? L.nhi[pb + pos] : -inf;
                kk[u] = in ? L.sk[pb + pos] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (!(af[u] < inf)) continue;                      // dead or past the end
                lo = fminf(lo, nl[u]);
                hi = fmaxf(hi, nh[u]);
                km = fmaxf(km, kk[u]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
                km = fmaxf(km, __shfl_xor_sync(0xffffffffu, km, o));
            }
            if (lane == 0) {
                blo[b] = lo; bhi[b] = hi; bkm[b] = km;
                if (brng != nullptr) brng[b] = make_float4(lo, hi, km, 0.0f);
            }
        }
    }
    if (threadIdx.x == 0) { base = 0; s_useful = 0; }
    __syncthreads();
    // a unit (I, Jp) may hold a pair below the threshold (empty blocks:
    // infinite gap, dropped)
    auto unit_kept = [&](int I, int Jp) -> bool {
        if (!ranges) return true;
        for (int c = 0; c < 2; c++) {
            const int J = 2 * Jp + c;
            if (J >= nb) continue;
            const float gap = fmaxf(0.0f, fmaxf(__fsub_rd(blo[J], bhi[I]), __fsub_rd(blo[I], bhi[J])));
            const float klo = __fdiv_rd(__fmul_rd(gap, gap), __fadd_ru(bkm[I], bkm[J]));
            if (!(klo >= Tf)) return true;
        }
        return false;
    };
    int32_t *ul = L.ulist + (int64_t)sec * L.ucap;
    if (L.tc_pair) {
        // CTA-pair form: the kept units of each column block Jp, in
        // increasing I, paired two by two into (I0, I1) (an odd last unit
        // with I1 = -1), listed column by column as two words,
        // (I0 << 16) | Jp and I1.  A pair shares the B block Jp, so the two
        // CTAs of a cluster can run it as one M = 256 MMA.
        __shared__ int32_t pbase[UL_MAX_BLOCKS / 2 + 1];
        int npairs;
        if (ranges) {
            for (int Jp = wid; Jp < nbp; Jp += nw) {             // pairs per column
                const int ni = min(2 * Jp + 2, nb);
                int c = 0;
                for (int i0 = 0; i0 < ni; i0 += 32) {
                    const int I = i0 + lane;
                    c += __popc(__ballot_sync(0xffffffffu, I < ni && unit_kept(I, Jp)));
                }
                if (lane == 0) pbase[Jp] = (c + 1) >> 1;
            }
            __syncthreads();
            if (threadIdx.x == 0) {                              // exclusive prefix (nbp <= 256)
                int acc = 0;
                for (int j = 0; j < nbp; j++) { const int v = pbase[j]; pbase[j] = acc; acc += v; }
                pbase[nbp] = acc;
            }
            __syncthreads();
            for (int Jp = wid; Jp < nbp; Jp += nw) {
                const int ni = min(2 * Jp + 2, nb);
                const int64_t b0 = pbase[Jp];
                int c = 0;
                for (int i0 = 0; i0 < ni; i0 += 32) {
                    const int I = i0 + lane;
                    const bool k = I < ni && unit_kept(I, Jp);
                    const unsigned m = __ballot_sync(0xffffffffu, k);
                    if (k) {
                        if (L.count_useful) atomicAdd(&s_useful, (unsigned long long)pairs_upper(I * 128ll, min(I * 128ll + 128, (long long)mc),
                                                                             Jp * 256ll, min(Jp * 256ll + 256, (long long)mc)));
                        const int r = c + __popc(m & ((1u << lane) - 1u));
                        const int64_t e = 2 * (b0 + (r >> 1));
                        if (r & 1) ul[e + 1] = I;
                        else ul[e] = (I << 16) | Jp;
                    }
                    c += __popc(m);
                }
                if ((c & 1) && lane == 0) ul[2 * (b0 + (c >> 1)) + 1] = -1;
            }
            npairs = pbase[nbp];
        } else {
            // every unit kept: the two halves of each tile (Ip, Jp), Ip <= Jp
            npairs = nbp * (nbp + 1) / 2;
            for (int t = threadIdx.x; t < npairs; t += blockDim.x) {
                int Ip, Jp;
                tri_decode(t, nbp, Ip, Jp);
                for (int hh = 0; hh < 2; hh++)
                    if (L.count_useful) atomicAdd(&s_useful, (unsigned long long)pairs_upper((2 * Ip + hh) * 128ll,
                                                                         min((2 * Ip + hh) * 128ll + 128, (long long)mc),
                                                                         Jp * 256ll, min(Jp * 256ll + 256, (long long)mc)));
                ul[2 * (int64_t)t] = ((2 * Ip) << 16) | Jp;
                ul[2 * (int64_t)t + 1] = (2 * Ip + 1 < nb) ? 2 * Ip + 1 : -1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            st.ranges_stale = 0;
            st.nunits = npairs;
            st.evaluated += (int64_t)npairs * 256 * 256;
            st.useful += (int64_t)s_useful;
        }
        return;
    }
    // one-CTA form: units (I, Jp) with 2 Jp + 1 >= I (the two 128-row halves
    // of every upper-triangle tile of 256-row blocks), listed row block by
    // row block (I, then Jp)
    const int nall = nb * nbp;
    for (int t0 = 0; t0 < nall; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        int keep = 0, entry = 0;
        if (t < nall) {
            const int I = t / nbp, Jp = t - I * nbp;
            if (2 * Jp + 1 >= I) {
                keep = unit_kept(I, Jp) ? 1 : 0;
                entry = (I << 16) | Jp;
                if (keep && L.count_useful)
                    atomicAdd(&s_useful, (unsigned long long)pairs_upper(I * 128ll, min(I * 128ll + 128, (long long)mc),
                                                                         Jp * 256ll, min(Jp * 256ll + 256, (long long)mc)));
            }
        }
        int incl = keep;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        int off = 0, tot = 0;
        for (int k2 = 0; k2 < nw; k2++) { if (k2 < wid) off += wsum[k2]; tot += wsum[k2]; }
        if (keep) ul[base + off + incl - 1] = entry;
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
    if (L.count_useful) __syncthreads();     // uniform
    if (threadIdx.x == 0) {
        st.ranges_stale = 0;
        st.nunits = base;
        st.evaluated += (int64_t)base * 128 * 256;
        st.useful += (int64_t)s_useful;
    }
}

// Level start with the norm-ordered screen: the positions in norm order,
// once the first operand rows (identity positions) exist.
__global__ void __launch_bounds__(STEP_THREADS) k_sort_positions(LevelDev L)
{
    const int sec = blockIdx.x;
    if (sec >= L.nsec) return;
    __shared__ SecState st;
    if (threadIdx.x == 0) st = L.st[sec];
    __syncthreads();
    if (st.done) return;
    block_sort_positions(L, sec, st);
    if (threadIdx.x == 0) L.st[sec] = st;
}

// Step 2 of HSEG: merge the adjacent pair of minimum key.
template <bool CSR>
__global__ void __launch_bounds__(STEP_THREADS, 2) k_adj_step(LevelDev L, ScreenConst sc)
{
    const int sec = blockIdx.x;
    // a new iteration: the list of sections whose rows are to be rewritten
    // starts empty (the previous iteration's k_write_rows has finished)
    if (blockIdx.x == 0 && threadIdx.x == 0 && L.wcount != nullptr) *L.wcount = 0;
    if (sec >= L.nsec) return;
    __shared__ StepSmem sm;
    if (threadIdx.x == 0) sm.st = L.st[sec];
    __syncthreads();
    SecState &st = sm.st;
    if (st.done) return;
    if (st.count <= st.target) {
        if (threadIdx.x == 0) { st.done = 1; st.spec_pending = 0; st.rows_from = 0; L.st[sec] = st; }
        return;
    }
    const int64_t ro = L.roff[sec];
    const int m0 = st.m0;
    __syncthreads();
    if (threadIdx.x == 0) { st.iter += 1; st.pairs += st.nadj; st.rows_from = 0; }
    __syncthreads();
    PairKey best = pk_none();
    if (!L.multi) {
        for (int i0 = threadIdx.x; i0 < m0; i0 += 8 * blockDim.x) {
            // eight slots per thread loaded together; absorbed slots carry RHSEG_KEY_NONE
            uint64_t kk[8];
            int32_t bp[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int i = i0 + u * blockDim.x;
                kk[u] = (i < m0) ? L.bestK[ro + i] : RHSEG_KEY_NONE;
                bp[u] = (i < m0) ? L.bestP[ro + i] : -1;
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                if (kk[u] == RHSEG_KEY_NONE) continue;
                const PairKey c = pk_make(kk[u], i0 + u * blockDim.x, bp[u]);
                if (pk_less(c, best)) best = c;
            }
        }
        best = block_min_pk(best, sm.pk);
    }
    __syncthreads();
    int merged = 0;
    double Kadj = __longlong_as_double(0x7FF0000000000000ll);
    if (L.multi) {
        // reading R12: every mutually best adjacent pair; the threshold of the
        // spectral stage comes from the first (smallest) of them
        double k0;
        if (block_merge_mutual<CSR>(L, sec, st, L.bestK, L.bestP, 0, sc, sm, &k0) > 0) { merged = 1; Kadj = k0; }
    } else if (best.k != RHSEG_KEY_NONE) {
        Kadj = __longlong_as_double((long long)best.k);
        block_merge<CSR>(L, sec, st, (int)best.lo, (int)best.hi, Kadj, 0, sc, sm);
        merged = 1;
        if (L.incremental && threadIdx.x == 0) {      // rows to recompute for the spectral minima
            st.pm_a[st.npm] = (int)best.lo;
            st.pm_b[st.npm] = (int)best.hi;
            st.npm += 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st.merged_adj = merged;
        st.Kadj = Kadj;
        if (merged && st.count <= st.target) {
            st.done = 1;
            st.spec_pending = 0;
        } else if (L.w > 0.0) {
            st.spec_pending = 1;
            st.tthr = merged ? L.ww * Kadj : Kadj;
            st.ncand = 0;
        } else {
            st.spec_pending = 0;
            if (!merged) { st.stalled = 1; st.done = 1; }
        }
    }
    __syncthreads();
    // per-row threshold terms of this step's tensor-core screen
    if (L.H != nullptr && st.spec_pending) {
        const float Tf = __double2float_ru(st.tthr);
        const int mc = st.mc;
        const int pend = ((mc + 255) / 256) * 256;      // the screen reads 256-row column blocks
        const int64_t pb = L.poff[sec];
        const float inf = __int_as_float(0x7f800000);
        for (int p0 = threadIdx.x; p0 < pend; p0 += 4 * blockDim.x) {
            float a4[4], k4[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int pos = p0 + u * blockDim.x;
                a4[u] = (pos < mc) ? L.Af[pb + pos] : 0.0f;
                k4[u] = (pos < mc) ? L.kf[pb + pos] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int pos = p0 + u * blockDim.x;
                if (pos < pend) L.H[pb + pos] = (pos < mc) ? 0.5f * (a4[u] - Tf * k4[u]) : inf;
            }
        }
        if (L.ulist != nullptr) block_unit_list(L, sec, st, Tf);
    }
    __syncthreads();
    if (threadIdx.x == 0) L.st[sec] = st;
}

// Screening error of the tensor-core screen on the re-checked candidates of
// one chunk (entries e < np of sm, keys in sm.pkey): the screen's estimate
// K~ = c 4^s (q_i + q_j - 2 g) with c = n_i n_j / (n_i + n_j), q the binary32
// ||x^||^2 of each operand row and g the candidate's binary32 Gram value
// (the screen stores g - h_j as it tested it; h_j is added back), against
// the exact K.  The bound on |K~ - K| is
// c 4^s [gamma (||x^_i|| + ||x^_j||)^2 + e (2 ||x_i - x_j|| + e)], where
// e = e_i + e_j bounds ||(x^_i - x^_j) - (x_i - x_j)|| (e_i = u ||x^_i|| +
// eta sqrt(B)) and ||x_i - x_j|| = sqrt(K / c) 2^-s.  The per-section maxima
// of |K~ - K| / K and |K~ - K| / bound go to st (a report only; no decision
// uses them).
__device__ void block_screen_error(const LevelDev &L, int sec, SecState &st, const uint32_t *cand, uint32_t c0,
                                   int np, StepSmem &sm)
{
    const int64_t ro = L.roff[sec], pb = L.poff[sec];
    const float *g = L.candg + (int64_t)sec * L.cand_cap;
    const double s4 = (L.sigma_shift && L.precision == 1) ? 4.0 : 1.0;     // 4^sigma (FP16 scaling only)
    const double sx = (L.sigma_shift && L.precision == 1) ? 0.5 : 1.0;     // 2^-sigma
    float rel = 0.0f, bnd = 0.0f;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        // every quantity scaled by n_i + n_j (no binary64 division); the two
        // ratios and the square roots in binary32 (a report, not a decision)
        const uint32_t c = c0 + (uint32_t)sm.prow[e];
        const int pi = (int)cand[2 * c], pj = (int)cand[2 * c + 1];
        const double K = __longlong_as_double((long long)sm.pkey[e]);
        const double ni = (double)L.n[ro + sm.pi[e]], nj = (double)L.n[ro + sm.pj[e]];
        const double nn = ni + nj, pp = ni * nj;
        const float qi = L.qf[pb + pi], qj = L.qf[pb + pj];
        // the screen's g: its tested value g - h_j plus h_j (binary64 sum; the
        // binary32 rounding of g - h_j is far below the bound's gamma term)
        const double gij = (double)g[c] + (double)L.H[pb + pj];
        const double Ktn = pp * s4 * ((double)qi + (double)qj - 2.0 * gij);           // K~ (n_i + n_j)
        const double Kn = K * nn;                                                     // K (n_i + n_j)
        const float dn = (float)fabs(Ktn - Kn);
        const float ri = sqrtf(qi), rj = sqrtf(qj);
        const float ee = (float)L.err_u * (ri + rj) + 2.0f * (float)L.err_etaB;
        const float dist = sqrtf(__fdiv_ru((float)Kn, (float)pp)) * (float)sx;          // ||x_i - x_j||
        const float bn = (float)(pp * s4) * ((float)L.err_gamma * (ri + rj) * (ri + rj) + ee * (2.0f * dist + ee));
        if (K > 0.0) rel = fmaxf(rel, __fdiv_ru(dn, (float)Kn));
        if (bn > 0.0f) bnd = fmaxf(bnd, __fdiv_ru(dn, bn));
    }
    // non-negative binary32 values order as their bits
    const unsigned rb = __float_as_uint(rel), bb = __float_as_uint(bnd);
    if (rb) atomicMax(&st.err_rel_bits, rb);
    if (bb) atomicMax(&st.err_bnd_bits, bb);
    if (threadIdx.x == 0) st.err_pairs += np;
    __syncthreads();
}

// Step 3 of HSEG: exact re-check of the screen's candidates (or of every
// non-adjacent pair when no finite threshold exists or the candidate buffer
// overflowed), merge of the minimum if below the threshold; then, when
// enough regions died, a new compact position list for the screen.
template <bool CSR>
__global__ void __launch_bounds__(STEP_THREADS, 2) k_spec_step(LevelDev L, ScreenConst sc)
{
    const int sec = blockIdx.x;
    if (sec >= L.nsec) return;
    __shared__ StepSmem sm;
    if (threadIdx.x == 0) sm.st = L.st[sec];
    __syncthreads();
    SecState &st = sm.st;
    if (!st.spec_pending) return;
    const int64_t ro = L.roff[sec];
    const int m0 = st.m0;
    constexpr bool csr = CSR;
    const int W = csr ? 0 : L.W[sec];
    const uint32_t *A = L.adj + (csr ? 0 : L.aoff[sec]);
    const double t = st.tthr;
    const int count = st.count;
    const int mc = st.mc;
    const uint32_t ncand = st.ncand;
    const bool finite = t < __longlong_as_double(0x7FF0000000000000ll);
    const bool exhaustive = !finite || (int64_t)ncand > L.cand_cap;
    const int tid = threadIdx.x, nt = blockDim.x, wid = tid >> 5, nw = nt >> 5;
    const uint64_t tbits = dbits(t);
    PairKey best = pk_none();
    long long ntrue = 0;
    // reading R12: pass 0 takes every slot's smallest below-threshold key,
    // pass 1 the smallest partner among the pairs with that key (for a fixed
    // slot, the (K, lo, hi) order of its pairs is the order of the partner)
    if (L.multi) {
        for (int i = tid; i < m0; i += nt) { L.mK[ro + i] = RHSEG_KEY_NONE; L.mP[ro + i] = ~0u; }
        __syncthreads();
    }
    const int npass = L.multi ? 2 : 1;
    for (int pass = 0; pass < npass; pass++) {
        if (!exhaustive) {
            const uint32_t *cand = L.cand + (int64_t)sec * L.cand_cap * 2;
            const int32_t *sop = L.slot_of_pos + L.poff[sec];
            for (uint32_t c0 = 0; c0 < ncand; c0 += PAIR_CAP) {
                __syncthreads();
                if (tid == 0) sm.npair = 0;
                __syncthreads();
                for (uint32_t c = c0 + tid; c < min(ncand, c0 + PAIR_CAP); c += nt) {
                    const int i = sop[cand[2 * c]], j = sop[cand[2 * c + 1]];
                    if (i == j || !L.alive[ro + i] || !L.alive[ro + j]) continue;
                    if (csr ? csr_adjacent(L, sec, st.phalf, ro, i, j) : ((A[(int64_t)i * W + (j >> 5)] >> (j & 31)) & 1))
                        continue;
                    const int idx = atomicAdd(&sm.npair, 1);
                    sm.pi[idx] = min(i, j);
                    sm.pj[idx] = max(i, j);
                    sm.prow[idx] = (int16_t)(c - c0);       // the entry's candidate
                }
                __syncthreads();
                const int np = sm.npair;
                block_keys(L, ro, sm.pi, sm.pj, sm.pkey, np);
                __syncthreads();
                if (L.candg != nullptr && pass == 0)
                    block_screen_error(L, sec, st, cand, c0, np, sm);
                for (int e = tid; e < np; e += nt) {
                    const uint64_t kb = sm.pkey[e];
                    if (!(kb < tbits)) continue;          // K < t (both non-negative binary64)
                    const int i = sm.pi[e], j = sm.pj[e];
                    if (!L.multi) {
                        ntrue++;
                        const PairKey pc = pk_make(kb, i, j);
                        if (pk_less(pc, best)) best = pc;
                    } else if (pass == 0) {
                        ntrue++;
                        atomicMin((unsigned long long *)L.mK + ro + i, (unsigned long long)kb);
                        atomicMin((unsigned long long *)L.mK + ro + j, (unsigned long long)kb);
                    } else {
                        if (kb == __ldcg((const unsigned long long *)L.mK + ro + i)) atomicMin(L.mP + ro + i, (uint32_t)j);
                        if (kb == __ldcg((const unsigned long long *)L.mK + ro + j)) atomicMin(L.mP + ro + j, (uint32_t)i);
                    }
                }
            }
        } else {
            // every unordered pair of live, non-adjacent slots
            const int lane = tid & 31;
            const int64_t npair = (int64_t)m0 * (m0 - 1) / 2;
            for (int64_t e = wid; e < npair; e += nw) {
                int64_t i = (int64_t)((2.0 * m0 - 1 - sqrt((2.0 * m0 - 1) * (2.0 * m0 - 1) - 8.0 * e)) / 2);
                while (i > 0 && i * (2 * m0 - i - 1) / 2 > e) i--;
                while ((i + 1) * (2 * m0 - i - 2) / 2 <= e) i++;
                const int64_t j = e - i * (2 * m0 - i - 1) / 2 + i + 1;
                if (!L.alive[ro + i] || !L.alive[ro + j]) continue;
                if (csr ? csr_adjacent(L, sec, st.phalf, ro, (int)i, (int)j) : ((A[i * W + (j >> 5)] >> (j & 31)) & 1))
                    continue;
                const double K = warp_key(L.S + (ro + i) * L.Bs, L.n[ro + i], L.S + (ro + j) * L.Bs, L.n[ro + j], L.B, L.err);
                if (!(K < t)) continue;
                const uint64_t kb = dbits(K);
                if (!L.multi) {
                    const PairKey pc = pk_make(kb, (int)i, (int)j);
                    if (pk_less(pc, best)) best = pc;
                } else if (lane == 0) {
                    if (pass == 0) {
                        atomicMin((unsigned long long *)L.mK + ro + i, (unsigned long long)kb);
                        atomicMin((unsigned long long *)L.mK + ro + j, (unsigned long long)kb);
                    } else {
                        if (kb == __ldcg((const unsigned long long *)L.mK + ro + i)) atomicMin(L.mP + ro + i, (uint32_t)j);
                        if (kb == __ldcg((const unsigned long long *)L.mK + ro + j)) atomicMin(L.mP + ro + j, (uint32_t)i);
                    }
                }
            }
        }
        __syncthreads();
    }
    ntrue = block_sum_ll(ntrue, sm.ll);
    best = block_min_pk(best, sm.pk);
    __syncthreads();
    if (tid == 0) {
        st.pairs += (int64_t)count * (count - 1) / 2 - st.nadj;
        st.cands += exhaustive ? 0 : (int64_t)ncand;
        st.cands_true += ntrue;
        st.fallbacks += exhaustive ? 1 : 0;
        if (!exhaustive) st.screened += (int64_t)mc * (mc - 1) / 2;
    }
    int merged = 0;
    if (L.multi) {
        double k0;
        merged = block_merge_mutual<CSR>(L, sec, st, L.mK, (const int32_t *)L.mP, 1, sc, sm, &k0) > 0;
    } else if (best.k != RHSEG_KEY_NONE) {
        block_merge<CSR>(L, sec, st, (int)best.lo, (int)best.hi, __longlong_as_double((long long)best.k), 1, sc, sm);
        merged = 1;
    }
    __syncthreads();
    if (tid == 0) {
        st.spec_pending = 0;
        st.ncand = 0;
        if (!merged && !st.merged_adj) { st.stalled = 1; st.done = 1; }
        if (st.count <= st.target) st.done = 1;
    }
    __syncthreads();
    // the screen's work depends on the number of 128-position blocks only
    if (!st.done && (st.count + 127) / 128 < (st.mc + 127) / 128) block_compact_positions(L, sec, st);
    __syncthreads();
    if (tid == 0) L.st[sec] = st;
}

// ---------------------------------------------------------------------------
// Level transitions
// ---------------------------------------------------------------------------

// Resolve each slot's root in the merge forest (pointer jumping in place;
// parent pointers are global slot indices).
__global__ void k_resolve_roots(int32_t *parent, const int64_t *roff, const SecState *st, int32_t nsec)
{
    int sec = blockIdx.x;
    if (sec >= nsec) return;
    int m0 = st[sec].m0;
    int64_t ro = roff[sec];
    __shared__ int changed;
    for (int it = 0; it < 40; it++) {
        __syncthreads();
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < m0; i += blockDim.x) {
            int p = parent[ro + i];
            int pp = parent[p];
            if (pp != p) { parent[ro + i] = pp; changed = 1; }
        }
        __syncthreads();
        if (!changed) break;
    }
}

// Pixel labels after a level: the ID of the root of the pixel's region.
__global__ void k_relabel(int64_t P, uint32_t *label, const int32_t *slot_of_id, const int32_t *parent,
                          const uint32_t *rid)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t l = label[p];
        if (!l) continue;
        label[p] = rid[parent[slot_of_id[l - 1]]];
    }
}

// ---------------------------------------------------------------------------
// Seam pass (boundary-artifact removal, Section 6.2 future work; reading R7)
// ---------------------------------------------------------------------------

struct SeamGeom {
    const int32_t *rb_c, *cb_c;   // row / column band at the child level
    int nbits_p;                  // split bits of the parent level
    int conn;
};

__device__ __forceinline__ void parent_and_quad(const SeamGeom &sg, int y, int x, int32_t &par, int &quad)
{
    int rb = sg.rb_c[y], cb = sg.cb_c[x];
    par = morton2(rb >> 1, cb >> 1, sg.nbits_p);
    quad = ((rb & 1) << 1) | (cb & 1);
}

__device__ __forceinline__ int nb_dy(int conn, int k)
{
    const int d8[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    const int d4[4] = {-1, 0, 0, 1};
    return conn == 8 ? d8[k] : d4[k];
}
__device__ __forceinline__ int nb_dx(int conn, int k)
{
    const int d8[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    const int d4[4] = {0, -1, 1, 0};
    return conn == 8 ? d8[k] : d4[k];
}

// Seam pixels: unmasked, with a neighbour in the same parent section but in
// another child quadrant.
__global__ void k_seam_detect(PixGeom g, SeamGeom sg, const uint32_t *label, int32_t *seam_list,
                              int32_t *nseam, int32_t seam_cap)
{
    int64_t P = (int64_t)g.rows * g.cols;
    int nn = sg.conn == 8 ? 8 : 4;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        if (!label[p]) continue;
        int y = (int)(p / g.cols), x = (int)(p % g.cols);
        int32_t par; int qd;
        parent_and_quad(sg, y, x, par, qd);
        bool seam = false;
        for (int k = 0; k < nn && !seam; k++) {
            int yy = y + nb_dy(sg.conn, k), xx = x + nb_dx(sg.conn, k);
            if (yy < 0 || yy >= g.rows || xx < 0 || xx >= g.cols) continue;
            int64_t q = (int64_t)yy * g.cols + xx;
            if (!label[q]) continue;
            int32_t par2; int qd2;
            parent_and_quad(sg, yy, xx, par2, qd2);
            if (par2 == par && qd2 != qd) seam = true;
        }
        if (seam) {
            int k = atomicAdd(nseam, 1);
            if (k < seam_cap) seam_list[k] = (int32_t)p;
        }
    }
}

// K({p}, region) for a one-pixel region p (warp-cooperative, exact).
__device__ __forceinline__ double warp_key_pixel(const uint16_t *xp, const int64_t *Sj, int64_t nj, int B,
                                                 int32_t *err)
{
    int lane = threadIdx.x & 31;
    u128 acc = {0, 0};
    for (int b = lane; b < B; b += 32) {
        int64_t d = nj * (int64_t)xp[b] - Sj[b];
        uint64_t a = (uint64_t)(d < 0 ? -d : d);
        acc = u128_add(acc, u128_sq(a));
    }
    acc = warp_sum_u128(acc);
    double K = 0.0;
    if (lane == 0) {
        u128 D = u128_mul64((uint64_t)nj, (uint64_t)(nj + 1));
        K = div_rn_u128(acc, D, err);
    }
    return __shfl_sync(0xffffffffu, K, 0);
}

// Split decisions against the pre-pass state (warp per seam pixel).
__global__ void k_seam_decide(PixGeom g, SeamGeom sg, const uint32_t *label, const int32_t *slot_of_id,
                              const int64_t *S, const int64_t *n, const uint32_t *rid,
                              const int32_t *seam_list, const int32_t *nseam, int32_t seam_cap, uint8_t *split,
                              double *split_key, uint32_t *split_from, int32_t *err)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int ns = min(*nseam, seam_cap);
    if (*nseam > seam_cap && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(err, 0x5345414d);  // seam list overflow
    int nn = sg.conn == 8 ? 8 : 4;
    for (int64_t t = warp; t < ns; t += nwarps) {
        int64_t p = seam_list[t];
        int y = (int)(p / g.cols), x = (int)(p % g.cols);
        int32_t par; int qd;
        parent_and_quad(sg, y, x, par, qd);
        const uint16_t *xp = g.img + p * g.B;
        int64_t R = slot_of_id[label[p] - 1];
        double kr = warp_key_pixel(xp, S + R * g.Bs, n[R], g.B, err);
        double best = __longlong_as_double(0x7FF0000000000000ll);
        int64_t seen[8];
        int nseen = 0;
        for (int k = 0; k < nn; k++) {
            int yy = y + nb_dy(sg.conn, k), xx = x + nb_dx(sg.conn, k);
            if (yy < 0 || yy >= g.rows || xx < 0 || xx >= g.cols) continue;
            int64_t q = (int64_t)yy * g.cols + xx;
            if (!label[q]) continue;
            int32_t par2; int qd2;
            parent_and_quad(sg, yy, xx, par2, qd2);
            if (par2 != par || qd2 == qd) continue;
            int64_t Q = slot_of_id[label[q] - 1];
            bool dup = false;
            for (int i = 0; i < nseen; i++) dup |= (seen[i] == Q);
            if (dup) continue;
            seen[nseen++] = Q;
            double kq = warp_key_pixel(xp, S + Q * g.Bs, n[Q], g.B, err);
            best = fmin(best, kq);
        }
        if (lane == 0) {
            bool sp = best < kr;
            split[p] = sp ? 1 : 0;
            if (sp) { split_key[p] = kr; split_from[p] = rid[R]; }
        }
    }
}

// Apply every split together: the pixel leaves its region (exact integer
// subtraction) and becomes a one-pixel region with ID p+1.
__global__ void k_seam_apply(PixGeom g, uint32_t *label, const int32_t *slot_of_id, int64_t *S, int64_t *n,
                             uint32_t *rid, uint8_t *lostid, const int32_t *seam_list, const int32_t *nseam,
                             int32_t seam_cap, const uint8_t *split)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int ns = min(*nseam, seam_cap);
    for (int64_t t = warp; t < ns; t += nwarps) {
        int64_t p = seam_list[t];
        if (!split[p]) continue;
        int64_t R = slot_of_id[label[p] - 1];
        const uint16_t *xp = g.img + p * g.B;
        for (int b = lane; b < g.B; b += 32)
            atomicAdd((unsigned long long *)&S[R * g.Bs + b], (unsigned long long)(-(long long)xp[b]));
        if (lane == 0) {
            atomicAdd((unsigned long long *)&n[R], (unsigned long long)(-1ll));
            if (rid[R] == (uint32_t)(p + 1)) lostid[R] = 1;
        }
    }
}

// Split pixels carry their own ID from now on.
__global__ void k_seam_label_singletons(const int32_t *seam_list, const int32_t *nseam, int32_t seam_cap,
                                        const uint8_t *split, uint32_t *label)
{
    int ns = min(*nseam, seam_cap);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ns; t += gridDim.x * blockDim.x) {
        int64_t p = seam_list[t];
        if (split[p]) label[p] = (uint32_t)(p + 1);
    }
}

// Regions that lost the pixel carrying their ID get ID = 1 + smallest
// raster index of the pixels they keep (reading R5).
__global__ void k_lost_reset(int64_t nslots, const uint8_t *lostid, uint32_t *rid)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nslots; g += (int64_t)gridDim.x * blockDim.x)
        if (lostid[g]) rid[g] = 0xffffffffu;
}

__global__ void k_lost_min(int64_t P, const uint32_t *label, const uint8_t *split, const int32_t *slot_of_id,
                           const uint8_t *lostid, uint32_t *rid)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t l = label[p];
        if (!l || split[p]) continue;
        int64_t g = slot_of_id[l - 1];
        if (lostid[g]) atomicMin(&rid[g], (uint32_t)(p + 1));
    }
}

__global__ void k_lost_relabel(int64_t P, uint32_t *label, const uint8_t *split, const int32_t *slot_of_id,
                               const uint8_t *lostid, const uint32_t *rid)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t l = label[p];
        if (!l || split[p]) continue;
        int64_t g = slot_of_id[l - 1];
        if (lostid[g]) label[p] = rid[g];
    }
}

// Region sources of the next level: surviving regions (by their possibly
// re-derived ID) and the one-pixel regions of the seam pass.
__global__ void k_mark_ids_upper(const int64_t *roff_prev, const SecState *st_prev,
                                 int32_t nsec_prev, const uint8_t *alive, const int64_t *n, const uint32_t *rid,
                                 uint8_t *isid, int32_t *srcslot)
{
    int sec = blockIdx.y;
    if (sec >= nsec_prev) return;
    int m0 = st_prev[sec].m0;
    int64_t ro = roff_prev[sec];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m0; i += gridDim.x * blockDim.x) {
        int64_t gsl = ro + i;
        if (!alive[gsl] || n[gsl] <= 0) continue;
        uint32_t id = rid[gsl];
        isid[id - 1] = 1;
        srcslot[id - 1] = (int32_t)gsl;
    }
}

__global__ void k_mark_singletons(const int32_t *seam_list, const int32_t *nseam, int32_t seam_cap,
                                  const uint8_t *split, uint8_t *isid, int32_t *srcslot)
{
    int ns = min(*nseam, seam_cap);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ns; t += gridDim.x * blockDim.x) {
        int64_t p = seam_list[t];
        if (!split[p]) continue;
        isid[p] = 1;
        srcslot[p] = -1;
    }
}

// ---------------------------------------------------------------------------
// Root hierarchy snapshots (reading R9)
// ---------------------------------------------------------------------------

// canon[g] = 1-based rank (slot order = ID order) of slots alive after
// merge ordinal M, 0 otherwise.  Single block.
__global__ void k_snap_canon(int m0, const int32_t *absorbed_at, int32_t M, int32_t *canon, int32_t *R_out)
{
    __shared__ int32_t wcnt[32];
    __shared__ int32_t base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = 0; c < m0; c += blockDim.x) {
        int i = c + threadIdx.x;
        int f = (i < m0) ? (absorbed_at[i] > M) : 0;
        unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wcnt[wid] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int k = 0; k < nw; k++) { if (k < wid) off += wcnt[k]; tot += wcnt[k]; }
        if (i < m0) canon[i] = f ? base + off + __popc(bal & ((1u << lane) - 1)) + 1 : 0;
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *R_out = base;
}

__device__ __forceinline__ int32_t snap_walk(int32_t g, const int32_t *parent, const int32_t *absorbed_at, int32_t M)
{
    for (int it = 0; it < (1 << 30) && absorbed_at[g] <= M; it++) g = parent[g];
    return g;
}

__global__ void k_snap_labels(int64_t P, const uint32_t *label, const int32_t *slot_of_id, const int32_t *parent,
                              const int32_t *absorbed_at, int32_t M, const int32_t *canon, int32_t *out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t l = label[p];
        out[p] = l ? canon[snap_walk(slot_of_id[l - 1], parent, absorbed_at, M)] : 0;
    }
}

__global__ void k_snap_tables(int m0, int B, int Bs, const int64_t *S0, const int64_t *n0, const int32_t *parent,
                              const int32_t *absorbed_at, int32_t M, const int32_t *canon, int64_t *sums,
                              int64_t *counts)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g0 = warp; g0 < m0; g0 += nwarps) {
        int c = canon[snap_walk((int32_t)g0, parent, absorbed_at, M)] - 1;
        for (int b = lane; b < B; b += 32)
            atomicAdd((unsigned long long *)&sums[(int64_t)c * B + b], (unsigned long long)S0[g0 * Bs + b]);
        if (lane == 0) atomicAdd((unsigned long long *)&counts[c], (unsigned long long)n0[g0]);
    }
}

// As k_snap_tables, for a caller that wants only the band sums or only the
// counts (the other pointer is null).
__global__ void k_snap_tables_part(int m0, int B, int Bs, const int64_t *S0, const int64_t *n0, const int32_t *parent,
                                   const int32_t *absorbed_at, int32_t M, const int32_t *canon, int64_t *sums,
                                   int64_t *counts)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g0 = warp; g0 < m0; g0 += nwarps) {
        int c = canon[snap_walk((int32_t)g0, parent, absorbed_at, M)] - 1;
        if (sums)
            for (int b = lane; b < B; b += 32)
                atomicAdd((unsigned long long *)&sums[(int64_t)c * B + b], (unsigned long long)S0[g0 * Bs + b]);
        if (counts && lane == 0) atomicAdd((unsigned long long *)&counts[c], (unsigned long long)n0[g0]);
    }
}

}  // namespace rhseg
