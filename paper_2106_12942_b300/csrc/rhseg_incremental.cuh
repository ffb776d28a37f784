// rhseg_incremental.cuh -- incremental spectral minima (exact).
//
// HSEG's spectral step (Section 4.1, step 3) takes the minimum key over all
// non-adjacent region pairs.  The thesis recomputes every pair each
// iteration ("Approach 2"); its conclusions (Chapter 7) point to reusing
// dissimilarities between iterations.  This file keeps, for every live
// region i, its exact best non-adjacent partner
//      (sbK[i], sbP[i]) = min over live non-adjacent j != i of (K_ij, lo, hi)
// in the same (key, lower slot, higher slot) order as the step's argmin, so
// the step's pair is the minimum of the per-region bests and the merges are
// identical to the all-pairs form.  After a merge of b into a only the rows
// whose best was a or b, and a itself, are recomputed; every other row's
// best can only improve through the pair with the new a, which is pushed to
// it while a's row is evaluated.
//
// A row is evaluated against all live positions with the binary32 operand
// rows x^ (region means relative to the section reference): s = sum over
// bands of fl(x^_i - x^_j)^2 gives the approximate key s / (k_i + k_j),
// k = 4^-sigma / n, and a certified lower bound of the exact key,
//      K_ij >= max(0, ||d^|| (1 - 2^-23) - e_i - e_j)^2 / (k_i + k_j),
// ||d^|| >= sqrt(s / (1 + gamma_B)), e_i >= ||x^_i - x_i|| (the operand
// error norm), every operation rounded in the safe direction.  The
// approximate argmin gives one exact key U (an upper bound of the row's
// minimum); every pair whose lower bound is <= U is then re-checked exactly,
// which decides the row.  The same bound against a neighbour's own best
// selects the pairs pushed to it.  (The differences avoid the cancellation
// of q_i + q_j - 2 g, so the bound is within ~1e-4 of the key.)
#pragma once
#include "rhseg_screen_simt.cuh"

namespace rhseg {

constexpr int INC_TILE = 64;
constexpr int INC_KC = 16;
constexpr int INC_RC = 8;               // rows evaluated per pass over a section's operand rows
constexpr int INC_RCAP = 32;            // rows of one update evaluated by the many-block sums pass

__device__ __forceinline__ unsigned long long inc_pack_pair(int i, int j)
{
    const uint32_t lo = (uint32_t)min(i, j), hi = (uint32_t)max(i, j);
    return ((unsigned long long)lo << 32) | hi;
}

// Certified lower bound of K_ij from s = fl(sum fl(x^_i - x^_j)^2) (Bpad
// fma steps), the operand error norms e and k = 4^-sigma / n (all rounded
// up); the result is rounded down.
__device__ __forceinline__ float inc_klo(float s, float ei, float ej, float ki, float kj, float onepg)
{
    float L = __fmul_rd(__fsqrt_rd(__fdiv_rd(s, onepg)), 1.0f - 0x1p-23f);
    L = __fsub_rd(L, __fadd_ru(ei, ej));
    if (!(L > 0.0f)) return 0.0f;
    return __fmul_rd(__fdiv_rd(1.0f, __fadd_ru(ki, kj)), __fmul_rd(L, L));
}

// binary32 threshold for "K <= U": the next binary64 above U, rounded up.
__device__ __forceinline__ float inc_thr_le(uint64_t Ubits)
{
    if (Ubits == RHSEG_KEY_NONE) return __int_as_float(0x7f800000);            // no best: every pair
    const double T = __longlong_as_double((long long)(Ubits + 1));              // K >= 0: next double up
    return __double2float_ru(T);
}

// Approximate key (only to choose a good U).
__device__ __forceinline__ float inc_khat(float s, float ki, float kj) { return s / (ki + kj); }

__device__ __forceinline__ unsigned long long inc_pack_apx(float khat, int slot)
{
    return ((unsigned long long)(uint32_t)__float_as_int(khat) << 32) | (uint32_t)slot;
}

template <typename TS> __device__ __forceinline__ float inc_ld(const TS *p);
template <> __device__ __forceinline__ float inc_ld<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float inc_ld<__half>(const __half *p) { return __half2float(*p); }
template <> __device__ __forceinline__ float inc_ld<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// ---------------------------------------------------------------------------
// Level start: every row's best, by 64x64 tiles of positions (positions are
// the slots at level start).  PASS 0: approximate argmin per row.  PASS 1:
// candidates of every row at its own threshold.
// ---------------------------------------------------------------------------
template <typename TS, int PASS>
__global__ void __launch_bounds__(256) k_sinit_tile(LevelDev L)
{
    __shared__ long long pre[MAX_SECTIONS + 1];
    __shared__ float As[INC_KC][INC_TILE + 1];
    __shared__ float Bsm[INC_KC][INC_TILE + 1];
    __shared__ float rA[INC_TILE], rk[INC_TILE], rT[INC_TILE], cA[INC_TILE], ck[INC_TILE], cT[INC_TILE];   // A: error norm e
    __shared__ uint32_t adjw[INC_TILE][3];
    block_tile_prefix(L, -INC_TILE, pre);
    const long long total = pre[L.nsec];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int sec = find_section(pre, L.nsec, t);
        const SecState *st = &L.st[sec];
        const int mc = st->mc;
        const long long nb = (mc + INC_TILE - 1) / INC_TILE;
        int I, J;
        tri_decode(t - pre[sec], nb, I, J);
        const int64_t pb = L.poff[sec];
        const int W = L.W[sec];
        const uint32_t *Aj = L.adj + L.aoff[sec];
        const TS *X = (const TS *)L.X;
        const TS *XA = X + (pb + (int64_t)I * INC_TILE) * L.Bpad;
        const TS *XB = X + (pb + (int64_t)J * INC_TILE) * L.Bpad;
        const float nan = __int_as_float(0x7fc00000);
        __syncthreads();
        if (threadIdx.x < 2 * INC_TILE) {
            const int r = threadIdx.x & (INC_TILE - 1);
            const bool row = threadIdx.x < INC_TILE;
            const int pos = (row ? I : J) * INC_TILE + r;
            float a = nan, k = nan, T = nan;
            if (pos < mc) {
                a = L.sE[pb + pos];
                k = L.sk[pb + pos];
                if (PASS == 1) T = L.sT[pb + pos];
            }
            if (row) { rA[r] = a; rk[r] = k; rT[r] = T; } else { cA[r] = a; ck[r] = k; cT[r] = T; }
        }
        if (threadIdx.x < INC_TILE) {
            // adjacency bits of row I*64 + r for columns J*64 .. J*64 + 63 (positions are slots here)
            const int i = I * INC_TILE + threadIdx.x;
            const int w0 = (J * INC_TILE) >> 5;
            for (int q = 0; q < 3; q++)
                adjw[threadIdx.x][q] = (i < mc && w0 + q < W) ? Aj[(int64_t)i * W + w0 + q] : 0u;
        }
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[a][c] = 0.0f;
        for (int k0 = 0; k0 < L.Bpad; k0 += INC_KC) {
            __syncthreads();
            for (int e = threadIdx.x; e < INC_TILE * INC_KC; e += blockDim.x) {
                const int r = e / INC_KC, k = e % INC_KC;
                As[k][r] = inc_ld<TS>(XA + (int64_t)r * L.Bpad + k0 + k);
                Bsm[k][r] = inc_ld<TS>(XB + (int64_t)r * L.Bpad + k0 + k);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < INC_KC; k++) {
                float av[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; a++) av[a] = As[k][ty * 4 + a];
#pragma unroll
                for (int c = 0; c < 4; c++) bv[c] = Bsm[k][tx * 4 + c];
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const float d = av[a] - bv[c];
                        acc[a][c] = fmaf(d, d, acc[a][c]);
                    }
            }
        }
        if (PASS == 0) {
            unsigned long long rbest[4] = {~0ull, ~0ull, ~0ull, ~0ull}, cbest[4] = {~0ull, ~0ull, ~0ull, ~0ull};
#pragma unroll
            for (int a = 0; a < 4; a++) {
                const int li = ty * 4 + a, i = I * INC_TILE + li;
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const int lj = tx * 4 + c, j = J * INC_TILE + lj;
                    if (!(i < j && j < mc)) continue;
                    const int bit = j - ((J * INC_TILE) & ~31);
                    if ((adjw[li][bit >> 5] >> (bit & 31)) & 1) continue;
                    const float kh = inc_khat(acc[a][c], rk[li], ck[lj]);
                    const unsigned long long pr = inc_pack_apx(kh, j), pc = inc_pack_apx(kh, i);
                    if (pr < rbest[a]) rbest[a] = pr;
                    if (pc < cbest[c]) cbest[c] = pc;
                }
            }
            // rows: the 16 threads of a row group (same ty) share rows ty*4 + a
#pragma unroll
            for (int a = 0; a < 4; a++) {
                unsigned long long v = rbest[a];
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) {
                    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o, 16);
                    v = w < v ? w : v;
                }
                if (tx == 0 && v != ~0ull) atomicMin(&L.sinit[pb + I * INC_TILE + ty * 4 + a], v);
            }
            // columns: reduce over ty through shared memory
            __shared__ unsigned long long colbest[INC_TILE];
            __syncthreads();
            if (threadIdx.x < INC_TILE) colbest[threadIdx.x] = ~0ull;
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 4; c++)
                if (cbest[c] != ~0ull) atomicMin(&colbest[tx * 4 + c], cbest[c]);
            __syncthreads();
            if (threadIdx.x < INC_TILE && colbest[threadIdx.x] != ~0ull)
                atomicMin(&L.sinit[pb + J * INC_TILE + threadIdx.x], colbest[threadIdx.x]);
        } else {
            SecState *stw = &L.st[sec];
#pragma unroll
            for (int a = 0; a < 4; a++) {
                const int li = ty * 4 + a, i = I * INC_TILE + li;
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const int lj = tx * 4 + c, j = J * INC_TILE + lj;
                    if (!(i < j && j < mc)) continue;
                    const int bit = j - ((J * INC_TILE) & ~31);
                    if ((adjw[li][bit >> 5] >> (bit & 31)) & 1) continue;
                    // row i at its threshold, row j at its threshold (NaN: the row has none)
                    const float kl = inc_klo(acc[a][c], rA[li], cA[lj], rk[li], ck[lj], L.inc_onepg);
                    const bool ci = kl <= rT[li];
                    const bool cj = kl <= cT[lj];
                    if (!(ci || cj)) continue;
                    const uint32_t idx = atomicAdd(&stw->ncand, 1u);
                    if ((int64_t)idx < L.cand_cap) {
                        uint32_t *cd = L.cand + ((int64_t)sec * L.cand_cap + idx) * 2;
                        cd[0] = (uint32_t)i | (ci ? 0x40000000u : 0u) | (cj ? 0x80000000u : 0u);
                        cd[1] = (uint32_t)j;
                    }
                }
            }
        }
    }
    (void)0;
}

// Level start, after PASS 0: the exact key of each row's approximate best
// (an upper bound U of its minimum) and the row's binary32 threshold.
__global__ void __launch_bounds__(256) k_sinit_exact(LevelDev L)
{
    const int sec = blockIdx.y;
    const SecState &st = L.st[sec];
    if (st.done) return;
    const int mc = st.mc;
    const int64_t ro = L.roff[sec], pb = L.poff[sec];
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < mc; i += gridDim.x * wpb) {
        const unsigned long long apx = L.sinit[pb + i];
        uint64_t U = RHSEG_KEY_NONE;
        int j = -1;
        if (apx != ~0ull) {
            j = (int)(uint32_t)apx;
            const double K = warp_key(L.S + (ro + i) * L.Bs, L.n[ro + i], L.S + (ro + j) * L.Bs, L.n[ro + j], L.B, L.err);
            U = dbits(K);
        }
        if (lane == 0) {
            L.sbK[ro + i] = U;
            L.sbP[ro + i] = j;
            L.stie[ro + i] = (j >= 0) ? inc_pack_pair(i, j) : ~0ull;
            L.sinit[pb + i] = U;                       // kept: the row's bound before the candidates
            L.sT[pb + i] = (j >= 0) ? inc_thr_le(U) : __int_as_float(0x7fc00000);   // none: no pair passes
        }
    }
}

// Exact keys of `cnt` (row, partner) slot pairs staged from a section's
// candidate list, with the keys written back to ckey (whole block).
__device__ void inc_keys_from_list(const LevelDev &L, int sec, uint32_t c0, uint32_t cnt, StepSmem &sm)
{
    const int64_t ro = L.roff[sec];
    const uint32_t *cand = L.cand + (int64_t)sec * L.cand_cap * 2;
    unsigned long long *ck = L.ckey + (int64_t)sec * L.cand_cap;
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < cnt; c += blockDim.x) {
        const uint32_t a = cand[2 * (c0 + c)] & 0x3fffffffu, b = cand[2 * (c0 + c) + 1];
        sm.pi[c] = (int32_t)a;
        sm.pj[c] = (int32_t)b;
    }
    __syncthreads();
    block_keys(L, ro, sm.pi, sm.pj, sm.pkey, (int)cnt);
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < cnt; c += blockDim.x) ck[c0 + c] = sm.pkey[c];
    __syncthreads();
}

// Full exact scan of row r over all live non-adjacent slots (one warp);
// the fallback when a candidate list overflowed.
__device__ void warp_spectral_row_exact(const LevelDev &L, int sec, int r, int m0)
{
    const int lane = threadIdx.x & 31;
    const int64_t ro = L.roff[sec];
    const int W = L.W[sec];
    const uint32_t *row = L.adj + L.aoff[sec] + (int64_t)r * W;
    PairKey best = pk_none();
    for (int j = 0; j < m0; j++) {
        if (j == r || !L.alive[ro + j]) continue;
        if ((row[j >> 5] >> (j & 31)) & 1) continue;
        const double K = warp_key(L.S + (ro + r) * L.Bs, L.n[ro + r], L.S + (ro + j) * L.Bs, L.n[ro + j], L.B, L.err);
        const PairKey c = pk_make(dbits(K), r, j);
        if (pk_less(c, best)) best = c;
    }
    if (lane == 0) {
        L.sbK[ro + r] = best.k;
        L.sbP[ro + r] = (best.k == RHSEG_KEY_NONE) ? -1 : (int32_t)(best.lo == (uint32_t)r ? best.hi : best.lo);
    }
}

// Level start, after PASS 1: exact keys of the candidates and every row's
// exact best (one block per section).
__global__ void __launch_bounds__(STEP_THREADS) k_sinit_final(LevelDev L)
{
    const int sec = blockIdx.x;
    __shared__ StepSmem sm;
    SecState *stg = &L.st[sec];
    if (stg->done) return;
    const int64_t ro = L.roff[sec];
    const int mc = stg->mc;
    const uint32_t ncand = stg->ncand;
    const uint32_t *cand = L.cand + (int64_t)sec * L.cand_cap * 2;
    const unsigned long long *ck = L.ckey + (int64_t)sec * L.cand_cap;
    const bool overflow = (int64_t)ncand > L.cand_cap;
    if (overflow) {
        const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r = wid; r < mc; r += nw) warp_spectral_row_exact(L, sec, r, stg->m0);
        __syncthreads();
        if (threadIdx.x == 0) { stg->fallbacks += 1; stg->ncand = 0; }
        return;
    }
    // keys: each candidate carries flags for the rows it serves (bit 30: row
    // i = cand[0], bit 31: row j = cand[1]); one key serves both
    for (uint32_t c0 = 0; c0 < ncand; c0 += PAIR_CAP) inc_keys_from_list(L, sec, c0, min((uint32_t)PAIR_CAP, ncand - c0), sm);
    // phase 1: minimum key per row
    for (uint32_t c = threadIdx.x; c < ncand; c += blockDim.x) {
        const uint32_t w0 = cand[2 * c], j = cand[2 * c + 1], i = w0 & 0x3fffffffu;
        if (w0 & 0x40000000u) atomicMin((unsigned long long *)&L.sbK[ro + i], ck[c]);
        if (w0 & 0x80000000u) atomicMin((unsigned long long *)&L.sbK[ro + j], ck[c]);
    }
    __syncthreads();
    // the bound's own pair keeps its tie word only if the minimum is still U
    for (int i = threadIdx.x; i < mc; i += blockDim.x)
        if (L.sbK[ro + i] != L.sinit[L.poff[sec] + i]) L.stie[ro + i] = ~0ull;
    __syncthreads();
    // phase 2: lowest slot pair among the minimum keys
    for (uint32_t c = threadIdx.x; c < ncand; c += blockDim.x) {
        const uint32_t w0 = cand[2 * c], j = cand[2 * c + 1], i = w0 & 0x3fffffffu;
        const unsigned long long p = inc_pack_pair((int)i, (int)j);
        if ((w0 & 0x40000000u) && ck[c] == L.sbK[ro + i]) atomicMin(&L.stie[ro + i], p);
        if ((w0 & 0x80000000u) && ck[c] == L.sbK[ro + j]) atomicMin(&L.stie[ro + j], p);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < mc; i += blockDim.x) {
        const unsigned long long p = L.stie[ro + i];
        if (L.sbK[ro + i] == RHSEG_KEY_NONE || p == ~0ull) { L.sbP[ro + i] = -1; continue; }
        const uint32_t lo = (uint32_t)(p >> 32), hi = (uint32_t)p;
        L.sbP[ro + i] = (int32_t)(lo == (uint32_t)i ? hi : lo);
    }
    __syncthreads();
    if (threadIdx.x == 0) { stg->cands += ncand; stg->ncand = 0; }
}

// ---------------------------------------------------------------------------
// Per iteration: rows to recompute after the pending merges, evaluated in
// passes of up to INC_RC rows over the section's live positions.
// ---------------------------------------------------------------------------

// Pass A over the live positions of a section: s[r] = sum over bands of
// fl(x^_r - x^_j)^2 for the rows r of the chunk (binary32 rows, float4
// loads), stored per position in sbuf, and each row's approximate argmin.
template <int RC>
__device__ void inc_pass_sums(const LevelDev &L, int sec, const int32_t *rows, int nr, const float *xs,
                              const float *rAk, unsigned long long *apx, int p_lo, int p_hi, int sb_off)
{
    const int64_t ro = L.roff[sec], pb = L.poff[sec];
    const int W = L.W[sec];
    const uint32_t *A = L.adj + L.aoff[sec];
    const int mc = L.st[sec].mc;
    const float *X = (const float *)L.X;
    unsigned long long lbest[RC];
#pragma unroll
    for (int r = 0; r < RC; r++) lbest[r] = ~0ull;
    (void)mc;
    for (int p = p_lo + (int)threadIdx.x; p < p_hi; p += blockDim.x) {
        const int j = L.slot_of_pos[pb + p];
        if (!L.alive[ro + j]) continue;
        const float4 *xj = (const float4 *)(X + (pb + p) * L.Bpad);
        float g[RC];
#pragma unroll
        for (int r = 0; r < RC; r++) g[r] = 0.0f;
        for (int b4 = 0; b4 < L.Bpad / 4; b4++) {
            const float4 v = __ldg(xj + b4);
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const float *xb = xs + (b4 * 4 + e) * INC_RC;
#pragma unroll
                for (int r = 0; r < RC; r++) {
                    const float d = xb[r] - vv[e];
                    g[r] = fmaf(d, d, g[r]);
                }
            }
        }
        float *sb = L.sbuf + (pb + p) * INC_RCAP + sb_off;
#pragma unroll
        for (int r = 0; r < RC; r++) sb[r] = g[r];
        const float kj = L.sk[pb + p];
#pragma unroll
        for (int r = 0; r < RC; r++) {
            if (r >= nr) break;
            const int rs = rows[r];
            if (rs == j) continue;
            if ((A[(int64_t)rs * W + (j >> 5)] >> (j & 31)) & 1) continue;
            const unsigned long long v = inc_pack_apx(inc_khat(g[r], rAk[2 * r + 1], kj), j);
            if (v < lbest[r]) lbest[r] = v;
        }
    }
#pragma unroll
    for (int r = 0; r < RC; r++) {
        unsigned long long v = lbest[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w < v ? w : v;
        }
        if ((threadIdx.x & 31) == 0 && r < nr && v != ~0ull) atomicMin(&apx[r], v);
    }
}

// Pass B: the certified lower bounds from the stored sums; candidates for
// each row's own minimum (bound <= its U) and, for the merged rows, for the
// partners whose best they may improve (bound <= the partner's best).
__device__ void inc_pass_test(const LevelDev &L, int sec, const int32_t *rows, int nr, int nprop, const float *rAk,
                              const float *rT, uint32_t *ncand_s, int sb_off)
{
    const int64_t ro = L.roff[sec], pb = L.poff[sec];
    const int W = L.W[sec];
    const uint32_t *A = L.adj + L.aoff[sec];
    const int mc = L.st[sec].mc;
    uint32_t *cand = L.cand + (int64_t)sec * L.cand_cap * 2;
    for (int p = threadIdx.x; p < mc; p += blockDim.x) {
        const int j = L.slot_of_pos[pb + p];
        if (!L.alive[ro + j]) continue;
        const float *sb = L.sbuf + (pb + p) * INC_RCAP + sb_off;
        const float Ej = L.sE[pb + p], kj = L.sk[pb + p];
        float Tj = 0.0f;
        bool inr = false;
        if (nprop > 0) {
            inr = L.inR[ro + j] != 0;
            Tj = inc_thr_le(L.sbK[ro + j]);
        }
        for (int r = 0; r < nr; r++) {
            const int rs = rows[r];
            if (rs == j) continue;
            if ((A[(int64_t)rs * W + (j >> 5)] >> (j & 31)) & 1) continue;
            const float kl = inc_klo(sb[r], rAk[2 * r], Ej, rAk[2 * r + 1], kj, L.inc_onepg);
            const bool own = kl <= rT[r];
            const bool prop = (r < nprop) && !inr && (kl <= Tj);
            if (!(own || prop)) continue;
            const uint32_t idx = atomicAdd(ncand_s, 1u);
            if ((int64_t)idx < L.cand_cap) {
                cand[2 * idx] = (uint32_t)r | (own ? 0x40000000u : 0u) | (prop ? 0x80000000u : 0u);
                cand[2 * idx + 1] = (uint32_t)j;
            }
        }
    }
}


// Shared memory of the update kernels: staged row vectors [Bpad][INC_RC]
// (binary32).
__host__ __device__ constexpr int inc_dyn_smem(int Bpad) { return Bpad * INC_RC * 4; }

constexpr int INC_SUM_BLOCKS = 8;      // blocks per section of the sums pass

// Per-section state of one row update, between its three kernels.
struct IncInfo {
    int32_t nrows, nmerged, nstaged;          // rows to recompute; merged survivors; rows staged (<= INC_RCAP)
    int32_t active;
    int32_t crow[INC_RCAP];
    float rAk[2 * INC_RCAP];
    unsigned long long apx[INC_RCAP];
};

// Exact bound, pass B, exact keys, minima and pushes of a chunk whose sums
// are in sbuf and approximate argmins in apx_in (whole block).
__device__ long long inc_chunk_finish(const LevelDev &L, int sec, StepSmem &sm, int m0, const int32_t *crow_s,
                                      int nr, int nprop, const float *rAk_s, const unsigned long long *apx_s,
                                      float *rT, unsigned long long *rK, unsigned long long *rTie,
                                      unsigned long long *rU, uint32_t *ncand_s, int64_t &fallbacks, int sb_off)
{
    const int64_t ro = L.roff[sec];
    // exact key of each row's approximate best: the bound U
    {
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (wid < nr) {
            const int r = crow_s[wid];
            const unsigned long long a = apx_s[wid];
            uint64_t U = RHSEG_KEY_NONE;
            int j = -1;
            if (a != ~0ull) {
                j = (int)(uint32_t)a;
                U = dbits(warp_key(L.S + (ro + r) * L.Bs, L.n[ro + r], L.S + (ro + j) * L.Bs, L.n[ro + j], L.B, L.err));
            }
            if (lane == 0) {
                rU[wid] = U;
                rK[wid] = U;
                rTie[wid] = (j >= 0) ? inc_pack_pair(r, j) : ~0ull;
                rT[wid] = (j >= 0) ? inc_thr_le(U) : __int_as_float(0x7fc00000);
            }
        }
        if (threadIdx.x == 0) *ncand_s = 0;
    }
    __syncthreads();
    // pass B: candidates for each row's own minimum, and the merged rows'
    // keys that may improve another row's best
    inc_pass_test(L, sec, crow_s, nr, nprop, rAk_s, rT, ncand_s, sb_off);
    __syncthreads();
    const uint32_t nc = *ncand_s;
    if ((int64_t)nc > L.cand_cap) {
        // overflow: exact scans (merged rows push to every row, one row at a time)
        const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r = wid; r < nr; r += nw) warp_spectral_row_exact(L, sec, crow_s[r], m0);
        __syncthreads();
        for (int r = 0; r < nprop; r++) {
            const int a = crow_s[r];
            const uint32_t *rowA = L.adj + L.aoff[sec] + (int64_t)a * L.W[sec];
            for (int j = wid; j < m0; j += nw) {
                if (j == a || !L.alive[ro + j] || L.inR[ro + j]) continue;
                if ((rowA[j >> 5] >> (j & 31)) & 1) continue;
                const double K = warp_key(L.S + (ro + a) * L.Bs, L.n[ro + a], L.S + (ro + j) * L.Bs, L.n[ro + j], L.B, L.err);
                if ((threadIdx.x & 31) == 0) {
                    const PairKey old = pk_make(L.sbK[ro + j], j, L.sbP[ro + j] < 0 ? j : L.sbP[ro + j]);
                    const PairKey nc2 = pk_make(dbits(K), j, a);
                    if (L.sbK[ro + j] == RHSEG_KEY_NONE || pk_less(nc2, old)) { L.sbK[ro + j] = nc2.k; L.sbP[ro + j] = a; }
                }
            }
            __syncthreads();
        }
        fallbacks += 1;
        __syncthreads();
        return 0;
    }
    // exact keys of the candidates (row index r in the low bits -> slot)
    const uint32_t *cand = L.cand + (int64_t)sec * L.cand_cap * 2;
    unsigned long long *ck = L.ckey + (int64_t)sec * L.cand_cap;
    for (uint32_t q0 = 0; q0 < nc; q0 += PAIR_CAP) {
        const uint32_t cnt = min((uint32_t)PAIR_CAP, nc - q0);
        __syncthreads();
        for (uint32_t c = threadIdx.x; c < cnt; c += blockDim.x) {
            sm.pi[c] = crow_s[cand[2 * (q0 + c)] & 0xffu];
            sm.pj[c] = (int32_t)cand[2 * (q0 + c) + 1];
        }
        __syncthreads();
        block_keys(L, ro, sm.pi, sm.pj, sm.pkey, (int)cnt);
        __syncthreads();
        for (uint32_t c = threadIdx.x; c < cnt; c += blockDim.x) ck[q0 + c] = sm.pkey[c];
    }
    __syncthreads();
    // own minima: key, then slot pair
    for (uint32_t c = threadIdx.x; c < nc; c += blockDim.x)
        if (cand[2 * c] & 0x40000000u) atomicMin(&rK[cand[2 * c] & 0xffu], ck[c]);
    __syncthreads();
    if (threadIdx.x < nr && rK[threadIdx.x] != rU[threadIdx.x]) rTie[threadIdx.x] = ~0ull;
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < nc; c += blockDim.x) {
        const uint32_t w0 = cand[2 * c];
        const int r = (int)(w0 & 0xffu);
        if ((w0 & 0x40000000u) && ck[c] == rK[r]) atomicMin(&rTie[r], inc_pack_pair(crow_s[r], (int)cand[2 * c + 1]));
    }
    __syncthreads();
    if (threadIdx.x < nr) {
        const int r = threadIdx.x, s2 = crow_s[r];
        const unsigned long long p = rTie[r];
        L.sbK[ro + s2] = rK[r];
        if (rK[r] == RHSEG_KEY_NONE || p == ~0ull) {
            L.sbP[ro + s2] = -1;
        } else {
            const uint32_t lo = (uint32_t)(p >> 32), hi = (uint32_t)p;
            L.sbP[ro + s2] = (int32_t)(lo == (uint32_t)s2 ? hi : lo);
        }
    }
    __syncthreads();
    // pushes of the merged rows' keys, one merged row at a time (each
    // partner appears once per merged row)
    for (int r = 0; r < nprop; r++) {
        const int a = crow_s[r];
        for (uint32_t c = threadIdx.x; c < nc; c += blockDim.x) {
            const uint32_t w0 = cand[2 * c];
            if ((int)(w0 & 0xffu) != r || !(w0 & 0x80000000u)) continue;
            const int j = (int)cand[2 * c + 1];
            const uint64_t K = ck[c];
            const uint64_t oldK = L.sbK[ro + j];
            const int op = L.sbP[ro + j];
            const bool better = (oldK == RHSEG_KEY_NONE) ||
                                pk_less(pk_make(K, j, a), pk_make(oldK, j, op < 0 ? j : op));
            if (better) { L.sbK[ro + j] = K; L.sbP[ro + j] = a; }
        }
        __syncthreads();
    }
    return (long long)nc;
}

// Row update, step 1 (one block per section): the rows to recompute
// (merged survivors first, then the rows whose best was a merged slot) and
// the first chunk's row terms; the pending merges are consumed.
__global__ void __launch_bounds__(STEP_THREADS) k_srow_begin(LevelDev L)
{
    const int sec = blockIdx.x;
    if (sec >= L.nsec) return;
    __shared__ int32_t nR, nM;
    __shared__ SecState st;
    IncInfo *info = L.sinfo + sec;
    SecState *stg = &L.st[sec];
    if (threadIdx.x == 0) st = *stg;
    __syncthreads();
    if (st.done || st.npm == 0) {
        if (threadIdx.x == 0) {
            info->active = 0;
            if (st.npm != 0) stg->npm = 0;
        }
        return;
    }
    const int64_t ro = L.roff[sec], pb = L.poff[sec];
    const int m0 = st.m0;
    int32_t *R = L.srow + ro;
    if (threadIdx.x == 0) {
        int n = 0;
        for (int k = 0; k < st.npm; k++) {
            const int a = st.pm_a[k];
            if (!L.alive[ro + a] || L.inR[ro + a]) continue;
            L.inR[ro + a] = 1;
            R[n++] = a;
        }
        nM = n;
        nR = n;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < m0; j += blockDim.x) {
        if (!L.alive[ro + j] || L.inR[ro + j]) continue;
        const int bp = L.sbP[ro + j];
        bool hit = false;
        for (int k = 0; k < st.npm; k++) hit |= (bp == st.pm_a[k] || bp == st.pm_b[k]);
        if (!hit) continue;
        L.inR[ro + j] = 1;
        R[atomicAdd(&nR, 1)] = j;
    }
    __syncthreads();
    const int nrows = nR, nmerged = nM;
    const int ns = min(INC_RCAP, nrows);
    for (int r = threadIdx.x; r < INC_RCAP; r += blockDim.x) {
        if (r < ns) {
            const int s = R[r];
            const int p = L.pos_of_slot[ro + s];
            info->crow[r] = s;
            info->rAk[2 * r] = L.sE[pb + p];
            info->rAk[2 * r + 1] = L.sk[pb + p];
        } else {
            info->crow[r] = -1;
            info->rAk[2 * r] = 0.0f;
            info->rAk[2 * r + 1] = 1.0f;
        }
        info->apx[r] = ~0ull;
    }
    // the staged rows' vectors, per chunk of INC_RC rows [Bpad][INC_RC]
    float *xg = L.srowx + (int64_t)sec * L.Bpad * INC_RCAP;
    const int nchunk = (ns + INC_RC - 1) / INC_RC;
    for (int e = threadIdx.x; e < nchunk * L.Bpad * INC_RC; e += blockDim.x) {
        const int c = e / (L.Bpad * INC_RC), rem = e % (L.Bpad * INC_RC);
        const int b = rem / INC_RC, r = c * INC_RC + rem % INC_RC;
        float v = 0.0f;
        if (r < ns) v = ((const float *)L.X)[(pb + L.pos_of_slot[ro + R[r]]) * L.Bpad + b];
        xg[e] = v;
    }
    if (threadIdx.x == 0) {
        info->nrows = nrows;
        info->nmerged = nmerged;
        info->nstaged = ns;
        info->active = nrows > 0 ? 1 : 0;
        stg->npm = 0;
    }
}

// Row update, step 2: pass A of the first chunk, INC_SUM_BLOCKS blocks per
// section over slices of the positions.
__global__ void __launch_bounds__(STEP_THREADS) k_srow_sums(LevelDev L)
{
    const int sec = blockIdx.y;
    if (sec >= L.nsec) return;
    IncInfo *info = L.sinfo + sec;
    if (!info->active) return;
    __shared__ int32_t crow[INC_RC];
    __shared__ float rAk[2 * INC_RC];
    __shared__ unsigned long long apx[INC_RC];
    extern __shared__ float xs[];
    const int ns = info->nstaged;
    const int mc = L.st[sec].mc;
    const int per = (mc + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * per, hi = min(mc, lo + per);
    for (int c0 = 0; c0 < ns; c0 += INC_RC) {
        const int nr = min(INC_RC, ns - c0);
        __syncthreads();
        if (threadIdx.x < INC_RC) {
            crow[threadIdx.x] = info->crow[c0 + threadIdx.x];
            rAk[2 * threadIdx.x] = info->rAk[2 * (c0 + threadIdx.x)];
            rAk[2 * threadIdx.x + 1] = info->rAk[2 * (c0 + threadIdx.x) + 1];
            apx[threadIdx.x] = ~0ull;
        }
        const float *xg = L.srowx + ((int64_t)sec * INC_RCAP + c0) * L.Bpad;
        for (int e = threadIdx.x; e < L.Bpad * INC_RC; e += blockDim.x) xs[e] = xg[e];
        __syncthreads();
        switch (nr) {
        case 1: inc_pass_sums<1>(L, sec, crow, nr, xs, rAk, apx, lo, hi, c0); break;
        case 2: inc_pass_sums<2>(L, sec, crow, nr, xs, rAk, apx, lo, hi, c0); break;
        case 3: inc_pass_sums<3>(L, sec, crow, nr, xs, rAk, apx, lo, hi, c0); break;
        case 4: inc_pass_sums<4>(L, sec, crow, nr, xs, rAk, apx, lo, hi, c0); break;
        case 5: case 6: inc_pass_sums<6>(L, sec, crow, nr, xs, rAk, apx, lo, hi, c0); break;
        default: inc_pass_sums<8>(L, sec, crow, nr, xs, rAk, apx, lo, hi, c0); break;
        }
        __syncthreads();
        if (threadIdx.x < nr && apx[threadIdx.x] != ~0ull) atomicMin(&info->apx[c0 + threadIdx.x], apx[threadIdx.x]);
    }
}

// Row update, step 3 (one block per section): the first chunk's exact
// minima and pushes; further chunks (rows past INC_RC) in-block.
__global__ void __launch_bounds__(STEP_THREADS) k_srow_finish(LevelDev L)
{
    const int sec = blockIdx.x;
    if (sec >= L.nsec) return;
    __shared__ StepSmem sm;
    __shared__ int32_t crow[INC_RC];
    __shared__ float rAk[2 * INC_RC], rT[INC_RC];
    __shared__ unsigned long long apx[INC_RC], rK[INC_RC], rTie[INC_RC], rU[INC_RC];
    __shared__ uint32_t ncand_s;
    extern __shared__ float xs[];
    const IncInfo *info = L.sinfo + sec;
    if (!info->active) return;
    SecState *stg = &L.st[sec];
    const int64_t ro = L.roff[sec], pb = L.poff[sec];
    const int m0 = stg->m0;
    const int32_t *R = L.srow + ro;
    const int nrows = info->nrows, nmerged = info->nmerged;
    int64_t fallbacks = 0;
    long long keys = 0;
    for (int c0 = 0; c0 < nrows; c0 += INC_RC) {
        const int nr = min(INC_RC, nrows - c0);
        const int nprop = max(0, min(nr, nmerged - c0));
        __syncthreads();
        int sb_off = c0;
        if (c0 < info->nstaged) {
            if (threadIdx.x < INC_RC) {
                crow[threadIdx.x] = info->crow[c0 + threadIdx.x];
                rAk[2 * threadIdx.x] = info->rAk[2 * (c0 + threadIdx.x)];
                rAk[2 * threadIdx.x + 1] = info->rAk[2 * (c0 + threadIdx.x) + 1];
                apx[threadIdx.x] = info->apx[c0 + threadIdx.x];
            }
            __syncthreads();
        } else {
            sb_off = 0;                            // the staged chunks are finished: reuse their scratch
            // a further chunk: stage and pass A in this block
            if (threadIdx.x < INC_RC) {
                const int r = threadIdx.x;
                if (r < nr) {
                    const int s2 = R[c0 + r];
                    const int p = L.pos_of_slot[ro + s2];
                    crow[r] = s2;
                    rAk[2 * r] = L.sE[pb + p];
                    rAk[2 * r + 1] = L.sk[pb + p];
                } else {
                    crow[r] = -1;
                    rAk[2 * r] = 0.0f;
                    rAk[2 * r + 1] = 1.0f;
                }
                apx[r] = ~0ull;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < L.Bpad * INC_RC; e += blockDim.x) {
                const int b = e / INC_RC, r = e % INC_RC;
                float v = 0.0f;
                if (r < nr) v = ((const float *)L.X)[(pb + L.pos_of_slot[ro + crow[r]]) * L.Bpad + b];
                xs[b * INC_RC + r] = v;
            }
            __syncthreads();
            inc_pass_sums<8>(L, sec, crow, nr, xs, rAk, apx, 0, stg->mc, 0);
            __syncthreads();
        }
        const long long nc = inc_chunk_finish(L, sec, sm, m0, crow, nr, nprop, rAk, apx, rT, rK, rTie, rU, &ncand_s,
                                              fallbacks, sb_off);
        if (threadIdx.x == 0) keys += nc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nrows; k += blockDim.x) L.inR[ro + R[k]] = 0;
    if (threadIdx.x == 0) {
        stg->cands += keys;
        stg->fallbacks += fallbacks;
        stg->screened += (int64_t)nrows * stg->count;     // row x position evaluations of this update
        stg->cands_true += nrows;                         // rows recomputed
    }
}

// Step 3 of HSEG with incremental minima: the pair of minimum key over the
// per-row spectral bests, merged if below the threshold.
__global__ void __launch_bounds__(STEP_THREADS, 2) k_spec_inc(LevelDev L, ScreenConst sc)
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
    const double t = st.tthr;
    const uint64_t tbits = dbits(t);
    const int count = st.count;
    PairKey best = pk_none();
    for (int i = threadIdx.x; i < m0; i += blockDim.x) {
        if (!L.alive[ro + i]) continue;
        const uint64_t k = L.sbK[ro + i];
        if (k == RHSEG_KEY_NONE) continue;
        const PairKey c = pk_make(k, i, L.sbP[ro + i]);
        if (pk_less(c, best)) best = c;
    }
    best = block_min_pk(best, sm.pk);
    __syncthreads();
    if (threadIdx.x == 0) st.pairs += (int64_t)count * (count - 1) / 2 - st.nadj;
    int merged = 0;
    if (best.k != RHSEG_KEY_NONE && best.k < tbits) {      // K < t (non-negative binary64)
        const int a = (int)best.lo, b = (int)best.hi;
        block_merge<false>(L, sec, st, a, b, __longlong_as_double((long long)best.k), 1, sc, sm);
        merged = 1;
        if (threadIdx.x == 0) {
            st.pm_a[st.npm] = a;
            st.pm_b[st.npm] = b;
            st.npm += 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st.spec_pending = 0;
        if (!merged && !st.merged_adj) { st.stalled = 1; st.done = 1; }
        if (st.count <= st.target) st.done = 1;
    }
    __syncthreads();
    if (!st.done && (st.count + 127) / 128 < (st.mc + 127) / 128) block_compact_positions(L, sec, st);
    __syncthreads();
    if (threadIdx.x == 0) L.st[sec] = st;
}

}  // namespace rhseg
