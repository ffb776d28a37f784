// rhseg_screen_simt.cuh -- spectral-step screen on CUDA cores (FP64 or FP32).
//
// For every unordered pair of compact positions (i < j) of every section
// with a pending spectral step, the Gram entry g_ij = <x_i, x_j> of the
// region-mean rows is accumulated and the separable test
//      g_ij > h_i + h_j,   h_i = (A_i - T k_i) / 2
// passes the pair to the exact re-check.  With A_i and k_i built as in
// warp_write_row this test keeps every pair with K_ij < T (no false
// negatives), where K_ij = n_i n_j / (n_i + n_j) ||mu_i - mu_j||^2 (Eq. 1).
#pragma once
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include "rhseg_kernels.cuh"

namespace rhseg {

constexpr int SIMT_TILE = 64;
constexpr int SIMT_KC = 16;
constexpr int MAX_SECTIONS = 1024;

// Work units of the tensor-core screen for a section of mc positions:
// 128-row blocks I against 256-row blocks Jp with 2*Jp + 1 >= I, i.e. the
// two 128-row halves of every upper-triangle tile of 256-row blocks, less
// the half past the last row block when the number of 128-row blocks is odd.
__host__ __device__ __forceinline__ long long tc_section_units(long long mc)
{
    const long long nb = (mc + 127) / 128, nbp = (nb + 1) / 2;
    return nbp * (nbp + 1) - (nb & 1);
}

// Exclusive prefix over sections of the number of upper-triangle tiles of
// each pending section (tile edge `tile`; tile == 0 counts the tensor-core
// screen's units instead; tile < 0 counts tiles of edge -tile of every
// section still running).  Whole block; result in pre[0..nsec].
__device__ void block_tile_prefix(const LevelDev &L, int tile, long long *pre)
{
    int nsec = L.nsec;
    int per = (nsec + blockDim.x - 1) / blockDim.x;      // <= 16 (nsec <= 1024, >= 64 threads)
    int s0 = threadIdx.x * per;
    long long cnt[16];
    long long loc = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        int s = s0 + k;
        long long t = 0;
        if (k < per && s < nsec) {
            const SecState &st = L.st[s];
            if (tile < 0) {
                if (!st.done) {
                    long long nb = (st.mc + (-tile) - 1) / (-tile);
                    t = nb * (nb + 1) / 2;
                }
            } else if (st.spec_pending && st.tthr < __longlong_as_double(0x7FF0000000000000ll)) {
                if (tile == 0) {
                    t = (L.ulist != nullptr) ? st.nunits : tc_section_units(st.mc);
                } else {
                    long long nb = (st.mc + tile - 1) / tile;
                    t = nb * (nb + 1) / 2;
                }
            }
        }
        cnt[k] = t;
        loc += t;
    }
    __shared__ long long wsum[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    __syncthreads();
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    long long woff = 0, tot = 0;
    for (int k = 0; k < nw; k++) { if (k < wid) woff += wsum[k]; tot += wsum[k]; }
    long long run = woff + incl - loc;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        int s = s0 + k;
        if (k < per && s < nsec) { pre[s] = run; run += cnt[k]; }
    }
    if (threadIdx.x == 0) pre[nsec] = tot;
    __syncthreads();
}

__device__ __forceinline__ int find_section(const long long *pre, int nsec, long long t)
{
    int lo = 0, hi = nsec;       // pre[lo] <= t < pre[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename TA> __device__ __forceinline__ TA cvt_acc(double v) { return (TA)v; }
template <typename TA> __device__ __forceinline__ TA cvt_acc(float v) { return (TA)v; }
template <typename TA> __device__ __forceinline__ TA cvt_acc(__half v) { return (TA)__half2float(v); }
template <typename TA> __device__ __forceinline__ TA cvt_acc(__nv_bfloat16 v) { return (TA)__bfloat162float(v); }

// TS: operand storage type, T: accumulation type (products of TS values are
// exact in T for the half/bf16 -> float and float -> float, double -> double
// pairs used here except float x float, whose rounding is in the bound).
template <typename TS, typename T>
__global__ void __launch_bounds__(256) k_screen_simt(LevelDev L)
{
    __shared__ long long pre[MAX_SECTIONS + 1];
    __shared__ T As[SIMT_KC][SIMT_TILE + 1];
    __shared__ T Bsm[SIMT_KC][SIMT_TILE + 1];
    __shared__ T hr[SIMT_TILE], hc[SIMT_TILE];
    block_tile_prefix(L, SIMT_TILE, pre);
    long long total = pre[L.nsec];
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        int sec = find_section(pre, L.nsec, t);
        SecState *st = &L.st[sec];
        int mc = st->mc;
        long long nb = (mc + SIMT_TILE - 1) / SIMT_TILE;
        int I, J;
        tri_decode(t - pre[sec], nb, I, J);
        int64_t pb = L.poff[sec];
        const TS *X = (const TS *)L.X;
        const TS *XA = X + (pb + (int64_t)I * SIMT_TILE) * L.Bpad;
        const TS *XB = X + (pb + (int64_t)J * SIMT_TILE) * L.Bpad;
        double tthr = st->tthr;
        __syncthreads();
        if (threadIdx.x < 2 * SIMT_TILE) {
            int r = threadIdx.x & (SIMT_TILE - 1);
            int pos = (threadIdx.x < SIMT_TILE ? I : J) * SIMT_TILE + r;
            T h;
            if (pos < mc) {
                if (sizeof(T) == 8) {
                    double A = L.Ad[pb + pos], k = L.kd[pb + pos];
                    h = (T)(0.5 * (A - tthr * k));
                } else {
                    float Tf = __double2float_ru(tthr);
                    float A = L.Af[pb + pos], k = L.kf[pb + pos];
                    h = (T)(0.5f * (A - Tf * k));
                }
            } else {
                h = (T)__longlong_as_double(0x7FF0000000000000ll);
            }
            if (threadIdx.x < SIMT_TILE) hr[r] = h; else hc[r] = h;
        }
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[a][c] = (T)0;
        for (int k0 = 0; k0 < L.Bpad; k0 += SIMT_KC) {
            __syncthreads();
            for (int e = threadIdx.x; e < SIMT_TILE * SIMT_KC; e += blockDim.x) {
                int r = e / SIMT_KC, k = e % SIMT_KC;
                As[k][r] = cvt_acc<T>(XA[(int64_t)r * L.Bpad + k0 + k]);
                Bsm[k][r] = cvt_acc<T>(XB[(int64_t)r * L.Bpad + k0 + k]);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < SIMT_KC; k++) {
                T av[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; a++) av[a] = As[k][ty * 4 + a];
#pragma unroll
                for (int c = 0; c < 4; c++) bv[c] = Bsm[k][tx * 4 + c];
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
            }
        }
        // epilogue: separable threshold test, emission of candidates
#pragma unroll
        for (int a = 0; a < 4; a++) {
            int li = ty * 4 + a;
            int i = I * SIMT_TILE + li;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                int lj = tx * 4 + c;
                int j = J * SIMT_TILE + lj;
                if (i < j && j < mc && acc[a][c] > hr[li] + hc[lj]) {
                    uint32_t idx = atomicAdd(&st->ncand, 1u);
                    if ((int64_t)idx < L.cand_cap) {
                        uint32_t *cd = L.cand + ((int64_t)sec * L.cand_cap + idx) * 2;
                        cd[0] = (uint32_t)i;
                        cd[1] = (uint32_t)j;
                    }
                }
            }
        }
    }
}

}  // namespace rhseg
