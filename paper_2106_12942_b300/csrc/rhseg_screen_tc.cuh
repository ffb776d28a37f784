// rhseg_screen_tc.cuh -- spectral-step screen on the 5th-generation tensor
// cores (tcgen05, sm_103a).
//
// The all-pairs part of HSEG step 3 (Section 4.1; the thesis's "spectral
// kernel", Fig. 4.8, evaluates every region pair each iteration) is written
// as a dense contraction: for region-mean rows x_i (FP16 or BF16, relative
// to a per-section reference spectrum) the Gram block G = X_I X_J^T of two
// 128-row blocks is accumulated in FP32 in tensor memory, and the epilogue
// applies the separable test g_ij > h_i + h_j that keeps every pair whose
// exact key could be below the step's threshold (see warp_write_row for the
// error bound behind h).  The N^2 matrix is never stored: passing pairs are
// appended to the section's candidate list for the exact re-check.
//
// Roles (192 threads): warp 0 issues TMA loads of 128x32 operand boxes
// (64-byte swizzle, two per operand per stage, so K pads only to 32) into a
// 3-stage shared-memory ring; warp 1 owns the
// tensor memory (2 accumulators x 128 columns) and issues tcgen05.mma
// (M=128, N=128, K=16) from one thread; warps 2-5 read the accumulator with
// tcgen05.ld (32 lanes each) and run the test.  Persistent CTAs walk the
// upper-triangle tiles of every pending section.  Every mbarrier wait is
// bounded; a wait that gives up sets the device error word and all roles
// leave their loops, so the tensor memory is always released.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include "rhseg_screen_simt.cuh"

namespace rhseg {

constexpr int TC_TILE = 128;
constexpr int TC_KATOM = 32;                  // 16-bit elements per 64-byte swizzle row (one TMA box)
constexpr int TC_ATOM_BYTES = TC_TILE * TC_KATOM * 2;        // 8 KB: 128 rows x 64 bytes
constexpr int TC_ATOMS_PER_STAGE = 2;                        // K = 64 per pipeline stage
constexpr int TC_STAGES = 3;
constexpr int TC_STAGE_BYTES = 2 * TC_ATOMS_PER_STAGE * TC_ATOM_BYTES;   // A + B
constexpr int TC_THREADS = 192;
constexpr long long TC_WAIT_CYCLES = 4000000000ll;           // about 2 s at 2 GHz
struct TcShared {
    uint64_t full[TC_STAGES], empty[TC_STAGES];
    uint64_t tfull[2], tempty[2];
    uint32_t tmem_base;
    int abort;
    alignas(16) float hc[2][TC_TILE];
    long long pre[MAX_SECTIONS + 1];
};
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 + (int)((sizeof(TcShared) + 127) / 128 * 128);

// Barrier 1 over the 128 epilogue threads with an OR-reduction of `v`:
// every participant gets the same answer.
__device__ __forceinline__ bool epi_bar_or(bool v)
{
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred q, p;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)v)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when the CTA aborted or the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort, int32_t *err)
{
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            *abort = 1;
            if (err) atomicExch(err, 0x54435754);   // screen wait timed out
            return false;
        }
    }
    return true;
}

// L2 policy for the streamed operand rows: evicted before other lines, so
// that the streaming does not push the region tables of the step kernels
// out of L2 between iterations.
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                            uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
        "%3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows
// of 64 bytes in groups of 8 (512-byte stride between groups).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address
    d |= (uint64_t)1 << 16;                          // leading offset (unused with this swizzle)
    d |= (uint64_t)(512 >> 4) << 32;                 // stride offset between 8-row groups
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)4 << 61;                          // 64-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, A/B in FP16 (fmt 0)
// or BF16 (fmt 1), both K-major, M = N = 128.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_TILE >> 3) << 17) | ((uint32_t)(TC_TILE >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Tile enumeration shared by all roles.  Screen mode: upper-triangle tiles
// of every section with a pending spectral step and a finite threshold.
// Gram mode (diagnostic): every (I, J) tile of one block of `gram_rows`.
struct TcJob {
    int gram_rows;            // > 0: Gram mode
    float *gram_out;          // [gram_rows][gram_rows]
};

__device__ __forceinline__ bool tc_tile(const LevelDev &L, const TcJob &job, const long long *pre, long long t,
                                        long long total, int &sec, int &I, int &J, int64_t &rowA, int64_t &rowB)
{
    if (t >= total) return false;
    if (job.gram_rows > 0) {
        int nb = job.gram_rows / TC_TILE;
        sec = 0;
        I = (int)(t / nb);
        J = (int)(t % nb);
        rowA = (int64_t)I * TC_TILE;
        rowB = (int64_t)J * TC_TILE;
        return true;
    }
    sec = find_section(pre, L.nsec, t);
    int mc = L.st[sec].mc;
    long long nb = (mc + TC_TILE - 1) / TC_TILE;
    tri_decode(t - pre[sec], nb, I, J);
    rowA = L.poff[sec] + (int64_t)I * TC_TILE;
    rowB = L.poff[sec] + (int64_t)J * TC_TILE;
    return true;
}

// tc_tile computed by lane 0 and broadcast to the warp.
__device__ __forceinline__ bool tc_tile_warp(const LevelDev &L, const TcJob &job, const long long *pre, long long t,
                                             long long total, int &sec, int &I, int &J, int64_t &rowA, int64_t &rowB)
{
    int have = 0;
    if ((threadIdx.x & 31) == 0) have = tc_tile(L, job, pre, t, total, sec, I, J, rowA, rowB) ? 1 : 0;
    have = __shfl_sync(0xffffffffu, have, 0);
    sec = __shfl_sync(0xffffffffu, sec, 0);
    I = __shfl_sync(0xffffffffu, I, 0);
    J = __shfl_sync(0xffffffffu, J, 0);
    rowA = __shfl_sync(0xffffffffu, rowA, 0);
    rowB = __shfl_sync(0xffffffffu, rowB, 0);
    return have != 0;
}

template <int FMT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_screen_tc(LevelDev L, const __grid_constant__ CUtensorMap tmap,
                                                             TcJob job)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *ring = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcShared &sh = *(TcShared *)(ring + TC_STAGES * TC_STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int natoms = L.Bpad / TC_KATOM;                       // 32-element K atoms
    const int nk = (natoms + TC_ATOMS_PER_STAGE - 1) / TC_ATOMS_PER_STAGE;   // pipeline stages per tile

    long long total;
    if (job.gram_rows > 0) {
        long long nb = job.gram_rows / TC_TILE;
        total = nb * nb;
    } else {
        block_tile_prefix(L, TC_TILE, sh.pre);
        total = sh.pre[L.nsec];
    }
    if (blockIdx.x >= total) return;     // uniform: this CTA has no tile

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; s++) { mbar_init(&sh.full[s], 1); mbar_init(&sh.empty[s], 1); }
        for (int b = 0; b < 2; b++) { mbar_init(&sh.tfull[b], 1); mbar_init(&sh.tempty[b], 4 * 32); }
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sh.tmem_base;
    volatile int *abort = &sh.abort;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            const uint64_t pol = l2_evict_first_policy();
            for (long long t = blockIdx.x; !*abort; t += gridDim.x) {
                int sec, I, J;
                int64_t rowA, rowB;
                if (!tc_tile(L, job, sh.pre, t, total, sec, I, J, rowA, rowB)) break;
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_wait(&sh.empty[stage], phase ^ 1, abort, L.err)) break;
                    uint8_t *a = ring + stage * TC_STAGE_BYTES;                  // A atoms, then B atoms
                    uint8_t *b = a + TC_ATOMS_PER_STAGE * TC_ATOM_BYTES;
                    const int na = min(TC_ATOMS_PER_STAGE, natoms - kc * TC_ATOMS_PER_STAGE);
                    mbar_expect_tx(&sh.full[stage], (uint32_t)(2 * na * TC_ATOM_BYTES));
                    for (int u = 0; u < na; u++) {
                        const int x = (kc * TC_ATOMS_PER_STAGE + u) * TC_KATOM;
                        tma_load_2d(a + u * TC_ATOM_BYTES, &tmap, x, (int)rowA, &sh.full[stage], pol);
                        tma_load_2d(b + u * TC_ATOM_BYTES, &tmap, x, (int)rowB, &sh.full[stage], pol);
                    }
                    if (++stage == TC_STAGES) { stage = 0; phase ^= 1; }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(FMT);
            int stage = 0;
            uint32_t phase = 0;
            int tcount = 0;
            for (long long t = blockIdx.x; !*abort; t += gridDim.x, tcount++) {
                int sec, I, J;
                int64_t rowA, rowB;
                if (!tc_tile(L, job, sh.pre, t, total, sec, I, J, rowA, rowB)) break;
                int buf = tcount & 1;
                if (!mbar_wait(&sh.tempty[buf], ((tcount >> 1) & 1) ^ 1, abort, L.err)) break;
                tc_fence_after();
                uint32_t dt = tbase + (uint32_t)(buf * TC_TILE);
                bool ok = true;
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_wait(&sh.full[stage], phase, abort, L.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a = smem_u32(ring + stage * TC_STAGE_BYTES);
                    const uint32_t b = a + TC_ATOMS_PER_STAGE * TC_ATOM_BYTES;
                    const int na = min(TC_ATOMS_PER_STAGE, natoms - kc * TC_ATOMS_PER_STAGE);
                    for (int u = 0; u < na; u++) {
                        const uint64_t ad = sdesc_sw64(a + u * TC_ATOM_BYTES), bd = sdesc_sw64(b + u * TC_ATOM_BYTES);
#pragma unroll
                        for (int k = 0; k < TC_KATOM / 16; k++)
                            tc_mma(dt, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                                   (kc > 0 || u > 0 || k > 0) ? 1u : 0u);
                    }
                    tc_commit(&sh.empty[stage]);
                    if (++stage == TC_STAGES) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                tc_commit(&sh.tfull[buf]);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 2..5 ----------------
        // Each thread owns one accumulator row (TMEM lane).  The per-row
        // terms h of the next tile are fetched while the current tile is
        // tested; the test runs as max_j (g_ij - h_j) > h_i over 32 columns
        // and only a passing chunk is examined element by element.
        const int q = warp & 3;                     // tensor-memory lane quarter of this warp
        const int row = q * 32 + lane;              // accumulator row = TMEM lane
        const int et = threadIdx.x - 64;            // 0..127, column index for h
        const float inf = __int_as_float(0x7f800000);
        int tcount = 0;
        float hc_next = inf, hr_next = inf;
        {
            int sec = 0, I = 0, J = 0;
            int64_t rowA = 0, rowB = 0;
            if (tc_tile_warp(L, job, sh.pre, blockIdx.x, total, sec, I, J, rowA, rowB) && job.gram_rows == 0) {
                hc_next = L.H[rowB + et];
                hr_next = L.H[rowA + row];
            }
        }
        for (long long t = blockIdx.x;; t += gridDim.x, tcount++) {
            int sec = 0, I = 0, J = 0;
            int64_t rowA = 0, rowB = 0;
            bool have = tc_tile_warp(L, job, sh.pre, t, total, sec, I, J, rowA, rowB);
            if (epi_bar_or(!have || *abort)) break;          // uniform over the 128 threads
            const int buf = tcount & 1;
            sh.hc[buf][et] = hc_next;
            const float hr = hr_next;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (job.gram_rows == 0) {
                int s2 = 0, I2 = 0, J2 = 0;
                int64_t rA2 = 0, rB2 = 0;
                if (tc_tile_warp(L, job, sh.pre, t + gridDim.x, total, s2, I2, J2, rA2, rB2)) {
                    hc_next = L.H[rB2 + et];
                    hr_next = L.H[rA2 + row];
                }
            }
            bool ok = mbar_wait(&sh.tfull[buf], (tcount >> 1) & 1, abort, L.err);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) continue;                               // the next loop top stops every warp
            tc_fence_after();
            const uint32_t taddr = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TC_TILE);
            const bool diag = (I == J);
            const float *hcs = sh.hc[buf];
            SecState *st = (job.gram_rows == 0) ? &L.st[sec] : nullptr;
            // two halves of 64 columns: two loads, one wait each; the
            // accumulator is released once the second half is in registers
            for (int h = 0; h < 2; h++) {
                uint32_t r[64];
                tmem_ld32_nowait(taddr + (uint32_t)(h * 64), r);
                tmem_ld32_nowait(taddr + (uint32_t)(h * 64 + 32), r + 32);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (h == 1) {
                    tc_fence_before();
                    mbar_arrive(&sh.tempty[buf]);
                }
                if (job.gram_rows > 0) {
                    float *o = job.gram_out + ((int64_t)I * TC_TILE + row) * job.gram_rows + (int64_t)J * TC_TILE + h * 64;
#pragma unroll
                    for (int c = 0; c < 64; c++) o[c] = __uint_as_float(r[c]);
                    continue;
                }
#pragma unroll
                for (int c0 = 0; c0 < 64; c0 += 32) {
                    float m = -inf;
#pragma unroll
                    for (int c = 0; c < 32; c++) m = fmaxf(m, __uint_as_float(r[c0 + c]) - hcs[h * 64 + c0 + c]);
                    if (m > hr) {
                        for (int c = 0; c < 32; c++) {
                            const int cc = h * 64 + c0 + c;
                            if (!(__uint_as_float(r[c0 + c]) - hcs[cc] > hr)) continue;
                            if (diag && cc <= row) continue;
                            uint32_t idx = atomicAdd(&st->ncand, 1u);
                            if ((int64_t)idx < L.cand_cap) {
                                uint32_t *cd = L.cand + ((int64_t)sec * L.cand_cap + idx) * 2;
                                cd[0] = (uint32_t)(I * TC_TILE + row);
                                cd[1] = (uint32_t)(J * TC_TILE + cc);
                            }
                        }
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(256) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Host side: tensor map over the operand rows and the launch.
// ---------------------------------------------------------------------------

typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline PFN_encodeTiled get_encode_tiled()
{
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

// Tensor map over X [rows][Bpad] of 16-bit elements, box 128 rows x 32.
inline int make_operand_map(CUtensorMap *map, const void *X, int64_t rows, int Bpad, int precision)
{
    PFN_encodeTiled enc = get_encode_tiled();
    if (!enc) return -1;
    if (((uintptr_t)X & 15) || (Bpad % TC_KATOM) != 0 || rows <= 0) return -2;
    cuuint64_t gdim[2] = {(cuuint64_t)Bpad, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)Bpad * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_KATOM, (cuuint32_t)TC_TILE};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, precision == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                     const_cast<void *>(X), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -3;
}

inline bool screen_uses_tcgen05(int precision) { return precision == 1 || precision == 2; }

// Launch the screen for a level.  `map` must describe L.X.
inline cudaError_t launch_screen_tc_map(const LevelDev &L, const CUtensorMap &map, int precision, int n_sm,
                                        cudaStream_t s, TcJob job)
{
    static bool attr_done[2] = {false, false};
    int fi = precision == 2 ? 1 : 0;
    if (!attr_done[fi]) {
        cudaError_t e = (precision == 2)
                            ? cudaFuncSetAttribute(k_screen_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   TC_SMEM_BYTES)
                            : cudaFuncSetAttribute(k_screen_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   TC_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_done[fi] = true;
    }
    // two persistent CTAs per SM (shared memory 106 KB, tensor memory 256 columns each)
    if (precision == 2) k_screen_tc<1><<<2 * n_sm, TC_THREADS, TC_SMEM_BYTES, s>>>(L, map, job);
    else k_screen_tc<0><<<2 * n_sm, TC_THREADS, TC_SMEM_BYTES, s>>>(L, map, job);
    return cudaGetLastError();
}

}  // namespace rhseg
