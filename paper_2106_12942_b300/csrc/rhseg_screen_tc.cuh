// rhseg_screen_tc.cuh -- spectral-step screen on the 5th-generation tensor
// cores (tcgen05, sm_103a).
//
// The all-pairs part of HSEG step 3 (Section 4.1; the thesis's "spectral
// kernel", Fig. 4.8, evaluates every region pair each iteration) is written
// as a dense contraction: for region-mean rows x_i (FP16 or BF16, relative
// to a per-section reference spectrum) the Gram block G = X_I X_J^T of a
// 128-row block I against a 256-row block Jp is accumulated in FP32 in
// tensor memory, and the epilogue applies the separable test
// g_ij > h_i + h_j that keeps every pair whose exact key could be below the
// step's threshold (see warp_write_row for the error bound behind h).  The
// N^2 matrix is never stored: passing pairs are appended to the section's
// candidate list for the exact re-check.
//
// Roles (416 threads, one CTA per SM): warps 0-3 issue TMA loads of one
// 32-element K slice per pipeline stage (a 128x32 box of A, two of B;
// 64-byte swizzle, so K pads only to 32) into an 8-stage shared-memory ring
// (192 KB in flight; one TMA-issuing thread per SM delivers only a fraction
// of what four do); warp 4 owns the tensor memory (2 accumulators x 256
// columns) and issues tcgen05.mma (M=128, N=256, K=16) from one thread,
// committing once per group of K slices (each commit costs the tensor pipe
// about one MMA); warps 5-12 read the accumulator with tcgen05.ld (two
// warps per 32-lane quarter, 128 columns each) and run the test.  An
// M=128 MMA costs the tensor pipe about the same time for N=128 as for
// N=256, so the 128x256 unit doubles the work per instruction.  Persistent
// CTAs walk the units each section lists for the step (units whose
// certified norm ranges prove every pair's key above the threshold are not
// listed, see block_unit_list).  Every mbarrier wait is bounded; a wait that
// gives up sets the device error word and all roles leave their loops, so
// the tensor memory is always released.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include "rhseg_screen_simt.cuh"

namespace rhseg {

constexpr int TC_TILE = 128;                  // rows of an A block (M)
constexpr int TC_N = 256;                     // rows of a B block (N)
constexpr int TC_KATOM = 32;                  // 16-bit elements per 64-byte swizzle row (one TMA box)
constexpr int TC_A_BYTES = TC_TILE * TC_KATOM * 2;           // 8 KB: 128 rows x 64 bytes
constexpr int TC_B_BYTES = TC_N * TC_KATOM * 2;              // 16 KB: 256 rows x 64 bytes
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;      // one K slice of 32
constexpr int TC_STAGES = 8;
constexpr int TC_GROUP = 4;                   // K slices per tcgen05.commit (a commit costs ~1 MMA of pipe time)
constexpr int TC_PROD_WARPS = 4;              // TMA issuing warps (one thread each; TMA rate grows with issuers)
constexpr int TC_NGBAR = 32;                  // group-completion barriers, used round-robin
constexpr int TC_NDESC = 16;                  // unit descriptors published ahead by the producer
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_MMA_WARP = TC_PROD_WARPS;
constexpr int TC_EPI_WARP0 = TC_PROD_WARPS + 1;
constexpr int TC_THREADS = 32 * (TC_PROD_WARPS + 1 + TC_EPI_WARPS);
static_assert(TC_STAGES % TC_PROD_WARPS == 0, "each producer owns whole ring slots");
static_assert((TC_STAGES & (TC_STAGES - 1)) == 0, "ring slot by mask");
constexpr uint32_t TC_TMEM_COLS = 2 * TC_N;
constexpr long long TC_WAIT_CYCLES = 4000000000ll;           // default wait bound: about 2 s at 2 GHz

// One work unit: rows [rowA, rowA + 128) against rows [rowB, rowB + 256).
struct TcUnit {
    int sec, I, Jp, pad;
    int64_t rowA, rowB;
};

struct TcShared {
    uint64_t full[TC_STAGES];                 // K slice landed (TMA transaction count)
    uint64_t gbar[TC_NGBAR];                  // MMAs of a group of K slices complete
    uint64_t tempty[2];                       // accumulator buffer read out by the epilogue
    uint64_t dfull[TC_NDESC], dempty[TC_NDESC];
    uint64_t drain;                           // MMAs of an aborted launch complete
    uint32_t tmem_base;
    int abort;
    long long slot_q[TC_STAGES];              // producer only: group that last read each ring slot
    int slot_fills[TC_STAGES];                // producer only: loads issued into each ring slot
    TcUnit desc[TC_NDESC];
    alignas(16) float hc[2][TC_N];
    long long pre[MAX_SECTIONS + 1];
    int smc[MAX_SECTIONS];                    // per section: positions this step
    int spoff[MAX_SECTIONS];                  // per section: first operand row
};
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 + (int)((sizeof(TcShared) + 127) / 128 * 128);
static_assert(TC_SMEM_BYTES <= 227 * 1024, "screen shared memory");
static_assert(TC_SMEM_BYTES > 227 * 1024 / 2, "one CTA per SM: the tensor memory is allocated whole");

// Barrier 1 over the epilogue threads with an OR-reduction of `v`: every
// participant gets the same answer.
__device__ __forceinline__ bool epi_bar_or(bool v)
{
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred q, p;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, 256, q;\n\t"
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
// Bounded wait of the pipeline (at most `cycles` clock cycles): false when
// the CTA aborted or the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort, int32_t *err,
                                          long long cycles)
{
    if (mbar_try_wait(bar, parity)) return true;     // the usual case: no clock read
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > cycles) {
            *abort = 1;
            if (err) atomicExch(err, 0x54435754);   // screen wait timed out
            return false;
        }
    }
    return true;
}

// Bounded wait that ignores the abort flag: used only to let this CTA's own
// TMA copies land, and its own MMAs complete, before it exits (always the
// default bound: these always finish, and the CTA must not leave before).
__device__ __forceinline__ void mbar_wait_landed(uint64_t *bar, uint32_t parity, int32_t *err)
{
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            if (err) atomicExch(err, 0x54434c44);   // copies still in flight at exit
            return;
        }
    }
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
// or BF16 (fmt 1), both K-major, M = 128, N = 256.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_TILE >> 4) << 24);
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

// Three-input maximum and a packed pair difference (both exact IEEE
// operations: max, and subtraction rounded to nearest, lane by lane).
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ void sub2f(float a0, float a1, float b0, float b1, float &d0, float &d1)
{
    asm("{\n\t.reg .b64 a, b, d;\n\t"
        "mov.b64 a, {%2, %3};\n\t"
        "mov.b64 b, {%4, %5};\n\t"
        "sub.rn.f32x2 d, a, b;\n\t"
        "mov.b64 {%0, %1}, d;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// Separable test of 64 accumulator columns of one thread's row (half h of
// its 128 columns of block J): max_j (g_ij - h_j) > h_i over 32 columns at a
// time (packed differences, 3-input maxima); only a passing chunk is
// examined element by element, and its passing pairs (upper triangle only
// on a diagonal block) are appended to the section's candidate list with
// their tested value g - h_j.
__device__ __forceinline__ void screen_test_64(const LevelDev &L, SecState *st, int sec, int I, int J, int row,
                                               bool diag, int h, const uint32_t (&r)[64], const float *hcs, float hr)
{
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
        const float4 *h4 = (const float4 *)(hcs + h * 64 + c0);
        float d[32];
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
            const float4 hv = h4[c / 4];
            sub2f(__uint_as_float(r[c0 + c]), __uint_as_float(r[c0 + c + 1]), hv.x, hv.y, d[c], d[c + 1]);
            sub2f(__uint_as_float(r[c0 + c + 2]), __uint_as_float(r[c0 + c + 3]), hv.z, hv.w, d[c + 2], d[c + 3]);
        }
        if (diag) {
            // on a diagonal block only the upper triangle holds pairs: the
            // self pair (which always passes) and the lower triangle are
            // masked before the test, so their chunks take the fast path
#pragma unroll
            for (int c = 0; c < 32; c++)
                if (h * 64 + c0 + c <= row) d[c] = -__int_as_float(0x7f800000);
        }
        float m0 = max3f(d[0], d[1], d[2]), m1 = max3f(d[3], d[4], d[5]);
        m0 = max3f(m0, d[6], d[7]);   m1 = max3f(m1, d[8], d[9]);
        m0 = max3f(m0, d[10], d[11]); m1 = max3f(m1, d[12], d[13]);
        m0 = max3f(m0, d[14], d[15]); m1 = max3f(m1, d[16], d[17]);
        m0 = max3f(m0, d[18], d[19]); m1 = max3f(m1, d[20], d[21]);
        m0 = max3f(m0, d[22], d[23]); m1 = max3f(m1, d[24], d[25]);
        m0 = max3f(m0, d[26], d[27]); m1 = max3f(m1, d[28], d[29]);
        const float m = max3f(m0, m1, fmaxf(d[30], d[31]));
        if (m > hr) {
            for (int c = 0; c < 32; c++) {
                const int cc = h * 64 + c0 + c;
                if (!(d[c] > hr)) continue;
                uint32_t idx = atomicAdd(&st->ncand, 1u);
                if ((int64_t)idx < L.cand_cap) {
                    uint32_t *cd = L.cand + ((int64_t)sec * L.cand_cap + idx) * 2;
                    cd[0] = (uint32_t)(I * TC_TILE + row);
                    cd[1] = (uint32_t)(J * TC_TILE + cc);
                    // g - h_j as tested (the re-check adds h_j back for the error report;
                    // storing g itself would keep all 64 accumulator registers live here)
                    if (L.candg != nullptr) L.candg[(int64_t)sec * L.cand_cap + idx] = d[c];
                }
            }
        }
    }
}

// Work-unit enumeration shared by all roles.  Screen mode: the units of
// every section with a pending spectral step and a finite threshold (see
// tc_section_units; unit u of a section is half u & 1 of upper-triangle
// tile u >> 1 of its 256-row blocks).  Gram mode (diagnostic): every
// (I, Jp) unit of one block of `gram_rows`.
struct TcJob {
    int gram_rows;            // > 0: Gram mode
    float *gram_out;          // [gram_rows][gram_rows]
};

// Unit t of this launch.  `cursor` is the section of the caller's previous
// unit (units are visited in increasing order, so the section only moves
// forward); the per-section data come from shared memory.
__device__ __forceinline__ bool tc_unit(const TcShared &sh, const TcJob &job, long long t, long long total, int &cursor,
                                        TcUnit &u, const int32_t *L_ulist = nullptr, int L_ucap = 0)
{
    if (t >= total) return false;
    if (job.gram_rows > 0) {
        const int nbp = (job.gram_rows + TC_N - 1) / TC_N;
        u.sec = 0;
        u.I = (int)(t / nbp);
        u.Jp = (int)(t % nbp);
        u.rowA = (int64_t)u.I * TC_TILE;
        u.rowB = (int64_t)u.Jp * TC_N;
        return true;
    }
    int s = cursor;
    while (sh.pre[s + 1] <= t) s++;
    cursor = s;
    u.sec = s;
    const long long local = t - sh.pre[s];
    if (L_ulist != nullptr) {                    // the step's kept units, listed per section
        const int32_t e = L_ulist[(int64_t)s * L_ucap + local];
        u.I = e >> 16;
        u.Jp = e & 0xffff;
    } else {
        const long long nb = (sh.smc[s] + TC_TILE - 1) / TC_TILE, nbp = (nb + 1) / 2;
        int Ip;
        tri_decode(local >> 1, nbp, Ip, u.Jp);
        u.I = 2 * Ip + (int)(local & 1);
    }
    u.rowA = sh.spoff[s] + (int64_t)u.I * TC_TILE;
    u.rowB = sh.spoff[s] + (int64_t)u.Jp * TC_N;
    return true;
}

template <int FMT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_screen_tc(LevelDev L, const __grid_constant__ CUtensorMap tmap,
                                                             TcJob job)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *ring = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcShared &sh = *(TcShared *)(ring + TC_STAGES * TC_STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int natoms = L.Bpad / TC_KATOM;                       // K slices (pipeline stages) per unit
    const long long wc = L.wait_cycles > 0 ? L.wait_cycles : TC_WAIT_CYCLES;   // bound of every pipeline wait

    long long total;
    if (job.gram_rows > 0) {
        total = (long long)(job.gram_rows / TC_TILE) * ((job.gram_rows + TC_N - 1) / TC_N);
    } else {
        block_tile_prefix(L, 0, sh.pre);
        total = sh.pre[L.nsec];
    }
    if (blockIdx.x >= total) return;     // uniform: this CTA has no unit
    const long long my_units = (total - blockIdx.x + gridDim.x - 1) / gridDim.x;
    int cursor0 = 0;
    if (job.gram_rows == 0) {
        for (int s = threadIdx.x; s < L.nsec; s += blockDim.x) {
            sh.smc[s] = L.st[s].mc;
            sh.spoff[s] = (int)L.poff[s];
        }
        cursor0 = find_section(sh.pre, L.nsec, blockIdx.x);
    }

    // K slices per commit: TC_GROUP, widened for very wide rows so that a
    // unit never spans more than 16 groups (the group barriers are reused
    // after TC_NGBAR groups; the epilogue trails the MMAs by at most one unit).
    // This form keeps the grouping fixed: taking the tuned L.tc_group here
    // (same value, 4) made the screen 12 % slower as compiled.
    const int G = max(TC_GROUP, (natoms + 15) / 16);
    const int gpu = (natoms + G - 1) / G;                    // groups per unit
    if (G > TC_STAGES) {                 // a group must fit the ring (rows of at most 4096 elements)
        if (threadIdx.x == 0 && L.err) atomicExch(L.err, 0x54434752);
        return;                          // uniform: before any barrier or tensor-memory use
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; s++) { mbar_init(&sh.full[s], 1); sh.slot_q[s] = -1; sh.slot_fills[s] = 0; }
        for (int g = 0; g < TC_NGBAR; g++) mbar_init(&sh.gbar[g], 1);
        for (int b = 0; b < 2; b++) mbar_init(&sh.tempty[b], TC_EPI_WARPS);
        for (int d = 0; d < TC_NDESC; d++) { mbar_init(&sh.dfull[d], 1); mbar_init(&sh.dempty[d], TC_EPI_WARPS); }
        mbar_init(&sh.drain, 1);
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == TC_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sh.tmem_base;
    volatile int *abort = &sh.abort;

    if (warp < TC_PROD_WARPS) {
        // ---------------- producers: unit decode + TMA ----------------
        // Producer p streams the K slices c = p, p + 4, ... of this CTA's
        // sequence (slot c mod 8, so each producer owns two ring slots); the
        // producer of a unit's first slice publishes the unit's descriptor
        // for the epilogue.  A slot is refilled once the commit group that
        // read it has completed.
        if (lane == 0) {
            const int p = warp;
            const uint64_t pol = l2_evict_first_policy();
            int cursor = cursor0;
            long long kdec = -1;
            TcUnit u{};
            const long long nslices = my_units * natoms;
            long long k = p / natoms;                        // unit and K slice of slice c
            int kc = p - (int)k * natoms;
            for (long long c = p; c < nslices && !*abort; c += TC_PROD_WARPS) {
                const int slot = (int)(c & (TC_STAGES - 1));
                if (k != kdec) {
                    tc_unit(sh, job, blockIdx.x + k * gridDim.x, total, cursor, u, job.gram_rows > 0 ? nullptr : L.ulist,
                            L.ucap);
                    kdec = k;
                }
                if (kc == 0) {
                    const int ds = (int)(k % TC_NDESC);
                    if (k >= TC_NDESC && !mbar_wait(&sh.dempty[ds], (uint32_t)((k / TC_NDESC - 1) & 1), abort, L.err, wc))
                        break;
                    sh.desc[ds] = u;
                    mbar_arrive(&sh.dfull[ds]);
                }
                const long long qo = sh.slot_q[slot];
                if (qo >= 0 && !mbar_wait(&sh.gbar[qo % TC_NGBAR], (uint32_t)((qo / TC_NGBAR) & 1), abort, L.err, wc)) break;
                uint8_t *a = ring + slot * TC_STAGE_BYTES;                       // A slice, then B slice
                uint8_t *b = a + TC_A_BYTES;
                const int x = kc * TC_KATOM;
                mbar_expect_tx(&sh.full[slot], (uint32_t)TC_STAGE_BYTES);
                tma_load_2d(a, &tmap, x, (int)u.rowA, &sh.full[slot], pol);
                tma_load_2d(b, &tmap, x, (int)u.rowB, &sh.full[slot], pol);
                tma_load_2d(b + TC_A_BYTES, &tmap, x, (int)u.rowB + TC_TILE, &sh.full[slot], pol);
                sh.slot_q[slot] = k * gpu + kc / G;
                sh.slot_fills[slot]++;
                kc += TC_PROD_WARPS;
                while (kc >= natoms) { kc -= natoms; k++; }
            }
            // every load this producer issued has landed before the CTA may
            // exit (immediate unless the CTA aborted with copies in flight)
            for (int sl = p; sl < TC_STAGES; sl += TC_PROD_WARPS)
                if (sh.slot_fills[sl] > 0) mbar_wait_landed(&sh.full[sl], (uint32_t)((sh.slot_fills[sl] - 1) & 1), L.err);
        }
        __syncwarp();
    } else if (warp == TC_MMA_WARP) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(FMT);
            int slot = 0;
            uint32_t phase = 0;
            long long q = 0;                                     // commit groups issued
            bool issued = false;
            for (long long k = 0; k < my_units && !*abort; k++) {
                const int buf = (int)(k & 1);
                if (!mbar_wait(&sh.tempty[buf], (uint32_t)(((k >> 1) & 1) ^ 1), abort, L.err, wc)) break;
                tc_fence_after();
                const uint32_t dt = tbase + (uint32_t)(buf * TC_N);
                bool ok = true;
                int ing = 0;                                 // K slices in the open commit group
                for (int kc = 0; kc < natoms; kc++) {
                    if (!mbar_wait(&sh.full[slot], phase, abort, L.err, wc)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a = smem_u32(ring + slot * TC_STAGE_BYTES);
                    const uint64_t ad = sdesc_sw64(a), bd = sdesc_sw64(a + TC_A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TC_KATOM / 16; kk++)
                        tc_mma(dt, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                    issued = true;
                    if (++slot == TC_STAGES) { slot = 0; phase ^= 1; }
                    if (++ing == G || kc + 1 == natoms) {
                        tc_commit(&sh.gbar[q % TC_NGBAR]);          // releases the group's slots; the
                        q++;                                         // unit's last group also readies D
                        ing = 0;
                    }
                }
                if (!ok) break;
            }
            // an aborted launch may leave MMAs in flight: they complete
            // before the tensor memory is released
            if (*abort && issued) {
                tc_commit(&sh.drain);
                mbar_wait_landed(&sh.drain, 0, L.err);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 5..12 ----------------
        // Each thread owns one accumulator row (TMEM lane) and one half of
        // the 256 columns: 128-row block J = 2 Jp + ch of the unit.  The h
        // terms of the next unit are fetched while the current one is
        // tested; the test runs as max_j (g_ij - h_j) > h_i over 32 columns
        // and only a passing chunk is examined element by element.
        const int q4 = warp & 3;                    // tensor-memory lane quarter of this warp
        const int ch = (warp - TC_EPI_WARP0) >> 2;  // column half
        const int row = q4 * 32 + lane;             // accumulator row = TMEM lane
        const int et = threadIdx.x - 32 * TC_EPI_WARP0;   // 0..255, column index for h
        const float inf = __int_as_float(0x7f800000);
        float hc_next = inf, hr_next = inf;
        TcUnit nxt{};
        bool ok0 = mbar_wait(&sh.dfull[0], 0, abort, L.err, wc);
        if (ok0) {
            nxt = sh.desc[0];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.dempty[0]);
            if (job.gram_rows == 0) {
                hc_next = L.H[nxt.rowB + et];
                hr_next = L.H[nxt.rowA + row];
            }
        }
        for (long long k = 0; k < my_units; k++) {
            if (epi_bar_or(*abort != 0)) break;              // uniform over the epilogue threads
            const int buf = (int)(k & 1);
            const TcUnit cur = nxt;
            sh.hc[buf][et] = hc_next;
            const float hr = hr_next;
            asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI_WARPS * 32) : "memory");
            if (k + 1 < my_units) {
                const int ds = (int)((k + 1) % TC_NDESC);
                if (mbar_wait(&sh.dfull[ds], (uint32_t)(((k + 1) / TC_NDESC) & 1), abort, L.err, wc)) {
                    nxt = sh.desc[ds];
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh.dempty[ds]);
                    if (job.gram_rows == 0) {
                        hc_next = L.H[nxt.rowB + et];
                        hr_next = L.H[nxt.rowA + row];
                    }
                }
            }
            const long long ql = k * gpu + gpu - 1;          // the unit's last commit group
            bool ok = mbar_wait(&sh.gbar[ql % TC_NGBAR], (uint32_t)((ql / TC_NGBAR) & 1), abort, L.err, wc);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) continue;                               // the next loop top stops every warp
            tc_fence_after();
            const int J = 2 * cur.Jp + ch;                   // 128-row block of this thread's columns
            const bool skip = (job.gram_rows > 0) ? (J * TC_TILE >= job.gram_rows) : (J < cur.I);
            if (skip) {                                      // past the Gram rows, or a lower-triangle block
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.tempty[buf]);
                continue;
            }
            const uint32_t taddr = tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * TC_N + ch * TC_TILE);
            const bool diag = (J == cur.I);
            const float *hcs = sh.hc[buf] + ch * TC_TILE;
            SecState *st = (job.gram_rows == 0) ? &L.st[cur.sec] : nullptr;
            // two halves of 64 columns: two loads, one wait each; the
            // accumulator is released once the second half is in registers
            for (int h = 0; h < 2; h++) {
                uint32_t r[64];
                tmem_ld32_nowait(taddr + (uint32_t)(h * 64), r);
                tmem_ld32_nowait(taddr + (uint32_t)(h * 64 + 32), r + 32);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (h == 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh.tempty[buf]);
                }
                if (job.gram_rows > 0) {
                    float *o = job.gram_out + ((int64_t)cur.I * TC_TILE + row) * job.gram_rows + (int64_t)J * TC_TILE + h * 64;
#pragma unroll
                    for (int c = 0; c < 64; c++) o[c] = __uint_as_float(r[c]);
                    continue;
                }
                screen_test_64(L, st, cur.sec, cur.I, J, row, diag, h, r, hcs, hr);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == TC_MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TC_TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// CTA-pair form (tcgen05 cta_group::2).  Two CTAs of a cluster share one
// 256x256 tile (Ip, Jp) of 256-row blocks: CTA rank r holds the 128 A rows
// of block I = 2 Ip + r and the B rows [128 r, 128 r + 128) of block Jp,
// and one thread of rank 0 issues M=256, N=256, K=16 MMAs that read both
// CTAs' shared memory and write each CTA's 128x256 accumulator into its own
// tensor memory.  Per K slice a CTA loads 16 KB instead of 24 KB, so the
// same shared memory holds a 12-slot ring: 1.5x the MMA work in flight for
// the same bytes.  Both CTAs' TMA copies of a K slice complete on rank 0's
// barrier for that slot (the peer's copies with the cta_group::2 form of
// the TMA load; rank 0 expects the bytes of both), so rank 0's MMAs start
// as soon as the slice is whole.  Before leaving, rank 0 balances any slot
// that only one CTA refilled (an aborted launch) and waits until every
// copy into either CTA has landed.  Commit groups arrive on both CTAs'
// barriers (multicast); rank 0's MMAs wait until both epilogues have read
// an accumulator buffer.  Epilogue and test are those of the one-CTA form,
// per CTA.
// ---------------------------------------------------------------------------
constexpr int TC2_BH_BYTES = TC_TILE * TC_KATOM * 2;            // 8 KB: this CTA's 128 rows of the B block
constexpr int TC2_STAGE_BYTES = TC_A_BYTES + TC2_BH_BYTES;      // 16 KB per K slice and CTA
constexpr int TC2_STAGES = 12;
static_assert(TC2_STAGES % TC_PROD_WARPS == 0, "each producer owns whole ring slots");

struct TcShared2 {
    uint64_t full[TC2_STAGES];                // rank 0: both CTAs' K slice landed (TMA transaction count)
    uint64_t gbar[TC_NGBAR];                  // MMAs of a group of K slices complete (both CTAs)
    uint64_t tempty[2];                       // rank 0: accumulator buffer read out by both epilogues
    uint64_t dfull[TC_NDESC], dempty[TC_NDESC];
    uint64_t drain;                           // rank 0: MMAs of an aborted launch complete
    uint32_t tmem_base;
    int abort;
    long long slot_q[TC2_STAGES];
    int slot_fills[TC2_STAGES];
    int peer_fills[TC2_STAGES];               // rank 0: loads the peer issued into each slot (written at the end)
    TcUnit desc[TC_NDESC];
    alignas(16) float hc[2][TC_N];
    long long pre[MAX_SECTIONS + 1];
    int smc[MAX_SECTIONS];
    int spoff[MAX_SECTIONS];
};
constexpr int TC2_SMEM_BYTES = TC2_STAGES * TC2_STAGE_BYTES + 1024 + (int)((sizeof(TcShared2) + 127) / 128 * 128);
static_assert(TC2_SMEM_BYTES <= 227 * 1024, "screen shared memory");
static_assert(TC2_SMEM_BYTES > 227 * 1024 / 2, "one CTA per SM: the tensor memory is allocated whole");

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Address of the same shared-memory variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cl_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_addr) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cl_addr, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cl_addr), "r"(v) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Whole-cluster barrier (every thread of both CTAs).
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Bounded wait of the pair's pipeline: like mbar_wait, and a wait that
// gives up also stops the peer CTA.  CL: the barrier receives arrivals
// from the peer (acquire at cluster scope).
template <bool CL>
__device__ __forceinline__ bool mbar_wait_pair(uint64_t *bar, uint32_t parity, volatile int *abort, uint32_t peer_abort,
                                               int32_t *err, long long cycles)
{
    long long t0 = clock64();
    while (!(CL ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity))) {
        if (*abort) return false;
        if (clock64() - t0 > cycles) {
            *abort = 1;
            st_cluster_u32(peer_abort, 1u);
            if (err) atomicExch(err, 0x54435754);   // screen wait timed out
            return false;
        }
    }
    return true;
}

// TMA load into this CTA's shared memory whose completion (bytes) is
// reported on a barrier of either CTA of the pair (`cl_bar`: a shared::cluster
// address, here rank 0's).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int x, int y, uint32_t cl_bar,
                                                 uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
        "[%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(cl_bar), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void mbar_complete_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Instruction descriptor of the pair's MMA: kind::f16, FP32 accumulator,
// A/B FP16 (fmt 0) or BF16 (fmt 1), K-major, M = 256, N = 256.
__host__ __device__ constexpr uint32_t idesc_f16_pair(uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)((2 * TC_TILE) >> 4) << 24);
}
__device__ __forceinline__ void tc2_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// Arrive on the barrier at this offset in every CTA of `mask` once the
// issuing thread's earlier MMAs are complete.
__device__ __forceinline__ void tc2_commit(uint64_t *bar, uint16_t mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
        : "memory");
}

// Pair unit t of this launch: A blocks (I0, I1) against the 256-row block
// Jp; this CTA (rank r) takes I_r.  u.pad = 1 when this CTA's block is real
// (screen mode: I1 = -1 pads an odd column with a copy of I0, whose
// results are not tested; Gram mode: the block lies inside the rows).
// u.rowB is the first row of the whole 256-row block.
__device__ __forceinline__ void tc2_unit(const TcShared2 &sh, const TcJob &job, long long t, int &cursor,
                                         uint32_t rank, TcUnit &u, const int32_t *ulist, int ucap)
{
    if (job.gram_rows > 0) {
        const int nbp = (job.gram_rows + TC_N - 1) / TC_N;
        u.sec = 0;
        const int Ip = (int)(t / nbp);
        u.Jp = (int)(t % nbp);
        u.I = 2 * Ip + (int)rank;
        u.pad = (u.I * TC_TILE < job.gram_rows) ? 1 : 0;
        u.rowA = (int64_t)u.I * TC_TILE;
        u.rowB = (int64_t)u.Jp * TC_N;
        return;
    }
    int s = cursor;
    while (sh.pre[s + 1] <= t) s++;
    cursor = s;
    u.sec = s;
    const int32_t *e = ulist + (int64_t)s * ucap + 2 * (t - sh.pre[s]);
    const int32_t e0 = e[0], e1 = e[1];
    u.Jp = e0 & 0xffff;
    u.I = (rank == 0 || e1 < 0) ? (e0 >> 16) : e1;
    u.pad = (rank == 0 || e1 >= 0) ? 1 : 0;
    u.rowA = sh.spoff[s] + (int64_t)u.I * TC_TILE;
    u.rowB = sh.spoff[s] + (int64_t)u.Jp * TC_N;
}

template <int FMT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
    k_screen_tc2(LevelDev L, const __grid_constant__ CUtensorMap tmap, TcJob job)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *ring = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcShared2 &sh = *(TcShared2 *)(ring + TC2_STAGES * TC2_STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();                    // 0 issues the MMAs
    const long long cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
    const int natoms = L.Bpad / TC_KATOM;
    const long long wc = L.wait_cycles > 0 ? L.wait_cycles : TC_WAIT_CYCLES;

    long long total;
    if (job.gram_rows > 0) {
        const long long nbp = (job.gram_rows + TC_N - 1) / TC_N;
        total = nbp * nbp;
    } else {
        block_tile_prefix(L, 0, sh.pre);
        total = sh.pre[L.nsec];
    }
    if (cid >= total) return;            // uniform over the pair: neither CTA has a unit
    const long long my_units = (total - cid + ncl - 1) / ncl;
    int cursor0 = 0;
    if (job.gram_rows == 0) {
        for (int s = threadIdx.x; s < L.nsec; s += blockDim.x) {
            sh.smc[s] = L.st[s].mc;
            sh.spoff[s] = (int)L.poff[s];
        }
        cursor0 = find_section(sh.pre, L.nsec, cid);
    }
    const int G = max(min(L.tc_group > 0 ? L.tc_group : TC_GROUP, TC2_STAGES), (natoms + 15) / 16);
    const int gpu = (natoms + G - 1) / G;
    if (G > TC2_STAGES) {
        if (threadIdx.x == 0 && L.err) atomicExch(L.err, 0x54434752);
        return;                          // uniform over the pair, before any barrier
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC2_STAGES; s++) {
            mbar_init(&sh.full[s], 1);
            sh.slot_q[s] = -1;
            sh.slot_fills[s] = 0;
            sh.peer_fills[s] = 0;
        }
        for (int g = 0; g < TC_NGBAR; g++) mbar_init(&sh.gbar[g], 1);
        for (int b = 0; b < 2; b++) mbar_init(&sh.tempty[b], 2 * TC_EPI_WARPS);
        for (int d = 0; d < TC_NDESC; d++) { mbar_init(&sh.dfull[d], 1); mbar_init(&sh.dempty[d], TC_EPI_WARPS); }
        mbar_init(&sh.drain, 1);
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == TC_MMA_WARP) {           // one warp of each CTA, together
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();                  // both CTAs' barriers exist before any remote arrive
    tc_fence_after();
    const uint32_t tbase = sh.tmem_base;
    volatile int *abort = &sh.abort;
    const uint32_t peer_abort = mapa_shared(smem_u32(&sh.abort), rank ^ 1u);

    if (warp < TC_PROD_WARPS) {
        // ---------------- producers: unit decode + TMA (both CTAs) ----------------
        if (lane == 0) {
            const int p = warp;
            const uint64_t pol = l2_evict_first_policy();
            int cursor = cursor0;
            long long kdec = -1;
            TcUnit u{};
            const uint32_t full0 = mapa_shared(smem_u32(&sh.full[0]), 0u);     // rank 0's slot barriers
            const long long nslices = my_units * natoms;
            long long k = p / natoms;                        // unit and K slice of slice c
            int kc = p - (int)k * natoms;
            int slot = p;
            for (long long c = p; c < nslices && !*abort; c += TC_PROD_WARPS) {
                if (k != kdec) {
                    tc2_unit(sh, job, cid + k * ncl, cursor, rank, u, L.ulist, L.ucap);
                    kdec = k;
                }
                if (kc == 0) {
                    const int ds = (int)(k % TC_NDESC);
                    if (k >= TC_NDESC &&
                        !mbar_wait_pair<false>(&sh.dempty[ds], (uint32_t)((k / TC_NDESC - 1) & 1), abort, peer_abort, L.err, wc))
                        break;
                    sh.desc[ds] = u;
                    mbar_arrive(&sh.dfull[ds]);
                }
                const long long qo = sh.slot_q[slot];
                if (qo >= 0 &&
                    !mbar_wait_pair<false>(&sh.gbar[qo % TC_NGBAR], (uint32_t)((qo / TC_NGBAR) & 1), abort, peer_abort, L.err, wc))
                    break;
                uint8_t *a = ring + slot * TC2_STAGE_BYTES;                      // A slice, then the B half
                const int x = kc * TC_KATOM;
                if (rank == 0) {
                    mbar_expect_tx(&sh.full[slot], (uint32_t)(2 * TC2_STAGE_BYTES));    // both CTAs' bytes
                    tma_load_2d(a, &tmap, x, (int)u.rowA, &sh.full[slot], pol);
                    tma_load_2d(a + TC_A_BYTES, &tmap, x, (int)u.rowB, &sh.full[slot], pol);
                } else {
                    const uint32_t fb = full0 + (uint32_t)(slot * 8);
                    tma_load_2d_pair(a, &tmap, x, (int)u.rowA, fb, pol);
                    tma_load_2d_pair(a + TC_A_BYTES, &tmap, x, (int)(u.rowB + TC_TILE), fb, pol);
                }
                sh.slot_q[slot] = k * gpu + kc / G;
                sh.slot_fills[slot]++;
                kc += TC_PROD_WARPS;
                while (kc >= natoms) { kc -= natoms; k++; }
                slot += TC_PROD_WARPS;
                if (slot >= TC2_STAGES) slot -= TC2_STAGES;
            }
            // the peer's loads per slot, for rank 0's balance at the end
            if (rank == 1) {
                const uint32_t pf0 = mapa_shared(smem_u32(&sh.peer_fills[0]), 0u);
                for (int sl = p; sl < TC2_STAGES; sl += TC_PROD_WARPS)
                    st_cluster_u32(pf0 + (uint32_t)(sl * 4), (uint32_t)sh.slot_fills[sl]);
            }
        }
        __syncwarp();
    } else if (warp == TC_MMA_WARP) {
        if (lane == 0 && rank == 0) {
            // ---------------- MMA issuer (rank 0) ----------------
            const uint32_t idesc = idesc_f16_pair(FMT);
            int slot = 0;
            uint32_t phase = 0;
            long long q = 0;
            bool issued = false;
            for (long long k = 0; k < my_units && !*abort; k++) {
                const int buf = (int)(k & 1);
                if (!mbar_wait_pair<true>(&sh.tempty[buf], (uint32_t)(((k >> 1) & 1) ^ 1), abort, peer_abort, L.err, wc))
                    break;
                tc_fence_after();
                const uint32_t dt = tbase + (uint32_t)(buf * TC_N);
                bool ok = true;
                for (int kc = 0; kc < natoms; kc++) {
                    if (!mbar_wait_pair<true>(&sh.full[slot], phase, abort, peer_abort, L.err, wc)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = smem_u32(ring + slot * TC2_STAGE_BYTES);
                    const uint64_t ad = sdesc_sw64(a), bd = sdesc_sw64(a + TC_A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TC_KATOM / 16; kk++)
                        tc2_mma(dt, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                    issued = true;
                    if (++slot == TC2_STAGES) { slot = 0; phase ^= 1; }
                    if ((kc + 1) % G == 0 || kc + 1 == natoms) {
                        tc2_commit(&sh.gbar[q % TC_NGBAR], (uint16_t)0x3);
                        q++;
                    }
                }
                if (!ok) break;
            }
            if (*abort && issued) {
                tc2_commit(&sh.drain, (uint16_t)0x1);
                mbar_wait_landed(&sh.drain, 0, L.err);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warps 5..12 of each CTA ----------------
        const int q4 = warp & 3;
        const int ch = (warp - TC_EPI_WARP0) >> 2;
        const int row = q4 * 32 + lane;
        const int et = threadIdx.x - 32 * TC_EPI_WARP0;
        const float inf = __int_as_float(0x7f800000);
        const uint32_t te0 = mapa_shared(smem_u32(&sh.tempty[0]), 0u);   // rank 0's accumulator-empty barriers
        float hc_next = inf, hr_next = inf;
        TcUnit nxt{};
        bool ok0 = mbar_wait_pair<false>(&sh.dfull[0], 0, abort, peer_abort, L.err, wc);
        if (ok0) {
            nxt = sh.desc[0];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.dempty[0]);
            if (job.gram_rows == 0) {
                hc_next = L.H[nxt.rowB + et];
                hr_next = L.H[nxt.rowA + row];
            }
        }
        for (long long k = 0; k < my_units; k++) {
            if (epi_bar_or(*abort != 0)) break;
            const int buf = (int)(k & 1);
            const TcUnit cur = nxt;
            sh.hc[buf][et] = hc_next;
            const float hr = hr_next;
            asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI_WARPS * 32) : "memory");
            if (k + 1 < my_units) {
                const int ds = (int)((k + 1) % TC_NDESC);
                if (mbar_wait_pair<false>(&sh.dfull[ds], (uint32_t)(((k + 1) / TC_NDESC) & 1), abort, peer_abort, L.err, wc)) {
                    nxt = sh.desc[ds];
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh.dempty[ds]);
                    if (job.gram_rows == 0) {
                        hc_next = L.H[nxt.rowB + et];
                        hr_next = nxt.pad ? L.H[nxt.rowA + row] : inf;
                    }
                }
            }
            const long long ql = k * gpu + gpu - 1;
            bool ok = mbar_wait_pair<false>(&sh.gbar[ql % TC_NGBAR], (uint32_t)((ql / TC_NGBAR) & 1), abort, peer_abort, L.err, wc);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) continue;
            tc_fence_after();
            const int J = 2 * cur.Jp + ch;
            const bool skip = !cur.pad || ((job.gram_rows > 0) ? (J * TC_TILE >= job.gram_rows) : (J < cur.I));
            if (skip) {
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(te0 + (uint32_t)(buf * 8));
                continue;
            }
            const uint32_t taddr = tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * TC_N + ch * TC_TILE);
            const bool diag = (J == cur.I);
            const float *hcs = sh.hc[buf] + ch * TC_TILE;
            SecState *st = (job.gram_rows == 0) ? &L.st[cur.sec] : nullptr;
            for (int h = 0; h < 2; h++) {
                uint32_t r[64];
                tmem_ld32_nowait(taddr + (uint32_t)(h * 64), r);
                tmem_ld32_nowait(taddr + (uint32_t)(h * 64 + 32), r + 32);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (h == 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_cluster(te0 + (uint32_t)(buf * 8));
                }
                if (job.gram_rows > 0) {
                    float *o = job.gram_out + ((int64_t)cur.I * TC_TILE + row) * job.gram_rows + (int64_t)J * TC_TILE + h * 64;
#pragma unroll
                    for (int c = 0; c < 64; c++) o[c] = __uint_as_float(r[c]);
                    continue;
                }
                screen_test_64(L, st, cur.sec, cur.I, J, row, diag, h, r, hcs, hr);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync_all();                  // both CTAs stopped issuing; the peer's load counts are in place
    // Every copy into either CTA completes on rank 0's slot barriers.  A
    // slot refilled by one CTA only (a launch that stopped early) is
    // balanced first: the missing CTA's bytes are marked done, or rank 0's
    // arrival is added; then rank 0 waits for each slot's last phase.  The
    // two counts differ by at most one (a slot is refilled only after both
    // CTAs' previous loads into it were consumed).
    if (rank == 0 && warp < TC_PROD_WARPS && lane == 0) {
        for (int sl = warp; sl < TC2_STAGES; sl += TC_PROD_WARPS) {
            const int lf = sh.slot_fills[sl], pf = sh.peer_fills[sl];
            if (lf == pf + 1) mbar_complete_tx(&sh.full[sl], (uint32_t)TC2_STAGE_BYTES);
            else if (pf == lf + 1) mbar_expect_tx(&sh.full[sl], (uint32_t)TC2_STAGE_BYTES);
            const int nf = max(lf, pf);
            if (nf > 0) mbar_wait_landed(&sh.full[sl], (uint32_t)((nf - 1) & 1), L.err);
        }
    }
    __syncthreads();
    cluster_sync_all();                  // rank 0's MMAs, every copy and every remote arrive are complete
    if (warp == TC_MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TC_TMEM_COLS) : "memory");
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

// Launch the screen for a level.  `map` must describe L.X.  One persistent
// CTA per SM (the shared memory admits no second one); `n_cta` caps the
// grid (the units are dealt out round-robin).
// The screen's shared-memory size attribute (set once per format, before
// any launch; also called before a stream capture).
inline cudaError_t screen_tc_prepare(int precision)
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
        e = (precision == 2) ? cudaFuncSetAttribute(k_screen_tc2<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    TC2_SMEM_BYTES)
                             : cudaFuncSetAttribute(k_screen_tc2<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    TC2_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_done[fi] = true;
    }
    return cudaSuccess;
}

// CTAs of the pair form's grid: two per cluster that can be resident at
// once (clusters need two free SMs of one GPU processing cluster).
inline int screen_tc2_grid(int n_sm)
{
    static int cached = 0;
    if (cached == 0) {
        (void)screen_tc_prepare(1);      // the shared-memory size the query assumes
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(n_sm & ~1));
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = TC2_SMEM_BYTES;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, k_screen_tc2<0>, &cfg) != cudaSuccess || ncl <= 0) {
            (void)cudaGetLastError();
            ncl = n_sm / 2;
        }
        cached = 2 * std::min(ncl, n_sm / 2);
    }
    return cached;
}

inline cudaError_t launch_screen_tc_map(const LevelDev &L, const CUtensorMap &map, int precision, int n_cta,
                                        cudaStream_t s, TcJob job, bool pair = false)
{
    cudaError_t e = screen_tc_prepare(precision);
    if (e != cudaSuccess) return e;
    if (pair) {
        const int grid = std::max(2, n_cta & ~1);
        if (precision == 2) k_screen_tc2<1><<<grid, TC_THREADS, TC2_SMEM_BYTES, s>>>(L, map, job);
        else k_screen_tc2<0><<<grid, TC_THREADS, TC2_SMEM_BYTES, s>>>(L, map, job);
    } else {
        if (precision == 2) k_screen_tc<1><<<n_cta, TC_THREADS, TC_SMEM_BYTES, s>>>(L, map, job);
        else k_screen_tc<0><<<n_cta, TC_THREADS, TC_SMEM_BYTES, s>>>(L, map, job);
    }
    return cudaGetLastError();
}

}  // namespace rhseg
