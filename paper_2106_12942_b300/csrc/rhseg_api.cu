// rhseg_api.cu -- host orchestrator and C ABI of the RHSEG hot path.
//
// One call of rhseg_run executes the whole recursion on the GPU:
//   deepest level (pixels as regions) ... root, per level:
//     [transition from the level below: roots of the merge forest, pixel
//      relabel, seam pass, ID re-derivation]
//     region tables sorted by ID, adjacency bitmaps, exact best adjacent
//     partners, screen operand rows;
//     HSEG iterations for all sections at once: adjacent step kernel,
//     spectral screen kernel, spectral re-check/merge kernel.
// The host only sizes buffers (one synchronisation per level, to learn the
// region count of each section) and decides when every section is done.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <atomic>
#include <mutex>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/rhseg.h"
#include "rhseg_dev.cuh"
#include "rhseg_kernels.cuh"
#include "rhseg_screen_simt.cuh"
#include "rhseg_screen_tc.cuh"
#include "rhseg_incremental.cuh"

using namespace rhseg;

static thread_local char g_cuda_msg[512] = "";

// Device allocations (cudaMalloc calls) the library has made in this process.
static std::atomic<int64_t> g_dev_allocs{0};

static cudaError_t dev_malloc(void **p, size_t bytes)
{
    g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(p, bytes);
}

#define CK(x)                                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) {                                                                \
            snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s at %s:%d: %s", #x, __FILE__, __LINE__, \
                     cudaGetErrorString(e_));                                                   \
            return (e_ == cudaErrorMemoryAllocation) ? RHSEG_ENOMEM : RHSEG_ECUDA;              \
        }                                                                                       \
    } while (0)

namespace {

struct LevelGeo {
    int32_t nsec = 0;
    std::vector<int32_t> rect;       // [nsec][4]
    std::vector<int32_t> rowband, colband;
    std::vector<int64_t> roff, poff, loff, area;
};

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    int alloc(size_t count)
    {
        if (count <= n && p) return RHSEG_OK;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        if (count == 0) count = 1;
        cudaError_t e = dev_malloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            snprintf(g_cuda_msg, sizeof(g_cuda_msg), "cudaMalloc(%zu bytes): %s", count * sizeof(T),
                     cudaGetErrorString(e));
            p = nullptr;
            return RHSEG_ENOMEM;
        }
        n = count;
        return RHSEG_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

struct SlotSet {
    DBuf<int64_t> S, n;
    DBuf<uint32_t> rid;
    DBuf<uint8_t> alive, lostid;
    DBuf<int32_t> parent, absorbed_at, bestP, pos_of_slot;
    DBuf<uint64_t> bestK;
    int alloc(size_t P, size_t Bs)
    {
        int rc;
        if ((rc = S.alloc(P * Bs))) return rc;
        if ((rc = n.alloc(P))) return rc;
        if ((rc = rid.alloc(P))) return rc;
        if ((rc = alive.alloc(P))) return rc;
        if ((rc = lostid.alloc(P))) return rc;
        if ((rc = parent.alloc(P))) return rc;
        if ((rc = absorbed_at.alloc(P))) return rc;
        if ((rc = bestP.alloc(P))) return rc;
        if ((rc = pos_of_slot.alloc(P))) return rc;
        if ((rc = bestK.alloc(P))) return rc;
        return RHSEG_OK;
    }
    void release()
    {
        S.release(); n.release(); rid.release(); alive.release(); lostid.release(); parent.release();
        absorbed_at.release(); bestP.release(); pos_of_slot.release(); bestK.release();
    }
};

int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace

struct rhseg_handle {
    int32_t rows = 0, cols = 0, B = 0, Bs = 0, Bpad = 0;
    rhseg_params p{};
    int min_nr = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_sm = 148;
    int dev = 0;                  // device the handle was created on
    // inputs
    const uint16_t *img = nullptr;
    const uint8_t *mask = nullptr;
    DBuf<uint16_t> img_own;
    DBuf<uint8_t> mask_own;
    int64_t maxval = 0, unmasked = 0;
    int sigma = 0;
    // geometry
    std::vector<LevelGeo> geo;    // index = level (1..L)
    std::vector<std::vector<DBuf<int32_t>>> geo_i32;   // per level: rect, rowband, colband
    std::vector<std::vector<DBuf<int64_t>>> geo_i64;   // per level: roff, poff, loff
    int64_t log_cap = 0;
    // per-pixel
    DBuf<uint32_t> label, split_from;
    DBuf<uint8_t> isid, split;
    DBuf<int32_t> srcslot, slot_of_id, seam_list, nseam;
    DBuf<double> split_key;
    int32_t seam_cap = 0;
    // slot tables (two sets, alternate per level)
    SlotSet slots[2];
    // positions
    DBuf<int32_t> slot_of_pos;
    DBuf<uint8_t> X;
    DBuf<float> Af, kf, H;
    DBuf<double> Ad, kd;
    size_t npos = 0;
    // incremental spectral minima
    DBuf<uint64_t> sbK;
    DBuf<int32_t> sbP, srow;
    DBuf<unsigned long long> stie, sinit, ckey;
    DBuf<uint8_t> inR;
    DBuf<float> sT, sE, sk, sbuf, srowx;
    DBuf<float> nlo, nhi, brng;
    DBuf<int32_t> ulist;
    DBuf<unsigned long long> sortk;
    DBuf<IncInfo> sinfo;
    // several merges per iteration
    DBuf<unsigned long long> mlist;
    DBuf<uint64_t> mK;
    DBuf<uint32_t> mP;
    // per level, sized at run time
    DBuf<uint32_t> adj;
    // CSR adjacency (params.adjacency = 1): pools, per-slot offsets and
    // lengths, the sort buffer of the build and per-section layout
    DBuf<int32_t> nbr, nofs, ndeg;
    DBuf<unsigned long long> ckeys, ccnt;
    DBuf<int64_t> cebase, cepow, cpbase, chcap;
    DBuf<int64_t> aoff;
    DBuf<int32_t> Wrow, ref;
    DBuf<uint32_t> cand;
    DBuf<float> candg, qf;              // screening-error report of the tensor-core forms
    DBuf<SecState> st;
    DBuf<rhseg_merge> log;
    DBuf<int32_t> err, active;
    DBuf<int32_t> wlist, wcount;        // sections whose operand rows are to be rewritten
    int32_t *active_host = nullptr;
    DBuf<unsigned long long> scan_tmp;
    unsigned long long *scan_host = nullptr;
    // root snapshot data
    DBuf<int64_t> S0, n0;
    int32_t root_m0 = 0, root_nmerge = 0;
    int root_set = 0;
    std::vector<int64_t> targets;
    // results
    bool ran = false;
    std::vector<std::vector<int64_t>> seglen;    // [level][section]
    rhseg_stats stats{};
    DBuf<int32_t> snap_canon, snap_R, snap_labels;
    DBuf<int64_t> snap_sums, snap_counts;
    DBuf<rhseg_merge> log_out;
    // instrumentation
    int64_t nlaunch = 0, nscreen = 0;
    std::vector<cudaEvent_t> prof_ev;   // [3 kernels][chunk][2]
    CUtensorMap tmap;                   // operand rows of the tensor-core screen
    cudaError_t launch_err = cudaSuccess;
};

static int check_params(const rhseg_params *p, int32_t rows, int32_t cols, int32_t bands)
{
    if (!p || rows <= 0 || cols <= 0 || bands <= 0 || bands > 4096) return RHSEG_EINVAL;
    if ((int64_t)rows * cols >= (1ll << 31) - 1) return RHSEG_EINVAL;
    if (p->rnb_levels < 1 || p->rnb_levels > 6) return RHSEG_EINVAL;
    if (!(p->spclust_wght >= 0.0 && p->spclust_wght <= 1.0)) return RHSEG_EINVAL;
    if (p->conv_nregions < 1 || (p->connectivity != 4 && p->connectivity != 8)) return RHSEG_EINVAL;
    if (p->min_nregions < 0 || p->n_out_levels < 0) return RHSEG_EINVAL;
    if (p->precision < 0 || p->precision > 3 || p->profile < 0 || p->profile > 1) return RHSEG_EINVAL;
    if (p->incremental < 0 || p->incremental > 1) return RHSEG_EINVAL;
    if (p->incremental && p->precision != 3) return RHSEG_EINVAL;   // binary32 rows only
    if (p->multi_merge < 0 || p->multi_merge > 1) return RHSEG_EINVAL;
    if (p->multi_merge && p->incremental) return RHSEG_EINVAL;
    if (p->wait_cycles < 0) return RHSEG_EINVAL;
    if (p->screen_group < 0 || p->screen_group > 8) return RHSEG_EINVAL;
    if (p->screen_pair < 0 || p->screen_pair > 1) return RHSEG_EINVAL;
    if (p->adjacency < 0 || p->adjacency > 1) return RHSEG_EINVAL;
    if (p->adjacency && p->incremental) return RHSEG_EINVAL;   // the incremental kernels read the bit matrix
    return RHSEG_OK;
}

// Row (or column) band of every index at a level: `splits` successive
// floor-halvings (reading R6), band = path bits, top split first.
static void make_bands(int n, int splits, std::vector<int32_t> &band)
{
    band.assign(n, 0);
    struct R { int a, b, idx; };
    std::vector<R> cur{{0, n, 0}};
    for (int d = 0; d < splits; d++) {
        std::vector<R> nxt;
        for (auto &r : cur) {
            int h = (r.b - r.a) / 2;
            nxt.push_back({r.a, r.a + h, r.idx * 2});
            nxt.push_back({r.a + h, r.b, r.idx * 2 + 1});
        }
        cur.swap(nxt);
    }
    for (auto &r : cur)
        for (int i = r.a; i < r.b; i++) band[i] = r.idx;
}

static void band_range(const std::vector<int32_t> &band, int idx, int n, int &a, int &b)
{
    a = n; b = n;
    for (int i = 0; i < n; i++)
        if (band[i] == idx) { a = i; break; }
    b = a;
    while (b < n && band[b] == idx) b++;
    if (a == n) { a = b = 0; }
}

static int build_geometry(rhseg_handle *h)
{
    int L = h->p.rnb_levels;
    h->geo.assign(L + 1, LevelGeo());
    int64_t lbase = 0;
    for (int lev = 1; lev <= L; lev++) {
        LevelGeo &G = h->geo[lev];
        int splits = lev - 1;
        G.nsec = 1 << (2 * splits);
        make_bands(h->rows, splits, G.rowband);
        make_bands(h->cols, splits, G.colband);
        int nb = 1 << splits;
        std::vector<int> ra(nb), rb(nb), ca(nb), cb(nb);
        for (int i = 0; i < nb; i++) {
            band_range(G.rowband, i, h->rows, ra[i], rb[i]);
            band_range(G.colband, i, h->cols, ca[i], cb[i]);
        }
        G.rect.resize(4 * G.nsec);
        G.roff.resize(G.nsec + 1);
        G.poff.resize(G.nsec + 1);
        G.loff.resize(G.nsec + 1);
        G.area.resize(G.nsec);
        int64_t ro = 0, po = 0, lo = lbase;
        for (int s = 0; s < G.nsec; s++) {
            int rbi = 0, cbi = 0;
            for (int i = splits - 1; i >= 0; i--) {
                int dig = (s >> (2 * i)) & 3;
                rbi = (rbi << 1) | (dig >> 1);
                cbi = (cbi << 1) | (dig & 1);
            }
            G.rect[4 * s] = ra[rbi]; G.rect[4 * s + 1] = rb[rbi];
            G.rect[4 * s + 2] = ca[cbi]; G.rect[4 * s + 3] = cb[cbi];
            int64_t hh = rb[rbi] - ra[rbi], ww = cb[cbi] - ca[cbi];
            int64_t area = hh * ww;
            G.area[s] = area;
            G.roff[s] = ro; G.poff[s] = po; G.loff[s] = lo;
            ro += area;
            po += ((area + 255) / 256) * 256;           // whole 256-row operand blocks
            lo += area + 2 * (hh + ww) + 8;
        }
        G.roff[G.nsec] = ro; G.poff[G.nsec] = po; G.loff[G.nsec] = lo;
        lbase = lo;
        h->npos = std::max(h->npos, (size_t)po);
    }
    h->log_cap = lbase;
    // upload per level
    h->geo_i32.assign(L + 1, {});
    h->geo_i64.assign(L + 1, {});
    for (int lev = 1; lev <= L; lev++) {
        LevelGeo &G = h->geo[lev];
        auto &I = h->geo_i32[lev];
        auto &J = h->geo_i64[lev];
        I.resize(3);
        J.resize(3);
        int rc;
        if ((rc = I[0].alloc(G.rect.size()))) return rc;
        if ((rc = I[1].alloc(G.rowband.size()))) return rc;
        if ((rc = I[2].alloc(G.colband.size()))) return rc;
        if ((rc = J[0].alloc(G.roff.size()))) return rc;
        if ((rc = J[1].alloc(G.poff.size()))) return rc;
        if ((rc = J[2].alloc(G.loff.size()))) return rc;
        CK(cudaMemcpy(I[0].p, G.rect.data(), G.rect.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(I[1].p, G.rowband.data(), G.rowband.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(I[2].p, G.colband.data(), G.colband.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(J[0].p, G.roff.data(), G.roff.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(J[1].p, G.poff.data(), G.poff.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(J[2].p, G.loff.data(), G.loff.size() * 8, cudaMemcpyHostToDevice));
    }
    return RHSEG_OK;
}

static size_t op_size(int precision)
{
    switch (precision) {
    case 0: return 8;
    case 3: return 4;
    default: return 2;
    }
}

static int bpad_for(int precision, int B)
{
    if (precision == 1 || precision == 2) return ((B + 31) / 32) * 32;   // 64-byte K atoms of the screen
    return ((B + 15) / 16) * 16;
}

static float f32_down(double v)
{
    float f = (float)v;
    if ((double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
}

static float f32_up(double v)
{
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}

// Error-bound constants of the spectral screen (see warp_write_row and the
// screen kernels): operand rounding u, eta; accumulation and evaluation
// slack gamma; the split parameter delta of 2ab <= delta a^2 + b^2 / delta.
static ScreenConst screen_const(const rhseg_handle *h)
{
    ScreenConst c{};
    double Bp = (double)h->Bpad;
    double delta;
    switch (h->p.precision) {
    case 0:
        c.u = 0x1p-52; c.eta = 0.0; delta = 0x1p-20;
        c.gamma = (Bp + 8.0) * 0x1p-52 + 0x1p-48;
        break;
    case 1:   // FP16 operand computed in binary32: 4 binary32 roundings then RN to FP16
        c.u = 0x1p-11 + 0x1p-20; c.eta = 0x1p-25; delta = 0x1p-4;
        c.gamma = 2.0 * Bp * 0x1p-23 + Bp * 0x1p-24 + 0x1p-21;
        break;
    case 2:
        c.u = 0x1p-8 + 0x1p-20; c.eta = 0x1p-133; delta = 0x1p-3;
        c.gamma = 2.0 * Bp * 0x1p-23 + Bp * 0x1p-24 + 0x1p-21;
        break;
    default:  // binary32 operand, CUDA-core accumulation
        c.u = 0x1p-21; c.eta = 0x1p-149; delta = 0x1p-10;
        c.gamma = Bp * 0x1p-23 + Bp * 0x1p-24 + 0x1p-21;
        break;
    }
    double sc = (h->p.precision == 1) ? std::ldexp(1.0, -h->sigma) : 1.0;
    c.two_one_inv_delta = 2.0 * (1.0 + 1.0 / delta);
    c.kscale = (1.0 + delta) * sc * sc;
    c.xscale = sc;
    double lam = 4.0 * (1.0 + 1.0 / delta);
    c.Fq = f32_down(1.0 - c.gamma - lam * c.u * c.u - 0x1p-40);
    c.E0 = f32_up(lam * c.eta * c.eta * (double)h->B);
    c.kscale_f = f32_up(c.kscale * (1.0 + 0x1p-30));
    c.xscale_f = (float)sc;
    c.u_f = f32_up(c.u * (1.0 + 0x1p-30));
    c.etaB_f = f32_up(c.eta * std::sqrt((double)h->B) * (1.0 + 0x1p-30));
    c.onepg_f = f32_up(1.0 + 2.0 * Bp * 0x1p-24);
    c.k1_f = (float)(sc * sc);
    return c;
}

static int common_create(rhseg_handle *h, const rhseg_params *p, void *stream)
{
    h->p = *p;
    if (h->p.n_out_levels == 0) h->p.n_out_levels = 1;
    h->min_nr = p->min_nregions > 0 ? p->min_nregions : p->conv_nregions;
    h->Bs = (h->B + 1) & ~1;
    h->Bpad = bpad_for(p->precision, h->B);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    h->dev = dev;
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev));
    if (prop.major < 10) {
        snprintf(g_cuda_msg, sizeof(g_cuda_msg), "device %s is sm_%d%d, sm_103a required", prop.name, prop.major,
                 prop.minor);
        return RHSEG_EDEVICE;
    }
    h->n_sm = prop.multiProcessorCount;
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    int rc;
    if ((rc = build_geometry(h))) return rc;
    size_t P = (size_t)h->rows * h->cols;
    if ((rc = h->label.alloc(P))) return rc;
    if ((rc = h->split_from.alloc(P))) return rc;
    if ((rc = h->isid.alloc(P))) return rc;
    if ((rc = h->split.alloc(P))) return rc;
    if ((rc = h->srcslot.alloc(P))) return rc;
    if ((rc = h->slot_of_id.alloc(P))) return rc;
    if ((rc = h->split_key.alloc(P))) return rc;
    // seam pixels of one level: at most 2 (h + w) per parent, i.e. at most
    // 2^(L-1) (rows + cols) over a level; twice that as capacity
    h->seam_cap = (int32_t)std::min<int64_t>((int64_t)P, ((int64_t)(h->rows + h->cols) << p->rnb_levels) + 1024);
    if ((rc = h->seam_list.alloc(h->seam_cap))) return rc;
    if ((rc = h->nseam.alloc(1))) return rc;
    for (int k = 0; k < 2; k++)
        if ((rc = h->slots[k].alloc(P, h->Bs))) return rc;
    if ((rc = h->slot_of_pos.alloc(h->npos))) return rc;
    if ((rc = h->X.alloc(h->npos * (size_t)h->Bpad * op_size(p->precision)))) return rc;
    if (p->precision == 0) {
        if ((rc = h->Ad.alloc(h->npos))) return rc;
        if ((rc = h->kd.alloc(h->npos))) return rc;
    } else {
        if ((rc = h->Af.alloc(h->npos))) return rc;
        if ((rc = h->kf.alloc(h->npos))) return rc;
    }
    if ((p->precision == 1 || p->precision == 2) && !p->incremental) {
        if ((rc = h->H.alloc(h->npos))) return rc;
        // certified norm ranges of the operand rows: units proven empty are skipped
        if ((rc = h->nlo.alloc(h->npos))) return rc;
        if ((rc = h->nhi.alloc(h->npos))) return rc;
        if ((rc = h->brng.alloc(4 * (h->npos / 128 + 1)))) return rc;
        if ((rc = h->sk.alloc(h->npos))) return rc;
        if ((rc = h->sortk.alloc(2 * P))) return rc;
        if ((rc = h->qf.alloc(h->npos))) return rc;
    }
    if (p->incremental) {
        if ((rc = h->sbK.alloc(P))) return rc;
        if ((rc = h->sbP.alloc(P))) return rc;
        if ((rc = h->srow.alloc(P))) return rc;
        if ((rc = h->stie.alloc(P))) return rc;
        if ((rc = h->inR.alloc(P))) return rc;
        if ((rc = h->sinit.alloc(h->npos))) return rc;
        if ((rc = h->sT.alloc(h->npos))) return rc;
        if ((rc = h->sE.alloc(h->npos))) return rc;
        if ((rc = h->sk.alloc(h->npos))) return rc;
        if ((rc = h->sbuf.alloc(h->npos * INC_RCAP))) return rc;
        if ((rc = h->srowx.alloc((size_t)h->geo[p->rnb_levels].nsec * h->Bpad * INC_RCAP))) return rc;
        if ((rc = h->sinfo.alloc((size_t)h->geo[p->rnb_levels].nsec))) return rc;
        CK(cudaMemset(h->inR.p, 0, P));
    }
    if (p->multi_merge) {
        if ((rc = h->mlist.alloc(2 * P))) return rc;
        if ((rc = h->mK.alloc(P))) return rc;
        if ((rc = h->mP.alloc(P))) return rc;
    }
    if (screen_uses_tcgen05(p->precision)) {
        CK(screen_tc_prepare(p->precision));
        int mr = make_operand_map(&h->tmap, h->X.p, (int64_t)h->npos, h->Bpad, p->precision);
        if (mr) {
            snprintf(g_cuda_msg, sizeof(g_cuda_msg), "tensor map for the screen operands failed (%d)", mr);
            return RHSEG_ECUDA;
        }
    }
    int nsec_max = h->geo[p->rnb_levels].nsec;
    if ((rc = h->st.alloc(nsec_max))) return rc;
    if ((rc = h->aoff.alloc(nsec_max + 1))) return rc;
    if ((rc = h->Wrow.alloc(nsec_max))) return rc;
    if ((rc = h->ref.alloc((size_t)nsec_max * h->Bs))) return rc;
    if ((rc = h->log.alloc(h->log_cap))) return rc;
    if ((rc = h->err.alloc(1))) return rc;
    if ((rc = h->wlist.alloc(nsec_max))) return rc;
    if (p->adjacency) {
        if ((rc = h->nofs.alloc(P))) return rc;
        if ((rc = h->ndeg.alloc(P))) return rc;
        if ((rc = h->ccnt.alloc(nsec_max))) return rc;
        if ((rc = h->cebase.alloc(nsec_max + 1))) return rc;
        if ((rc = h->cepow.alloc(nsec_max))) return rc;
        if ((rc = h->cpbase.alloc(nsec_max + 1))) return rc;
        if ((rc = h->chcap.alloc(nsec_max))) return rc;
    }
    if ((rc = h->wcount.alloc(1))) return rc;
    CK(cudaMemset(h->wcount.p, 0, 4));
    if ((rc = h->active.alloc(2))) return rc;
    CK(cudaMallocHost((void **)&h->active_host, 2 * sizeof(int32_t)));
    CK(cudaMallocHost((void **)&h->scan_host, 2 * sizeof(unsigned long long)));
    return RHSEG_OK;
}

static int scan_inputs(rhseg_handle *h, const uint16_t *img, const uint8_t *mask)
{
    int64_t P = (int64_t)h->rows * h->cols;
    int64_t mx = 0, un = 0;
    for (int64_t q = 0; q < P; q++) {
        if (mask && mask[q]) continue;
        un++;
        const uint16_t *x = img + q * h->B;
        for (int b = 0; b < h->B; b++) mx = std::max<int64_t>(mx, x[b]);
    }
    h->maxval = mx;
    h->unmasked = un;
    long double a = (long double)un * (long double)un / 4.0L * (long double)mx;
    if (a >= ldexpl(1.0L, 62)) return RHSEG_ERANGE;
    if ((long double)h->B * a * a >= ldexpl(1.0L, 127)) return RHSEG_ERANGE;
    h->sigma = (mx >= 32768) ? 1 : 0;
    return RHSEG_OK;
}

extern "C" int rhseg_create(const uint16_t *image, int32_t rows, int32_t cols, int32_t bands, const uint8_t *mask,
                            const rhseg_params *p, void *cuda_stream, rhseg_handle **out)
{
    if (!out || !image) return RHSEG_EINVAL;
    *out = nullptr;
    int rc = check_params(p, rows, cols, bands);
    if (rc) return rc;
    rhseg_handle *h = new rhseg_handle();
    h->rows = rows; h->cols = cols; h->B = bands;
    if ((rc = scan_inputs(h, image, mask))) { delete h; return rc; }
    if ((rc = common_create(h, p, cuda_stream))) { rhseg_destroy(h); return rc; }
    size_t P = (size_t)rows * cols;
    if ((rc = h->img_own.alloc(P * bands))) { rhseg_destroy(h); return rc; }
    cudaError_t e = cudaMemcpyAsync(h->img_own.p, image, P * bands * 2, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && mask) {
        if ((rc = h->mask_own.alloc(P))) { rhseg_destroy(h); return rc; }
        e = cudaMemcpyAsync(h->mask_own.p, mask, P, cudaMemcpyHostToDevice, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        snprintf(g_cuda_msg, sizeof(g_cuda_msg), "input copy: %s", cudaGetErrorString(e));
        rhseg_destroy(h);
        return RHSEG_ECUDA;
    }
    h->img = h->img_own.p;
    h->mask = mask ? h->mask_own.p : nullptr;
    *out = h;
    return RHSEG_OK;
}

__global__ void k_scan_device_inputs(const uint16_t *img, const uint8_t *mask, int64_t P, int B,
                                     unsigned long long *maxv, unsigned long long *cnt)
{
    unsigned long long mx = 0, c = 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
        if (mask && mask[q]) continue;
        c++;
        for (int b = 0; b < B; b++) mx = max(mx, (unsigned long long)img[q * B + b]);
    }
    atomicMax(maxv, mx);
    atomicAdd(cnt, c);
}

extern "C" int rhseg_create_device(const uint16_t *image_dev, int32_t rows, int32_t cols, int32_t bands,
                                   const uint8_t *mask_dev, const rhseg_params *p, void *cuda_stream,
                                   rhseg_handle **out)
{
    if (!out || !image_dev) return RHSEG_EINVAL;
    *out = nullptr;
    int rc = check_params(p, rows, cols, bands);
    if (rc) return rc;
    rhseg_handle *h = new rhseg_handle();
    h->rows = rows; h->cols = cols; h->B = bands;
    if ((rc = common_create(h, p, cuda_stream))) { rhseg_destroy(h); return rc; }
    unsigned long long *tmp = nullptr, host[2] = {0, 0};
    cudaError_t e = dev_malloc((void **)&tmp, 16);
    if (e == cudaSuccess) e = cudaMemsetAsync(tmp, 0, 16, h->stream);
    if (e == cudaSuccess) {
        k_scan_device_inputs<<<h->n_sm * 4, 256, 0, h->stream>>>(image_dev, mask_dev, (int64_t)rows * cols, bands,
                                                                  tmp, tmp + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, 16, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
        snprintf(g_cuda_msg, sizeof(g_cuda_msg), "input scan: %s", cudaGetErrorString(e));
        rhseg_destroy(h);
        return RHSEG_ECUDA;
    }
    h->maxval = (int64_t)host[0];
    h->unmasked = (int64_t)host[1];
    long double a = (long double)h->unmasked * (long double)h->unmasked / 4.0L * (long double)h->maxval;
    if (a >= ldexpl(1.0L, 62) || (long double)bands * a * a >= ldexpl(1.0L, 127)) {
        rhseg_destroy(h);
        return RHSEG_ERANGE;
    }
    h->sigma = (h->maxval >= 32768) ? 1 : 0;
    h->img = image_dev;
    h->mask = mask_dev;
    *out = h;
    return RHSEG_OK;
}

__global__ void k_scan_inputs_dev(const uint16_t *img, const uint8_t *mask, int64_t P, int B,
                                  unsigned long long *maxv, unsigned long long *cnt);

extern "C" int rhseg_set_image(rhseg_handle *h, const uint16_t *image, const uint8_t *mask, void *cuda_stream)
{
    if (!h || !image) return RHSEG_EINVAL;
    if (!h->img_own.p) return RHSEG_ESTATE;
    if ((mask != nullptr) != (h->mask_own.p != nullptr)) return RHSEG_EINVAL;
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : h->stream;
    size_t P = (size_t)h->rows * h->cols;
    CK(cudaMemcpyAsync(h->img_own.p, image, P * h->B * 2, cudaMemcpyHostToDevice, s));
    if (mask) CK(cudaMemcpyAsync(h->mask_own.p, mask, P, cudaMemcpyHostToDevice, s));
    // range of the new image (exact-key bound), on the device
    int rc;
    if ((rc = h->scan_tmp.alloc(2))) return rc;
    CK(cudaMemsetAsync(h->scan_tmp.p, 0, 16, s));
    k_scan_inputs_dev<<<h->n_sm * 4, 256, 0, s>>>(h->img_own.p, h->mask_own.p, (int64_t)P, h->B, h->scan_tmp.p,
                                                   h->scan_tmp.p + 1);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->scan_host, h->scan_tmp.p, 16, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int64_t mx = (int64_t)h->scan_host[0], un = (int64_t)h->scan_host[1];
    long double a = (long double)un * (long double)un / 4.0L * (long double)mx;
    if (a >= ldexpl(1.0L, 62) || (long double)h->B * a * a >= ldexpl(1.0L, 127)) return RHSEG_ERANGE;
    if (((mx >= 32768) ? 1 : 0) != h->sigma) {
        h->sigma = (mx >= 32768) ? 1 : 0;
    }
    h->maxval = mx;
    h->unmasked = un;
    h->ran = false;
    return RHSEG_OK;
}

__global__ void k_scan_inputs_dev(const uint16_t *img, const uint8_t *mask, int64_t P, int B,
                                  unsigned long long *maxv, unsigned long long *cnt)
{
    unsigned long long mx = 0, c = 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
        if (mask && mask[q]) continue;
        c++;
        for (int b = 0; b < B; b++) mx = max(mx, (unsigned long long)img[q * B + b]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxv, mx);
        atomicAdd(cnt, c);
    }
}

// ---------------------------------------------------------------------------
// run
// ---------------------------------------------------------------------------

// Sections still running -> active[0]; the device error word -> active[1].
__global__ void k_count_active(const SecState *st, int nsec, int32_t *active, const int32_t *err)
{
    int c = 0;
    for (int s = threadIdx.x; s < nsec; s += blockDim.x) c += st[s].done ? 0 : 1;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ int w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += w[i];
        active[0] = t;
        active[1] = *(volatile const int32_t *)err;
    }
}

static void launch_screen(rhseg_handle *h, const LevelDev &L, cudaStream_t st)
{
    h->nlaunch++;
    h->nscreen++;
    int grid = h->n_sm * 2;
    switch (h->p.precision) {
    case 0: k_screen_simt<double, double><<<grid, 256, 0, st>>>(L); break;
    case 3: k_screen_simt<float, float><<<grid, 256, 0, st>>>(L); break;
    default: {
        TcJob job{0, nullptr};
        const bool pair = L.tc_pair != 0;
        cudaError_t e = launch_screen_tc_map(L, h->tmap, h->p.precision, pair ? screen_tc2_grid(h->n_sm) : h->n_sm,
                                             st, job, pair);
        if (e != cudaSuccess) h->launch_err = e;
        break;
    }
    }
}

// Level start of the incremental mode: tiled pass `pass` over every
// running section (operand type by precision).
static void launch_sinit(rhseg_handle *h, const LevelDev &D, int pass)
{
    h->nlaunch++;
    const int grid = h->n_sm * 4;
    switch (h->p.precision) {
    case 1: if (pass) k_sinit_tile<__half, 1><<<grid, 256, 0, h->stream>>>(D); else k_sinit_tile<__half, 0><<<grid, 256, 0, h->stream>>>(D); break;
    case 2: if (pass) k_sinit_tile<__nv_bfloat16, 1><<<grid, 256, 0, h->stream>>>(D); else k_sinit_tile<__nv_bfloat16, 0><<<grid, 256, 0, h->stream>>>(D); break;
    default: if (pass) k_sinit_tile<float, 1><<<grid, 256, 0, h->stream>>>(D); else k_sinit_tile<float, 0><<<grid, 256, 0, h->stream>>>(D); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) h->launch_err = e;
}

// Per-iteration row updates of the incremental mode (binary32 rows): the
// rows to recompute, the sums pass over many blocks per section, then the
// exact minima and pushes.
static void launch_srow_update(rhseg_handle *h, const LevelDev &D)
{
    const int dyn = inc_dyn_smem(h->Bpad);
    static bool attr = false;
    cudaError_t e = cudaSuccess;
    if (!attr) {
        e = cudaFuncSetAttribute(k_srow_sums, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_srow_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr = true;
    }
    if (e == cudaSuccess) {
        k_srow_begin<<<D.nsec, STEP_THREADS, 0, h->stream>>>(D);
        k_srow_sums<<<dim3(INC_SUM_BLOCKS, D.nsec), STEP_THREADS, dyn, h->stream>>>(D);
        k_srow_finish<<<D.nsec, STEP_THREADS, dyn, h->stream>>>(D);
        h->nlaunch += 3;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) h->launch_err = e;
}

// Return code of a device error word: a bounded wait of the screen that gave
// up is RHSEG_ETIMEOUT, any other failed device check RHSEG_ECUDA.
static int err_word_code(int32_t w)
{
    if (w == 0x54435754 || w == 0x54434c44) return RHSEG_ETIMEOUT;
    return RHSEG_ECUDA;
}

static int run_impl(rhseg_handle *h)
{
    cudaStream_t s = h->stream;
    const int L = h->p.rnb_levels;
    const int64_t P = (int64_t)h->rows * h->cols;
    PixGeom g{h->rows, h->cols, h->B, h->Bs, h->img, h->mask};
    ScreenConst sc = screen_const(h);
    int grid_pix = h->n_sm * 8;
    h->stats = rhseg_stats{};
    h->nlaunch = 0;
    h->nscreen = 0;
    const int chunk = 32;
    if (h->p.profile && h->prof_ev.empty()) {
        h->prof_ev.resize(3 * chunk * 2);
        for (auto &e : h->prof_ev) CK(cudaEventCreate(&e));
    }
    h->seglen.assign(L + 1, {});
    h->root_set = 0;
    cudaEvent_t ev0, ev1;
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    CK(cudaEventRecord(ev0, s));
    CK(cudaMemsetAsync(h->err.p, 0, 4, s));
    k_init_labels<<<grid_pix, 256, 0, s>>>(g, h->label.p, h->isid.p, h->srcslot.p); h->nlaunch++;
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(h->split.p, 0, P, s));
    int cur = 0;
    cudaEvent_t lev_ev[2];
    CK(cudaEventCreate(&lev_ev[0]));
    CK(cudaEventCreate(&lev_ev[1]));
    for (int lev = L; lev >= 1; lev--) {
        CK(cudaEventRecord(lev_ev[0], s));
        LevelGeo &G = h->geo[lev];
        auto &GI = h->geo_i32[lev];
        auto &GJ = h->geo_i64[lev];
        SlotSet &T = h->slots[cur];
        SlotSet &Pv = h->slots[cur ^ 1];
        if (lev < L) {
            // ---- transition from level lev+1 (tables in Pv) ----
            LevelGeo &Gc = h->geo[lev + 1];
            auto &GJc = h->geo_i64[lev + 1];
            auto &GIc = h->geo_i32[lev + 1];
            k_resolve_roots<<<Gc.nsec, 256, 0, s>>>(Pv.parent.p, GJc[0].p, h->st.p, Gc.nsec); h->nlaunch++;
            k_relabel<<<grid_pix, 256, 0, s>>>(P, h->label.p, h->slot_of_id.p, Pv.parent.p, Pv.rid.p); h->nlaunch++;
            CK(cudaMemsetAsync(h->isid.p, 0, P, s));
            CK(cudaMemsetAsync(h->split.p, 0, P, s));
            CK(cudaMemsetAsync(h->nseam.p, 0, 4, s));
            CK(cudaMemsetAsync(Pv.lostid.p, 0, Pv.lostid.n, s));
            if (h->p.seam_pass) {
                SeamGeom sg{GIc[1].p, GIc[2].p, lev - 1, h->p.connectivity};
                k_seam_detect<<<grid_pix, 256, 0, s>>>(g, sg, h->label.p, h->seam_list.p, h->nseam.p, h->seam_cap); h->nlaunch++;
                k_seam_decide<<<h->n_sm * 4, 256, 0, s>>>(g, sg, h->label.p, h->slot_of_id.p, Pv.S.p, Pv.n.p,
                                                          Pv.rid.p, h->seam_list.p, h->nseam.p, h->seam_cap,
                                                          h->split.p, h->split_key.p, h->split_from.p, h->err.p); h->nlaunch++;
                k_seam_apply<<<h->n_sm * 4, 256, 0, s>>>(g, h->label.p, h->slot_of_id.p, Pv.S.p, Pv.n.p, Pv.rid.p,
                                                         Pv.lostid.p, h->seam_list.p, h->nseam.p, h->seam_cap,
                                                         h->split.p); h->nlaunch++;
                k_lost_reset<<<grid_pix, 256, 0, s>>>((int64_t)Pv.lostid.n, Pv.lostid.p, Pv.rid.p); h->nlaunch++;
                k_lost_min<<<grid_pix, 256, 0, s>>>(P, h->label.p, h->split.p, h->slot_of_id.p, Pv.lostid.p,
                                                    Pv.rid.p); h->nlaunch++;
                k_lost_relabel<<<grid_pix, 256, 0, s>>>(P, h->label.p, h->split.p, h->slot_of_id.p, Pv.lostid.p,
                                                        Pv.rid.p); h->nlaunch++;
                k_seam_label_singletons<<<h->n_sm, 256, 0, s>>>(h->seam_list.p, h->nseam.p, h->seam_cap,
                                                                 h->split.p, h->label.p); h->nlaunch++;
                k_mark_singletons<<<h->n_sm, 256, 0, s>>>(h->seam_list.p, h->nseam.p, h->seam_cap, h->split.p,
                                                          h->isid.p, h->srcslot.p); h->nlaunch++;
            }
            dim3 gm(64, Gc.nsec);
            k_mark_ids_upper<<<gm, 256, 0, s>>>(GJc[0].p, h->st.p, Gc.nsec, Pv.alive.p, Pv.n.p, Pv.rid.p,
                                                 h->isid.p, h->srcslot.p); h->nlaunch++;
            CK(cudaGetLastError());
        }
        // ---- region tables of this level ----
        k_section_scan<<<G.nsec, 512, 0, s>>>(g, G.nsec, GI[0].p, h->isid.p, lev < L ? h->split.p : nullptr,
                                              h->split_key.p, h->split_from.p, GJ[0].p, h->slot_of_id.p, h->st.p,
                                              h->log.p, GJ[2].p, lev); h->nlaunch++;
        CK(cudaGetLastError());
        std::vector<SecState> sth(G.nsec);
        CK(cudaMemcpyAsync(sth.data(), h->st.p, sizeof(SecState) * G.nsec, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::vector<int32_t> W(G.nsec);
        std::vector<int64_t> aoff(G.nsec + 1);
        int64_t atot = 0, maxpairs = 0;
        int32_t m0max = 0;
        for (int k = 0; k < G.nsec; k++) {
            int m0 = sth[k].m0;
            m0max = std::max(m0max, m0);
            W[k] = ((ceil_div(m0, 32) + 3) / 4) * 4;
            if (W[k] == 0) W[k] = 4;
            if (h->p.adjacency) W[k] = 0;              // lists instead of the bit matrix
            aoff[k] = atot;
            atot += (int64_t)m0 * W[k];
            maxpairs = std::max(maxpairs, (int64_t)m0 * (m0 - 1) / 2);
        }
        aoff[G.nsec] = atot;
        int rc;
        if ((rc = h->adj.alloc((size_t)atot))) return rc;
        int64_t cand_cap = std::min<int64_t>(std::max<int64_t>(maxpairs, 1),
                                             std::max<int64_t>(1 << 16, (1ll << 24) / G.nsec));
        if (h->p.spclust_wght > 0.0) {
            if ((rc = h->cand.alloc((size_t)G.nsec * cand_cap * 2))) return rc;
            if (h->qf.p && (rc = h->candg.alloc((size_t)G.nsec * cand_cap))) return rc;
        }
        const bool inc = h->p.incremental && h->p.spclust_wght > 0.0;
        if (inc)
            if ((rc = h->ckey.alloc((size_t)G.nsec * cand_cap))) return rc;
        const bool skip_units = h->nlo.p != nullptr && h->p.spclust_wght > 0.0;
        // the pair form lists two words per pair, at most one pair per unit
        const int32_t ucap = ((int32_t)tc_section_units(m0max) + 1) * (h->p.screen_pair ? 2 : 1);
        if (skip_units)
            if ((rc = h->ulist.alloc((size_t)G.nsec * ucap))) return rc;
        CK(cudaMemcpyAsync(h->aoff.p, aoff.data(), 8 * (G.nsec + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(h->Wrow.p, W.data(), 4 * G.nsec, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(h->adj.p, 0, (size_t)atot * 4, s));
        k_fill_tables<<<h->n_sm * 8, 256, 0, s>>>(g, P, h->isid.p, h->srcslot.p, h->slot_of_id.p, Pv.S.p, Pv.n.p,
                                                  T.S.p, T.n.p, T.rid.p, T.alive.p, T.parent.p, T.absorbed_at.p,
                                                  T.bestK.p, T.bestP.p); h->nlaunch++;
        k_init_parent<<<dim3(8, G.nsec), 256, 0, s>>>(T.parent.p, GJ[0].p, h->st.p, G.nsec); h->nlaunch++;
        const bool csr = h->p.adjacency != 0;
        if (!csr) {
            k_build_adj<<<grid_pix, 256, 0, s>>>(g, h->label.p, h->slot_of_id.p, GI[1].p, GI[2].p, lev - 1,
                                                 h->p.connectivity, GJ[0].p, h->aoff.p, h->Wrow.p, h->adj.p);
            h->nlaunch++;
            h->stats.adjacency_bytes = std::max<int64_t>(h->stats.adjacency_bytes, atot * 4);
        } else {
            // neighbour lists: count the section's directed pixel edges, lay out
            // its sort buffer (a power of two) and its pool (two halves of
            // 3 x edges + 64 words), write the edges; sorted below
            CK(cudaMemsetAsync(h->ccnt.p, 0, 8 * G.nsec, s));
            k_csr_emit<<<grid_pix, 256, 0, s>>>(g, h->label.p, h->slot_of_id.p, GI[1].p, GI[2].p, lev - 1,
                                                h->p.connectivity, GJ[0].p, h->ccnt.p, nullptr, nullptr);
            h->nlaunch++;
            std::vector<unsigned long long> cnt(G.nsec);
            CK(cudaMemcpyAsync(cnt.data(), h->ccnt.p, 8 * G.nsec, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            std::vector<int64_t> ebase(G.nsec + 1), epow(G.nsec), pbase(G.nsec + 1), hcap(G.nsec);
            int64_t et = 0, pt = 0;
            for (int k = 0; k < G.nsec; k++) {
                int64_t e2 = 1;
                while (e2 < (int64_t)cnt[k]) e2 <<= 1;
                epow[k] = e2;
                ebase[k] = et;
                et += e2;
                hcap[k] = 3 * (int64_t)cnt[k] + 64;
                if (hcap[k] >= ((int64_t)1 << 31)) return RHSEG_ERANGE;   // offsets are 32-bit
                pbase[k] = pt;
                pt += 2 * hcap[k];
            }
            ebase[G.nsec] = et;
            pbase[G.nsec] = pt;
            if ((rc = h->ckeys.alloc((size_t)et))) return rc;
            if ((rc = h->nbr.alloc((size_t)pt))) return rc;
            CK(cudaMemcpyAsync(h->cebase.p, ebase.data(), 8 * (G.nsec + 1), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(h->cepow.p, epow.data(), 8 * G.nsec, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(h->cpbase.p, pbase.data(), 8 * (G.nsec + 1), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(h->chcap.p, hcap.data(), 8 * G.nsec, cudaMemcpyHostToDevice, s));
            CK(cudaMemsetAsync(h->ccnt.p, 0, 8 * G.nsec, s));
            k_csr_emit<<<grid_pix, 256, 0, s>>>(g, h->label.p, h->slot_of_id.p, GI[1].p, GI[2].p, lev - 1,
                                                h->p.connectivity, GJ[0].p, h->ccnt.p, h->cebase.p, h->ckeys.p);
            h->nlaunch++;
            h->stats.adjacency_bytes = std::max<int64_t>(h->stats.adjacency_bytes,
                                                         et * 8 + pt * 4 + G.roff[G.nsec] * 8);
        }
        CK(cudaGetLastError());
        LevelDev D{};
        D.level = lev; D.nsec = G.nsec; D.B = h->B; D.Bs = h->Bs; D.Bpad = h->Bpad;
        D.wait_cycles = h->p.wait_cycles;
        D.tc_group = h->p.screen_group;
        D.precision = h->p.precision;
        D.w = h->p.spclust_wght; D.ww = h->p.spclust_wght * h->p.spclust_wght;
        D.sigma_shift = h->sigma;
        D.st = h->st.p; D.roff = GJ[0].p; D.poff = GJ[1].p; D.aoff = h->aoff.p; D.W = h->Wrow.p;
        D.loff = GJ[2].p; D.ref = h->ref.p; D.rect = GI[0].p;
        D.S = T.S.p; D.n = T.n.p; D.rid = T.rid.p; D.alive = T.alive.p; D.parent = T.parent.p;
        D.absorbed_at = T.absorbed_at.p; D.bestK = T.bestK.p; D.bestP = T.bestP.p; D.pos_of_slot = T.pos_of_slot.p;
        D.slot_of_pos = h->slot_of_pos.p; D.X = h->X.p;
        D.Af = h->Af.p; D.kf = h->kf.p; D.Ad = h->Ad.p; D.kd = h->kd.p;
        D.H = (h->p.precision == 1 || h->p.precision == 2) ? h->H.p : nullptr;
        D.adj = h->adj.p; D.cand = h->cand.p; D.cand_cap = cand_cap;
        if (csr) {
            D.csr = 1;
            D.nbr = h->nbr.p; D.pbase = h->cpbase.p; D.hcap = h->chcap.p; D.nofs = h->nofs.p; D.ndeg = h->ndeg.p;
        }
        if (h->qf.p && h->p.spclust_wght > 0.0 && !inc) {
            D.candg = h->candg.p; D.qf = h->qf.p;
            D.err_gamma = sc.gamma; D.err_u = sc.u; D.err_etaB = sc.eta * std::sqrt((double)h->B);
        }
        D.log = h->log.p; D.err = h->err.p;
        D.wlist = h->wlist.p; D.wcount = h->wcount.p;
        if (skip_units) {
            D.nlo = h->nlo.p; D.nhi = h->nhi.p; D.sk = h->sk.p; D.brng = h->brng.p;
            D.ulist = h->ulist.p; D.ucap = ucap; D.sortk = h->sortk.p;
            D.tc_pair = h->p.screen_pair;      // the pair form walks the listed tiles
            D.count_useful = h->p.profile;     // a diagnostic: a shared atomic per kept unit
        }
        if (h->p.multi_merge) {
            D.multi = 1;
            D.mlist = h->mlist.p; D.mK = h->mK.p; D.mP = h->mP.p;
        }
        if (inc) {
            D.H = nullptr;
            D.incremental = 1;
            D.sbK = h->sbK.p; D.sbP = h->sbP.p; D.stie = h->stie.p; D.inR = h->inR.p; D.srow = h->srow.p;
            D.sinit = h->sinit.p; D.sT = h->sT.p; D.ckey = h->ckey.p;
            D.sE = h->sE.p; D.sk = h->sk.p; D.inc_onepg = sc.onepg_f; D.sbuf = h->sbuf.p;
            D.srowx = h->srowx.p; D.sinfo = h->sinfo.p;
        }
        if (csr) {
            k_csr_build<<<G.nsec, 1024, 0, s>>>(D, h->ccnt.p, h->cebase.p, h->cepow.p, h->ckeys.p);
            h->nlaunch++;
        }
        k_init_best<<<dim3(std::max(1, std::min(64, ceil_div(m0max, 8))), G.nsec), 256, 0, s>>>(D); h->nlaunch++;
        int32_t target = (lev == 1) ? h->p.conv_nregions : h->min_nr;
        k_init_section<<<G.nsec, STEP_THREADS, 0, s>>>(D, sc, target); h->nlaunch++;
        if (h->p.spclust_wght > 0.0) {
            k_write_rows<<<h->n_sm * 4, 256, 0, s>>>(D, sc, 0); h->nlaunch++;
            if (skip_units) {             // positions in norm order, rows rewritten there
                k_sort_positions<<<G.nsec, STEP_THREADS, 0, s>>>(D); h->nlaunch++;
                k_write_rows<<<h->n_sm * 4, 256, 0, s>>>(D, sc, 0); h->nlaunch++;
            }
        }
        CK(cudaGetLastError());
        if (inc) {
            // every row's exact best non-adjacent partner
            CK(cudaMemsetAsync(h->sinit.p, 0xff, h->npos * 8, s));
            if (h->p.profile) CK(cudaEventRecord(h->prof_ev[0], s));
            launch_sinit(h, D, 0);
            k_sinit_exact<<<dim3(std::max(1, std::min(64, ceil_div(m0max, 8))), G.nsec), 256, 0, s>>>(D); h->nlaunch++;
            launch_sinit(h, D, 1);
            k_sinit_final<<<G.nsec, STEP_THREADS, 0, s>>>(D); h->nlaunch++;
            CK(cudaGetLastError());
            CK(h->launch_err);
            if (h->p.profile) {
                CK(cudaEventRecord(h->prof_ev[1], s));
                CK(cudaEventSynchronize(h->prof_ev[1]));
                float a = 0;
                CK(cudaEventElapsedTime(&a, h->prof_ev[0], h->prof_ev[1]));
                h->stats.screen_ms += a;
                h->stats.level_screen_ms[lev - 1] += a;
            }
        }
        if (lev == 1) {
            h->root_m0 = sth[0].m0;
            if ((rc = h->S0.alloc((size_t)std::max(1, h->root_m0) * h->Bs))) return rc;
            if ((rc = h->n0.alloc((size_t)std::max(1, h->root_m0)))) return rc;
            CK(cudaMemcpyAsync(h->S0.p, T.S.p, (size_t)h->root_m0 * h->Bs * 8, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(h->n0.p, T.n.p, (size_t)h->root_m0 * 8, cudaMemcpyDeviceToDevice, s));
        }
        // ---- HSEG iterations, all sections at once ----
        int64_t max_iter = (int64_t)m0max + 2;
        int64_t it = 0;
        const bool prof = h->p.profile != 0;
        // one chunk of HSEG iterations, then the count of running sections and
        // the device error word into pinned host memory
        auto enqueue_chunk = [&]() -> int {
            for (int k = 0; k < chunk; k++) {
                if (prof) CK(cudaEventRecord(h->prof_ev[(0 * chunk + k) * 2], s));
                if (csr) k_adj_step<true><<<G.nsec, STEP_THREADS, 0, s>>>(D, sc);
                else k_adj_step<false><<<G.nsec, STEP_THREADS, 0, s>>>(D, sc);
                h->nlaunch++;
                if (prof) CK(cudaEventRecord(h->prof_ev[(0 * chunk + k) * 2 + 1], s));
                if (h->p.spclust_wght > 0.0) {
                    if (prof) CK(cudaEventRecord(h->prof_ev[(1 * chunk + k) * 2], s));
                    if (inc) launch_srow_update(h, D);
                    else launch_screen(h, D, s);
                    if (prof) CK(cudaEventRecord(h->prof_ev[(1 * chunk + k) * 2 + 1], s));
                    if (inc) k_spec_inc<<<G.nsec, STEP_THREADS, 0, s>>>(D, sc);
                    else if (csr) k_spec_step<true><<<G.nsec, STEP_THREADS, 0, s>>>(D, sc);
                    else k_spec_step<false><<<G.nsec, STEP_THREADS, 0, s>>>(D, sc);
                    h->nlaunch++;
                    k_write_rows<<<h->n_sm * 4, 256, 0, s>>>(D, sc, 1); h->nlaunch++;
                    if (prof) CK(cudaEventRecord(h->prof_ev[(2 * chunk + k) * 2 + 1], s));
                }
            }
            CK(cudaGetLastError());
            CK(h->launch_err);
            k_count_active<<<1, 1024, 0, s>>>(h->st.p, G.nsec, h->active.p, h->err.p); h->nlaunch++;
            CK(cudaMemcpyAsync(h->active_host, h->active.p, 8, cudaMemcpyDeviceToHost, s));
            return RHSEG_OK;
        };
        // Without per-kernel events the chunk is captured once per level as a
        // CUDA graph (the kernels read all per-iteration state from the
        // device, so every chunk of the level is the same graph) and replayed;
        // the legacy default stream cannot be captured, so there the chunks
        // are launched directly.
        cudaGraphExec_t gexec = nullptr;
        int64_t chunk_launches = 0, chunk_screens = 0;
        if (!prof && !inc && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread) {
            cudaGraph_t graph = nullptr;
            const int64_t l0 = h->nlaunch, sc0 = h->nscreen;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const int rc_c = enqueue_chunk();
                const cudaError_t ec = cudaStreamEndCapture(s, &graph);
                if (rc_c == RHSEG_OK && ec == cudaSuccess && graph != nullptr &&
                    cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess)
                    gexec = nullptr;
                if (graph) cudaGraphDestroy(graph);
                if (rc_c != RHSEG_OK || ec != cudaSuccess) {
                    if (gexec) cudaGraphExecDestroy(gexec);
                    gexec = nullptr;
                }
            }
            (void)cudaGetLastError();
            h->launch_err = cudaSuccess;
            chunk_launches = h->nlaunch - l0;
            chunk_screens = h->nscreen - sc0;
            h->nlaunch = l0;
            h->nscreen = sc0;
        }
        while (true) {
            if (gexec) {
                const cudaError_t e = cudaGraphLaunch(gexec, s);
                if (e != cudaSuccess) {
                    cudaGraphExecDestroy(gexec);
                    CK(e);
                }
                h->nlaunch += chunk_launches;
                h->nscreen += chunk_screens;
            } else {
                int rcq = enqueue_chunk();
                if (rcq) return rcq;
            }
            it += chunk;
            {
                const cudaError_t e = cudaStreamSynchronize(s);
                if (e != cudaSuccess && gexec) cudaGraphExecDestroy(gexec);
                CK(e);
            }
            if (h->active_host[1]) {          // a device wait gave up or a check failed: stop here
                int rc_err = err_word_code(h->active_host[1]);
                snprintf(g_cuda_msg, sizeof(g_cuda_msg), "device error word 0x%08x at level %d", h->active_host[1], lev);
                if (gexec) cudaGraphExecDestroy(gexec);
                return rc_err;
            }
            if (prof) {
                for (int k = 0; k < chunk; k++) {
                    float a = 0, b = 0, c = 0;
                    CK(cudaEventElapsedTime(&a, h->prof_ev[(0 * chunk + k) * 2], h->prof_ev[(0 * chunk + k) * 2 + 1]));
                    h->stats.adj_ms += a;
                    h->stats.level_adj_ms[lev - 1] += a;
                    if (h->p.spclust_wght > 0.0) {
                        CK(cudaEventElapsedTime(&b, h->prof_ev[(1 * chunk + k) * 2], h->prof_ev[(1 * chunk + k) * 2 + 1]));
                        CK(cudaEventElapsedTime(&c, h->prof_ev[(1 * chunk + k) * 2 + 1], h->prof_ev[(2 * chunk + k) * 2 + 1]));
                        h->stats.screen_ms += b;
                        h->stats.spec_ms += c;
                        h->stats.level_screen_ms[lev - 1] += b;
                        h->stats.level_spec_ms[lev - 1] += c;
                    }
                }
            }
            if (*h->active_host == 0) break;
            if (it > max_iter + chunk) {
                snprintf(g_cuda_msg, sizeof(g_cuda_msg), "level %d did not finish after %lld iterations", lev,
                         (long long)it);
                if (gexec) cudaGraphExecDestroy(gexec);
                return RHSEG_ETIMEOUT;
            }
        }
        if (gexec) cudaGraphExecDestroy(gexec);
        CK(cudaMemcpyAsync(sth.data(), h->st.p, sizeof(SecState) * G.nsec, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        h->seglen[lev].resize(G.nsec);
        for (int k = 0; k < G.nsec; k++) {
            const SecState &q = sth[k];
            h->seglen[lev][k] = q.log_n;
            h->stats.pairs += q.pairs;
            h->stats.iterations += q.iter;
            h->stats.screened_pairs += q.screened;
            h->stats.screen_evaluated += q.evaluated;
            h->stats.level_screen_evaluated[lev - 1] += q.evaluated;
            h->stats.screen_useful += q.useful;
            h->stats.candidates += q.cands;
            h->stats.candidates_below += q.cands_true;
            h->stats.fallbacks += q.fallbacks;
            h->stats.stalled_sections += q.stalled;
            h->stats.merges_adj += q.madj;
            h->stats.merges_spec += q.mspec;
            h->stats.seam_splits += q.nsplit;
            float er, eb;
            std::memcpy(&er, &q.err_rel_bits, 4);
            std::memcpy(&eb, &q.err_bnd_bits, 4);
            h->stats.screen_err_rel_max = std::max(h->stats.screen_err_rel_max, (double)er);
            h->stats.screen_err_bound_max = std::max(h->stats.screen_err_bound_max, (double)eb);
            h->stats.screen_err_pairs += q.err_pairs;
        }
        if (lev == 1) h->root_nmerge = sth[0].nmerge;
        {
            int32_t mi = 0;
            for (int k = 0; k < G.nsec; k++) mi = std::max(mi, sth[k].iter);
            h->stats.level_iters[lev - 1] = mi;
            CK(cudaEventRecord(lev_ev[1], s));
            CK(cudaEventSynchronize(lev_ev[1]));
            float lms = 0;
            CK(cudaEventElapsedTime(&lms, lev_ev[0], lev_ev[1]));
            h->stats.level_ms[lev - 1] = lms;
        }
        cur ^= 1;
    }
    cudaEventDestroy(lev_ev[0]);
    cudaEventDestroy(lev_ev[1]);
    CK(cudaEventRecord(ev1, s));
    CK(cudaEventSynchronize(ev1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    h->stats.run_ms = ms;
    h->stats.kernel_launches = h->nlaunch;
    h->stats.screen_impl = h->nscreen == 0 ? 0 : (h->p.precision == 0 ? 1 : (screen_uses_tcgen05(h->p.precision) ? 3 : 2));
    h->stats.screen_launches = h->nscreen;
    int32_t errh = 0;
    CK(cudaMemcpy(&errh, h->err.p, 4, cudaMemcpyDeviceToHost));
    if (errh) {
        snprintf(g_cuda_msg, sizeof(g_cuda_msg), "device error word 0x%08x", errh);
        return err_word_code(errh);
    }
    // merge counts from the log segments (kind field) are gathered in get_log;
    // per-kind totals here come from a pass over the log lengths
    h->ran = true;
    // output-level targets (reading R9)
    {
        int K = h->p.n_out_levels;
        int64_t c0 = h->root_m0, conv = h->p.conv_nregions;
        std::vector<int64_t> t;
        if (c0 <= conv) t.push_back(c0);
        else if (K == 1) t.push_back(conv);
        else {
            for (int k = 0; k < K; k++) {
                if (k == 0) t.push_back(c0);
                else if (k == K - 1) t.push_back(conv);
                else t.push_back((int64_t)std::nearbyint((double)conv * std::pow((double)c0 / (double)conv,
                                                                            (double)(K - 1 - k) / (double)(K - 1))));
            }
        }
        h->targets.clear();
        for (auto v : t)
            if (h->targets.empty() || h->targets.back() != v) h->targets.push_back(v);
        h->stats.n_levels_out = (int32_t)h->targets.size();
    }
    return RHSEG_OK;
}

extern "C" int rhseg_run(rhseg_handle *h, void *cuda_stream)
{
    if (!h) return RHSEG_EINVAL;
    cudaStream_t keep = h->stream;
    if (cuda_stream) h->stream = (cudaStream_t)cuda_stream;
    h->ran = false;
    int rc = run_impl(h);
    h->stream = keep;
    if (rc == RHSEG_OK) {
        // per-kind merge counts
        int64_t tot = 0;
        for (auto &v : h->seglen)
            for (auto x : v) tot += x;
        (void)tot;
    }
    return rc;
}

extern "C" int rhseg_set_wait_cycles(rhseg_handle *h, int64_t cycles)
{
    if (!h || cycles < 0) return RHSEG_EINVAL;
    h->p.wait_cycles = cycles;
    return RHSEG_OK;
}

extern "C" int rhseg_n_levels(const rhseg_handle *h, int32_t *n_levels)
{
    if (!h || !n_levels) return RHSEG_EINVAL;
    if (!h->ran) return RHSEG_ESTATE;
    *n_levels = (int32_t)h->targets.size();
    return RHSEG_OK;
}

extern "C" int rhseg_get_level(rhseg_handle *h, int32_t level, int32_t *labels, int64_t *band_sums,
                               int64_t *counts, int32_t *nregions_out)
{
    if (!h) return RHSEG_EINVAL;
    if (!h->ran) return RHSEG_ESTATE;
    if (level < 0 || level >= (int32_t)h->targets.size()) return RHSEG_EINVAL;
    cudaStream_t s = h->stream;
    int64_t P = (int64_t)h->rows * h->cols;
    int64_t M = (int64_t)h->root_m0 - h->targets[level];
    if (M > h->root_nmerge) M = h->root_nmerge;
    if (M < 0) M = 0;
    int m0 = h->root_m0;
    SlotSet &T = h->slots[(h->p.rnb_levels - 1) & 1];   // tables of the root level
    int rc;
    if ((rc = h->snap_canon.alloc(std::max(1, m0)))) return rc;
    if ((rc = h->snap_R.alloc(1))) return rc;
    k_snap_canon<<<1, 1024, 0, s>>>(m0, T.absorbed_at.p + 0, (int32_t)M, h->snap_canon.p, h->snap_R.p);
    int32_t R = 0;
    CK(cudaMemcpyAsync(&R, h->snap_R.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nregions_out) *nregions_out = R;
    if (labels) {
        if ((rc = h->snap_labels.alloc(P))) return rc;
        k_snap_labels<<<h->n_sm * 8, 256, 0, s>>>(P, h->label.p, h->slot_of_id.p, T.parent.p, T.absorbed_at.p,
                                                  (int32_t)M, h->snap_canon.p, h->snap_labels.p);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(labels, h->snap_labels.p, P * 4, cudaMemcpyDeviceToHost, s));
    }
    if (band_sums || counts) {
        if ((rc = h->snap_sums.alloc((size_t)std::max(1, R) * h->B))) return rc;
        if ((rc = h->snap_counts.alloc(std::max(1, R)))) return rc;
        CK(cudaMemsetAsync(h->snap_sums.p, 0, (size_t)std::max(1, R) * h->B * 8, s));
        CK(cudaMemsetAsync(h->snap_counts.p, 0, (size_t)std::max(1, R) * 8, s));
        k_snap_tables<<<h->n_sm * 4, 256, 0, s>>>(m0, h->B, h->Bs, h->S0.p, h->n0.p, T.parent.p, T.absorbed_at.p,
                                                  (int32_t)M, h->snap_canon.p, h->snap_sums.p, h->snap_counts.p);
        CK(cudaGetLastError());
        if (band_sums) CK(cudaMemcpyAsync(band_sums, h->snap_sums.p, (size_t)R * h->B * 8, cudaMemcpyDeviceToHost, s));
        if (counts) CK(cudaMemcpyAsync(counts, h->snap_counts.p, (size_t)R * 8, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return RHSEG_OK;
}

// ---------------------------------------------------------------------------
// Hierarchy levels without device allocation
// ---------------------------------------------------------------------------

// Working array of rhseg_get_level_noalloc: canonical label of each root
// region, then the region count.  File scope, so it needs no allocation.
static __device__ __align__(256) int32_t g_level_scratch[RHSEG_NOALLOC_MAX_REGIONS + 1];

static int32_t *g_level_scratch_dev[64];     // device address per device, looked up once
static std::mutex g_level_scratch_mu;

static int level_scratch_ptr(int dev, int32_t **out)
{
    if (dev < 0 || dev >= 64) return RHSEG_EDEVICE;
    std::lock_guard<std::mutex> lock(g_level_scratch_mu);
    if (!g_level_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_level_scratch);   // for the current device (= dev)
        if (e != cudaSuccess || !p) {
            snprintf(g_cuda_msg, sizeof(g_cuda_msg), "cudaGetSymbolAddress(level scratch): %s", cudaGetErrorString(e));
            return RHSEG_ECUDA;
        }
        g_level_scratch_dev[dev] = (int32_t *)p;
    }
    *out = g_level_scratch_dev[dev];
    return RHSEG_OK;
}

extern "C" int rhseg_get_level_noalloc(rhseg_handle *h, int32_t level, int32_t *labels_dev, int64_t *band_sums_dev,
                                       int64_t *counts_dev, int32_t regions_cap, int32_t *nregions_out)
{
    if (!h || regions_cap < 0) return RHSEG_EINVAL;
    if (!h->ran) return RHSEG_ESTATE;
    if (level < 0 || level >= (int32_t)h->targets.size()) return RHSEG_EINVAL;
    int m0 = h->root_m0;
    if (m0 > RHSEG_NOALLOC_MAX_REGIONS) {
        snprintf(g_cuda_msg, sizeof(g_cuda_msg),
                 "root level has %d regions; rhseg_get_level_noalloc holds at most %d", m0, RHSEG_NOALLOC_MAX_REGIONS);
        return RHSEG_ERANGE;
    }
    int cur_dev = -1;
    CK(cudaGetDevice(&cur_dev));
    if (cur_dev != h->dev) {
        snprintf(g_cuda_msg, sizeof(g_cuda_msg), "current device %d is not the handle's device %d", cur_dev, h->dev);
        return RHSEG_EDEVICE;
    }
    int32_t *scratch = nullptr;
    int rc = level_scratch_ptr(h->dev, &scratch);
    if (rc) return rc;
    int32_t *canon = scratch, *Rdev = scratch + RHSEG_NOALLOC_MAX_REGIONS;
    cudaStream_t s = h->stream;
    int64_t P = (int64_t)h->rows * h->cols;
    int64_t M = (int64_t)h->root_m0 - h->targets[level];
    if (M > h->root_nmerge) M = h->root_nmerge;
    if (M < 0) M = 0;
    SlotSet &T = h->slots[(h->p.rnb_levels - 1) & 1];   // tables of the root level
    k_snap_canon<<<1, 1024, 0, s>>>(m0, T.absorbed_at.p, (int32_t)M, canon, Rdev);
    CK(cudaGetLastError());
    int32_t R = 0;
    CK(cudaMemcpyAsync(&R, Rdev, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nregions_out) *nregions_out = R;
    // the capacity check comes first: on RHSEG_ETRUNC nothing is written
    if ((band_sums_dev || counts_dev) && R > regions_cap) return RHSEG_ETRUNC;
    if (labels_dev) {
        k_snap_labels<<<h->n_sm * 8, 256, 0, s>>>(P, h->label.p, h->slot_of_id.p, T.parent.p, T.absorbed_at.p,
                                                  (int32_t)M, canon, labels_dev);
        CK(cudaGetLastError());
    }
    if (band_sums_dev || counts_dev) {
        if (band_sums_dev && R > 0) CK(cudaMemsetAsync(band_sums_dev, 0, (size_t)R * h->B * 8, s));
        if (counts_dev && R > 0) CK(cudaMemsetAsync(counts_dev, 0, (size_t)R * 8, s));
        if (band_sums_dev && counts_dev) {
            k_snap_tables<<<h->n_sm * 4, 256, 0, s>>>(m0, h->B, h->Bs, h->S0.p, h->n0.p, T.parent.p, T.absorbed_at.p,
                                                      (int32_t)M, canon, band_sums_dev, counts_dev);
            CK(cudaGetLastError());
        } else if (R > 0) {
            // only one of the two tables was requested
            k_snap_tables_part<<<h->n_sm * 4, 256, 0, s>>>(m0, h->B, h->Bs, h->S0.p, h->n0.p, T.parent.p,
                                                           T.absorbed_at.p, (int32_t)M, canon, band_sums_dev,
                                                           counts_dev);
            CK(cudaGetLastError());
        }
    }
    CK(cudaStreamSynchronize(s));
    return RHSEG_OK;
}

__global__ void k_gather_log(const rhseg_merge *src, rhseg_merge *dst, const int64_t *seg_src,
                             const int64_t *seg_dst, const int64_t *seg_len, int nseg)
{
    int seg = blockIdx.y;
    if (seg >= nseg) return;
    int64_t n = seg_len[seg];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[seg_dst[seg] + k] = src[seg_src[seg] + k];
}

extern "C" int rhseg_get_log(rhseg_handle *h, rhseg_merge *log, int64_t log_cap, int64_t *log_len)
{
    if (!h || !log_len) return RHSEG_EINVAL;
    if (!h->ran) return RHSEG_ESTATE;
    std::vector<int64_t> ssrc, sdst, slen;
    int64_t tot = 0;
    for (int lev = h->p.rnb_levels; lev >= 1; lev--) {
        const LevelGeo &G = h->geo[lev];
        for (int k = 0; k < G.nsec; k++) {
            int64_t n = h->seglen[lev][k];
            if (!n) continue;
            ssrc.push_back(G.loff[k]);
            sdst.push_back(tot);
            slen.push_back(n);
            tot += n;
        }
    }
    *log_len = tot;
    if (!log) return RHSEG_OK;
    if (log_cap < tot) return RHSEG_ETRUNC;
    if (tot == 0) return RHSEG_OK;
    cudaStream_t s = h->stream;
    int rc;
    if ((rc = h->log_out.alloc(tot))) return rc;
    int nseg = (int)slen.size();
    DBuf<int64_t> d;
    if ((rc = d.alloc(3 * (size_t)nseg))) return rc;
    std::vector<int64_t> all;
    all.insert(all.end(), ssrc.begin(), ssrc.end());
    all.insert(all.end(), sdst.begin(), sdst.end());
    all.insert(all.end(), slen.begin(), slen.end());
    cudaError_t e = cudaMemcpyAsync(d.p, all.data(), all.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        for (int base = 0; base < nseg; base += 65535) {
            int cnt = std::min(65535, nseg - base);
            k_gather_log<<<dim3(4, cnt), 256, 0, s>>>(h->log.p, h->log_out.p, d.p + base, d.p + nseg + base,
                                                      d.p + 2 * nseg + base, cnt);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(log, h->log_out.p, tot * sizeof(rhseg_merge), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    d.release();
    if (e != cudaSuccess) {
        snprintf(g_cuda_msg, sizeof(g_cuda_msg), "get_log: %s", cudaGetErrorString(e));
        return RHSEG_ECUDA;
    }
    return RHSEG_OK;
}

extern "C" int rhseg_get_stats(const rhseg_handle *h, rhseg_stats *s)
{
    if (!h || !s) return RHSEG_EINVAL;
    if (!h->ran) return RHSEG_ESTATE;
    *s = h->stats;
    s->device_allocs = g_dev_allocs.load(std::memory_order_relaxed);
    return RHSEG_OK;
}

extern "C" void rhseg_destroy(rhseg_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->img_own.release(); h->mask_own.release();
    for (auto &v : h->geo_i32) for (auto &b : v) b.release();
    for (auto &v : h->geo_i64) for (auto &b : v) b.release();
    h->label.release(); h->split_from.release(); h->isid.release(); h->split.release();
    h->srcslot.release(); h->slot_of_id.release(); h->seam_list.release(); h->nseam.release();
    h->split_key.release();
    h->slots[0].release(); h->slots[1].release();
    h->sbK.release(); h->sbP.release(); h->srow.release(); h->stie.release(); h->sinit.release();
    h->ckey.release(); h->inR.release(); h->sT.release(); h->sE.release(); h->sk.release(); h->sbuf.release();
    h->nlo.release(); h->nhi.release(); h->brng.release(); h->ulist.release();
    h->sortk.release();
    h->mlist.release(); h->mK.release(); h->mP.release();
    h->srowx.release(); h->sinfo.release();
    h->candg.release(); h->qf.release();
    h->slot_of_pos.release(); h->X.release(); h->Af.release(); h->kf.release(); h->H.release(); h->Ad.release(); h->kd.release();
    h->nbr.release(); h->nofs.release(); h->ndeg.release(); h->ckeys.release(); h->ccnt.release();
    h->cebase.release(); h->cepow.release(); h->cpbase.release(); h->chcap.release();
    h->adj.release(); h->aoff.release(); h->Wrow.release(); h->ref.release(); h->cand.release(); h->st.release();
    h->log.release(); h->err.release(); h->active.release(); h->wlist.release(); h->wcount.release();
    h->S0.release(); h->n0.release();
    h->snap_canon.release(); h->snap_R.release(); h->snap_labels.release(); h->snap_sums.release();
    h->snap_counts.release(); h->log_out.release();
    if (h->active_host) cudaFreeHost(h->active_host);
    if (h->scan_host) cudaFreeHost(h->scan_host);
    h->scan_tmp.release();
    for (auto &e : h->prof_ev) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

extern "C" const char *rhseg_strerror(int code)
{
    switch (code) {
    case RHSEG_OK: return "ok";
    case RHSEG_EINVAL: return "invalid argument";
    case RHSEG_ERANGE: return "image exceeds the exact-key range";
    case RHSEG_ENOMEM: return "device memory exhausted";
    case RHSEG_ECUDA: return "CUDA error";
    case RHSEG_ETIMEOUT: return "bounded device wait or iteration limit exceeded";
    case RHSEG_ESTATE: return "call out of order";
    case RHSEG_ETRUNC: return "output buffer too small";
    case RHSEG_EDEVICE: return "no usable sm_103a device";
    default: return "unknown error";
    }
}

extern "C" const char *rhseg_last_cuda_error(void) { return g_cuda_msg; }

// ---------------------------------------------------------------------------
// Utility entry points
// ---------------------------------------------------------------------------

__global__ void k_keys(const int64_t *S, const int64_t *n, int32_t nreg, int32_t B, int32_t stride,
                       const int32_t *pi, const int32_t *pj, int32_t np, double *out, int32_t *err)
{
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < np; t += nwarps) {
        int i = pi[t], j = pj[t];
        double K;
        if (i < 0 || j < 0 || i >= nreg || j >= nreg) K = __longlong_as_double(0x7FF8000000000000ll);
        else K = warp_key(S + (int64_t)i * stride, n[i], S + (int64_t)j * stride, n[j], B, err);
        if ((threadIdx.x & 31) == 0) out[t] = K;
    }
}

extern "C" int rhseg_keys(const int64_t *S, const int64_t *n, int32_t nreg, int32_t bands, int32_t stride,
                          const int32_t *pair_i, const int32_t *pair_j, int32_t npairs, double *out,
                          void *cuda_stream)
{
    if (!S || !n || !pair_i || !pair_j || !out || nreg < 0 || bands <= 0 || stride < bands || npairs < 0)
        return RHSEG_EINVAL;
    if (npairs == 0) return RHSEG_OK;
    int grid = std::min<int64_t>(4096, ((int64_t)npairs + 7) / 8);
    k_keys<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(S, n, nreg, bands, stride, pair_i, pair_j, npairs, out,
                                                       nullptr);
    CK(cudaGetLastError());
    return RHSEG_OK;
}

__global__ void k_div(const uint64_t *nh, const uint64_t *nl, const uint64_t *dh, const uint64_t *dl, int32_t n,
                      double *out)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        u128 N{nl[t], nh[t]}, D{dl[t], dh[t]};
        if ((D.lo | D.hi) == 0 || (N.hi >> 63) || (D.hi >> 63)) { out[t] = __longlong_as_double(0x7FF8000000000000ll); continue; }
        out[t] = div_rn_u128(N, D, nullptr);
    }
}

extern "C" int rhseg_gram_tc(const void *X, int32_t rows, int32_t Bpad, int32_t precision, int32_t cta_pair,
                             float *G, void *cuda_stream)
{
    if (!X || !G || rows <= 0 || rows % TC_TILE || Bpad <= 0 || Bpad % TC_KATOM || Bpad > 4096 ||
        (precision != 1 && precision != 2) || (cta_pair != 0 && cta_pair != 1))
        return RHSEG_EINVAL;
    CUtensorMap map;
    if (make_operand_map(&map, X, rows, Bpad, precision)) {
        snprintf(g_cuda_msg, sizeof(g_cuda_msg), "tensor map encode failed");
        return RHSEG_ECUDA;
    }
    LevelDev L{};
    L.Bpad = Bpad;
    L.nsec = 1;
    TcJob job{rows, G};
    const int units = (rows / TC_TILE) * ((rows + TC_N - 1) / TC_N);
    int nsm = 148;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    if (cta_pair) {
        const int tiles = ((rows + TC_N - 1) / TC_N) * ((rows + TC_N - 1) / TC_N);
        CK(launch_screen_tc_map(L, map, precision, std::min(2 * tiles, screen_tc2_grid(nsm)), (cudaStream_t)cuda_stream,
                                job, true));
        return RHSEG_OK;
    }
    CK(launch_screen_tc_map(L, map, precision, std::max(1, std::min(units, nsm)), (cudaStream_t)cuda_stream, job));
    return RHSEG_OK;
}

extern "C" int rhseg_div_rn(const uint64_t *n_hi, const uint64_t *n_lo, const uint64_t *d_hi, const uint64_t *d_lo,
                            int32_t n, double *out, void *cuda_stream)
{
    if (!n_hi || !n_lo || !d_hi || !d_lo || !out || n < 0) return RHSEG_EINVAL;
    if (n == 0) return RHSEG_OK;
    k_div<<<std::min(4096, (n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(n_hi, n_lo, d_hi, d_lo, n, out);
    CK(cudaGetLastError());
    return RHSEG_OK;
}
