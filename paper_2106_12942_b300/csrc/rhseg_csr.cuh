// rhseg_csr.cuh -- compressed-row adjacency of the regions of a section
// (params.adjacency = 1).
//
// Section 4.1 keeps, for every region, the regions it touches; the thesis's
// GPU program stores them in fixed-size lists (MAX_ADJACENCIES, a limit its
// Section 6.2 names).  The default form here is a dense bit matrix per
// section (m0^2 / 8 bytes).  This form takes memory in proportion to the
// edges: each slot's neighbour slots, sorted ascending, in a per-section
// pool of two halves of hcap words (hcap = 3 x the directed pixel edges of
// the section + 64, which bounds the number of list entries, plus room for
// one union and its scratch).  A merge writes the survivor's new list at the
// top of the pool; when the pool is full, the live lists are copied densely
// into the other half first.  Both forms give identical merges.
#pragma once
#include "rhseg_dev.cuh"

namespace rhseg {

// Slot r's neighbour list and its length.
__device__ __forceinline__ int32_t *csr_row(const LevelDev &L, int sec, int phalf, int64_t ro, int r, int &deg)
{
    deg = L.ndeg[ro + r];
    return L.nbr + L.pbase[sec] + (int64_t)phalf * L.hcap[sec] + L.nofs[ro + r];
}

// First index i of the ascending v[0..n) with v[i] >= x (n when none).
__device__ __forceinline__ int csr_lower_bound(const int32_t *v, int n, int x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (v[m] < x) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// Slots i and j adjacent (binary search in the shorter list).
__device__ __forceinline__ bool csr_adjacent(const LevelDev &L, int sec, int phalf, int64_t ro, int i, int j)
{
    int di, dj;
    const int32_t *li = csr_row(L, sec, phalf, ro, i, di);
    const int32_t *lj = csr_row(L, sec, phalf, ro, j, dj);
    if (dj < di) { li = lj; di = dj; j = i; }
    const int k = csr_lower_bound(li, di, j);
    return k < di && li[k] == j;
}

// Exclusive prefix sum of v over the block; *total = the sum (every thread).
__device__ __forceinline__ int csr_scan(int v, int *total)
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

// Directed pixel edges between different regions of one section (4 or 8
// connectivity, both pixels unmasked): counted per section (keys null, cnt
// += 2 per neighbouring pixel pair) or written as (slot p << 32) | slot q in
// both directions at keys[ebase[k] + atomicAdd(cnt[k], 2)].
__global__ void k_csr_emit(PixGeom g, const uint32_t *label, const int32_t *slot_of_id, const int32_t *rowband,
                           const int32_t *colband, int nbits, int conn, const int64_t *roff, unsigned long long *cnt,
                           const int64_t *ebase, unsigned long long *keys)
{
    const int64_t P = (int64_t)g.rows * g.cols;
    const int dy8[4] = {0, 1, 1, 1}, dx8[4] = {1, -1, 0, 1};
    const int dy4[2] = {0, 1}, dx4[2] = {1, 0};
    const int nn = conn == 8 ? 4 : 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t lp = label[p];
        if (lp == 0) continue;
        const int y = (int)(p / g.cols), x = (int)(p % g.cols);
        const int sp = morton2(rowband[y], colband[x], nbits);
        for (int k = 0; k < nn; k++) {
            const int yy = y + (conn == 8 ? dy8[k] : dy4[k]);
            const int xx = x + (conn == 8 ? dx8[k] : dx4[k]);
            if (yy < 0 || yy >= g.rows || xx < 0 || xx >= g.cols) continue;
            const int64_t q = (int64_t)yy * g.cols + xx;
            const uint32_t lq = label[q];
            if (lq == 0 || lq == lp) continue;
            if (morton2(rowband[yy], colband[xx], nbits) != sp) continue;
            const unsigned long long i = atomicAdd(&cnt[sp], 2ull);
            if (keys == nullptr) continue;
            const unsigned long long a = (unsigned long long)(slot_of_id[lp - 1] - roff[sp]);
            const unsigned long long b = (unsigned long long)(slot_of_id[lq - 1] - roff[sp]);
            keys[ebase[sp] + (int64_t)i] = (a << 32) | b;
            keys[ebase[sp] + (int64_t)i + 1] = (b << 32) | a;
        }
    }
}

// One block per section: sort the section's edge keys (bitonic network over
// epow[k] entries, a power of two, the tail filled with ~0), drop repeats,
// and lay the lists out in half 0 of the pool; ndeg and nofs of every slot,
// ptop and phalf of the section.
__global__ void k_csr_build(LevelDev L, const unsigned long long *cnt, const int64_t *ebase, const int64_t *epow,
                            unsigned long long *keys)
{
    const int sec = blockIdx.x;
    if (sec >= L.nsec) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t n = (int64_t)cnt[sec], n2 = epow[sec];
    unsigned long long *k = keys + ebase[sec];
    const int64_t ro = L.roff[sec];
    const int m0 = L.st[sec].m0;
    for (int64_t i = n + tid; i < n2; i += nt) k[i] = ~0ull;
    for (int s = tid; s < m0; s += nt) { L.ndeg[ro + s] = 0; L.nofs[ro + s] = 0; }
    __syncthreads();
    for (int64_t size = 2; size <= n2; size <<= 1) {
        for (int64_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (int64_t i = tid; i < (n2 >> 1); i += nt) {
                const int64_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const unsigned long long x = k[lo], y = k[hi];
                if ((x > y) == asc) { k[lo] = y; k[hi] = x; }
            }
            __syncthreads();
        }
    }
    int32_t *pool = L.nbr + L.pbase[sec];
    int64_t base = 0;
    for (int64_t c0 = 0; c0 < n; c0 += nt) {
        const int64_t i = c0 + tid;
        unsigned long long key = 0, prev = ~0ull;
        int f = 0;
        if (i < n) {
            key = k[i];
            if (i > 0) prev = k[i - 1];
            f = (i == 0 || prev != key) ? 1 : 0;
        }
        int tot;
        const int off = csr_scan(f, &tot);
        if (f) {
            const int p = (int)(key >> 32), q = (int)(key & 0xffffffffull);
            const int64_t w = base + off;
            pool[w] = q;
            atomicAdd(&L.ndeg[ro + p], 1);
            if (i == 0 || (int)(prev >> 32) != p) L.nofs[ro + p] = (int32_t)w;
        }
        base += tot;
    }
    if (tid == 0) {
        L.st[sec].ptop = (int32_t)base;
        L.st[sec].phalf = 0;
    }
}

// Block-wide: copy the live lists of the section densely (slot order) into
// the other half of its pool and switch to it.  st is the block's shared
// copy of the section state.
__device__ void csr_compact(const LevelDev &L, int sec, SecState &st)
{
    const int64_t ro = L.roff[sec];
    const int m0 = st.m0;
    const int64_t hc = L.hcap[sec];
    const int32_t *src = L.nbr + L.pbase[sec] + (int64_t)st.phalf * hc;
    int32_t *dst = L.nbr + L.pbase[sec] + (int64_t)(st.phalf ^ 1) * hc;
    int base = 0;
    for (int s0 = 0; s0 < m0; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        const int d = (s < m0) ? L.ndeg[ro + s] : 0;
        int tot;
        const int off = csr_scan(d, &tot);
        if (d > 0) {
            const int32_t *from = src + L.nofs[ro + s];
            int32_t *to = dst + base + off;
            for (int e = 0; e < d; e++) to[e] = from[e];
            L.nofs[ro + s] = base + off;
        }
        base += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st.phalf ^= 1;
        st.ptop = base;
    }
    __syncthreads();
}

// One warp: in the ascending list l[0..d), which holds b, replace b by a
// (a < b) keeping the order when ins, else remove b.  Returns false when b
// is missing (the list is then left as it was).
__device__ bool csr_warp_replace(int32_t *l, int d, int b, int a, bool ins)
{
    const int lane = threadIdx.x & 31;
    int ib = -1, ia = 0;
    for (int e0 = 0; e0 < d; e0 += 32) {
        const int e = e0 + lane;
        const int v = (e < d) ? l[e] : 0x7fffffff;
        const unsigned mb = __ballot_sync(0xffffffffu, e < d && v == b);
        if (mb && ib < 0) ib = e0 + __ffs(mb) - 1;
        ia += __popc(__ballot_sync(0xffffffffu, e < d && v < a));
    }
    __syncwarp();
    if (ib < 0) return false;
    if (ins) {
        // l[ia .. ib) moves up by one (top chunk first), then a goes to ia
        for (int hi = ib - 1; hi >= ia; hi -= 32) {
            const int e = hi - lane;
            const int v = (e >= ia) ? l[e] : 0;
            __syncwarp();
            if (e >= ia) l[e + 1] = v;
            __syncwarp();
        }
        if (lane == 0) l[ia] = a;
    } else {
        // l[ib + 1 .. d) moves down by one (bottom chunk first)
        for (int lo = ib; lo < d - 1; lo += 32) {
            const int e = lo + lane;
            const int v = (e < d - 1) ? l[e + 1] : 0;
            __syncwarp();
            if (e < d - 1) l[e] = v;
            __syncwarp();
        }
    }
    __syncwarp();
    return true;
}

// Block-wide adjacency update of merging slot b into slot a (a < b):
// a's new list is (list_a \ {b}) U (list_b \ {a}) in order, written at the
// top of the pool (the pool is compacted first when the union and its
// scratch would not fit); every other neighbour r of b gets a in place of b
// (b just removed where a was already a neighbour).  Outputs the old degrees
// of a and b, whether they were adjacent, and a's new degree.
__device__ void csr_merge(const LevelDev &L, int sec, SecState &st, int a, int b, int &pa_o, int &pb_o, int &ab_o,
                          int &pn_o)
{
    const int64_t ro = L.roff[sec];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const int64_t hc = L.hcap[sec];
    const int pa = L.ndeg[ro + a], pb = L.ndeg[ro + b];
    __syncthreads();
    if ((int64_t)st.ptop + pa + 2 * (int64_t)pb + 1 > hc) csr_compact(L, sec, st);
    if ((int64_t)st.ptop + pa + 2 * (int64_t)pb + 1 > hc) {
        // cannot happen (the live lists take at most a third of a half);
        // reported rather than written past the pool
        if (tid == 0 && L.err) atomicExch(L.err, 0x43535232);
        pa_o = pa; pb_o = pb; ab_o = 0; pn_o = pa;
        __syncthreads();
        return;
    }
    int32_t *half = L.nbr + L.pbase[sec] + (int64_t)st.phalf * hc;
    const int32_t *LA = half + L.nofs[ro + a];
    const int32_t *LB = half + L.nofs[ro + b];
    int32_t *NEW = half + st.ptop;                 // the union, pa + pb words reserved
    int32_t *PB = NEW + pa + pb;                   // pb + 1 words: scan of list_b's joining members
    __shared__ int s_bin, s_miss;
    if (tid == 0) {
        const int k = csr_lower_bound(LA, pa, b);
        s_bin = (k < pa && LA[k] == b) ? 1 : 0;
        s_miss = 0;
    }
    for (int j = tid; j < pb; j += nt) {
        const int y = LB[j];
        const int k = csr_lower_bound(LA, pa, y);
        PB[j] = (y != a && !(k < pa && LA[k] == y)) ? 1 : 0;
    }
    __syncthreads();
    int base = 0;
    for (int j0 = 0; j0 < pb; j0 += nt) {          // in place: each thread reads its entry before the scan
        const int j = j0 + tid;
        const int f = (j < pb) ? PB[j] : 0;
        int tot;
        const int off = csr_scan(f, &tot);
        if (j < pb) PB[j] = base + off;
        base += tot;
    }
    if (tid == 0) PB[pb] = base;
    __syncthreads();
    const int bin = s_bin;
    for (int i = tid; i < pa; i += nt) {
        const int x = LA[i];
        if (x == b) continue;
        NEW[i - ((bin && b < x) ? 1 : 0) + PB[csr_lower_bound(LB, pb, x)]] = x;
    }
    for (int j = tid; j < pb; j += nt) {
        if (PB[j + 1] == PB[j]) continue;
        const int y = LB[j];
        NEW[csr_lower_bound(LA, pa, y) - ((bin && b < y) ? 1 : 0) + PB[j]] = y;
    }
    for (int j = wid; j < pb; j += nw) {
        const int r = LB[j];
        if (r == a) continue;
        const bool ins = PB[j + 1] != PB[j];
        int32_t *lr = half + L.nofs[ro + r];
        const int dr = L.ndeg[ro + r];
        const bool ok = csr_warp_replace(lr, dr, b, a, ins);
        if (lane == 0) {
            if (!ok) s_miss = 1;
            else if (!ins) L.ndeg[ro + r] = dr - 1;
        }
    }
    __syncthreads();
    const int pn = pa - bin + base;
    if (tid == 0) {
        L.nofs[ro + a] = st.ptop;
        L.ndeg[ro + a] = pn;
        L.ndeg[ro + b] = 0;
        st.ptop += pn;
        if (s_miss && L.err) atomicExch(L.err, 0x43535231);   // a neighbour list lacked its symmetric entry
    }
    __syncthreads();
    pa_o = pa;
    pb_o = pb;
    ab_o = bin;
    pn_o = pn;
}

}  // namespace rhseg
