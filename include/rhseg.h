/*
 * rhseg.h -- C ABI of the B300 (sm_103a) RHSEG/HSEG hot path.
 *
 * The method: recursive hierarchical segmentation of a hyperspectral image
 * (thesis "High Performance Hyperspectral Image Classification using
 * Graphics Processing Units", 2015, Section 4.1).  HSEG (Section 4.1, steps
 * 1-4) starts from one region per pixel and repeats: merge the spatially
 * adjacent pair of minimum dissimilarity; then merge the non-adjacent pair of
 * minimum dissimilarity if it is below the adjacent minimum scaled by the
 * spectral clustering weight; until the target region count.  The
 * dissimilarity is the square root of the band-sum mean squared error
 * (Eq. 1).  RHSEG (Section 4.1, Fig. 4.3/4.4) runs HSEG on 4^(L-1) sections,
 * reassembles them four at a time (regions on the seams linked across,
 * 8-neighbourhood) and runs HSEG again up to the whole image.
 *
 * Conventions the thesis leaves open, fixed here (identical in every
 * precision form; results are bit-exact across forms):
 *   - K = d^2 = N / D, N = sum_b (n_j S_ib - n_i S_jb)^2, D = n_i n_j (n_i+n_j)
 *     from exact int64 band sums S and counts n; K is the correctly rounded
 *     binary64 of the exact rational; dissim = sqrt(K).
 *   - ties broken on (K, smaller region ID, larger region ID); region ID =
 *     1 + smallest raster index (row * cols + col) of its pixels; the
 *     survivor of a merge keeps the smaller ID.
 *   - spectral step on the state after the adjacent merge of the same
 *     iteration, non-adjacent pairs only, merge iff K < (w*w) * K_adj
 *     (binary64; +inf when no adjacent pair is left; w = 0: no spectral step).
 *   - stop test before each iteration and after every merge; an iteration
 *     that merges nothing stalls the section (not an error).
 *   - sections split at floor(h/2), floor(w/2), children in Z order.
 *   - seam pass at each reassembly (the boundary-artifact removal that
 *     Section 6.2 names as future work): a pixel with a neighbour in another
 *     child section leaves its region R and becomes a one-pixel region iff
 *     min over those neighbours' regions Q of K({p}, Q) < K({p}, R); all
 *     tests on the pre-pass state, applied together, IDs re-derived.
 *   - output levels: c_0 = count at the start of the root HSEG,
 *     c_{K-1} = conv_nregions, geometric in between (nearest-even),
 *     duplicates removed; labels renumbered 1..R in raster order of first
 *     appearance (= ID order).
 *
 * Error behaviour: every call returns 0 (RHSEG_OK) or a negative code;
 * rhseg_strerror() names it.  No call aborts the process.
 * Threading: a handle is not thread-safe; distinct handles are independent.
 */
#ifndef RHSEG_H
#define RHSEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RHSEG_OK = 0,
    RHSEG_EINVAL = -1,    /* bad dimensions or parameters                          */
    RHSEG_ERANGE = -2,    /* exact-key bound fails: B*(P^2/4*maxval)^2 >= 2^127 or
                             P^2/4*maxval >= 2^62 (P = unmasked pixels)           */
    RHSEG_ENOMEM = -3,    /* device allocation failed                              */
    RHSEG_ECUDA = -4,     /* a CUDA call failed (message via rhseg_last_cuda_error) */
    RHSEG_ETIMEOUT = -5,  /* a bounded device wait gave up                         */
    RHSEG_ESTATE = -6,    /* call out of order (e.g. get_level before run)          */
    RHSEG_ETRUNC = -7,    /* output buffer too small; the needed size is returned  */
    RHSEG_EDEVICE = -8    /* no usable sm_103a device                              */
};

/* Parameters (Section 4.1; L, spectral clustering weight and the number of
 * classes are the thesis's inputs). */
typedef struct rhseg_params {
    int32_t rnb_levels;    /* 1 <= L <= 6: the deepest level has 4^(L-1) sections   */
    int32_t conv_nregions; /* final region count of the root HSEG (>= 1)            */
    double  spclust_wght;  /* w in [0, 1]; 0 disables spectral merges (HSWO)        */
    int32_t connectivity;  /* 4 or 8 (8 is the thesis's reassembly neighbourhood)   */
    int32_t min_nregions;  /* per-section target below the root; 0 -> conv_nregions */
    int32_t n_out_levels;  /* hierarchy snapshots kept at the root; 0 -> 1          */
    int32_t seam_pass;     /* 1: boundary-artifact split pass at each reassembly    */
    int32_t precision;     /* screen of the spectral step (results identical):
                              0 = FP64 on CUDA cores (the plain form),
                              1 = FP16 region means on tcgen05 tensor cores, FP32 accumulate,
                              2 = BF16 region means on tcgen05 tensor cores, FP32 accumulate,
                              3 = FP32 on CUDA cores (the thesis kernel's arithmetic, Fig. 4.8).
                              There is no TF32 form: FP16 rows have TF32's unit roundoff
                              (2^-11) at twice its tensor rate and half its bytes, and the
                              operand scale 2^-s keeps them inside FP16's range. */
    int32_t profile;       /* 1: time every step kernel with CUDA events (stats *_ms) */
    int32_t incremental;   /* 1: keep every region's exact best non-adjacent partner and
                              recompute only the rows a merge touches, instead of screening
                              all pairs each iteration (results identical; needs the
                              binary32 rows, precision 3, else RHSEG_EINVAL).  The level-start pass and the row
                              updates are timed as the screen (stats screen_ms). */
    int32_t multi_merge;   /* 1: several merges per HSEG iteration (Section 6.2 names the
                              idea; reading R12): in each step every region takes its
                              best partner, and all mutually best pairs merge, smallest
                              key first, until the target.  The spectral threshold is
                              (w*w) times the iteration's smallest adjacent key.  Results
                              differ from the single-merge rule (0, default) and match
                              the oracle's multi-merge mode.  Not with incremental = 1
                              (RHSEG_EINVAL). */
    int64_t wait_cycles;   /* bound, in SM clock cycles, of every wait inside the
                              tensor-core screen's pipeline (a load or MMA that never
                              completes, a stalled partner warp); 0 = the default,
                              4e9 cycles (about 2 s).  A wait that runs out makes the
                              screen stop, release its tensor memory and set an error
                              that rhseg_run returns as RHSEG_ETIMEOUT; the handle stays
                              usable (the next run starts over from the image). */
    int32_t screen_group;  /* CTA-pair form of the tensor-core screen: K slices (32
                              bands each) whose MMAs share one tcgen05.commit, 1..8,
                              0 = the default (4); a choice of the autotuner (results
                              identical).  The one-CTA form always groups 4 */
    int32_t screen_pair;   /* tensor-core screen: 1 = CTA-pair form (two CTAs of a cluster
                              share each 256x256 tile through tcgen05 cta_group::2 MMAs,
                              M = 256: each CTA loads 16 KB per K slice instead of 24 KB);
                              0 = one CTA per 128x256 unit.  Results identical; a
                              schedule choice of the autotuner */
    int32_t adjacency;     /* region adjacency of a section (Section 4.1): 0 = dense bit
                              matrix, m0^2 / 8 bytes for m0 regions at the level start
                              (default); 1 = sorted neighbour lists in a per-section pool,
                              memory in proportion to the region edges (at most 10 words per
                              directed pixel edge, build scratch included), for large
                              sections.  Results identical.  Not with incremental = 1
                              (RHSEG_EINVAL) */
    int32_t reserved;      /* set to 0 */
} rhseg_params;

/* One merge-log record.  kind 0 = adjacent merge, 1 = spectral merge,
 * 2 = seam split (survivor_id = region the pixel left, absorbed_id = the new
 * one-pixel region's ID, key = K({p}, R), step = 0).  Canonical order:
 * levels deepest first, sections in Z order, within a section the seam
 * splits (raster order) then the HSEG merges in order; step counts HSEG
 * iterations from 1. */
typedef struct rhseg_merge {
    int32_t level, section, step, kind;
    int64_t survivor_id, absorbed_id;
    double  key;            /* K = d^2, correctly rounded binary64           */
    double  dissim;         /* sqrt(K), Eq. 1                                  */
    int32_t nregions_after; /* section's region count after this record      */
    int32_t pad;
} rhseg_merge;

typedef struct rhseg_stats {
    int64_t pairs;            /* dissimilarities the method defines: adjacent pairs
                                 of each adjacent step + non-adjacent pairs of each
                                 spectral step                                    */
    int64_t iterations;       /* HSEG iterations over all sections                */
    int64_t merges_adj, merges_spec, seam_splits;
    int64_t screened_pairs;   /* pairs the spectral screen evaluated              */
    int64_t candidates;       /* pairs the screen passed to the exact re-check    */
    int64_t fallbacks;        /* spectral steps resolved by exhaustive exact keys */
    int32_t stalled_sections, n_levels_out;
    double  run_ms;           /* device time of the last rhseg_run                */
    int64_t kernel_launches;  /* kernels launched by the last rhseg_run            */
    int64_t candidates_below; /* candidates that were non-adjacent with exact K below
                                 the threshold (the rest were screen false positives) */
    int64_t screen_launches;  /* spectral-screen launches                          */
    double  screen_ms, adj_ms, spec_ms;  /* summed device time per step kernel
                                            (profile = 1 only, else 0)            */
    int32_t screen_impl;      /* 0 none, 1 FP64 CUDA cores, 2 FP32-accumulate CUDA
                                 cores, 3 tcgen05 tensor cores                    */
    int32_t pad;
    double  level_ms[6];      /* device time of each recursion level (index
                                 level-1), set-up and HSEG iterations             */
    int32_t level_iters[6];   /* HSEG iterations run at each level (max over
                                 its sections)                                    */
    double  level_screen_ms[6], level_adj_ms[6], level_spec_ms[6];
                              /* per level split of screen_ms, adj_ms, spec_ms
                                 (profile = 1 only)                               */
    int64_t screen_evaluated; /* pairs the tensor-core screen's MMAs actually covered
                                 (whole 128x256 units; units whose norm ranges prove
                                 every pair's key >= the threshold are skipped)    */
    int64_t device_allocs;    /* device allocations (cudaMalloc calls) the library has
                                 made in this process so far, over all handles; read
                                 when rhseg_get_stats is called                    */
    double  screen_err_rel_max;   /* tensor-core screen (precision 1, 2): over the
                                     re-checked candidate pairs, max |K~ - K| / K, where
                                     K~ = c 4^s (q_i + q_j - 2 g) is the screen's own
                                     estimate of the key from its binary32 Gram value g
                                     and row norms q, and K the exact key; 0 otherwise */
    double  screen_err_bound_max; /* max |K~ - K| / bound over the same pairs: the
                                     screen's error model holds iff this is <= 1    */
    int64_t screen_err_pairs;     /* re-checked pairs the two maxima cover         */
    int64_t level_screen_evaluated[6];  /* per level (index level-1) split of
                                           screen_evaluated                    */
    int64_t adjacency_bytes;  /* largest device memory the region adjacency of one
                                 level took in the last rhseg_run (bit matrices, or
                                 lists, offsets and their build scratch)           */
    int64_t screen_useful;    /* of screen_evaluated, the pairs (i, j), i < j, of
                                 positions in use (the rest: the lower triangle of
                                 diagonal units, rows past the last position, and
                                 the CTA-pair form's padding halves); counted with
                                 profile = 1 only, else 0                          */
} rhseg_stats;

typedef struct rhseg_handle rhseg_handle;

/* Create from HOST buffers (the hyperspectral cube of Section 4.1, one
 * region per pixel at the start).  image: [rows][cols][bands] uint16 (copied);
 * mask: [rows][cols], nonzero = no data, or NULL.  Device memory is
 * allocated here (cudaMalloc) and owned by the handle.  The copy runs on
 * `cuda_stream` (a cudaStream_t, NULL = legacy default stream). */
int rhseg_create(const uint16_t *image, int32_t rows, int32_t cols, int32_t bands,
                 const uint8_t *mask, const rhseg_params *p, void *cuda_stream,
                 rhseg_handle **out);

/* Create from DEVICE buffers that stay owned by the caller and must outlive
 * the handle (same layouts as rhseg_create; read only). */
int rhseg_create_device(const uint16_t *image_dev, int32_t rows, int32_t cols, int32_t bands,
                        const uint8_t *mask_dev, const rhseg_params *p, void *cuda_stream,
                        rhseg_handle **out);

/* Replace the image (and mask) of a handle made by rhseg_create with new
 * HOST buffers of the same shape; the copy runs on `cuda_stream` (NULL = the
 * handle's stream) and is ordered before the next rhseg_run on that stream.
 * The mask must be given iff the handle was created with one.  Pinned host
 * memory makes the copy asynchronous; the buffers must stay valid until the
 * next rhseg_run returns.  RHSEG_ESTATE for handles of rhseg_create_device;
 * RHSEG_ERANGE if the new image breaks the exact-key bound. */
int rhseg_set_image(rhseg_handle *h, const uint16_t *image, const uint8_t *mask, void *cuda_stream);

/* Run the whole recursion (Section 4.1: HSEG steps 1-4 on every section of
 * the deepest level, then reassembly and HSEG at each level up to the whole
 * image; Fig. 4.3/4.4) on `cuda_stream` (NULL = the handle's stream) and wait
 * for it.  May be called again; each call recomputes from the image.
 * RHSEG_ETIMEOUT when a bounded device wait gave up (see wait_cycles); the
 * run stops at the next check (at most 32 HSEG iterations later) and its
 * results are not available (RHSEG_ESTATE from the getters). */
int rhseg_run(rhseg_handle *h, void *cuda_stream);

/* Change the wait bound of a handle (rhseg_params.wait_cycles; 0 = the
 * default) for its next runs.  No device work; the paper has no
 * counterpart (failure detection of this library). */
int rhseg_set_wait_cycles(rhseg_handle *h, int64_t cycles);

/* Number of hierarchy levels kept at the root (valid after run). */
int rhseg_n_levels(const rhseg_handle *h, int32_t *n_levels);

/* One hierarchy level (the output levels of hierarchical segmentation,
 * Section 4.1, Fig. 4.1:
 * coarser levels are unions of finer regions), 0 = finest kept ...
 * n_levels-1 = conv_nregions.
 * labels: host [rows*cols] int32 (0 = masked, 1..R canonical) or NULL;
 * band_sums: host [R*bands] int64 by canonical label or NULL;
 * counts: host [R] int64 or NULL; nregions_out: R (may be NULL).
 * Pass NULL outputs first to learn R. */
int rhseg_get_level(rhseg_handle *h, int32_t level, int32_t *labels, int64_t *band_sums,
                    int64_t *counts, int32_t *nregions_out);

/* Largest root-level region count rhseg_get_level_noalloc accepts. */
#define RHSEG_NOALLOC_MAX_REGIONS 65536

/* Same result as rhseg_get_level, written straight into caller-owned DEVICE
 * buffers, for callers that may not allocate device memory once they are
 * running: for example a service that reserves its whole device-memory
 * budget at start-up, or code embedded in a framework whose allocator owns
 * all of the device memory.  This call makes no device allocation of any
 * kind; the handle's own buffers were allocated by rhseg_create and
 * rhseg_run before.  The paper has no counterpart (it is an interface
 * choice of this library).
 *   labels_dev    [rows*cols] int32 or NULL
 *   band_sums_dev [regions_cap*bands] int64 or NULL (first R rows cleared, then filled)
 *   counts_dev    [regions_cap] int64 or NULL (first R entries cleared, then filled)
 *   nregions_out  host int32: R of this level (may be NULL)
 * The kernels run on the handle's stream, which does not wait for other
 * streams: the caller's earlier work on these buffers must be complete
 * (synchronise the stream that wrote them) before the call.  The current
 * device must be the one the handle was created on (else RHSEG_EDEVICE).
 * RHSEG_ETRUNC if R > regions_cap while sums or counts are requested: R is
 * still returned and no buffer is written.  The working array (one int32 per root region) is a
 * fixed, file-scope device array of RHSEG_NOALLOC_MAX_REGIONS + 1 entries
 * that every GPU using the library holds until the process exits; a root
 * level that started with more regions is rejected with RHSEG_ERANGE.  The
 * first call on a device looks up that array's device address once, so
 * make the first call before any stream capture.  All calls share the one
 * array: calls that overlap on the GPU (other host threads, other streams)
 * race on it.  Runs on the handle's stream and waits for completion. */
int rhseg_get_level_noalloc(rhseg_handle *h, int32_t level, int32_t *labels_dev, int64_t *band_sums_dev,
                            int64_t *counts_dev, int32_t regions_cap, int32_t *nregions_out);

/* Full canonical merge log (every merge of HSEG steps 2-3, Section 4.1, and
 * every seam split) into host `log` (capacity log_cap records).
 * *log_len receives the number of records; RHSEG_ETRUNC if log_cap is
 * smaller (nothing written).  log may be NULL to query the length. */
int rhseg_get_log(rhseg_handle *h, rhseg_merge *log, int64_t log_cap, int64_t *log_len);

int rhseg_get_stats(const rhseg_handle *h, rhseg_stats *s);

void rhseg_destroy(rhseg_handle *h);

const char *rhseg_strerror(int code);
const char *rhseg_last_cuda_error(void);

/* Exact keys (Eq. 1 squared) for explicit region pairs on the device: for t < npairs,
 * out[t] = K(pair_i[t], pair_j[t]) from band sums S (int64 [nreg][bands],
 * row stride `stride` elements) and counts n (int64 [nreg]).  All pointers
 * are device pointers; runs on `cuda_stream` and does not wait. */
int rhseg_keys(const int64_t *S, const int64_t *n, int32_t nreg, int32_t bands, int32_t stride,
               const int32_t *pair_i, const int32_t *pair_j, int32_t npairs, double *out,
               void *cuda_stream);

/* Correctly rounded binary64 of N/D for 128-bit N, D given as (hi, lo)
 * uint64 pairs, device pointers, n values (diagnostic of the key's final
 * rounding).  Does not wait. */
int rhseg_div_rn(const uint64_t *n_hi, const uint64_t *n_lo, const uint64_t *d_hi,
                 const uint64_t *d_lo, int32_t n, double *out, void *cuda_stream);

/* Diagnostic of the tensor-core screen's contraction: G = X X^T in FP32 for
 * X = [rows][Bpad] FP16 (precision 1) or BF16 (precision 2) device rows,
 * rows a multiple of 128, Bpad a multiple of 32 and at most 4096, cta_pair
 * 0 (one-CTA form) or 1 (CTA-pair form, as params.screen_pair) (else
 * RHSEG_EINVAL); G [rows][rows] device float.  Uses the same TMA/tcgen05
 * main loop as the spectral screen (Section 4.2's spectral kernel, here as
 * a Gram contraction).  Does not wait. */
int rhseg_gram_tc(const void *X, int32_t rows, int32_t Bpad, int32_t precision, int32_t cta_pair, float *G,
                  void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* RHSEG_H */
