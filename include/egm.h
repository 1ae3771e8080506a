/*
 * egm.h - exact epipolar-guided matching on NVIDIA GB300 (sm_103a).
 *
 * C ABI of libegm.so.  The library implements the matching hot path of
 * "Pixel-Accurate Epipolar Guided Matching" (arXiv 2603.18401):
 *
 *   1. epipole e2 = null(F^T)                                 (Algorithm 1)
 *   2. epipolar line l_i = F p~_i^1 of every image-1 query    (Sec. 3)
 *   3. the angle of every image-2 keypoint seen from e2 and the angular
 *      radius of its eps-circle                               (Sec. 4.2)
 *   4. keypoints ordered by (angular-radius level, angle bucket) with a
 *      device counting sort, the replacement of the paper's segment tree
 *                                                              (Sec. 4.2/4.4)
 *   5. stabbing: each query scans the angle window its line can reach and
 *      keeps exactly the keypoints with dist(l_i, p_j) <= eps_j (Eq. 3/4);
 *      or (the banded form) tiles of 128 angle-ordered queries against the
 *      band of keypoints their windows reach, distances on the tensor cores
 *   6. optional candidate lists in CSR form                   (Eq. 4)
 *   7. descriptor distances restricted to the candidates      (Sec. 4.3)
 *   8. best / second best by (distance, index) and Lowe's ratio test
 *      (tau = 0.8 in Sec. 5.1)                                 (Sec. 4.3)
 *
 * Exactness: the candidate set of a query is the set the plain definition
 * (Eq. 4, "<=" as printed) gives when evaluated in IEEE FP64 as
 *     a = (F00 x + F01 y) + F02,  b = ...,  c = ...
 *     dist = |(a x2 + b y2) + c| / sqrt(a a + b b)
 * with one rounding per operation and no fused multiply-add.  Keypoints whose
 * FP32 pre-test is not conclusive are decided by exactly that FP64
 * expression, so results are bit-identical to a brute-force evaluation.
 *
 * Conventions for every entry point:
 *   - Device pointers, unless the entry point's name ends in _host.  The
 *     caller owns every input and output buffer; the library owns only the
 *     scratch memory held by the context (grown on demand, or fixed in
 *     advance by egm_reserve).
 *   - Work is enqueued on the context's CUDA stream.  When params.sync is
 *     1 (the default) a call waits for its own completion and returns the
 *     device-side status; when 0 it returns after enqueueing and
 *     egm_sync() returns the device-side status later.
 *   - Errors never abort or trap the device: kernels record a status word.
 *   - Not thread-safe per context; use one context per host thread.
 */
#ifndef EGM_H
#define EGM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EGM_VERSION 1

typedef struct egm_ctx egm_ctx;

typedef enum egm_status {
    EGM_OK = 0,
    EGM_ERR_ARG = -1,            /* invalid argument (NULL, size, eps <= 0, alignment) */
    EGM_ERR_CUDA = -2,           /* a CUDA runtime call failed */
    EGM_ERR_NOMEM = -3,          /* scratch allocation failed */
    EGM_ERR_CAPACITY = -4,       /* cand_capacity too small; *cand_total holds the need */
    EGM_ERR_DEGENERATE_F = -5,   /* F is zero, or rank < 2 (no epipole) */
    EGM_ERR_NAN = -6,            /* NaN or Inf in F, keypoints or eps */
    EGM_ERR_TIMEOUT = -7,        /* a bounded device wait ran out */
    EGM_ERR_UNIMPLEMENTED = -8
} egm_status;

/* Descriptor kinds (Sec. 4.3 compares descriptors only within C_i). */
enum {
    EGM_DESC_U8_L2 = 0,   /* dim uint8 per row; squared L2, exact int32 */
    EGM_DESC_F32_L2 = 1,  /* dim float32 per row; squared L2 in FP32 */
    EGM_DESC_BIN = 2      /* dim bits per row (dim % 128 == 0); Hamming */
};

/* Per-query result flags. */
enum {
    EGM_FLAG_HAS_BEST = 1,         /* at least one candidate */
    EGM_FLAG_RATIO_PASS = 2,       /* accepted: ratio test passed or no second candidate */
    EGM_FLAG_NO_SECOND = 4,        /* exactly one candidate */
    EGM_FLAG_DEGENERATE_LINE = 8,  /* F p~ has a = b = 0: no line, empty set */
    EGM_FLAG_MUTUAL = 16,          /* egm_match_mutual: the best match's own best is this row */
    EGM_FLAG_GMS = 32              /* egm_gms: the match passed the grid motion-statistics filter */
};

/*
 * One image pair (Sec. 3 "Guided Matching": P1, P2, D1, D2 and F; the
 * tolerance eps of Eq. 4, per image-2 keypoint as in Sec. 4.2).
 *   xy1     [m][2] float64  image-1 keypoints (x, y) in pixels (queries)
 *   xy2     [n][2] float64  image-2 keypoints (references)
 *   F       [9]    float64  row-major fundamental matrix, p2^T F p1 = 0
 *   eps2    [n]    float64  per-keypoint tolerance in pixels, or NULL to
 *                           use eps_scalar for every keypoint; must be > 0
 *   desc1   [m][row]        image-1 descriptors, 16-byte aligned rows
 *   desc2   [n][row]        image-2 descriptors
 *           row = dim bytes (U8_L2), 4*dim bytes (F32_L2), dim/8 bytes (BIN);
 *           row % 16 == 0 and row <= 2048
 *   width, height           image-2 size in pixels.  Only a hint for the
 *                           angular key range; keypoints outside it are
 *                           still handled exactly.  Must be > 0.
 * desc1/desc2 may be NULL, in which case only candidate sets are produced
 * (egm_out.cand_offsets must then be set).
 */
typedef struct egm_pair {
    const double *xy1;
    const double *xy2;
    const double *F;
    const double *eps2;
    const void *desc1;
    const void *desc2;
    int32_t m;
    int32_t n;
    double eps_scalar;
    int32_t kind;
    int32_t dim;
    int32_t width;
    int32_t height;
} egm_pair;

/*
 * Outputs.  For a batch, per-query arrays hold the pairs' queries one pair
 * after another, in pair order (query k of pair p at sum_{q<p} m_q + k), and
 * reference indices are local to the pair's image 2.
 *   best, second   [M] int32   index j of the best / second-best candidate, -1 if none
 *   best_d, second_d [M] float  squared L2 distance (L2 kinds) or Hamming count;
 *                               +inf where there is no such candidate
 *   flags          [M] uint8    EGM_FLAG_* bits
 *   cand_offsets   [M+1] int64  optional (NULL: no candidate lists).  Row k of
 *                               the candidate CSR is cand_idx[off[k] .. off[k+1]),
 *                               ascending in j.
 *   cand_idx       [cand_capacity] int32
 *   cand_total     [1] int64    device: number of candidate entries written or
 *                               needed; required when cand_offsets is set
 * Any of best .. flags may be NULL to skip that output.
 */
typedef struct egm_out {
    int32_t *best;
    int32_t *second;
    float *best_d;
    float *second_d;
    uint8_t *flags;
    int64_t *cand_offsets;
    int32_t *cand_idx;
    int64_t cand_capacity;
    int64_t *cand_total;
} egm_out;

/* Matching forms. */
enum {
    EGM_FORM_AUTO = 0,     /* library choice: banded for batches with more than two
                              128-query tiles per SM, or when every pair has u8
                              descriptors, a scalar eps and an expected 32 or more
                              candidates per query (2 eps n / (W H) x 0.8 of the
                              image diagonal); plain otherwise */
    EGM_FORM_PLAIN = 1,    /* windowed stabbing + CUDA-core descriptor distances */
    EGM_FORM_BANDED = 2    /* angle-banded tiles, descriptor dot products on tensor cores */
};

/* Tensor-core pass of float descriptors in the banded form (Sec. 4.3 on the
 * tensor cores): rows rounded to BF16, or to FP8 E4M3 with one scale per row
 * (max |x| / 448).  Either pass bounds every distance it computes by the
 * rows' rounding errors; the candidates that can be among the best two are
 * then re-ranked in FP32, so both give the plain form's FP32 result. */
enum { EGM_FLOAT_PASS_BF16 = 0, EGM_FLOAT_PASS_FP8 = 1 };

typedef struct egm_params {
    int32_t ratio_num;     /* ratio test tau = num / den, default 4 / 5 (Sec. 5.1) */
    int32_t ratio_den;
    int32_t sync;          /* 1 (default): calls wait and return the device status */
    int32_t form;          /* EGM_FORM_* */
    int32_t band_tile;     /* banded form tile shape: 0 (default) chosen by the tuner (see tune);
                              k = 1..7: shape k - 1, (boxes of 32 references per tensor-core
                              chunk, resident CTAs per SM) = (4, 2), (2, 3), (1, 4), (1, 3),
                              (2, 2), (4, 1), (1, 2) */
    int32_t float_pass;    /* banded form, float descriptors: the tensor-core pass that brackets
                              the distances before the exact FP32 rerank (results are the same):
                              EGM_FLOAT_PASS_BF16 (default) or EGM_FLOAT_PASS_FP8 */
    int32_t timeout_check; /* 0 (default); 1: a check of the device timeout path (no results).
                              Every wait of the banded form's kernel on the device is bounded
                              (2 s); when one gives up, the kernel records EGM_ERR_TIMEOUT, lets
                              the copies and tensor-core operations it issued complete (again
                              bounded), releases its tensor memory and ends.  With 1, each CTA of
                              that kernel first waits 10 us on a barrier that nothing completes,
                              before it issues any copy: banded calls then return
                              EGM_ERR_TIMEOUT and the context stays usable */
    int32_t tune;          /* 1 (default): the library's tuner picks the form (EGM_FORM_AUTO) and the
                              band tile shape (band_tile 0) per call regime -- the number of 128-query
                              tiles (log2), one or several pairs, the descriptor kinds, the expected
                              candidates per query (log2) -- by timing the plain form and every band
                              tile shape on the first call of a regime (that call waits for the
                              device and runs the pipeline 32 times; results are the same in every
                              configuration) and caching the fastest in the context
                              (egm_tuner_export / egm_tuner_import); 0: no timing, a fixed rule */
    int32_t reserved[8];   /* zero */
} egm_params;

/* Context lifetime.  `stream` is a cudaStream_t (NULL: the legacy default stream). */
egm_status egm_create(egm_ctx **ctx, int device, void *stream);
egm_status egm_destroy(egm_ctx *ctx);
egm_status egm_set_stream(egm_ctx *ctx, void *stream);
egm_status egm_set_params(egm_ctx *ctx, const egm_params *params);
egm_status egm_get_params(egm_ctx *ctx, egm_params *params);
void egm_default_params(egm_params *params);

/* Grow the context's scratch to hold at least this many queries,
 * references and pairs per call, so that later calls allocate nothing.
 * Memory management of the library (no counterpart in the paper, whose
 * Algorithm 1 builds its index per call).  EGM_ERR_ARG for negative sizes,
 * EGM_ERR_NOMEM when the device memory is not available. */
egm_status egm_reserve(egm_ctx *ctx, int64_t queries, int64_t refs, int32_t pairs);

/* Match one pair (steps 1-8 above).  Device pointers.
 * Calls on a context are ordered on its stream, with one relaxation: when a
 * call directly follows another call of the context on the stream, its
 * first kernel may read the new F (9 doubles) while the previous call's last
 * kernel still runs; F must therefore not alias the previous call's output
 * arrays.  Every other input is read only after the previous call ended. */
egm_status egm_match_pair(egm_ctx *ctx, const egm_pair *pair, const egm_out *out);

/* Match npairs independent pairs in one pass (one launch per step for the
 * whole batch).  Algorithm 1 applied to each pair (its Match loop over the
 * queries of every pair at once); the pairs share nothing, so the results
 * equal npairs calls of egm_match_pair.  Device pointers; outputs
 * concatenated as described above.  Errors as for egm_match_pair; an invalid
 * pair rejects the whole call before any work. */
egm_status egm_match_batch(egm_ctx *ctx, const egm_pair *pairs, int32_t npairs,
                           const egm_out *out);

/*
 * A batch captured once as a CUDA graph and replayed many times (the same
 * pointers and sizes every time; the data behind the pointers may change).
 * The computation is egm_match_batch's (Algorithm 1 per pair); the graph is
 * a launch mechanism of the library with no counterpart in the paper.
 * The graph owns its own scratch, sized for this batch, and its own copy of
 * the pair table, so ordinary calls on the context in between do not
 * disturb it.  egm_graph_launch enqueues the whole pipeline with one graph
 * launch on the context's stream and, when params.sync is 1, waits and
 * returns the device status.  Device pointers.
 */
typedef struct egm_graph egm_graph;
egm_status egm_graph_create(egm_ctx *ctx, const egm_pair *pairs, int32_t npairs, const egm_out *out,
                            egm_graph **graph);
egm_status egm_graph_launch(egm_graph *graph);
egm_status egm_graph_destroy(egm_graph *graph);

/* As egm_match_pair, but every pointer in *pair and *out is HOST memory
 * (pinned memory gives the fastest copies).  The call stages the inputs to
 * the device, matches, copies the outputs back and waits for completion. */
egm_status egm_match_pair_host(egm_ctx *ctx, const egm_pair *pair, const egm_out *out);

/* Several pairs from HOST memory, each matched on its own as by
 * egm_match_pair (the same kernels, one pair per pipeline), with the copies
 * overlapped: every pair's inputs are queued for upload on a copy stream of
 * the context, and pair k is matched as soon as its inputs are on the device
 * while later pairs are still uploading; each pair's outputs are copied back
 * after its matching.  outs[k] holds pair k's outputs (host memory, m_k rows;
 * no candidate lists: cand_offsets must be NULL, and every pair needs
 * descriptors).  pairs, outs: npairs entries.  The device copies of all the
 * inputs are staged at once (grow-only context memory).  Host buffers should
 * be pinned for the copies to overlap.  The call returns after the last
 * output arrived, with the status of the batch.  EGM_ERR_ARG for invalid
 * pairs or requested candidate lists. */
egm_status egm_match_batch_host(egm_ctx *ctx, const egm_pair *pairs, int32_t npairs, const egm_out *outs);

/*
 * egm_match_pair without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory, e.g.
 * code running under a framework that owns the device allocator and its
 * budget, real-time loops that cannot afford cudaMalloc / cudaFree (which may
 * synchronise the whole device), or plug-ins handed a stream but no context.
 *
 * It takes no egm_ctx and calls no cudaMalloc, cudaFree, cudaMallocHost or
 * other allocating routine.  All scratch lives in one fixed file-scope device
 * array of about 2.4 MB that every GPU loading libegm.so keeps until the
 * process exits; it holds pairs of at most 16384 keypoints per image (m and
 * n); larger pairs are rejected with EGM_ERR_CAPACITY before any work.
 *   pair, out  as for egm_match_pair (device pointers)
 *   params     ratio test (ratio_num / ratio_den); NULL for 4 / 5.  The
 *              sync and form fields are ignored.
 *   stream     cudaStream_t to run on (NULL: the legacy default stream)
 * The call returns after the work finished on `stream`, with the device-side
 * status.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call uses the same array: calls that overlap on the GPU (other
 * streams, other host threads) race and corrupt each other's results.
 */
egm_status egm_match_pair_static(const egm_pair *pair, const egm_out *out, const egm_params *params,
                                 void *stream);

/*
 * The tuner's cache (egm_params.tune): one entry per call regime with the
 * timings of the plain form and of the fastest band tile shape, and the
 * choice.  egm_tuner_export writes it to `buf` (host memory, `capacity`
 * bytes) and *size receives the bytes it needs; with buf NULL only *size
 * is set; EGM_ERR_CAPACITY when capacity < *size.  egm_tuner_import
 * replaces the context's cache with an exported one (for example from an
 * earlier process on the same GPU model), so that calls of those regimes
 * are not timed again; EGM_ERR_ARG if the bytes are not an export of this
 * format.  Layout: a 16-byte header ("EGMT", version 1, entry count, SM
 * count of the device it was measured on, as uint32) and 24 bytes per entry
 * (uint64 regime key, int32 form, int32 shape, float ms_plain, float
 * ms_band).  A tuning method of the library, with no counterpart in the
 * paper.
 */
egm_status egm_tuner_export(egm_ctx *ctx, void *buf, int64_t capacity, int64_t *size);
egm_status egm_tuner_import(egm_ctx *ctx, const void *buf, int64_t size);

/* Wait for the context's stream and return (then clear) the device status. */
egm_status egm_sync(egm_ctx *ctx);

/*
 * Mutual (cross-check) matching: the matching step of Algorithm 1 run in both
 * directions; a match i -> j is kept as mutual when j's best match in the
 * other direction is i.  `fwd` is the pair as for egm_match_pair; `rev` the
 * same images with the roles swapped: xy1 / desc1 of image 2, xy2 / desc2 of
 * image 1, F transposed (p1^T F^T p2 = 0), the tolerance of the image-1
 * keypoints, and image 1's width and height.  rev->m must equal fwd->n and
 * rev->n fwd->m, with the same descriptor kind and dimension.  `out` has
 * fwd->m + fwd->n rows: [0, m) the forward results, [m, m + n) the reverse
 * ones (indices local to each direction); every row whose best match is
 * mutual gets EGM_FLAG_MUTUAL.  No candidate lists (cand_offsets NULL).
 */
egm_status egm_match_mutual(egm_ctx *ctx, const egm_pair *fwd, const egm_pair *rev, const egm_out *out);

/* egm_match_mutual from the forward pair alone: the library forms the
 * reverse direction itself (image-2 keypoints and descriptors as queries,
 * image 1's as references, F^T computed on the device into context scratch,
 * Sec. 3).  eps1 [m] float64 (device): the tolerance of each image-1
 * keypoint, or NULL to use eps1_scalar (> 0); width1, height1: image 1's
 * size in pixels.  out as for egm_match_mutual (m + n rows).  Errors as for
 * egm_match_mutual. */
egm_status egm_match_mutual_pair(egm_ctx *ctx, const egm_pair *fwd, const double *eps1, double eps1_scalar,
                                 int32_t width1, int32_t height1, const egm_out *out);

/*
 * The compact list of matches: (qi[k], rj[k]) = (i, best[i]) for every row
 * i < m whose flags contain every bit of `require` (for example
 * EGM_FLAG_RATIO_PASS | EGM_FLAG_MUTUAL), in ascending i; *count receives
 * their number.  flags, best: m entries; qi, rj: room for m; count: one
 * int64.  Device pointers.  This library extension has no counterpart in the
 * paper beyond its output "matches" (Algorithm 1).
 */
egm_status egm_compact_matches(egm_ctx *ctx, const uint8_t *flags, const int32_t *best, int64_t m,
                               uint32_t require, int32_t *qi, int32_t *rj, int64_t *count);

/*
 * Grid-based motion statistics filter (GMS, Bian et al. 2017), the filter the
 * paper applies to its guided matches by default with the neighbour
 * threshold 6 (Sec. 5.1; Sec. 4.3).  The input matches are the rows i < m
 * with 0 <= best[i] < n whose flags contain every bit of `require` (for
 * example EGM_FLAG_HAS_BEST: every query's best candidate).  Both images are
 * cut into grid x grid cells; a match from image-1 cell c to image-2 cell d
 * is kept when d is the cell receiving most of c's matches (the lowest
 * d = dy * grid + dx on ties) and the matches between the 3 x 3
 * neighbourhoods of c and d number more than alpha * sqrt(n / 9), n the
 * matches in c's neighbourhood; image-1 grids shifted by (0 or 1/2,
 * 0 or 1/2) cell are tried and their keeps united.  Cells are computed as
 * floor(x * grid / width) in FP64.
 *   xy1 [m][2], xy2 [n][2] float64; best [m] int32; flags [m] uint8, updated
 *   in place: EGM_FLAG_GMS set on kept input matches, cleared on every other
 *   row.  Device pointers, asynchronous on the context stream.
 *   width1 .. height2 > 0 (image sizes in pixels); 1 <= grid <= 48 (GMS
 *   uses 20); alpha > 0 (6).  m <= 2^31 - 1.  EGM_ERR_ARG otherwise.
 */
egm_status egm_gms(egm_ctx *ctx, const double *xy1, int64_t m, const double *xy2, int64_t n, const int32_t *best,
                   uint8_t *flags, int32_t width1, int32_t height1, int32_t width2, int32_t height2,
                   uint32_t require, int32_t grid, double alpha);

/* egm_gms over several pairs in one call (one set of launches; pairs are
 * filtered independently).  Each entry as the arguments of egm_gms, device
 * pointers; m <= 2^31 - 1 in total.  EGM_ERR_ARG if any entry is invalid
 * (nothing is launched then). */
typedef struct egm_gms_pair {
    const double *xy1;
    const double *xy2;
    const int32_t *best;
    uint8_t *flags;
    int64_t m, n;
    int32_t width1, height1, width2, height2;
} egm_gms_pair;

egm_status egm_gms_batch(egm_ctx *ctx, const egm_gms_pair *pairs, int32_t npairs, uint32_t require, int32_t grid,
                         double alpha);

/*
 * The paper's interval view, for inspection and tests (Sec. 4.2, Eq. theta
 * and delta; Algorithm 1 preprocessing), computed on the device in FP64:
 *   e3     [3] float64   epipole e2 = null(F^T), unit norm, e_w >= 0
 *   mode   [1] int32     0: finite epipole (angular), 1: epipole at or near
 *                        infinity (parallel lines; theta/delta not defined)
 *   theta  [n] float64   atan2(y_j - y_e, x_j - x_e) reduced to [0, pi)
 *   delta  [n] float64   asin(eps_j / ||p_j - e2||), or pi/2 when
 *                        ||p_j - e2|| <= eps_j (full interval)
 * In parallel mode theta/delta receive NaN.  Device pointers; any may be NULL.
 */
egm_status egm_intervals(egm_ctx *ctx, const egm_pair *pair, double *theta, double *delta,
                         double *e3, int32_t *mode);

/*
 * Learned per-keypoint tolerance.  The paper names per-point tolerances as a
 * promising direction (Sec. 6) without a model; this network, its features
 * and its loss are the library's reading:
 *   features  (ln s, orientation / 2 pi, ln response, x / W, y / H) computed
 *             on the device from raw [n][5] float32 rows
 *             (scale s > 0, orientation in radians, response > 0, x / W, y / H)
 *   network   5 -> 64 -> 64 -> 64 -> 1, GELU, eps = softplus(z) + 0.25 px;
 *             FP32 master weights rounded to BF16 for every product, FP32 sums
 *   training  pinball (quantile) loss of the residual r - eps at quantile q,
 *             Adam (0.9, 0.999, 1e-8); r = distance of a true match from its
 *             epipolar line (Eq. 3), see egm_pair_residuals
 * Parameters are a flat float32 vector of EGM_MLP_PARAMS values:
 * W1 (64x5), b1, W2 (64x64), b2, W3 (64x64), b3, W4 (1x64), b4, rows = outputs.
 * The object holds the parameters, the Adam moments and the step count on
 * the context's device; calls run on the context's stream and wait for it.
 */
#define EGM_MLP_PARAMS 8769
typedef struct egm_mlp egm_mlp;
egm_status egm_mlp_create(egm_ctx *ctx, const float *params, egm_mlp **mlp);   /* params: host */
egm_status egm_mlp_destroy(egm_mlp *mlp);
/* Checkpoint (host pointers, any may be NULL). */
egm_status egm_mlp_get_state(egm_mlp *mlp, float *params, float *adam_m, float *adam_v, int64_t *step);
egm_status egm_mlp_set_state(egm_mlp *mlp, const float *params, const float *adam_m, const float *adam_v,
                             int64_t step);
/* eps [n] float64 (device) for features [n][5] float32 (device); the output
 * can be passed as egm_pair.eps2.  Layers 2 and 3 run on the tensor cores
 * (tcgen05.mma, BF16 weights; each FP32 activation enters as the sum of two
 * BF16 parts, so results agree with FP32 products to about 1e-6 relative).
 * Fixed-tolerance fallback: a sample whose network output is not a finite
 * tolerance (NaN / Inf features, or weights that overflow) receives the
 * fallback tolerance (2 px, see egm_mlp_set_fallback) instead, so every
 * output is a valid egm_pair.eps2 entry.  EGM_ERR_TIMEOUT if a tensor-core
 * wait gave up: the samples of the blocks concerned receive the fallback. */
egm_status egm_mlp_infer(egm_mlp *mlp, const float *feat, int64_t n, double *eps);
/* The fallback tolerance of egm_mlp_infer in pixels (default 2, the fixed
 * tolerance the learned one is compared with).  EGM_ERR_ARG unless finite
 * and > 0. */
egm_status egm_mlp_set_fallback(egm_mlp *mlp, double eps_px);
/* Gradient of the mean pinball loss (device outputs: grad [EGM_MLP_PARAMS], loss [1]).
 * The forward pass of training runs as egm_mlp_infer's (layers 2 and 3 on
 * the tensor cores) and also keeps the pre-activations for the backward
 * pass (CUDA cores, FP32).  EGM_ERR_TIMEOUT if a tensor-core wait gave up in
 * this call or in an egm_mlp_train_step since the last report (the steps
 * concerned used stale activations); egm_mlp_get_state reports it too. */
egm_status egm_mlp_grad(egm_mlp *mlp, const float *feat, const float *resid, int64_t n, float quantile, float *grad,
                        float *loss);
/* One Adam step on a batch; loss [1] (device, may be NULL) receives the batch loss. */
egm_status egm_mlp_train_step(egm_mlp *mlp, const float *feat, const float *resid, int64_t n, float lr,
                              float quantile, float *loss);

/* Exact distances (Eq. 3, the brute force's FP64 evaluation) of the pairs
 * (qi[t], rj[t]) of one image pair: dist [k] float64.  Device pointers; only
 * xy1, xy2, F, m and n of the pair are read.  An index outside [0, m) or
 * [0, n) gives NaN; a degenerate line (a = b = 0) gives +inf. */
egm_status egm_pair_residuals(egm_ctx *ctx, const egm_pair *pair, const int32_t *qi, const int32_t *rj, int64_t k,
                              double *dist);

/* Work counters of the last match call, for metrics (host memory). */
typedef struct egm_stats {
    int64_t queries;        /* queries processed */
    int64_t refs;           /* reference keypoints processed */
    int64_t window_refs;    /* references visited inside the stabbing windows */
    int64_t candidates;     /* candidate pairs found */
    int64_t fp64_rechecks;  /* pairs decided by the FP64 exact test */
} egm_stats;

/* Enables (1) or disables (0, default) the work counters, then reads them.
 * Reading waits for the stream. */
egm_status egm_set_counters(egm_ctx *ctx, int32_t enable);
egm_status egm_get_stats(egm_ctx *ctx, egm_stats *stats);

/* Per-stage device time, measured with CUDA events that the library records
 * on its own stream around each stage of every match call while timing is
 * enabled.  Times are sums over the calls since the last egm_set_timing(1). */
typedef struct egm_timing {
    double geometry_ms;   /* epipole and key frame */
    double prep_ms;       /* reference keys, query lines, bucket tables zeroed */
    double sort_ms;       /* reference counting sort by (level, angle bucket):
                             bucket counts, scan, placement of the records */
    double post_sort_ms;  /* banded form: query order and operand packing;
                             plain form: nothing */
    double stab_ms;       /* the matching kernel (plain: stabbing, exact test,
                             descriptors, top-2, ratio; banded: the same on
                             tensor-core tiles) */
    double csr_ms;        /* candidate lists: count, scan, fill, row sort */
    int64_t calls;        /* match calls timed */
    int64_t banded_calls; /* of which ran the banded form */
} egm_timing;

/* Enables (1, also resets the sums) or disables (0) per-stage timing. */
egm_status egm_set_timing(egm_ctx *ctx, int32_t enable);
/* Waits for the stream and returns the sums. */
egm_status egm_get_timing(egm_ctx *ctx, egm_timing *timing);

const char *egm_status_string(egm_status status);
int32_t egm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EGM_H */
