// Internal declarations shared by the libegm translation units.
//
// Data layout in device memory (one call, `npairs` pairs):
//   PairDesc[npairs]   caller pointers, sizes and offsets into the scratch
//   PairGeom[npairs]   epipole, key frame, per-level statistics and tables
//   per reference (sum of n over pairs, pair p at r_off):
//     key_a/val_a      unsorted (level|angle-key, local index) pairs
//     key_c            scratch of the CSR long-row sort
//     rec              float4 (x - cx, y - cy, eps, index bits) in bucket order
//   tab                per (pair, level) bucket -> first sorted position
//   curs               bucket fill cursors while the records are placed
//   banded form: query order; for float pairs sorted query records and
//                packed operand rows
//   per query (sum of m, pair p at q_off):
//     QueryRec         FP32 line in the pair frame, window centre, pad terms
//     qcount           candidates per query (CSR path)
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <stdint.h>

#include "../../include/egm.h"

namespace egm {

// ------------------------------------------------------------ dependent launch
// The pipeline's kernels are launched with programmatic stream serialization:
// a kernel may be scheduled while its predecessor in the stream finishes.
// pdl_begin(), the first statement of every such kernel, waits until the
// predecessor has completed and its memory is visible (so no kernel touches
// global memory early) and then lets the successor be scheduled.  For a
// kernel launched without the attribute both instructions return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_begin() {
    pdl_wait();
    pdl_trigger();
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}


constexpr int kLevels = 32;        // angular-radius levels (5 bits of the sort key)
constexpr int kQBits = 22;         // quantised key bits within a level
constexpr uint32_t kQMax = (1u << kQBits) - 1u;
constexpr int kKeyBits = kQBits + 5;
constexpr float kPiF = 3.14159265358979f;
constexpr float kHalfPiF = 1.57079632679490f;

// Device status bits (combined with atomicOr, mapped to egm_status on the host).
enum : uint32_t {
    kStNan = 1u,
    kStArg = 2u,
    kStDegenerateF = 4u,
    kStCapacity = 8u,
    kStTimeout = 16u,
};

enum : int32_t { kModeAngular = 0, kModeParallel = 1 };

struct __align__(16) PairDesc {
    const double *xy1;
    const double *xy2;
    const double *F;
    const double *eps2;
    const uint8_t *desc1;
    const uint8_t *desc2;
    double eps_scalar;
    int32_t m, n;
    int32_t kind, dim, row_bytes;
    int32_t width, height;
    int32_t pad0;
    int64_t q_off;      // first query of this pair in per-query arrays
    int64_t r_off;      // first reference in per-reference arrays
    int64_t t_off;      // first bucket-table entry
    int64_t t_cap;      // bucket-table entries reserved for this pair
};

struct __align__(16) PairGeom {
    double ex, ey, ew;          // homogeneous epipole, unit norm, ew >= 0
    double xe, ye;              // Euclidean epipole (angular mode)
    double cx, cy;              // frame origin: image centre
    float ux, uy;               // angular: unit vector from the epipole to the centre; parallel: line direction
    float de;                   // angular: |centre - epipole|
    float kappa;                // angular: -u x (epipole - centre), the rounding residue of the frame
    float kmin, kscale;         // key quantisation q = clamp((k - kmin) * kscale)
    int32_t mode;               // kModeAngular / kModeParallel
    int32_t level_base;         // level = clamp(ilogb(d/eps) - level_base, 1, kLevels-1)
    float Ff[9];                // F rounded to FP32 (magnitudes for error terms)
    int32_t pad0;
    // per-level statistics, written with atomics by the prep kernel
    uint32_t cnt[kLevels];      // members
    uint32_t smax[kLevels];     // float bits: upper bound of eps/d (angular) or eps (parallel)
    uint32_t dmin[kLevels];     // float bits: lower bound of d (angular)
    uint32_t tmax[kLevels];     // float bits: upper bound of |p - c|
    // filled by the sort kernel
    uint32_t start[kLevels + 1];  // first sorted position of each level
    uint32_t tab[kLevels];        // table offset (relative to t_off)
    int32_t bits[kLevels];        // bucket bits of each level
    // extremes over the pair's queries with an FP32 view, written with atomics
    // by the prep kernel (float bits of non-negative values): the largest
    // aux0 (angular: r_i), the smallest aux0 and the largest aux1 (parallel:
    // cos phi and |sin phi|), the largest |key|
    uint32_t qa0max, qa0min, qa1max, qkabs;
    float cxf, cyf, xef, yef;     // cx, cy, xe, ye rounded to FP32 (for error terms)
    // angular: upper bounds of |v_k|, v = F^T (xe, ye, 1), the residual of the
    // computed epipole; p . v is the exact line of p = (x1, y1, 1) evaluated
    // at (xe, ye)
    float vb[3];
    int32_t pad1;
};

static_assert(sizeof(PairGeom) % 16 == 0, "PairGeom is copied in 16-byte units");
static_assert(sizeof(PairDesc) % 16 == 0, "PairDesc is copied in 16-byte units");

// Query flags beyond the public EGM_FLAG_* bits.
enum : uint32_t { kQExactOnly = 0x100u };  // FP32 view unusable: whole levels, FP64 decides every pair

// FP32 view of one query, written by the prep kernel.
struct __align__(16) QueryRec {
    float A, B, C;      // normalised line in the pair frame: dist = |A x' + B y' + C|
    float key;          // angular: folded line angle; parallel: offset along the normal
    float aux0;         // angular: r_i upper bound (px); parallel: cos(phi)
    float aux1;         // parallel: |sin(phi)|
    float E0, E1;       // line error terms of the pre-test: E0 + E1 (|x'| + |y'| + 2 eps)
    uint32_t flags;     // EGM_FLAG_DEGENERATE_LINE, kQExactOnly
    int32_t pair;       // pair of this query
    uint32_t pad[2];
};

// Queries per block of the stabbing kernel.
constexpr int kStabQB = 32;

struct Launch {
    const PairDesc *pairs;
    PairGeom *geom;
    int32_t npairs;
    int64_t nq, nr;               // total queries / references
    const int64_t *q_offs;        // npairs + 1 (device) for pair lookup
    const int64_t *r_offs;        // npairs + 1
    uint32_t *key_a, *val_a, *key_b, *val_b, *key_c, *val_c;
    float4 *rec;
    float4 *rtmp;                 // per reference in input order: its record (x - cx, y - cy, eps, index),
                                  //   written by the prep kernel, moved to its bucket by the sort
    uint32_t *tab;
    int64_t ntab;                 // table entries of the whole call (zeroed by the prep kernel)
    uint32_t *curs;               // bucket fill cursors (a copy of tab while the records are placed)
    uint32_t *prep_done;          // blocks of the prep kernel finished (the last one resets it)
    QueryRec *qrec;
    uint32_t *status;
    unsigned long long *counters;  // egm_stats fields, or NULL
    // outputs (concatenated over pairs)
    int32_t *best, *second;
    float *best_d, *second_d;
    uint8_t *flags;
    int64_t *cand_offsets;
    int32_t *cand_idx;
    int64_t cand_capacity;
    int64_t *cand_total;
    int64_t *qcount;              // per-query candidate counts (CSR path)
    int64_t *scan_tmp;            // scan partials
    int32_t *blkpair;             // pair of query kStabQB * b, written by the prep kernel
    int32_t ratio_num, ratio_den;
    int32_t max_n;                // largest reference count of the batch
    int32_t kind;                 // descriptor kind shared by every pair, or -1 when mixed
    uint32_t kinds;               // bit k set when some pair has descriptor kind k
    // banded form (tiles of 128 queries sorted by angle)
    uint32_t *qperm;              // sorted query slot -> pair-local query index
    uint16_t *qbkt;               // per query: its bucket of the angle order (written by the prep kernel)
    uint8_t *descA, *descB;       // float pairs: 256-byte operand rows of the sorted queries / references
    QueryRec *qsrt;               // float pairs: query records in sorted order, pad = (query index, norm
                                  //   bits), pair field = rounding error bits
    float4 *rnorm;                // float pairs, sorted references: (squared norm of the operand
                                  //   row; rounding error |r - r~|; row scale, 1 unless FP8; 0)
    float *qscale;                // float pairs, sorted queries: row scale of the operand row (1 unless FP8)
    int32_t fp8;                  // float rows packed as FP8 E4M3 with per-row scales
    const int64_t *tile_offs;     // npairs + 1: first tile of each pair
    const int2 *tile_seq;         // ntiles: (tile, pair) in the order tiles are handed out (costliest pairs first)
    uint32_t *work;               // tile dispenser (zeroed before the band kernel)
    int64_t ntiles;
    int32_t probe;                // timeout check: band CTAs first wait on a barrier nothing completes
    // a single pair's plan travels in the launch parameters: the geometry
    // kernel writes the pair table, offsets and tile order that the later
    // kernels read, so the call needs no host-to-device copy
    int32_t inl_use;
    PairDesc inl;
};

// The fields of pair p that the prep and sort kernels read, by value: from
// the launch parameters for a single pair (no dependent global load), else
// from the pair table.
struct PairView {
    const double *xy1, *xy2, *F, *eps2;
    double eps_scalar;
    int64_t q_off, r_off, t_off, t_cap;
    int32_t n;
};
__device__ __forceinline__ PairView pair_view(const Launch &L, int p) {
    if (L.inl_use)
        return PairView{L.inl.xy1, L.inl.xy2, L.inl.F, L.inl.eps2, L.inl.eps_scalar,
                        L.inl.q_off, L.inl.r_off, L.inl.t_off, L.inl.t_cap, L.inl.n};
    const PairDesc &P = L.pairs[p];
    return PairView{P.xy1, P.xy2, P.F, P.eps2, P.eps_scalar, P.q_off, P.r_off, P.t_off, P.t_cap, P.n};
}

// Level layout (first sorted position, bucket bits, table offset) from the
// level counts; every block that needs it computes the same values.  One warp,
// lane = level: a level of c > 1 members gets about two buckets per member
// (ceil(log2 c) + 1 bits, at most max_bits) and a table of 2^bits + 1
// entries; positions and table offsets are exclusive prefix sums.
constexpr int kMaxBucketBits = 16;  // the tables resolve at most 16 bits of a 22-bit angle key

__device__ __forceinline__ void level_layout_lane(uint32_t c, uint32_t *start, int32_t *bits, uint32_t *tab,
                                                  int max_bits, int lane) {
    int b = 0;
    if (c > 1) {
        b = 32 - __clz(c - 1) + 1;
        if (b > max_bits) b = max_bits;
    }
    const uint32_t sz = (1u << b) + 1u;
    uint32_t ic = c, is = sz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t tc = __shfl_up_sync(0xffffffffu, ic, o);
        const uint32_t ts = __shfl_up_sync(0xffffffffu, is, o);
        if (lane >= o) {
            ic += tc;
            is += ts;
        }
    }
    start[lane] = ic - c;
    bits[lane] = b;
    tab[lane] = is - sz;
    if (lane == kLevels - 1) start[kLevels] = ic;
}
static_assert(kLevels == 32, "one lane per level");

__device__ __forceinline__ void level_layout_warp(const uint32_t *cnt, uint32_t *start, int32_t *bits,
                                                  uint32_t *tab, int max_bits, int lane) {
    level_layout_lane(cnt[lane], start, bits, tab, max_bits, lane);
}

// The same search over offsets held in shared memory (plain loads).
__device__ __forceinline__ int pair_of_shared(const int64_t *offs, int npairs, int64_t g) {
    int lo = 0, hi = npairs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Pair offsets cached in a block's shared memory when the batch has at most
// kSmemPairs pairs (every thread calls load_offsets, then the block syncs).
constexpr int kSmemPairs = 512;

__device__ __forceinline__ bool load_offsets(int64_t *s_offs, const int64_t *offs, int npairs) {
    if (npairs > kSmemPairs) return false;
    for (int i = threadIdx.x; i <= npairs; i += blockDim.x) s_offs[i] = offs[i];
    return true;
}

// The pair of row g (references first, then queries) for every lane of a
// converged warp whose rows ascend with the lane, from offsets cached in
// shared memory (at most kSmemPairs pairs): the warp finds the pair of its
// first row in two rounds of the 32 lanes comparing offsets with it (the
// largest k with offs[k] <= row, as the binary search finds it); a lane
// whose row lies beyond that pair, or on the other side of the split,
// searches alone.
__device__ __forceinline__ int warp_pair(const int64_t *s_roffs, const int64_t *s_qoffs, int npairs, int64_t nr,
                                         int64_t g) {
    const int lane = threadIdx.x & 31;
    const bool isr = g < nr;
    const int64_t key = isr ? g : g - nr;
    const int64_t *own = isr ? s_roffs : s_qoffs;
    const bool r0 = __shfl_sync(0xffffffffu, isr, 0);
    const int64_t k0 = __shfl_sync(0xffffffffu, key, 0);
    const int64_t *o0 = r0 ? s_roffs : s_qoffs;
    const int c1 = lane * 16;
    const uint32_t b1 = __ballot_sync(0xffffffffu, c1 < npairs && o0[c1 < npairs ? c1 : 0] <= k0);
    const int seg = (__popc(b1) - 1) * 16;
    const int c2 = seg + lane;
    const bool in2 = lane < 16 && c2 < npairs;
    const uint32_t b2 = __ballot_sync(0xffffffffu, in2 && o0[in2 ? c2 : 0] <= k0);
    const int p0 = seg + __popc(b2) - 1;
    if (isr == r0 && (p0 + 1 >= npairs || key < own[p0 + 1])) return p0;
    return pair_of_shared(own, npairs, key);
}

// Index of the pair that owns flattened element g, given offs[0..npairs] in
// global memory.
__device__ __forceinline__ int pair_of(const int64_t *offs, int npairs, int64_t g) {
    int lo = 0, hi = npairs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(offs + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Monotone quantisation shared by references and windows.  Explicit
// round-to-nearest intrinsics keep the compiler from contracting the two
// operations differently at different call sites.
__device__ __forceinline__ uint32_t qmap(float k, float kmin, float kscale) {
    float t = __fmul_rn(__fsub_rn(k, kmin), kscale);
    t = fminf(fmaxf(t, 0.0f), (float)kQMax);
    return (uint32_t)t;
}

// FP64 classification on the integer pipes (the FP64 pipe is scarce on
// GB300): finite (exponent not all ones) and strictly positive.
__device__ __forceinline__ bool finite64(double v) { return (__double2hiint(v) & 0x7ff00000) != 0x7ff00000; }
__device__ __forceinline__ bool positive64(double v) { return __double_as_longlong(v) > 0; }

// The oracle's FP64 evaluation order, with one rounding per operation.
__device__ __forceinline__ void exact_line(const double *F, double x, double y, double &a, double &b,
                                           double &c) {
    a = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(F + 0), x), __dmul_rn(__ldg(F + 1), y)), __ldg(F + 2));
    b = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(F + 3), x), __dmul_rn(__ldg(F + 4), y)), __ldg(F + 5));
    c = __dadd_rn(__dadd_rn(__dmul_rn(__ldg(F + 6), x), __dmul_rn(__ldg(F + 7), y)), __ldg(F + 8));
}

__device__ __forceinline__ double exact_norm(double a, double b) {
    return __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)));
}

// Eq. 3 / Eq. 4 decided exactly as the brute-force definition: dist <= eps.
__device__ __forceinline__ bool exact_member(double a, double b, double c, double N, double x, double y,
                                             double eps) {
    double num = fabs(__dadd_rn(__dadd_rn(__dmul_rn(a, x), __dmul_rn(b, y)), c));
    return __ddiv_rn(num, N) <= eps;
}

// Bucket of a query in the angle order of the banded form: the top bits of
// its quantised line angle; lines without an FP32 view, or whose windows are
// whole levels, after every angle.
constexpr int kQSortBits = 11;
constexpr int kQBuckets = (1 << kQSortBits) + 2;

__device__ __forceinline__ uint32_t query_bucket(const PairGeom &G, const QueryRec &r) {
    if (r.flags & EGM_FLAG_DEGENERATE_LINE) return 1u << kQSortBits;
    if ((r.flags & kQExactOnly) || (G.mode == kModeParallel && !(r.aux0 >= 0.5f))) return (1u << kQSortBits) + 1;
    return qmap(r.key, G.kmin, G.kscale) >> (kQBits - kQSortBits);
}

// ---------------------------------------------------------------- windows
//
// The stabbing window of query r in level lv (Sec. 4.2): the keys of every
// reference of the level whose tolerance circle can meet the query's line.
// First in key space (KeyWin), then as bucket-table indices (WinKeys) so
// that the table loads of many windows can be issued together, then as
// sorted positions (Window).  A hull of several KeyWins (the windows of a
// tile of queries) goes through the same two last steps.

struct KeyWin {
    int kind;        // 0 empty, 1 the whole level, 2 keys in [lo, hi] (angular: may cross the seam)
    float lo, hi;
};

struct WinKeys {
    uint32_t s, e;   // the level's sorted positions [s, e)
    uint32_t ta, tb; // bucket-table indices
    int kind;        // 0 empty, 1 whole level, 2 [T[ta], T[tb]), 3 seam: [T[ta], e) and [s, T[tb])
};

struct Window {
    uint32_t b0, len0, b1, len1;  // up to two disjoint ranges of sorted positions (pair-relative)
};

__device__ __forceinline__ KeyWin key_window(const PairGeom &G, const QueryRec &r, int lv) {
    KeyWin w;
    w.kind = 0;
    w.lo = w.hi = 0.0f;
    if (lv >= kLevels || (r.flags & EGM_FLAG_DEGENERATE_LINE) || G.cnt[lv] == 0) return w;
    const float smax = __uint_as_float(G.smax[lv]);
    // R: largest |p - c| of the level; the FP32 keys of its members are the
    // exact keys of points moved by at most `dpos` pixels.
    const float R = __uint_as_float(G.tmax[lv]);
    const float u = 5.9604645e-8f;
    bool full = (r.flags & kQExactOnly) != 0;
    if (full) {
    } else if (G.mode == kModeAngular) {
        const float dpos = 8.0f * u * R + 4.0f * u * fminf(G.de, R) + 2.0f * u * fabsf(G.kappa) + 1e-9f;
        const float dmin = __uint_as_float(G.dmin[lv]);
        const float sigma = (dmin > 0.0f) ? (smax + (r.aux0 + dpos) / dmin) * 1.000001f : INFINITY;
        full = !(sigma < 1.0f);
        if (!full) {
            // pads: relative (asinf, atan2f, the 1.000001 factors) and absolute
            // (the FP32 line direction: roundings of a, b, of the normalisation
            // and of the turn into the frame of u, about 7 ulp of 1 in all,
            // 4.3e-7 rad; taken as 2e-6)
            const float wv = asinf(sigma) * 1.000001f + 1e-37f;
            const float hw = wv + (4e-6f * (fabsf(r.key) + wv) + 2e-6f);
            full = !(hw < kHalfPiF);
            w.lo = r.key - hw;
            w.hi = r.key + hw;
        }
    } else {
        full = !(r.aux0 >= 0.5f);
        if (!full) {
            const float wv = (smax + R * r.aux1 + 8.0f * u * R + 1e-9f) / r.aux0 * 1.000001f;
            const float hw = wv + (1e-6f * (fabsf(r.key) + wv) + 1e-6f);
            full = !isfinite(hw);
            w.lo = r.key - hw;
            w.hi = r.key + hw;
        }
    }
    w.kind = full ? 1 : 2;
    return w;
}

// One window containing the windows of several queries of a pair (a warp of
// the banded form): keys in [kmin, kmax], |key| <= kabs, and the pad argument
// a0 (angular: the largest r_i; parallel: the smallest cos phi) and a1
// (parallel: the largest |sin phi|).  The true half-width grows with r_i
// (angular) and with |sin phi| / cos phi (parallel), and the pads of
// key_window cover the FP32 evaluation for any argument, so the result
// contains every one of those queries' windows.  `exact`: some query has no
// FP32 view (every level whole).
__device__ __forceinline__ KeyWin key_window_span(const PairGeom &G, int lv, float kmin, float kmax, float kabs,
                                                  float a0, float a1, bool exact) {
    KeyWin w;
    w.kind = 0;
    w.lo = w.hi = 0.0f;
    if (lv >= kLevels || G.cnt[lv] == 0) return w;
    const float smax = __uint_as_float(G.smax[lv]);
    const float R = __uint_as_float(G.tmax[lv]);
    const float u = 5.9604645e-8f;
    bool full = exact;
    float hw = 0.0f;
    if (full) {
    } else if (G.mode == kModeAngular) {
        const float dpos = 8.0f * u * R + 4.0f * u * fminf(G.de, R) + 2.0f * u * fabsf(G.kappa) + 1e-9f;
        const float dmin = __uint_as_float(G.dmin[lv]);
        const float sigma = (dmin > 0.0f) ? (smax + (a0 + dpos) / dmin) * 1.000001f : INFINITY;
        full = !(sigma < 1.0f);
        if (!full) {
            const float wv = asinf(sigma) * 1.000001f + 1e-37f;
            hw = wv + (4e-6f * (kabs + wv) + 2e-6f);
            full = !(hw < kHalfPiF);
        }
    } else {
        full = !(a0 >= 0.5f);
        if (!full) {
            const float wv = (smax + R * a1 + 8.0f * u * R + 1e-9f) / a0 * 1.000001f;
            hw = wv + (1e-6f * (kabs + wv) + 1e-6f);
            full = !isfinite(hw);
        }
    }
    w.kind = full ? 1 : 2;
    w.lo = kmin - hw;
    w.hi = kmax + hw;
    return w;
}

__device__ __forceinline__ WinKeys win_buckets(const PairGeom &G, int lv, const KeyWin &w) {
    WinKeys k;
    k.kind = 0;
    k.s = k.e = k.ta = k.tb = 0;
    if (w.kind == 0 || lv >= kLevels || G.cnt[lv] == 0) return k;
    k.s = G.start[lv];
    k.e = G.start[lv + 1];
    const float lo = w.lo, hi = w.hi;
    const bool low = G.mode == kModeAngular && lo < -kHalfPiF;
    const bool high = G.mode == kModeAngular && hi >= kHalfPiF;
    if (w.kind == 1 || (low && high)) {
        k.kind = 1;
        return k;
    }
    // Whole buckets around the window: a superset of the keypoints whose key
    // lies in it (the exact test decides membership).
    const int sh = kQBits - G.bits[lv];
    if (low || high) {
        // the window crosses the seam of the [-pi/2, pi/2) domain (Sec. 4.4,
        // "Discontinuity at 0/pi"): the high part [qa, end) of the level and
        // the low part [start, qb]
        k.ta = qmap(low ? lo + kPiF : lo, G.kmin, G.kscale) >> sh;
        k.tb = (qmap(low ? hi : hi - kPiF, G.kmin, G.kscale) >> sh) + 1;
        k.kind = 3;
    } else {
        k.ta = qmap(lo, G.kmin, G.kscale) >> sh;
        k.tb = (qmap(hi, G.kmin, G.kscale) >> sh) + 1;
        k.kind = 2;
    }
    return k;
}

__device__ __forceinline__ WinKeys window_keys(const PairGeom &G, const QueryRec &r, int lv) {
    return win_buckets(G, lv, key_window(G, r, lv));
}

__device__ __forceinline__ Window window_ranges(const WinKeys &k, uint32_t pa, uint32_t pb) {
    Window w;
    w.b0 = w.len0 = w.b1 = w.len1 = 0;
    if (k.kind == 1) {
        w.b0 = k.s;
        w.len0 = k.e - k.s;
    } else if (k.kind == 2) {
        w.b0 = pa;
        w.len0 = pb > pa ? pb - pa : 0;
    } else if (k.kind == 3) {
        if (pb > pa) pb = pa;  // a shared edge bucket is visited once
        w.b0 = pa;
        w.len0 = k.e - pa;
        w.b1 = k.s;
        w.len1 = pb > k.s ? pb - k.s : 0;
    }
    return w;
}

// exact_member(a, b, c, exact_norm(a, b), x, y, eps), mostly without the
// square root and the division.  With num = |a x + b y + c| and S = a a + b b
// evaluated as the definition evaluates them, the definition's quotient is
// Q = RN(num / N), N = RN(sqrt(S)).  Let lhs = RN(num num), rhs = RN(RN(eps
// eps) S), all normal (u = 2^-53 the unit roundoff), so N^2 is within
// (1 +- 3u) of S.  If lhs <= RN(rhs (1 - 2^-48)) then num^2 < eps^2 S (1 -
// 2^-49) < eps^2 N^2: num / N < eps and Q <= eps.  If lhs >= RN(rhs (1 +
// 2^-48)) then num^2 > eps^2 N^2 (1 + 2^-50): num / N > eps (1 + 2^-52) >=
// eps + ulp(eps), and Q > eps.  Otherwise (and outside the normal range)
// the definition itself decides.
__device__ __forceinline__ bool exact_within(double a, double b, double c, double x, double y, double eps) {
    const double num = fabs(__dadd_rn(__dadd_rn(__dmul_rn(a, x), __dmul_rn(b, y)), c));
    const double S = __dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b));
    if (eps >= 1e-140 && eps <= 1e140 && num <= 1e145) {
        const double lhs = __dmul_rn(num, num);
        const double rhs = __dmul_rn(__dmul_rn(eps, eps), S);
        if (rhs >= 1e-290 && rhs <= 1e290) {
            if (lhs <= __dmul_rn(rhs, 1.0 - 0x1p-48)) return true;
            if (lhs >= __dmul_rn(rhs, 1.0 + 0x1p-48)) return false;
        }
    }
    return exact_member(a, b, c, exact_norm(a, b), x, y, eps);
}

// The brute-force FP64 decision for one (query, reference) pair.
__device__ __forceinline__ bool exact_pair_inline(const PairDesc &P, int64_t i, uint32_t j) {
    double a, b, c;
    exact_line(P.F, P.xy1[2 * i], P.xy1[2 * i + 1], a, b, c);
    const double eps = P.eps2 ? P.eps2[j] : P.eps_scalar;
    return exact_within(a, b, c, P.xy2[2 * (int64_t)j], P.xy2[2 * (int64_t)j + 1], eps);
}

// The same, kept out of line for the loops where it runs only when the FP32
// test is inconclusive.
static __device__ __noinline__ bool exact_pair(const PairDesc &P, int64_t i, uint32_t j) {
    return exact_pair_inline(P, i, j);
}

// Outputs of query gq from its best two (distance << 32 | index) keys:
// indices, distances, flags and the ratio test (Sec. 5.1) in exact integer
// form for integer distances.
__device__ __forceinline__ void store_match(const Launch &L, int64_t gq, const PairDesc &P, uint32_t qflags,
                                            unsigned long long b1, unsigned long long b2) {
    uint8_t fl = (uint8_t)(qflags & EGM_FLAG_DEGENERATE_LINE);
    int32_t jb = -1, js = -1;
    float db = INFINITY, ds = INFINITY;
    if (P.row_bytes > 0 && b1 != ~0ull) {
        const bool isf = P.kind == EGM_DESC_F32_L2;
        jb = (int32_t)(b1 & 0xffffffffu);
        const uint32_t d1 = (uint32_t)(b1 >> 32);
        db = isf ? __uint_as_float(d1) : (float)d1;
        fl |= EGM_FLAG_HAS_BEST;
        bool pass;
        if (b2 == ~0ull) {
            fl |= EGM_FLAG_NO_SECOND;
            pass = true;
        } else {
            js = (int32_t)(b2 & 0xffffffffu);
            const uint32_t d2 = (uint32_t)(b2 >> 32);
            ds = isf ? __uint_as_float(d2) : (float)d2;
            const long long nn = L.ratio_num, dn = L.ratio_den;
            if (P.kind == EGM_DESC_U8_L2)
                pass = (long long)d1 * dn * dn < (long long)d2 * nn * nn;
            else if (P.kind == EGM_DESC_BIN)
                pass = (long long)d1 * dn < (long long)d2 * nn;
            else
                pass = db * (float)(dn * dn) < ds * (float)(nn * nn);
        }
        if (pass) fl |= EGM_FLAG_RATIO_PASS;
    }
    if (L.best) L.best[gq] = jb;
    if (L.second) L.second[gq] = js;
    if (L.best_d) L.best_d[gq] = db;
    if (L.second_d) L.second_d[gq] = ds;
    if (L.flags) L.flags[gq] = fl;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_geometry(const Launch &L, cudaStream_t s);
bool band_supported(int kind, int dim);
int band_row_bytes();
int band_tile_queries();
cudaError_t launch_query_sort(const Launch &L, cudaStream_t s);
cudaError_t launch_pack(const Launch &L, cudaStream_t s);
int band_shapes();  // tile shapes of the band kernel (see band.cu)
cudaError_t launch_mutual(const int32_t *best, uint8_t *flags, int64_t m, int64_t n, cudaStream_t s);
cudaError_t launch_transpose3(const double *F, double *Ft, cudaStream_t s);
// GMS (gms.cu): one pair of a batch, as the kernels read it from the table
struct GmsPair {
    const double *xy1, *xy2;
    const int32_t *best;
    uint8_t *flags;
    int64_t m, n, row_off;   // rows, references, first row in the concatenated per-row arrays
    double w1, h1, w2, h2;
};
struct GmsLayout {
    size_t table, offs, ds, dec, c1, c2, total;
};
GmsLayout gms_layout(int npairs, int64_t rows, int grid);
// the pair table and row offsets are already in the scratch at l.table, l.offs
cudaError_t launch_gms(void *scratch, const GmsLayout &l, int npairs, int64_t rows, uint32_t require, int grid,
                       double alpha, cudaStream_t st);
int64_t compact_tiles(int64_t m);
cudaError_t launch_compact(const uint8_t *flags, const int32_t *best, int64_t m, uint32_t require,
                           uint32_t *tile_count, int32_t *qi, int32_t *rj, int64_t *count, cudaStream_t s);
// zero_work: reset the tile dispenser first (the pipeline's query-sort
// kernel resets it otherwise)
cudaError_t launch_band(const Launch &L, int sms, int shape, cudaStream_t s, bool zero_work = true);
// part: 0 every row, 1 the references, 2 the queries (prep_kernel)
cudaError_t launch_prep(const Launch &L, cudaStream_t s, int part = 0);
cudaError_t launch_sort(const Launch &L, cudaStream_t s);
cudaError_t launch_stab(const Launch &L, int mode, cudaStream_t s);  // 0 fused match, 1 count, 2 fill+match
cudaError_t launch_csr_offsets(const Launch &L, uint32_t *long_count, cudaStream_t s);
cudaError_t launch_csr_row_sort(const Launch &L, uint32_t *long_list, uint32_t *long_count, cudaStream_t s);
cudaError_t launch_long_row_sort(const Launch &L, const uint32_t *list, const uint32_t *count, cudaStream_t s);
cudaError_t launch_intervals(const Launch &L, double *theta, double *delta, double *e3, int32_t *mode,
                             cudaStream_t s);
int mlp_param_count();
cudaError_t launch_mlp_backward(const float *params, const float *feat, const float *resid, int64_t n, float q,
                                const float *pre, const float *z, float *grad, float *loss, cudaStream_t s);
cudaError_t launch_adam(float *p, float *g, float *m, float *v, float lr, int64_t step, cudaStream_t s);
cudaError_t launch_residuals(const double *xy1, const double *xy2, const double *F, int64_t m, int64_t n,
                             const int32_t *qi, const int32_t *rj, int64_t k, double *out, cudaStream_t s);

}  // namespace egm
