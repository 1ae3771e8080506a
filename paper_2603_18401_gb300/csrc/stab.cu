// Candidate retrieval and candidate-restricted matching.
//
//   post_sort_kernel  gathers the sorted references into FP32 records
//                     (x - cx, y - cy, eps, index) and fills, per level, a
//                     bucket table: entry b = first sorted position whose
//                     quantised angle has top bits >= b.
//   stab_kernel       one warp per query (Sec. 4.2 "query"; Algorithm 1,
//                     Match loop).  Lane l computes the angle window of level
//                     l, the largest angular radius among that level's
//                     keypoints widened by the line's distance from the
//                     epipole, then the warp walks the concatenated windows
//                     32 keypoints at a time.  Each keypoint in a window gets
//                     the point-to-line test of Eq. 3 / Eq. 4: an FP32 test
//                     with a rigorous error bound, and, only when that is not
//                     conclusive, the FP64 expression of the brute-force
//                     definition.  Candidates are compared by descriptor
//                     (Sec. 4.3) and the warp keeps the best two by
//                     (distance, index), then applies the ratio test.
//   scan / row sort   the CSR form of the candidate sets (Eq. 4).
#include <math.h>

#include "egm_internal.cuh"

namespace egm {

namespace {

__global__ void __launch_bounds__(256) post_sort_kernel(Launch L) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < L.nr;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int p = pair_of(L.r_offs, L.npairs, g);
        const PairDesc &P = L.pairs[p];
        if (P.n <= kClusterMaxN) continue;  // done by the cluster sort
        const PairGeom &G = L.geom[p];
        const uint32_t pos = (uint32_t)(g - P.r_off);
        const uint32_t key = L.key_b[g];
        const uint32_t j = L.val_b[g];
        const double x = P.xy2[2 * (int64_t)j], y = P.xy2[2 * (int64_t)j + 1];
        const double eps = P.eps2 ? P.eps2[j] : P.eps_scalar;
        L.rec[g] = make_float4((float)(x - G.cx), (float)(y - G.cy), (float)eps, __uint_as_float(j));

        const int lv = (int)(key >> kQBits);
        const uint32_t s = G.start[lv], e = G.start[lv + 1];
        const int sh = kQBits - G.bits[lv];
        uint32_t *T = L.tab + P.t_off + G.tab[lv];
        const int64_t b = (int64_t)((key & kQMax) >> sh);
        const int64_t bp = pos == s ? -1 : (int64_t)((L.key_b[g - 1] & kQMax) >> sh);
        for (int64_t bb = bp + 1; bb <= b; bb++) T[bb] = pos;
        if (pos == e - 1) {
            const int64_t nb = (int64_t)1 << G.bits[lv];
            for (int64_t bb = b + 1; bb <= nb; bb++) T[bb] = e;
        }
    }
}

// ------------------------------------------------------------ descriptors

template <int KIND>
__device__ __forceinline__ uint32_t desc_dist(const uint4 *__restrict__ q, const uint4 *__restrict__ r,
                                              int chunks) {
    if (KIND == EGM_DESC_U8_L2) {
        uint32_t acc = 0;
        for (int c = 0; c < chunks; c++) {
            const uint4 a = q[c];
            const uint4 b = __ldg(r + c);
            uint32_t d;
            d = __vabsdiffu4(a.x, b.x); acc = __dp4a(d, d, acc);
            d = __vabsdiffu4(a.y, b.y); acc = __dp4a(d, d, acc);
            d = __vabsdiffu4(a.z, b.z); acc = __dp4a(d, d, acc);
            d = __vabsdiffu4(a.w, b.w); acc = __dp4a(d, d, acc);
        }
        return acc;
    } else if (KIND == EGM_DESC_BIN) {
        uint32_t acc = 0;
        for (int c = 0; c < chunks; c++) {
            const uint4 a = q[c];
            const uint4 b = __ldg(r + c);
            acc += __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
        }
        return acc;
    } else {
        float acc = 0.0f;
        for (int c = 0; c < chunks; c++) {
            const float4 a = reinterpret_cast<const float4 *>(q)[c];
            const float4 b = __ldg(reinterpret_cast<const float4 *>(r) + c);
            float d;
            d = a.x - b.x; acc = fmaf(d, d, acc);
            d = a.y - b.y; acc = fmaf(d, d, acc);
            d = a.z - b.z; acc = fmaf(d, d, acc);
            d = a.w - b.w; acc = fmaf(d, d, acc);
        }
        return __float_as_uint(acc);  // non-negative: bit order = value order
    }
}

__device__ __forceinline__ void top2_insert(unsigned long long &b1, unsigned long long &b2, unsigned long long k) {
    if (k < b1) { b2 = b1; b1 = k; }
    else if (k < b2) { b2 = k; }
}

constexpr int kStabWarps = 8;
constexpr int kMaxRowBytes = 2048;

struct Window {
    uint32_t b0, len0, b1, len1;  // up to two disjoint ranges of sorted positions (pair-relative)
};

__device__ __forceinline__ void level_window(const Launch &L, const PairDesc &P, const PairGeom &G,
                                             const QueryRec &r, int lv, Window &w) {
    w.b0 = w.len0 = w.b1 = w.len1 = 0;
    if (lv >= kLevels) return;
    const uint32_t cnt = G.cnt[lv];
    if (cnt == 0) return;
    const uint32_t s = G.start[lv], e = G.start[lv + 1];
    const float smax = __uint_as_float(G.smax[lv]);
    // R: largest |p - c| of the level; the FP32 keys of its members are the
    // exact keys of points moved by at most `dpos` pixels.
    const float R = __uint_as_float(G.tmax[lv]);
    const float u = 5.9604645e-8f;
    bool full = (r.flags & kQExactOnly) != 0;
    float lo = 0.0f, hi = 0.0f;
    if (full) {
    } else if (G.mode == kModeAngular) {
        const float dpos = 8.0f * u * R + 4.0f * u * fminf(G.de, R) + 2.0f * u * fabsf(G.kappa) + 1e-9f;
        const float dmin = __uint_as_float(G.dmin[lv]);
        const float sigma = (dmin > 0.0f) ? (smax + (r.aux0 + dpos) / dmin) * 1.000001f : INFINITY;
        full = !(sigma < 1.0f);
        if (!full) {
            const float wv = asinf(sigma) * 1.000001f + 1e-37f;
            const float hw = wv + (4e-6f * (fabsf(r.key) + wv) + 1e-14f);
            full = !(hw < kHalfPiF);
            lo = r.key - hw;
            hi = r.key + hw;
        }
    } else {
        full = !(r.aux0 >= 0.5f);
        if (!full) {
            const float wv = (smax + R * r.aux1 + 8.0f * u * R + 1e-9f) / r.aux0 * 1.000001f;
            const float hw = wv + (1e-6f * (fabsf(r.key) + wv) + 1e-6f);
            full = !isfinite(hw);
            lo = r.key - hw;
            hi = r.key + hw;
        }
    }
    if (full) {
        w.b0 = s;
        w.len0 = e - s;
        return;
    }
    // Whole buckets around the window: a superset of the keypoints whose key
    // lies in it (the exact test decides membership).
    const int sh = kQBits - G.bits[lv];
    const uint32_t *T = L.tab + P.t_off + G.tab[lv];
    if (G.mode == kModeAngular && (lo < -kHalfPiF || hi >= kHalfPiF)) {
        // the window crosses the seam of the [-pi/2, pi/2) domain (Sec. 4.4,
        // "Discontinuity at 0/pi"): the high part [qa, end) of the level and
        // the low part [start, qb]
        const bool low = lo < -kHalfPiF;
        const uint32_t qa = qmap(low ? lo + kPiF : lo, G.kmin, G.kscale);
        const uint32_t qb = qmap(low ? hi : hi - kPiF, G.kmin, G.kscale);
        const uint32_t pa = __ldg(T + (qa >> sh));
        uint32_t pb = __ldg(T + (qb >> sh) + 1);
        if (pb > pa) pb = pa;  // a shared edge bucket is visited once
        w.b0 = pa;
        w.len0 = e - pa;
        w.b1 = s;
        w.len1 = pb > s ? pb - s : 0;
    } else {
        const uint32_t pa = __ldg(T + (qmap(lo, G.kmin, G.kscale) >> sh));
        const uint32_t pb = __ldg(T + (qmap(hi, G.kmin, G.kscale) >> sh) + 1);
        w.b0 = pa;
        w.len0 = pb > pa ? pb - pa : 0;
    }
}

// The brute-force FP64 decision for one (query, reference) pair, kept out of
// line: it runs only when the FP32 test is inconclusive.
__device__ __noinline__ bool exact_pair(const PairDesc &P, int64_t i, uint32_t j) {
    double a, b, c;
    exact_line(P.F, P.xy1[2 * i], P.xy1[2 * i + 1], a, b, c);
    const double N = exact_norm(a, b);
    const double eps = P.eps2 ? P.eps2[j] : P.eps_scalar;
    return exact_member(a, b, c, N, P.xy2[2 * (int64_t)j], P.xy2[2 * (int64_t)j + 1], eps);
}

// mode 0: fused matching; 1: count candidates; 2: write candidate rows and match.
template <int KIND>
__device__ void stab_query(const Launch &L, int mode, int64_t gq, uint4 *qbuf, int lane) {
    const int p = pair_of(L.q_offs, L.npairs, gq);
    const PairDesc &P = L.pairs[p];
    const PairGeom &G = L.geom[p];
    const int64_t i = gq - P.q_off;
    const QueryRec r = L.qrec[gq];
    const bool exact_only = (r.flags & kQExactOnly) != 0;
    const bool match = mode != 1 && P.row_bytes > 0;
    const int chunks = P.row_bytes >> 4;

    unsigned long long b1 = ~0ull, b2 = ~0ull;
    uint32_t ncand = 0, nwin = 0, nexact = 0;
    int64_t row_off = 0;
    if (mode == 2) row_off = L.cand_offsets[gq];
    const bool write_rows = mode == 2 && L.cand_offsets[L.nq] <= L.cand_capacity;

    if (!(r.flags & EGM_FLAG_DEGENERATE_LINE)) {
        if (match) {
            const uint4 *src = reinterpret_cast<const uint4 *>(P.desc1 + i * (int64_t)P.row_bytes);
            for (int c = lane; c < chunks; c += 32) qbuf[c] = __ldg(src + c);
            __syncwarp();
        }
        Window w;
        level_window(L, P, G, r, lane, w);
        const uint32_t len = w.len0 + w.len1;
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const float4 *srec = L.rec + P.r_off;
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t f = base + lane;
            // owner lane: number of lanes whose inclusive prefix is <= f
            int o = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const uint32_t v = __shfl_sync(0xffffffffu, incl, o + st - 1);
                if (v <= f) o += st;
            }
            const uint32_t excl = __shfl_sync(0xffffffffu, incl - len, o);
            const uint32_t ob0 = __shfl_sync(0xffffffffu, w.b0, o);
            const uint32_t ol0 = __shfl_sync(0xffffffffu, w.len0, o);
            const uint32_t ob1 = __shfl_sync(0xffffffffu, w.b1, o);
            bool cand = false;
            uint32_t jc = 0;
            if (f < total) {
                const uint32_t off = f - excl;
                const uint32_t pos = off < ol0 ? ob0 + off : ob1 + (off - ol0);
                {
                    nwin++;
                    const float4 rc = __ldg(srec + pos);
                    const float t = fmaf(r.A, rc.x, fmaf(r.B, rc.y, r.C));
                    const float d = fabsf(t);
                    const float S = fmaf(fabsf(r.A), fabsf(rc.x), fmaf(fabsf(r.B), fabsf(rc.y), fabsf(r.C)));
                    // FP32 rounding (16u S), the FP32 tolerance (2u eps) and the
                    // distance between this line and the brute force's FP64 line
                    const float lerr = fmaf(r.E1, fabsf(rc.x) + fabsf(rc.y) + 2.0f * rc.z, r.E0);
                    const float bound = fmaf(9.6e-7f, S, fmaf(1.2e-7f, rc.z, lerr + 1e-9f));
                    if (exact_only) {
                        cand = exact_pair(P, i, __float_as_uint(rc.w));
                        nexact++;
                    } else if (d <= rc.z - bound) {
                        cand = true;
                    } else if (!(d > rc.z + bound)) {
                        // FP32 inconclusive: the brute-force FP64 expression decides.
                        cand = exact_pair(P, i, __float_as_uint(rc.w));
                        nexact++;
                    }
                    if (cand) {
                        const uint32_t j = __float_as_uint(rc.w);
                        jc = j;
                        ncand++;
                        if (match) {
                            const uint4 *rr = reinterpret_cast<const uint4 *>(P.desc2 + (int64_t)j * P.row_bytes);
                            const uint32_t dd = desc_dist<KIND>(qbuf, rr, chunks);
                            top2_insert(b1, b2, ((unsigned long long)dd << 32) | j);
                        }
                    }
                }
            }
            if (mode == 2) {
                const uint32_t bal = __ballot_sync(0xffffffffu, cand);
                if (cand && write_rows) {
                    const uint32_t slot = __popc(bal & ((1u << lane) - 1u));
                    L.cand_idx[row_off + slot] = (int32_t)jc;
                }
                row_off += __popc(bal);
            }
        }
    }
    // warp reduction of the two best keys and the counters
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long o1 = __shfl_xor_sync(0xffffffffu, b1, o);
        const unsigned long long o2 = __shfl_xor_sync(0xffffffffu, b2, o);
        const unsigned long long n1 = b1 < o1 ? b1 : o1;
        const unsigned long long mx = b1 < o1 ? o1 : b1;
        const unsigned long long mn2 = b2 < o2 ? b2 : o2;
        b2 = mx < mn2 ? mx : mn2;
        b1 = n1;
        ncand += __shfl_xor_sync(0xffffffffu, ncand, o);
        nwin += __shfl_xor_sync(0xffffffffu, nwin, o);
        nexact += __shfl_xor_sync(0xffffffffu, nexact, o);
    }
    if (lane == 0) {
        if (mode == 1) {
            L.qcount[gq] = ncand;
        } else {
            uint8_t fl = (uint8_t)(r.flags & EGM_FLAG_DEGENERATE_LINE);
            int32_t jb = -1, js = -1;
            float db = INFINITY, ds = INFINITY;
            if (match && b1 != ~0ull) {
                jb = (int32_t)(b1 & 0xffffffffu);
                const uint32_t d1 = (uint32_t)(b1 >> 32);
                db = KIND == EGM_DESC_F32_L2 ? __uint_as_float(d1) : (float)d1;
                fl |= EGM_FLAG_HAS_BEST;
                bool pass;
                if (b2 == ~0ull) {
                    fl |= EGM_FLAG_NO_SECOND;
                    pass = true;
                } else {
                    js = (int32_t)(b2 & 0xffffffffu);
                    const uint32_t d2 = (uint32_t)(b2 >> 32);
                    ds = KIND == EGM_DESC_F32_L2 ? __uint_as_float(d2) : (float)d2;
                    const long long nn = L.ratio_num, dn = L.ratio_den;
                    if (KIND == EGM_DESC_U8_L2)
                        pass = (long long)d1 * dn * dn < (long long)d2 * nn * nn;
                    else if (KIND == EGM_DESC_BIN)
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
        if (L.counters) {
            atomicAdd(L.counters + 2, (unsigned long long)nwin);
            atomicAdd(L.counters + 3, (unsigned long long)ncand);
            atomicAdd(L.counters + 4, (unsigned long long)nexact);
        }
    }
}

__global__ void __launch_bounds__(kStabWarps * 32, 4) stab_kernel(Launch L, int mode) {
    __shared__ __align__(16) uint4 qbuf_all[kStabWarps][kMaxRowBytes / 16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint4 *qbuf = qbuf_all[warp];
    for (int64_t gq = (int64_t)blockIdx.x * kStabWarps + warp; gq < L.nq; gq += (int64_t)gridDim.x * kStabWarps) {
        const int p = pair_of(L.q_offs, L.npairs, gq);
        const int kind = L.pairs[p].kind;
        if (kind == EGM_DESC_U8_L2) stab_query<EGM_DESC_U8_L2>(L, mode, gq, qbuf, lane);
        else if (kind == EGM_DESC_BIN) stab_query<EGM_DESC_BIN>(L, mode, gq, qbuf, lane);
        else stab_query<EGM_DESC_F32_L2>(L, mode, gq, qbuf, lane);
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_post_sort(const Launch &L, cudaStream_t s) {
    if (L.nr == 0 || L.max_n <= kClusterMaxN) return cudaSuccess;
    int64_t blocks = (L.nr + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    post_sort_kernel<<<(int)blocks, 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_stab(const Launch &L, int mode, cudaStream_t s) {
    if (L.nq == 0) return cudaSuccess;
    int64_t blocks = (L.nq + kStabWarps - 1) / kStabWarps;
    if (blocks > 152 * 32) blocks = 152 * 32;
    stab_kernel<<<(int)blocks, kStabWarps * 32, 0, s>>>(L, mode);
    return cudaGetLastError();
}

}  // namespace egm
