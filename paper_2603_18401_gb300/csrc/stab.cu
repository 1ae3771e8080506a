// Candidate retrieval and candidate-restricted matching.
//
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

// ------------------------------------------------------------ descriptors

// ------------------------------------------------------------ stabbing
//
// One block takes kQB consecutive queries.  On GB300 a dependent global
// access costs about a microsecond, so the kernel is organised around the
// number of serial memory round trips per block:
//   phase 1  (2 trips)  query records and the block's pair geometry; then
//            the bucket-table loads of every window and the query
//            descriptors together.  Warp w handles queries 4w .. 4w+3,
//            lane = level; non-empty ranges are compacted into shared memory.
//   2a (1 trip)  the concatenated window elements, a contiguous chunk per
//            thread, record loads issued together; each passes the Eq. 3/4
//            test (FP32 with a rigorous bound, FP64 brute-force expression
//            when inconclusive); candidates are appended to a list with one
//            warp-aggregated atomic.
//   2a'      the list is counting-sorted by query into segments.
//   2b (1 trip per 128 candidates)  a group of G lanes per candidate
//            (G 16-byte chunks of its descriptor), four candidates per group
//            with all loads issued first; distances go to the segment.
//   2c       one warp per query reduces its segment into the query's best
//            two (distance, index) keys - a single writer, no atomics.
// Rounds of kRound elements repeat 2a-2c; the outputs follow the last round.
constexpr int kQB = kStabQB;
// the per-round segment scan gives one lane of warp 0 to each query of the block
static_assert(kQB == 32, "one lane per query in the segment scan");
constexpr int kStabThreads = 256;
constexpr int kRangesPerQuery = 2 * kLevels;
constexpr int kDescCache = 256;  // query descriptors up to this many bytes are staged in shared memory
// window elements a thread tests per batch of record loads, and candidates
// per lane group in the distance pass
constexpr int kBatch = 4;
constexpr int kU = 4;
// window elements tested per round (shared memory for occupancy)
constexpr int kRound = 1024;
constexpr int kQPerWarp = kQB / (kStabThreads / 32);

template <int kRound>
struct StabSmem {
    uint2 rng[kQB][kRangesPerQuery];  // (first sorted position, length) of each non-empty range
    QueryRec qr[kQB];
    PairGeom g;                       // geometry of the block's first pair
    PairDesc pd;                      //   and its descriptor
    unsigned long long b1[kQB], b2[kQB];
    uint32_t nrng[kQB];
    uint32_t tq[kQB];
    uint32_t eoff[kQB + 1];
    uint32_t cnt[kQB];                // candidates per query (all rounds)
    uint32_t rcnt[kQB];               // candidates per query in this round
    uint32_t roff[kQB + 1];           //   their segment offsets
    uint32_t rfill[kQB];
    uint32_t fill[kQB];               // CSR fill counters
    uint32_t nwin, nexact, ncand;
    int32_t gpair;
    uint32_t lj[kRound];              // append list: reference index
    uint8_t lq[kRound];               //   and query slot
    uint32_t sj[kRound];              // per-query segments: reference index
    uint8_t sq[kRound];               //   and query slot
    uint32_t sd[kRound];              //   and descriptor distance
    uint32_t rmask[kQB][2];           // non-empty ranges of each query (bit k: range k)
    int32_t lv[kLevels];              // non-empty levels of the block's pair
    int32_t nlev;
    uint4 qdesc[kQB][kDescCache / 16];
};

constexpr int kKindAny = -1;  // a launch that mixes descriptor kinds

// Contribution of one 16-byte chunk to a descriptor distance.
template <int KIND>
__device__ __forceinline__ void chunk_dist(int kind, uint4 a, uint4 b, uint32_t &acc, float &facc) {
    const int k = KIND == kKindAny ? kind : KIND;
    if (k == EGM_DESC_U8_L2) {
        uint32_t d;
        d = __vabsdiffu4(a.x, b.x); acc = __dp4a(d, d, acc);
        d = __vabsdiffu4(a.y, b.y); acc = __dp4a(d, d, acc);
        d = __vabsdiffu4(a.z, b.z); acc = __dp4a(d, d, acc);
        d = __vabsdiffu4(a.w, b.w); acc = __dp4a(d, d, acc);
    } else if (k == EGM_DESC_BIN) {
        acc += __popc(a.x ^ b.x) + __popc(a.y ^ b.y) + __popc(a.z ^ b.z) + __popc(a.w ^ b.w);
    } else {
        float d;
        d = __uint_as_float(a.x) - __uint_as_float(b.x); facc = fmaf(d, d, facc);
        d = __uint_as_float(a.y) - __uint_as_float(b.y); facc = fmaf(d, d, facc);
        d = __uint_as_float(a.z) - __uint_as_float(b.z); facc = fmaf(d, d, facc);
        d = __uint_as_float(a.w) - __uint_as_float(b.w); facc = fmaf(d, d, facc);
    }
}

__device__ __forceinline__ void top2_key(unsigned long long key, unsigned long long &b1, unsigned long long &b2) {
    if (key < b1) {
        b2 = b1;
        b1 = key;
    } else if (key < b2) {
        b2 = key;
    }
}

// 16-byte asynchronous copy global -> shared (no registers held while it is
// in flight); cp_async_wait() before the data is read
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void copy16(void *dst, const void *src, int bytes, int lane) {
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (int k = lane; k < bytes / 16; k += 32) d4[k] = __ldg(s4 + k);
}

// mode 0: fused matching; 1: count candidates; 2: write candidate rows and match.
// (A single pair with u8 or binary rows runs stab_pair_kernel instead.)
template <int KIND>
__global__ void __launch_bounds__(kStabThreads, 4) stab_kernel(Launch L, int mode) {
    pdl_begin();
    __shared__ __align__(16) StabSmem<kRound> S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const bool write_rows = mode == 2 && L.cand_offsets[L.nq] <= L.cand_capacity;
    uint32_t nwin = 0, nexact = 0;
    if (tid == 0) { S.nwin = 0; S.nexact = 0; S.ncand = 0; }
    for (int64_t q0 = (int64_t)blockIdx.x * kQB; q0 < L.nq; q0 += (int64_t)gridDim.x * kQB) {
        const int nqb = (int)min((int64_t)kQB, L.nq - q0);
        // ---- phase 1, trip 1: query records, and the first pair's geometry and descriptor
        const int qbase = warp * kQPerWarp;
        if (lane < 3 * kQPerWarp) {
            const int ql = qbase + lane / 3;
            if (ql < nqb)
                reinterpret_cast<uint4 *>(&S.qr[ql])[lane % 3] =
                    __ldg(reinterpret_cast<const uint4 *>(L.qrec + q0 + ql) + lane % 3);
        }
        if (warp == kStabThreads / 32 - 1) {
            const int p0 = L.npairs == 1 ? 0 : L.blkpair[q0 / kQB];
            copy16(&S.g, L.geom + p0, (int)sizeof(PairGeom), lane);
            copy16(&S.pd, L.pairs + p0, (int)sizeof(PairDesc), lane);
            if (lane == 0) S.gpair = p0;
        }
        __syncthreads();
        // ---- phase 1, trip 2: windows, their bucket-table loads and the query
        // descriptors issued together.  Lanes take (query, non-empty level)
        // slots of the block's pair, so a pair with two populated levels costs
        // two lanes per query, not 32; ranges go to fixed slots 2 i, 2 i + 1 of
        // level index i (empty ones have length 0).
        if (warp == 0) {
            const uint32_t nz = __ballot_sync(0xffffffffu, S.g.cnt[lane] > 0);
            if (nz & (1u << lane)) S.lv[__popc(nz & lt)] = lane;
            if (lane == 0) S.nlev = __popc(nz);
        }
        if (tid < kQB) {
            S.tq[tid] = 0;
            S.nrng[tid] = 0;
            S.b1[tid] = ~0ull;
            S.b2[tid] = ~0ull;
            S.cnt[tid] = 0;
            S.fill[tid] = 0;
            S.rmask[tid][0] = S.rmask[tid][1] = 0u;
        }
        __syncthreads();
        // the query descriptors, copied to shared memory while the windows are computed
        constexpr int kStage = kQPerWarp * kDescCache / 16 / 32;
#pragma unroll
        for (int k = 0; k < kStage; k++) {
            const int idx = lane + 32 * k;
            const int ql = qbase + idx / (kDescCache / 16);
            const int c = idx % (kDescCache / 16);
            if (mode != 1 && ql < nqb) {
                const int p = S.qr[ql].pair;
                const PairDesc &P = p == S.gpair ? S.pd : L.pairs[p];
                if (P.row_bytes > 0 && P.row_bytes <= kDescCache && c < (P.row_bytes >> 4))
                    cp_async16(&S.qdesc[ql][c], reinterpret_cast<const uint4 *>(P.desc1 + (q0 + ql - P.q_off) *
                                                                                         (int64_t)P.row_bytes) + c);
            }
        }
        {
            const int nlev = S.nlev;
            const int nslot = nqb * nlev;
            for (int g0 = warp * 32; g0 < nslot; g0 += kStabThreads) {
                const int sl = g0 + lane;
                WinKeys wk;
                wk.kind = 0;
                int ql = 0, li = 0;
                if (sl < nslot) {
                    ql = sl / nlev;
                    li = sl - ql * nlev;
                    if (S.qr[ql].pair == S.gpair) wk = window_keys(S.g, S.qr[ql], S.lv[li]);
                    else ql = -1;  // another pair: handled below
                }
                uint32_t a = 0, b = 0;
                if (wk.kind >= 2) {
                    const uint32_t *T = L.tab + S.pd.t_off + S.g.tab[S.lv[li]];
                    a = __ldg(T + wk.ta);
                    b = __ldg(T + wk.tb);
                }
                if (sl < nslot && ql >= 0) {
                    const Window w = window_ranges(wk, a, b);
                    S.rng[ql][2 * li] = make_uint2(w.b0, w.len0);
                    S.rng[ql][2 * li + 1] = make_uint2(w.b1, w.len1);
                    if (w.len0 + w.len1) {
                        atomicAdd(&S.tq[ql], w.len0 + w.len1);
                        const uint32_t bits = (w.len0 ? 1u : 0u) | (w.len1 ? 2u : 0u);
                        atomicOr(&S.rmask[ql][li >> 4], bits << (2 * (li & 15)));
                    }
                    if (li == 0) S.nrng[ql] = 2 * nlev;
                }
            }
            // queries of another pair than the block's first: one warp per query, lane = level
#pragma unroll 1
            for (int t = 0; t < kQPerWarp; t++) {
                const int ql = qbase + t;
                if (ql >= nqb || S.qr[ql].pair == S.gpair) continue;
                const int p = S.qr[ql].pair;
                const PairGeom &G = L.geom[p];
                const WinKeys wk = window_keys(G, S.qr[ql], lane);
                uint32_t a = 0, b = 0;
                if (wk.kind >= 2) {
                    const uint32_t *T = L.tab + L.pairs[p].t_off + G.tab[lane];
                    a = __ldg(T + wk.ta);
                    b = __ldg(T + wk.tb);
                }
                const Window w = window_ranges(wk, a, b);
                S.rng[ql][2 * lane] = make_uint2(w.b0, w.len0);
                S.rng[ql][2 * lane + 1] = make_uint2(w.b1, w.len1);
                const uint32_t bits = (w.len0 ? 1u : 0u) | (w.len1 ? 2u : 0u);
                const uint32_t lo16 = __reduce_or_sync(0xffffffffu, lane < 16 ? bits << (2 * lane) : 0u);
                const uint32_t hi16 = __reduce_or_sync(0xffffffffu, lane >= 16 ? bits << (2 * (lane - 16)) : 0u);
                if (lane == 0) { S.rmask[ql][0] = lo16; S.rmask[ql][1] = hi16; }
                uint32_t tot = w.len0 + w.len1;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
                if (lane == 0) {
                    S.tq[ql] = tot;
                    S.nrng[ql] = 2 * kLevels;
                }
            }
        }
        cp_async_wait();
        // every query of the block in the cached pair, descriptors of one kind
        // and staged: the pair's fields are block constants (the common case)
        const bool uni = __syncthreads_and(tid >= nqb || S.qr[tid].pair == S.gpair) && KIND != kKindAny &&
                         S.pd.row_bytes <= kDescCache;
        const float4 *recb = L.rec + S.pd.r_off;
        if (warp == 0) {
            uint32_t incl = S.tq[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            S.eoff[lane + 1] = incl;
            if (lane == 0) S.eoff[0] = 0;
        }
        __syncthreads();

        // ---- phase 2, in rounds of kRound window elements
        const uint32_t T = S.eoff[kQB];
        for (uint32_t base = 0; base < T; base += kRound) {
            // 2a: tests, candidates appended to the list
            if (tid < kQB) S.rcnt[tid] = 0;
            __syncthreads();
            const uint32_t Tr = min(T - base, (uint32_t)kRound);
            const uint32_t K = (Tr + kStabThreads - 1) / kStabThreads;  // the same for every thread
            uint32_t f = base + (uint32_t)tid * K;
            const uint32_t fend = min(f + K, base + Tr);
            int q = 0, k = 0;
            uint32_t rem = 0;
            // move (q, k, rem) forward to a real element: past exhausted or empty
            // ranges and past queries without elements
            auto settle = [&]() {
                while (q < kQB) {
                    // next non-empty range at or after k
                    const uint32_t m0 = k < 32 ? S.rmask[q][0] & (~0u << k) : 0u;
                    const uint32_t m1 = k >= 64 ? 0u : k <= 32 ? S.rmask[q][1] : S.rmask[q][1] & (~0u << (k - 32));
                    if (m0) k = __ffs(m0) - 1;
                    else if (m1) k = 32 + __ffs(m1) - 1;
                    else { q++; k = 0; continue; }
                    const uint32_t len = S.rng[q][k].y;
                    if (rem < len) break;
                    rem -= len;
                    k++;
                }
            };
            if (f < fend) {
#pragma unroll
                for (int st = 16; st > 0; st >>= 1)
                    if (S.eoff[q + st] <= f) q += st;
                rem = f - S.eoff[q];
                settle();
            }
            for (uint32_t kb = 0; kb < K; kb += kBatch) {
                int bq[kBatch];
                uint32_t bpos[kBatch];
                bool bv[kBatch];
#pragma unroll
                for (int t = 0; t < kBatch; t++) {
                    bv[t] = f < fend;
                    bq[t] = q;
                    bpos[t] = 0;
                    if (bv[t]) {
                        bpos[t] = S.rng[q][k].x + rem;
                        f++;
                        rem++;
                        if (f < fend) settle();
                    }
                }
                float4 rc[kBatch];
#pragma unroll
                for (int t = 0; t < kBatch; t++) {
                    if (bv[t]) {
                        if (uni) {
                            rc[t] = __ldg(recb + bpos[t]);
                        } else {
                            const int p = S.qr[bq[t]].pair;
                            const int64_t ro = p == S.gpair ? S.pd.r_off : L.pairs[p].r_off;
                            rc[t] = __ldg(L.rec + ro + bpos[t]);
                        }
                    }
                }
#pragma unroll 1
                for (int t = 0; t < kBatch; t++) {
                    // element t of the batch by register selects: a dynamic index into
                    // these arrays would place them in local memory
                    int qq = bq[0];
                    bool bvt = bv[0];
                    float4 rct = rc[0];
#pragma unroll
                    for (int u = 1; u < kBatch; u++)
                        if (t == u) {
                            qq = bq[u];
                            bvt = bv[u];
                            rct = rc[u];
                        }
                    uint32_t j = 0;
                    bool cand = false;
                    if (bvt) {
                        const QueryRec &r = S.qr[qq];
                        j = __float_as_uint(rct.w);
                        nwin++;
                        bool exact = (r.flags & kQExactOnly) != 0;
                        if (!exact) {
                            const float x = rct.x, y = rct.y, e = rct.z;
                            const float d = fabsf(fmaf(r.A, x, fmaf(r.B, y, r.C)));
                            const float Sm = fmaf(fabsf(r.A), fabsf(x), fmaf(fabsf(r.B), fabsf(y), fabsf(r.C)));
                            // FP32 rounding (16u S), the FP32 tolerance (2u eps) and the
                            // distance between this line and the brute force's FP64 line
                            const float lerr = fmaf(r.E1, fabsf(x) + fabsf(y) + 2.0f * e, r.E0);
                            const float bound = fmaf(9.6e-7f, Sm, fmaf(1.2e-7f, e, lerr + 1e-9f));
                            cand = d <= e - bound;
                            exact = !cand && !(d > e + bound);
                        }
                        if (exact) {
                            // FP32 inconclusive: the brute-force FP64 expression decides.
                            const PairDesc &P = L.pairs[r.pair];
                            cand = exact_pair(P, q0 + qq - P.q_off, j);
                            nexact++;
                        }
                    }
                    if (cand) atomicAdd(&S.cnt[qq], 1u);
                    if (cand && mode == 2) {
                        const uint32_t slot = atomicAdd(&S.fill[qq], 1u);
                        if (write_rows) L.cand_idx[L.cand_offsets[q0 + qq] + slot] = (int32_t)j;
                    }
                    if (mode != 1) {
                        // warp-aggregated append to the round's candidate list
                        const uint32_t m = __ballot_sync(0xffffffffu, cand);
                        if (m) {
                            const int leader = __ffs(m) - 1;
                            uint32_t c0 = 0;
                            if (lane == leader) c0 = atomicAdd(&S.ncand, (uint32_t)__popc(m));
                            c0 = __shfl_sync(0xffffffffu, c0, leader);
                            if (cand) {
                                const uint32_t c = c0 + __popc(m & lt);
                                S.lj[c] = j;
                                S.lq[c] = (uint8_t)qq;
                                atomicAdd(&S.rcnt[qq], 1u);
                            }
                        }
                    }
                }
            }
            __syncthreads();
            const uint32_t nc = S.ncand;
            if (mode != 1 && nc > 0) {
                // 2a': segments by query
                if (warp == 0) {
                    const uint32_t v = S.rcnt[lane];
                    uint32_t incl = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += t;
                    }
                    S.roff[lane] = incl - v;
                    S.rfill[lane] = incl - v;
                    if (lane == 31) S.roff[kQB] = incl;
                }
                __syncthreads();
                for (uint32_t c = tid; c < nc; c += kStabThreads) {
                    const int qq = S.lq[c];
                    const uint32_t pos = atomicAdd(&S.rfill[qq], 1u);
                    S.sj[pos] = S.lj[c];
                    S.sq[pos] = (uint8_t)qq;
                }
                __syncthreads();
                // 2b: G lanes per candidate read its descriptor row together (one
                // cache line per group of eight 16-byte chunks), four candidates per
                // group with the loads issued first; distances go to shared memory.
                const int rb0 = KIND != kKindAny ? S.pd.row_bytes : kDescCache;
                const int chunks0 = rb0 >> 4;
                const int G = chunks0 >= 32 ? 32 : chunks0 >= 16 ? 16 : chunks0 >= 8 ? 8 : chunks0 >= 4 ? 4
                            : chunks0 >= 2 ? 2 : 1;
                const int groups = kStabThreads / G;
                const int gl = tid % G;
                constexpr int U = kU;
                if (uni && chunks0 <= G) {
                    // block constants; one chunk per lane of each candidate
                    const uint4 *d2 = reinterpret_cast<const uint4 *>(S.pd.desc2);
                    const int rb16 = chunks0;
                    for (uint32_t cb = 0; cb < nc; cb += (uint32_t)(groups * U)) {
                        uint32_t cc[U];
                        uint4 rv[U];
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            cc[u] = cb + (uint32_t)(tid / G) + (uint32_t)(u * groups);
                            if (cc[u] < nc && gl < rb16) rv[u] = __ldg(d2 + (int64_t)S.sj[cc[u]] * rb16 + gl);
                        }
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            uint32_t acc = 0;
                            float facc = 0.0f;
                            if (cc[u] < nc && gl < rb16) chunk_dist<KIND>(KIND, S.qdesc[S.sq[cc[u]]][gl], rv[u], acc, facc);
                            if (KIND == EGM_DESC_F32_L2) {
                                for (int o = G >> 1; o > 0; o >>= 1) facc += __shfl_xor_sync(0xffffffffu, facc, o, G);
                                acc = __float_as_uint(facc);
                            } else {
                                for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
                            }
                            if (gl == 0 && cc[u] < nc) S.sd[cc[u]] = acc;
                        }
                    }
                } else
                for (uint32_t cb = 0; cb < nc; cb += (uint32_t)(groups * U)) {
                    uint32_t cc[U];
                    const uint4 *rrow[U];
                    const uint4 *qrow[U];
                    int chunks[U], kinds[U];
                    bool qsm[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        cc[u] = cb + (uint32_t)(tid / G) + (uint32_t)(u * groups);
                        chunks[u] = 0;
                        kinds[u] = KIND;
                        rrow[u] = qrow[u] = nullptr;
                        qsm[u] = true;
                        if (cc[u] < nc) {
                            const int qq = S.sq[cc[u]];
                            const int p = S.qr[qq].pair;
                            const PairDesc &P = p == S.gpair ? S.pd : L.pairs[p];
                            chunks[u] = P.row_bytes >> 4;
                            if (KIND == kKindAny) kinds[u] = P.kind;
                            rrow[u] = reinterpret_cast<const uint4 *>(P.desc2 + (int64_t)S.sj[cc[u]] * P.row_bytes);
                            qsm[u] = P.row_bytes <= kDescCache;
                            qrow[u] = qsm[u] ? S.qdesc[qq]
                                             : reinterpret_cast<const uint4 *>(P.desc1 + (q0 + qq - P.q_off) *
                                                                                         (int64_t)P.row_bytes);
                        }
                    }
                    uint32_t acc[U];
                    float facc[U];
#pragma unroll
                    for (int u = 0; u < U; u++) { acc[u] = 0; facc[u] = 0.0f; }
                    int maxch = 0;
#pragma unroll
                    for (int u = 0; u < U; u++) maxch = max(maxch, chunks[u]);
                    for (int ch0 = 0; ch0 < maxch; ch0 += G) {
                        const int ch = ch0 + gl;
                        uint4 rv[U];
#pragma unroll
                        for (int u = 0; u < U; u++)
                            if (ch < chunks[u]) rv[u] = __ldg(rrow[u] + ch);
#pragma unroll
                        for (int u = 0; u < U; u++)
                            if (ch < chunks[u])
                                chunk_dist<KIND>(kinds[u], qsm[u] ? qrow[u][ch] : __ldg(qrow[u] + ch), rv[u], acc[u],
                                                 facc[u]);
                    }
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const bool isf = (KIND == kKindAny ? kinds[u] : KIND) == EGM_DESC_F32_L2;
                        uint32_t v = isf ? __float_as_uint(facc[u]) : acc[u];
                        for (int o = G >> 1; o > 0; o >>= 1) {
                            if (isf) {
                                facc[u] += __shfl_xor_sync(0xffffffffu, facc[u], o, G);
                                v = __float_as_uint(facc[u]);
                            } else {
                                acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o, G);
                                v = acc[u];
                            }
                        }
                        if (gl == 0 && cc[u] < nc) S.sd[cc[u]] = v;
                    }
                }
                __syncthreads();
                // 2c: a thread per candidate, segmented best two per query within
                // the warp (a query's candidates are contiguous), merged by the
                // segment's first lane.  The merge keeps the minimum with one
                // atomicMin and offers min(the larger of the displaced and the
                // offered first, the offered second) to the second slot: every
                // value offered there is an element other than the minimum and
                // the true second is always offered, so the pair is exact under
                // any interleaving.
                for (uint32_t cb = 0; cb < nc; cb += kStabThreads) {
                    const uint32_t c = cb + (uint32_t)tid;
                    const bool valid = c < nc;
                    const int qq = valid ? (int)S.sq[c] : -1 - lane;
                    unsigned long long k1 = valid ? ((unsigned long long)S.sd[c] << 32) | S.sj[c] : ~0ull;
                    unsigned long long k2 = ~0ull;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned long long o1 = __shfl_down_sync(0xffffffffu, k1, o);
                        const unsigned long long o2 = __shfl_down_sync(0xffffffffu, k2, o);
                        const int oq = __shfl_down_sync(0xffffffffu, qq, o);
                        if (lane + o < 32 && oq == qq) {
                            const unsigned long long mx = k1 < o1 ? o1 : k1;
                            const unsigned long long mn2 = k2 < o2 ? k2 : o2;
                            k1 = k1 < o1 ? k1 : o1;
                            k2 = mx < mn2 ? mx : mn2;
                        }
                    }
                    const int pq = __shfl_up_sync(0xffffffffu, qq, 1);
                    if (valid && (lane == 0 || pq != qq)) {
                        const unsigned long long old = atomicMin(&S.b1[qq], k1);
                        const unsigned long long lose = old > k1 ? old : k1;
                        const unsigned long long offer = lose < k2 ? lose : k2;
                        if (offer != ~0ull) atomicMin(&S.b2[qq], offer);
                    }
                }
            }
            __syncthreads();
            if (tid == 0) S.ncand = 0;
        }
        if (L.counters) {
            atomicAdd(&S.nwin, nwin);
            atomicAdd(&S.nexact, nexact);
            nwin = nexact = 0;
        }
        __syncthreads();

        // ---- results
        if (tid < nqb) {
            const int64_t gq = q0 + tid;
            if (mode == 1) {
                L.qcount[gq] = S.cnt[tid];
            } else {
                const int p = S.qr[tid].pair;
                const PairDesc &P = p == S.gpair ? S.pd : L.pairs[p];
                store_match(L, gq, P, S.qr[tid].flags, S.b1[tid], S.b2[tid]);
            }
            if (L.counters) atomicAdd(L.counters + 3, (unsigned long long)S.cnt[tid]);
        }
        __syncthreads();
    }
    if (L.counters && tid == 0) {
        atomicAdd(L.counters + 2, (unsigned long long)S.nwin);
        atomicAdd(L.counters + 4, (unsigned long long)S.nexact);
    }
}

// ------------------------------------------------------------ one pair, a warp per query
//
// The queries of one pair share nothing but the pair's tables, so in this
// variant each warp takes one query at a time and needs no block-wide
// phase: lane l computes the window of the pair's l-th populated level and
// its two ranges of sorted positions (Sec. 4.2 query, split at the seam);
// the ranges are flattened by a prefix sum over the lanes, and the warp
// tests 32 window elements per step (each lane finds its element's range by
// a five-step search over the lanes' prefix sums).  Candidates go to a small
// per-warp ring in shared memory; every 32 of them are one batch of
// descriptor distances (Sec. 4.3): G lanes read one candidate's row (16
// bytes each, coalesced), G rounds are accumulated per lane and reduced by
// a transposed butterfly (G - 1 shuffles for the G rounds), after which
// each lane holds one candidate's distance.  Each lane keeps its best two
// (distance, index) keys; four warp reductions give the query's best two.
constexpr int kPairThreads = 64;
constexpr int kPairWarps = kPairThreads / 32;
constexpr int kRing = 64;  // candidate ring per warp: 32 waiting + 32 new
constexpr int kChunkQ = 8; // queries per warp whose windows are computed in one pass

// The window of a query in one level, from the level's half-width over all
// of the pair's queries (key_window_span with the pair's extremes of the pad
// arguments and of |key|, recorded by the prep kernel): a superset of each
// query's own window, so the exact test keeps the same candidates.
struct LevelWin {
    float hw;      // half-width of every window in the level's key space
    int whole;     // 1: every window covers the whole level
    uint32_t s, e; // sorted positions of the level
    int sh;        // key bits below the level's buckets
};

__device__ __forceinline__ LevelWin level_win(const PairGeom &G, int lv) {
    const float a0 = G.mode == kModeAngular ? __uint_as_float(G.qa0max) : __uint_as_float(G.qa0min);
    const KeyWin w = key_window_span(G, lv, 0.0f, 0.0f, __uint_as_float(G.qkabs), a0, __uint_as_float(G.qa1max),
                                     false);
    LevelWin c;
    c.hw = w.hi;
    c.whole = w.kind == 1 ? 1 : 0;
    c.s = G.start[lv];
    c.e = G.start[lv + 1];
    c.sh = kQBits - G.bits[lv];
    return c;
}

// The window of query r in the lane's level as bucket-table indices (the
// kinds of WinKeys).
__device__ __forceinline__ WinKeys level_window(const PairGeom &G, const LevelWin &c, const QueryRec &r) {
    WinKeys k;
    k.s = c.s;
    k.e = c.e;
    k.ta = k.tb = 0u;
    k.kind = 0;
    if (r.flags & EGM_FLAG_DEGENERATE_LINE) return k;
    const bool full = c.whole || (r.flags & kQExactOnly) != 0;
    const float lo = r.key - c.hw, hi = r.key + c.hw;
    const bool low = G.mode == kModeAngular && lo < -kHalfPiF;
    const bool high = G.mode == kModeAngular && hi >= kHalfPiF;
    if (full || (low && high)) {
        k.kind = 1;
    } else if (low || high) {
        // across the seam of the [-pi/2, pi/2) domain: [ta, end) and [start, tb)
        k.ta = qmap(low ? lo + kPiF : lo, G.kmin, G.kscale) >> c.sh;
        k.tb = (qmap(low ? hi : hi - kPiF, G.kmin, G.kscale) >> c.sh) + 1;
        k.kind = 3;
    } else {
        k.ta = qmap(lo, G.kmin, G.kscale) >> c.sh;
        k.tb = (qmap(hi, G.kmin, G.kscale) >> c.sh) + 1;
        k.kind = 2;
    }
    return k;
}

// The brute force's FP64 decision for one (query, reference) pair of a
// single-pair call, from plain pointers.
static __device__ __noinline__ bool exact_pair_p(const double *F, const double *xy1, const double *xy2,
                                                 const double *eps2, double eps_scalar, int64_t i, uint32_t j) {
    double a, b, c;
    exact_line(F, xy1[2 * i], xy1[2 * i + 1], a, b, c);
    const double eps = eps2 ? eps2[j] : eps_scalar;
    return exact_within(a, b, c, xy2[2 * (int64_t)j], xy2[2 * (int64_t)j + 1], eps);
}

// G lanes read a descriptor row, C 16-byte chunks each (a row is G C 16 bytes).
template <int KIND, int G, int C, int MODE>
__global__ void __launch_bounds__(kPairThreads, 12) stab_pair_kernel(Launch L) {
    static_assert(G >= 1 && G <= 16 && (G & (G - 1)) == 0, "lanes per descriptor row");
    constexpr int kPerRound = 32 / G;  // candidates per round of loads
    constexpr int kRow16 = G * C;      // 16-byte chunks per row
    constexpr bool kDesc = MODE != 1;  // descriptor distances (the launcher checks that rows exist)
    pdl_begin();
    __shared__ __align__(16) PairGeom sg;
    __shared__ int32_t slv[kLevels];
    __shared__ int32_t snlev;
    __shared__ uint32_t ring[kPairWarps][kRing];
    __shared__ LevelWin slc[kLevels];
    // a warp's chunk of queries: their records, descriptor rows and window ranges
    __shared__ __align__(16) QueryRec qchunk[kPairWarps][kChunkQ];
    __shared__ __align__(16) uint4 dchunk[kPairWarps][kChunkQ][kRow16];
    __shared__ __align__(16) uint4 wrng[kPairWarps][kChunkQ * kLevels];
    __shared__ __align__(16) uint4 res[kPairWarps][kChunkQ];   // best two (distance, index) of each query
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt = (1u << lane) - 1u;
    for (int k = tid; k < (int)(sizeof(PairGeom) / 16); k += kPairThreads)
        reinterpret_cast<uint4 *>(&sg)[k] = __ldg(reinterpret_cast<const uint4 *>(L.geom) + k);
    __syncthreads();
    if (warp == 0) {
        const uint32_t nz = __ballot_sync(0xffffffffu, sg.cnt[lane] > 0);
        const int idx = __popc(nz & lt);
        if (nz & (1u << lane)) {
            slv[idx] = lane;
            slc[idx] = level_win(sg, lane);
        }
        if (lane == 0) snlev = __popc(nz);
    }
    __syncthreads();
    // the pair's fields, by value from the launch parameters
    const double *Fp = L.inl.F, *xy1 = L.inl.xy1, *xy2 = L.inl.xy2, *eps2 = L.inl.eps2;
    const double eps_scalar = L.inl.eps_scalar;
    const int64_t q_off = L.inl.q_off;
    const int nlev = snlev;
    const bool haslev = lane < nlev;
    const float4 *recb = L.rec + L.inl.r_off;
    uint32_t *rg = ring[warp];
    const int sub = lane % G, grp = lane / G;
    const uint4 *d1 = reinterpret_cast<const uint4 *>(L.inl.desc1);
    const uint4 *d2 = reinterpret_cast<const uint4 *>(L.inl.desc2);
    const bool write_rows = MODE == 2 && L.cand_offsets[L.nq] <= L.cand_capacity;
    const int64_t rnum = L.ratio_num, rden = L.ratio_den;
    uint32_t nwin = 0, ncand = 0, nexact = 0;
    const int64_t nwarps = (int64_t)gridDim.x * kPairWarps;
    // The warp's queries come in chunks of up to kChunkQ (q = c0 + k nwarps):
    // their records and descriptor rows are copied at once, and the windows
    // of every (query, level) slot of the chunk are computed in one pass over
    // the lanes, with their table loads issued together.
    for (int64_t c0 = (int64_t)blockIdx.x * kPairWarps + warp; c0 < L.nq; c0 += (int64_t)kChunkQ * nwarps) {
    const int nk = (int)min((int64_t)kChunkQ, (L.nq - c0 + nwarps - 1) / nwarps);
    for (int t = lane; t < 3 * nk; t += 32)
        cp_async16(reinterpret_cast<uint4 *>(&qchunk[warp][t / 3]) + t % 3,
                   reinterpret_cast<const uint4 *>(L.qrec + c0 + (int64_t)(t / 3) * nwarps) + t % 3);
    if (kDesc)
        for (int t = lane; t < kRow16 * nk; t += 32)
            cp_async16(&dchunk[warp][t / kRow16][t % kRow16],
                       d1 + (c0 + (int64_t)(t / kRow16) * nwarps - q_off) * kRow16 + t % kRow16);
    cp_async_wait();
    __syncwarp();
    for (int s0 = 0; s0 < nk * nlev; s0 += 32) {
        const int sl = s0 + lane;
        if (sl < nk * nlev) {
            const int k = sl / nlev, l = sl - k * nlev;
            const WinKeys wk = level_window(sg, slc[l], qchunk[warp][k]);
            uint32_t a = 0, b = 0;
            if (wk.kind >= 2) {
                const uint32_t *Tl = L.tab + L.inl.t_off + sg.tab[slv[l]];
                a = __ldg(Tl + wk.ta);
                b = __ldg(Tl + wk.tb);
            }
            const Window wl = window_ranges(wk, a, b);
            wrng[warp][k * kLevels + l] = make_uint4(wl.b0, wl.len0, wl.b1, wl.len1);
        }
    }
    __syncwarp();
    for (int k = 0; k < nk; k++) {
        const int64_t q = c0 + (int64_t)k * nwarps;
        const int64_t qi = q - q_off;
        const QueryRec rq = qchunk[warp][k];
        uint4 qdq[C];
#pragma unroll
        for (int c = 0; c < C; c++) qdq[c] = kDesc ? dchunk[warp][k][sub * C + c] : make_uint4(0u, 0u, 0u, 0u);
        // the window of this lane's level as (at most) two ranges of sorted positions
        Window w;
        w.b0 = w.len0 = w.b1 = w.len1 = 0u;
        if (haslev) {
            const uint4 v = wrng[warp][k * kLevels + lane];
            w.b0 = v.x;
            w.len0 = v.y;
            w.b1 = v.z;
            w.len1 = v.w;
        }
        const uint32_t tl = w.len0 + w.len1;
        uint32_t incl = tl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        const uint32_t p0 = incl - tl;  // first flattened element of this lane's ranges
        const uint32_t E = __shfl_sync(0xffffffffu, incl, 31);
        const bool exact_only = (rq.flags & kQExactOnly) != 0;
        uint32_t count = 0, done = 0;  // candidates found / already in a distance batch (warp-uniform)
        unsigned long long k1 = ~0ull, k2 = ~0ull;

        // one batch of nb <= 32 candidates from the ring, starting at `start`
        auto batch = [&](uint32_t start, uint32_t nb) {
            __syncwarp();
            uint32_t acc[G];
#pragma unroll
            for (int u = 0; u < G; u++) acc[u] = 0u;
#pragma unroll
            for (int u = 0; u < G; u++) {
                if ((uint32_t)(u * kPerRound) >= nb) break;
                const uint32_t c = (uint32_t)(u * kPerRound + grp);
                if (c < nb) {
                    const uint32_t jj = rg[(start + c) % kRing];
                    const uint4 *row = d2 + (int64_t)jj * kRow16 + sub * C;
                    uint4 rv[C];
#pragma unroll
                    for (int cc = 0; cc < C; cc++) rv[cc] = __ldg(row + cc);
                    float unused = 0.0f;
#pragma unroll
                    for (int cc = 0; cc < C; cc++) chunk_dist<KIND>(KIND, qdq[cc], rv[cc], acc[u], unused);
                }
            }
            // transposed butterfly: after the step over lane bit h a lane keeps
            // the rounds whose bit h equals its own, summed with its partner's
#pragma unroll
            for (int h = G / 2; h >= 1; h >>= 1) {
                const bool up = (sub & h) != 0;
#pragma unroll
                for (int k = 0; k < h; k++) {
                    const uint32_t send = up ? acc[k] : acc[k + h];
                    const uint32_t keep = up ? acc[k + h] : acc[k];
                    acc[k] = keep + __shfl_xor_sync(0xffffffffu, send, h);
                }
            }
            // lane (grp, sub) now holds the full distance of round sub
            const uint32_t c = (uint32_t)(sub * kPerRound + grp);
            if (c < nb) top2_key(((unsigned long long)acc[0] << 32) | rg[(start + c) % kRing], k1, k2);
            __syncwarp();
        };

        for (uint32_t base = 0; base < E; base += 32) {
            const uint32_t e = base + (uint32_t)lane;
            // the lane whose ranges hold element e: the last one whose first
            // element is <= e (it has elements, since the next one starts after e)
            int o = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1)
                if (__shfl_sync(0xffffffffu, p0, o + st) <= e) o += st;
            const uint32_t ob0 = __shfl_sync(0xffffffffu, w.b0, o), ol0 = __shfl_sync(0xffffffffu, w.len0, o);
            const uint32_t ob1 = __shfl_sync(0xffffffffu, w.b1, o), op0 = __shfl_sync(0xffffffffu, p0, o);
            bool cand = false;
            uint32_t j = 0;
            if (e < E) {
                const uint32_t off = e - op0;
                const float4 rc = __ldg(recb + (off < ol0 ? ob0 + off : ob1 + (off - ol0)));
                j = __float_as_uint(rc.w);
                nwin++;
                bool exact = exact_only;
                if (!exact) {
                    const float x = rc.x, y = rc.y, ee = rc.z;
                    const float d = fabsf(fmaf(rq.A, x, fmaf(rq.B, y, rq.C)));
                    const float Sm = fmaf(fabsf(rq.A), fabsf(x), fmaf(fabsf(rq.B), fabsf(y), fabsf(rq.C)));
                    // FP32 rounding (16u S), the FP32 tolerance (2u eps) and the
                    // distance between this line and the brute force's FP64 line
                    const float lerr = fmaf(rq.E1, fabsf(x) + fabsf(y) + 2.0f * ee, rq.E0);
                    const float bound = fmaf(9.6e-7f, Sm, fmaf(1.2e-7f, ee, lerr + 1e-9f));
                    cand = d <= ee - bound;
                    exact = !cand && !(d > ee + bound);
                }
                if (exact) {
                    // FP32 inconclusive: the brute-force FP64 expression decides
                    cand = exact_pair_p(Fp, xy1, xy2, eps2, eps_scalar, qi, j);
                    nexact++;
                }
            }
            const uint32_t m = __ballot_sync(0xffffffffu, cand);
            if (cand) {
                const uint32_t slot = count + (uint32_t)__popc(m & lt);
                if (MODE == 2 && write_rows) L.cand_idx[L.cand_offsets[q] + slot] = (int32_t)j;
                if (kDesc) rg[slot % kRing] = j;
            }
            count += (uint32_t)__popc(m);
            if (kDesc && count - done >= 32u) {
                batch(done, 32u);
                done += 32u;
            }
        }
        if (kDesc && count > done) batch(done, count - done);
        ncand += count;
        if (MODE == 1) {
            if (lane == 0) L.qcount[q] = count;
            continue;
        }
        // the query's best two over the lanes' best two: (distance, index) minima
        const uint32_t dk1 = (uint32_t)(k1 >> 32), jk1 = (uint32_t)k1;
        const uint32_t md = __reduce_min_sync(0xffffffffu, dk1);
        const uint32_t mj = __reduce_min_sync(0xffffffffu, dk1 == md ? jk1 : 0xffffffffu);
        const unsigned long long c2 = (dk1 == md && jk1 == mj) ? k2 : k1;
        const uint32_t dk2 = (uint32_t)(c2 >> 32), jk2 = (uint32_t)c2;
        const uint32_t sd = __reduce_min_sync(0xffffffffu, dk2);
        const uint32_t sj = __reduce_min_sync(0xffffffffu, dk2 == sd ? jk2 : 0xffffffffu);
        // the query's best two wait in shared memory; lane k writes query k's
        // outputs after the chunk
        if (lane == 0) res[warp][k] = make_uint4(md, mj, sd, sj);
    }
    __syncwarp();
    if (MODE != 1 && lane < nk) {
        // outputs as store_match writes them (integer distances; Sec. 5.1 ratio
        // test in exact integer form)
        const int64_t q = c0 + (int64_t)lane * nwarps;
        const uint4 rr = res[warp][lane];
        const uint32_t md = rr.x, mj = rr.y, sd = rr.z, sj = rr.w;
        uint32_t fl = qchunk[warp][lane].flags & EGM_FLAG_DEGENERATE_LINE;
        const bool has1 = md != 0xffffffffu || mj != 0xffffffffu;
        const bool has2 = sd != 0xffffffffu || sj != 0xffffffffu;
        if (has1) {
            fl |= EGM_FLAG_HAS_BEST;
            bool pass;
            if (!has2) {
                fl |= EGM_FLAG_NO_SECOND;
                pass = true;
            } else if (KIND == EGM_DESC_U8_L2) {
                pass = (long long)md * rden * rden < (long long)sd * rnum * rnum;
            } else {
                pass = (long long)md * rden < (long long)sd * rnum;
            }
            if (pass) fl |= EGM_FLAG_RATIO_PASS;
        }
        if (L.best) L.best[q] = has1 ? (int32_t)mj : -1;
        if (L.second) L.second[q] = has2 ? (int32_t)sj : -1;
        if (L.best_d) L.best_d[q] = has1 ? (float)md : INFINITY;
        if (L.second_d) L.second_d[q] = has2 ? (float)sd : INFINITY;
        if (L.flags) L.flags[q] = (uint8_t)fl;
    }
    __syncwarp();  // the chunk's buffers are read before the next chunk's copies
    }
    if (L.counters) {
        const uint32_t a = __reduce_add_sync(0xffffffffu, nwin);
        const uint32_t b = __reduce_add_sync(0xffffffffu, lane == 0 ? ncand : 0u);
        const uint32_t c = __reduce_add_sync(0xffffffffu, nexact);
        if (lane == 0) {
            atomicAdd(L.counters + 2, (unsigned long long)a);
            atomicAdd(L.counters + 3, (unsigned long long)b);
            atomicAdd(L.counters + 4, (unsigned long long)c);
        }
    }
}

template <int KIND, int G, int C, int MODE>
cudaError_t launch_pair_mode(const Launch &L, int sms, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stab_pair_kernel<KIND, G, C, MODE>,
                                                                      kPairThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    int64_t blocks = (L.nq + kPairWarps - 1) / kPairWarps;
    blocks = std::min<int64_t>(blocks, (int64_t)per_sm * sms);
    return launch_pdl(stab_pair_kernel<KIND, G, C, MODE>, dim3((unsigned)blocks), dim3(kPairThreads), 0, s, L);
}

template <int KIND, int G, int C>
cudaError_t launch_pair(const Launch &L, int mode, int sms, cudaStream_t s) {
    switch (mode) {
        case 0: return launch_pair_mode<KIND, G, C, 0>(L, sms, s);
        case 1: return launch_pair_mode<KIND, G, C, 1>(L, sms, s);
        default: return launch_pair_mode<KIND, G, C, 2>(L, sms, s);
    }
}

}  // namespace

cudaError_t launch_stab(const Launch &L, int mode, cudaStream_t s) {
    if (L.nq == 0) return cudaSuccess;
    int64_t blocks = (L.nq + kQB - 1) / kQB;
    if (blocks > 152 * 8) blocks = 152 * 8;
    const dim3 g((unsigned)blocks), b(kStabThreads);
    // one pair with rows of 16..256 bytes, a power of two (u8 128-d, binary
    // 256-bit): the uniform variant
    const int rb = L.inl_use ? L.inl.row_bytes : 0;
    const bool one = L.npairs == 1 && L.inl_use && rb >= 16 && rb <= kDescCache && (rb & (rb - 1)) == 0;
    if (one && (L.kind == EGM_DESC_U8_L2 || L.kind == EGM_DESC_BIN)) {
        // one pair: a warp per query
        int sms = 0;
        cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
        if (e != cudaSuccess) return e;
        const bool u8 = L.kind == EGM_DESC_U8_L2;
        switch (rb >> 4) {
            // rows of 16 .. 256 bytes: a lane reads 32 bytes of a row (16 for 16-byte rows)
            case 1: return u8 ? launch_pair<EGM_DESC_U8_L2, 1, 1>(L, mode, sms, s) : launch_pair<EGM_DESC_BIN, 1, 1>(L, mode, sms, s);
            case 2: return u8 ? launch_pair<EGM_DESC_U8_L2, 1, 2>(L, mode, sms, s) : launch_pair<EGM_DESC_BIN, 1, 2>(L, mode, sms, s);
            case 4: return u8 ? launch_pair<EGM_DESC_U8_L2, 2, 2>(L, mode, sms, s) : launch_pair<EGM_DESC_BIN, 2, 2>(L, mode, sms, s);
            case 8: return u8 ? launch_pair<EGM_DESC_U8_L2, 4, 2>(L, mode, sms, s) : launch_pair<EGM_DESC_BIN, 4, 2>(L, mode, sms, s);
            default: return u8 ? launch_pair<EGM_DESC_U8_L2, 8, 2>(L, mode, sms, s) : launch_pair<EGM_DESC_BIN, 8, 2>(L, mode, sms, s);
        }
    }
    switch (L.kind) {
        case EGM_DESC_U8_L2: return launch_pdl(stab_kernel<EGM_DESC_U8_L2>, g, b, 0, s, L, mode);
        case EGM_DESC_BIN: return launch_pdl(stab_kernel<EGM_DESC_BIN>, g, b, 0, s, L, mode);
        case EGM_DESC_F32_L2: return launch_pdl(stab_kernel<EGM_DESC_F32_L2>, g, b, 0, s, L, mode);
        default: return launch_pdl(stab_kernel<kKindAny>, g, b, 0, s, L, mode);
    }
}

}  // namespace egm
