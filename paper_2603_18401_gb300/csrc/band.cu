// Banded matching on the tensor cores.
//
// Queries sorted by the angle of their epipolar line (Sec. 4.2, alpha_i) and
// references sorted by the angle of their tolerance interval (theta_j) make
// the candidate blocks of a tile of consecutive queries dense: the union of
// the tile's stabbing windows is a few contiguous runs of sorted references
// (one or two per level).  All descriptor dot products of the tile against
// those runs are one dense product on the tensor cores; the exact membership
// test of Eq. 3 / Eq. 4 then selects, per query, the entries that count.
//
//   query_sort_kernel  one block per pair: counting sort of the queries by
//                      the top bits of their quantised line angle; lines
//                      without an FP32 view (FP64-only, degenerate) last.
//   pack_kernel        float pairs only: descriptor rows of the sorted
//                      references and queries as 256-byte BF16 (or E4M3)
//                      operands, with the norm of the rounded row and the
//                      rounding error |x - x~|, and the sorted query records
//   band_kernel        persistent; one tile of 128 sorted queries at a time.
//                      Warps 0-3 (one thread per query) build the tile's band
//                      from the hull of their windows; warp 4 issues the bulk
//                      loads of the band's sorted records (32-row boxes) and
//                      the tcgen05.mma chain (M = 128, N = 32 per box, K = 128)
//                      into a double-buffered TMEM accumulator.  Operands:
//                        u8 rows     gathered by warps 0-3 straight from the
//                                    caller's descriptors (cp.async, 128 bytes
//                                    a row) and widened in shared memory to
//                                    FP16, exact (integers < 2^11)
//                        float rows  the packed BF16 / E4M3 rows, by TMA
//                        binary rows gathered as they are (32 bytes); no
//                                    product: Hamming distances are popcounts
//                      Warps 0-3 read their lanes back, run the exact test on
//                      the columns in their own windows, and keep the best two
//                      by (distance, index):
//                        L2^2    = |q|^2 + |r|^2 - 2 q.r   (integers < 2^24: exact in FP32)
//                        Hamming = popcount(q xor r)
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "egm_internal.cuh"
#include "tc.cuh"

namespace egm {

namespace {

// ------------------------------------------------------------ query order
constexpr int kQSortThreads = 1024;
constexpr int kQSortPer = 16;  // bucket loads a thread issues before its atomics

__global__ void __launch_bounds__(kQSortThreads) query_sort_kernel(Launch L) {
    pdl_begin();
    __shared__ uint32_t hist[kQBuckets];
    __shared__ uint32_t wsum[kQSortThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.x == 0 && tid == 0) *L.work = 0u;  // the band kernel's tile dispenser
    const PairDesc &P = L.pairs[blockIdx.x];
    const int m = P.m;
    if (m == 0) return;
    const uint16_t *bk = L.qbkt + P.q_off;
    for (int b = tid; b < kQBuckets; b += kQSortThreads) hist[b] = 0;
    __syncthreads();
    for (int i0 = 0; i0 < m; i0 += kQSortThreads * kQSortPer) {
        uint32_t v[kQSortPer];
#pragma unroll
        for (int k = 0; k < kQSortPer; k++) {
            const int i = i0 + k * kQSortThreads + tid;
            v[k] = i < m ? __ldg(bk + i) : 0xffffu;
        }
#pragma unroll
        for (int k = 0; k < kQSortPer; k++)
            if (v[k] != 0xffffu) atomicAdd(&hist[v[k]], 1u);
    }
    __syncthreads();
    // exclusive scan: thread t owns buckets [kPer t, kPer t + kPer)
    constexpr int kPer = (kQBuckets + kQSortThreads - 1) / kQSortThreads;
    uint32_t c[kPer], tot = 0;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        const int b = tid * kPer + k;
        c[k] = b < kQBuckets ? hist[b] : 0u;
        tot += c[k];
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = wsum[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += x;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - tot;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        const int b = tid * kPer + k;
        if (b < kQBuckets) hist[b] = run;
        run += c[k];
    }
    __syncthreads();
    for (int i0 = 0; i0 < m; i0 += kQSortThreads * kQSortPer) {
        uint32_t v[kQSortPer];
#pragma unroll
        for (int k = 0; k < kQSortPer; k++) {
            const int i = i0 + k * kQSortThreads + tid;
            v[k] = i < m ? __ldg(bk + i) : 0xffffu;
        }
#pragma unroll
        for (int k = 0; k < kQSortPer; k++) {
            const int i = i0 + k * kQSortThreads + tid;
            if (v[k] != 0xffffu) L.qperm[P.q_off + atomicAdd(&hist[v[k]], 1u)] = (uint32_t)i;
        }
    }
}

// ------------------------------------------------------------ packing
constexpr int kRowB = 256;  // packed operand row: 128 BF16 or 256 E4M3 values
constexpr int kBinRowB = 32;  // binary row (256 bits), kept as it is

// Float rows only (u8 and binary rows go to the band kernel as they are).
// 8 threads per row; thread part t writes output bytes [32 t, 32 t + 32).
// F8: float rows packed for the FP8 pass (a separate variant: its staged
// values would cost the common variant registers and occupancy).
template <bool F8>
__global__ void __launch_bounds__(256) pack_kernel(Launch L) {
    pdl_begin();
    const int64_t rows = L.nr + L.nq;
    const int part = threadIdx.x & 7;
    __shared__ int64_t s_roffs[kSmemPairs + 1], s_qoffs[kSmemPairs + 1];
    const bool cached = load_offsets(s_roffs, L.r_offs, L.npairs) && load_offsets(s_qoffs, L.q_offs, L.npairs);
    __syncthreads();
    for (int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3; g0 < ((rows + 3) / 4) * 4;
         g0 += ((int64_t)gridDim.x * blockDim.x) >> 3) {
        bool use = g0 < rows;  // a float row (every thread of the row's group agrees)
        const bool is_ref = g0 < L.nr;
        uint32_t qi = 0;
        float fnrm = 0.0f, ferr = 0.0f;  // squared norm of the rounded row, squared rounding error
        float xs8[16];                   // FP8 pass: this thread's 16 values, kept for the second step
        float amax = 0.0f;               //   and their largest magnitude
        uint4 o0 = make_uint4(0, 0, 0, 0), o1 = o0, qr = o0;
        uint8_t *dst = nullptr;
        const int64_t g = is_ref ? g0 : g0 - L.nr;
        const PairDesc *PP = nullptr;
        if (use) {
            const int p = cached ? pair_of_shared(is_ref ? s_roffs : s_qoffs, L.npairs, g)
                                 : pair_of(is_ref ? L.r_offs : L.q_offs, L.npairs, g);
            PP = L.pairs + p;
            use = PP->kind == EGM_DESC_F32_L2;
        }
        if (use) {
            const PairDesc &P = *PP;
            const uint8_t *src;
            if (is_ref) {
                const uint32_t j = __float_as_uint(L.rec[g].w);
                src = P.desc2 + (int64_t)j * P.row_bytes;
                dst = L.descB + g * kRowB;
            } else {
                qi = L.qperm[g];
                src = P.desc1 + (int64_t)qi * P.row_bytes;
                dst = L.descA + g * kRowB;
                if (part < 3) qr = __ldg(reinterpret_cast<const uint4 *>(L.qrec + P.q_off + qi) + part);
            }
            if (F8) {
                // FP8 pass, step 1: 16 values per thread and their largest magnitude
                // (the row's scale needs the maximum over its 8 threads)
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + 4 * part + c);
                    xs8[4 * c] = v.x;
                    xs8[4 * c + 1] = v.y;
                    xs8[4 * c + 2] = v.z;
                    xs8[4 * c + 3] = v.w;
                    amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
                }
            } else {
                // 16 values per thread: 64 bytes in, 32 bytes of BF16 out
                uint32_t out[8];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + 4 * part + c);
                    const float xs[4] = {v.x, v.y, v.z, v.w};
                    float b[4];
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        b[k] = __bfloat162float(__float2bfloat16_rn(xs[k]));
                        fnrm = fmaf(b[k], b[k], fnrm);
                        const float d = xs[k] - b[k];  // exact: b is x rounded to 8 bits
                        ferr = fmaf(d, d, ferr);
                    }
                    out[2 * c] = (__float_as_uint(b[0]) >> 16) | (__float_as_uint(b[1]) & 0xffff0000u);
                    out[2 * c + 1] = (__float_as_uint(b[2]) >> 16) | (__float_as_uint(b[3]) & 0xffff0000u);
                }
                o0 = make_uint4(out[0], out[1], out[2], out[3]);
                o1 = make_uint4(out[4], out[5], out[6], out[7]);
            }
        }
        // FP8 pass, step 2: the row's scale s = max |x| / 448 (E4M3's largest
        // value); the operand holds e4m3(x / s) in bytes 0..127 and zeros in
        // 128..255, and the squared norm and rounding error are those of
        // s e4m3(x / s), the row the tensor cores see
        float scale = 1.0f;
        if (F8) {
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o, 8));
        }
        if (F8 && use) {
            const float inv = amax > 0.0f ? 448.0f / amax : 1.0f;
            scale = amax > 0.0f ? amax / 448.0f : 1.0f;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const __nv_fp8_storage_t e = __nv_cvt_float_to_fp8(xs8[k] * inv, __NV_SATFINITE, __NV_E4M3);
                const float b = __half2float(__half(__nv_cvt_fp8_to_halfraw(e, __NV_E4M3))) * scale;
                fnrm = fmaf(b, b, fnrm);
                const float d = xs8[k] - b;
                ferr = fmaf(d, d, ferr);
                w[k >> 2] |= (uint32_t)e << (8 * (k & 3));
            }
            o0 = make_uint4(w[0], w[1], w[2], w[3]);
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            fnrm += __shfl_xor_sync(0xffffffffu, fnrm, o, 8);
            ferr += __shfl_xor_sync(0xffffffffu, ferr, o, 8);
        }
        // norm of the operand row and |x - x~|, rounded up
        const float err = sqrtf(ferr) * 1.0001f + 1e-30f;
        if (use) {
            if (F8) {
                // 16 bytes per thread: bytes [16 part, 16 part + 16), zeros above 128
                reinterpret_cast<uint4 *>(dst)[part] = o0;
                reinterpret_cast<uint4 *>(dst)[8 + part] = make_uint4(0u, 0u, 0u, 0u);
            } else {
                reinterpret_cast<uint4 *>(dst)[2 * part] = o0;
                reinterpret_cast<uint4 *>(dst)[2 * part + 1] = o1;
            }
            if (is_ref) {
                if (part == 0) L.rnorm[g0] = make_float4(fnrm, err, scale, 0.0f);
            } else if (part < 3) {
                if (part == 0) L.qscale[g0 - L.nr] = scale;
                // sorted query record; the padding carries the query index and the
                // norm, the pair field (the tile knows its pair) the rounding error
                if (part == 2) {
                    qr.y = __float_as_uint(err);
                    qr.z = qi;
                    qr.w = __float_as_uint(fnrm);
                }
                reinterpret_cast<uint4 *>(L.qsrt + (g0 - L.nr))[part] = qr;
            }
        }
    }
}

// ------------------------------------------------------------ band kernel
constexpr int kTM = 128;                 // queries per tile (MMA M, TMEM lanes)
constexpr int kBoxR = 32;                // reference rows per TMA box (N per box)
constexpr int kBandThreads = kTM + 32;   // four epilogue warps and the control warp
// Tile shapes (chosen per call regime by the tuner): CB boxes per MMA chunk
// (N = 32 CB) and CPS resident CTAs per SM, which size shared memory and TMEM.
//   0: CB 4, CPS 2   few tiles per SM (single pairs): fewer, larger chunks
//   1: CB 2, CPS 3   many tiles (batches): more CTAs in flight per SM
//   2: CB 1, CPS 4   many tiles: more CTAs still, more synchronisation per box
//   3: CB 1, CPS 3   4: CB 2, CPS 2   5: CB 4, CPS 1   6: CB 1, CPS 2
// Every shape whose CPS CTAs fit the SM's shared memory (CB 1: up to 4,
// CB 2: up to 3, CB 4: up to 2) except CPS 1 with CB 1 or 2.
constexpr int kGroup = 8;                // columns per TMEM load in the epilogue

struct __align__(16) Piece {
    uint32_t start, len, box0;
    int32_t li;
};

// A tile as the control thread hands it out: its pair, the pair's first
// query slot, the tile's first sorted slot and its query count.
struct TileDesc {
    int64_t q_off, q_first;
    int32_t pair, mt, kind;  // pair -1: no tile left
};

constexpr uint32_t kOperandArrivals = 5; // afull: the control thread and the four consumer warps
constexpr int kDeferCap = 16;            // FP64 tests a warp defers per tile (more: decided at once)
constexpr int kRS = 4;                   // record / norm / binary-row slots (chunk g in slot g mod kRS)

template <int CB, bool FLT, int NB>
struct BandSmem {
    static constexpr int kCN = kBoxR * CB;  // columns per chunk
    // query tile, K halves (1024-byte aligned); u8 tiles stage each query's
    // bytes in its own row of A[1] before widening them
    uint8_t A[2][kTM * 128];
    // band chunk: operand stage (NB of them), K half.  u8 tiles stage a chunk's
    // gathered bytes in K half 1 of its stage; binary tiles keep kRS chunks of
    // 32-byte rows (chunk g in slot g mod kRS) in B[0][0]
    uint8_t B[NB][2][kCN * 128];
    // The record slots are idle while a tile's windows are computed (every
    // chunk of the previous tile has been tested, and the next records are
    // copied after), so the per-warp hulls share their memory.
    union {
        struct {
            float4 rec[kRS][kCN];                  // (x - cx, y - cy, eps, index) of each column
            float4 rn[FLT ? kRS : 1][CB][kBoxR];   // float rows: (norm, rounding error, row scale, 0)
            float n8[kRS][kCN];                    // u8 rows: squared norms
        } io;
        struct {
            float wlo[4][kLevels], whi[4][kLevels];  // each consumer warp's hull per level index
            int32_t wkind[4][kLevels];
        } hull;
    } u;
    // fullR: a slot's records (and float norms) landed; rows: the producer has
    // written a chunk's rows (u8 norms, binary rows); rfree: the consumers have
    // finished a slot's chunk; sfree: the MMA that read an operand stage is
    // done; fullB: a stage's float rows landed (TMA); done: an accumulator is
    // ready; tfree: the consumers have read it
    uint64_t fullR[kRS], rows[kRS], rfree[kRS], sfree[NB], fullB[NB], done[4], tfree[4], afull;
    uint64_t probe;               // never arrived on: the wait of the timeout check (Launch::probe)
    PairGeom g;
    PairDesc pd;
    Piece pc[2 * kLevels];
    int32_t lv[kLevels];
    int32_t nlev, npc, nbox, gpair;
    TileDesc td, tdn, tdnn;       // the tile being processed; the next two
    // u8 and binary tiles: each consumer warp's pairs left to the FP64 test,
    // (distance key, reference, owner lane), decided together at the tile end
    uint4 xq[4][kDeferCap];
    uint32_t xn[4];
    uint32_t tmem;
    volatile uint32_t err;
};

template <int CB, int CPS, bool FLT>
struct BandShape {
    static constexpr int kCB = CB, kCN = kBoxR * CB;
    // accumulators: four where TMEM holds them for CPS CTAs, else two
    static constexpr int kNA = 512 / (CPS * kCN) >= 4 ? 4 : 2;
    static constexpr uint32_t kTmemCols = kNA * kCN;  // a power of two
    static constexpr size_t kSmPerSm = 228 * 1024;
    // operand stages: three where the shared memory holds them for CPS CTAs
    static constexpr int kNB = CPS * (sizeof(BandSmem<CB, FLT, 3>) + 2048) <= kSmPerSm ? 3 : 2;
    using Smem = BandSmem<CB, FLT, kNB>;
    static_assert(offsetof(Smem, B) % 1024 == 0, "operand tiles need 1024-byte alignment");
    static_assert(kTM * sizeof(QueryRec) <= sizeof(Smem::B[1]), "a tile's query records fit operand stage 1");
    static_assert(offsetof(Smem, u) % 16 == 0, "bulk copy destinations need 16-byte alignment");
    static_assert(kRS * kCN * kBinRowB <= sizeof(Smem::B[0][0]), "binary rows fit their slots");
    // CPS CTAs per SM share the 512 TMEM columns; the shared memory a CTA asks
    // for (its layout, 1 KB of alignment slack, the 1 KB the SM reserves per
    // CTA) keeps one more from becoming resident (its TMEM allocation would
    // wait for another CTA to end)
    static constexpr size_t kDynSmem = sizeof(Smem) + 1024 > kSmPerSm / (CPS + 1) + 1 - 1024
                                           ? sizeof(Smem) + 1024
                                           : kSmPerSm / (CPS + 1) + 1 - 1024;
    static_assert(CPS * (kDynSmem + 1024) <= kSmPerSm && (CPS + 1) * (kDynSmem + 1024) > kSmPerSm,
                  "shared memory admits exactly CPS CTAs per SM");
    static_assert(CPS * kTmemCols <= 512 && (kTmemCols & (kTmemCols - 1)) == 0, "TMEM columns");
};

__device__ __forceinline__ int sortable(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float unsortable(int b) { return __int_as_float(b >= 0 ? b : b ^ 0x7fffffff); }

// Walks the tile's boxes in order: piece k, box b within the piece.
struct BoxCursor {
    int k = 0;
    uint32_t b = 0;
    template <class SM>
    __device__ __forceinline__ void next(const SM &S, uint32_t &pos, uint32_t &len, int &li) {
        const Piece &pc = S.pc[k];
        pos = pc.start + b * kBoxR;
        len = min((uint32_t)kBoxR, pc.len - b * kBoxR);
        li = pc.li;
        if (++b * kBoxR >= pc.len) {
            k++;
            b = 0;
        }
    }
};

__device__ __forceinline__ void copy16(void *dst, const void *src, int bytes, int lane) {
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (int k = lane; k < bytes / 16; k += 32) d4[k] = __ldg(s4 + k);
}

// ---- float descriptors: BF16 tensor-core pass, FP32 rerank
//
// For rows q, r with BF16 roundings q~, r~ (|q - q~| <= eq, |r - r~| <= er) the
// squared distances d = |q - r|^2 and d~ = |q~ - r~|^2 satisfy
// |d - d~| <= 2 sqrt(d~) D + D^2 with D = eq + er.  d~ is evaluated as
// |q~|^2 + |r~|^2 - 2 q~.r~ in FP32 (products of BF16 values are exact; the
// sums of 128 terms are within 3e-5 (|q~|^2 + |r~|^2), a wide allowance for the
// tensor core's accumulation), and the rerank's FP32 evaluation of d is within
// 1e-4 relative of d.  A candidate whose lower bound exceeds the second
// smallest upper bound cannot be among the best two.
constexpr int kFBuf = 8;  // candidates kept per query for the rerank

__device__ __forceinline__ void float_bounds(float dt, float qn, float rn, float eq, float er, float &lo, float &hi) {
    const float efp = 3.0e-5f * (qn + rn) + 1e-30f;
    const float D = eq + er;
    const float sd = sqrtf(fmaxf(dt + efp, 0.0f));
    const float E = fmaf(2.0f * sd, D, fmaf(D, D, efp));
    hi = (dt + E) * 1.0001f + 1e-30f;
    lo = (dt - E) - 1.0e-4f * fabsf(dt + E) - 1e-30f;
}

// The candidates of one query that can still be among its best two: lower
// bounds (L, +inf when free) and indices, the two smallest upper bounds seen,
// and the smallest lower bound ever dropped for lack of room.
struct FBuf {
    float U1, U2, drop;
    float L[kFBuf];
    uint32_t J[kFBuf];
    __device__ __forceinline__ void init() {
        U1 = U2 = drop = INFINITY;
#pragma unroll
        for (int t = 0; t < kFBuf; t++) {
            L[t] = INFINITY;
            J[t] = 0u;
        }
    }
    __device__ __forceinline__ void insert(float lo, float up, uint32_t j) {
        if (up < U1) {
            U2 = U1;
            U1 = up;
        } else if (up < U2) {
            U2 = up;
        }
        if (!(lo <= U2)) return;
        int slot = -1, mxs = 0;
        float mx = -INFINITY;
#pragma unroll
        for (int t = 0; t < kFBuf; t++) {
            if (L[t] > U2) L[t] = INFINITY;  // out for good: U2 only decreases
            if (slot < 0 && L[t] == INFINITY) slot = t;
            if (L[t] > mx) {
                mx = L[t];
                mxs = t;
            }
        }
        if (slot < 0) {  // full: keep the smaller lower bounds
            if (lo < mx) {
                drop = fminf(drop, mx);
                slot = mxs;
            } else {
                drop = fminf(drop, lo);
                return;
            }
        }
#pragma unroll
        for (int t = 0; t < kFBuf; t++)
            if (t == slot) {
                L[t] = lo;
                J[t] = j;
            }
    }
    // every reference that can be among the best two is in the buffer
    __device__ __forceinline__ bool complete() const { return drop > U2; }
};

// FP32 squared distance of the query row (this lane's 16-byte chunk in qv)
// and the reference row at r, in the plain kernel's order: four fused
// multiply-adds per lane, then an XOR butterfly over the warp.
__device__ __forceinline__ float coop_dist(const float4 &qv, const uint8_t *r, int lane) {
    const float4 rv = __ldg(reinterpret_cast<const float4 *>(r) + lane);
    float acc = 0.0f, d;
    d = qv.x - rv.x; acc = fmaf(d, d, acc);
    d = qv.y - rv.y; acc = fmaf(d, d, acc);
    d = qv.z - rv.z; acc = fmaf(d, d, acc);
    d = qv.w - rv.w; acc = fmaf(d, d, acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// Eq. 3 / Eq. 4 in FP32 with the rigorous bound: 1 member, 0 not, 2 inconclusive.
__device__ __forceinline__ int member32(float A, float B, float C, float E0, float E1, const float4 &rc) {
    const float x = rc.x, y = rc.y, e = rc.z;
    const float d = fabsf(fmaf(A, x, fmaf(B, y, C)));
    const float Sm = fmaf(fabsf(A), fabsf(x), fmaf(fabsf(B), fabsf(y), fabsf(C)));
    const float lerr = fmaf(E1, fabsf(x) + fabsf(y) + 2.0f * e, E0);
    const float bound = fmaf(9.6e-7f, Sm, fmaf(1.2e-7f, e, lerr + 1e-9f));
    if (d <= e - bound) return 1;
    return d > e + bound ? 0 : 2;
}

__device__ __forceinline__ void top2(unsigned long long key, unsigned long long &b1, unsigned long long &b2) {
    if (key < b1) {
        b2 = b1;
        b1 = key;
    } else if (key < b2) {
        b2 = key;
    }
}

// ---- u8 rows as FP16 tensor-core operands.  For a byte b, the halfword
// 0x6400 | b is the FP16 number 1024 + b (spacing 1 in [1024, 2048)), so one
// packed subtraction of 1024 gives b exactly; products of such integers and
// their sums of 128 terms (below 2^24) are exact in the FP32 accumulator.
__device__ __forceinline__ uint32_t h2_minus_1024(uint32_t x) {
    uint32_t y;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(y) : "r"(x), "r"(0x64006400u));
    return y;
}

// 16 bytes in, their FP16 values out (o0: bytes 0-7, o1: bytes 8-15); adds
// the bytes' squared sum to nrm.
__device__ __forceinline__ void widen16(const uint4 w, uint4 &o0, uint4 &o1, uint32_t &nrm) {
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    uint32_t o[8];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        o[2 * k] = h2_minus_1024(__byte_perm(ws[k], 0x64u, 0x4140u));
        o[2 * k + 1] = h2_minus_1024(__byte_perm(ws[k], 0x64u, 0x4342u));
        nrm = __dp4a(ws[k], ws[k], nrm);
    }
    o0 = make_uint4(o[0], o[1], o[2], o[3]);
    o1 = make_uint4(o[4], o[5], o[6], o[7]);
}

// The k-th tile handed out (tile_seq holds each tile's index and pair).
__device__ __forceinline__ TileDesc fetch_tile(const Launch &L, uint32_t k) {
    TileDesc d;
    d.pair = -1;
    d.q_off = d.q_first = 0;
    d.mt = d.kind = 0;
    if (k >= (uint64_t)L.ntiles) return d;
    const int2 ts = L.tile_seq[k];
    const int p = ts.y;
    d.pair = p;
    d.q_off = L.q_offs[p];
    d.q_first = d.q_off + ((int64_t)ts.x - L.tile_offs[p]) * kTM;
    d.mt = (int)min((int64_t)kTM, L.q_offs[p + 1] - d.q_first);
    d.kind = L.pairs[p].kind;
    return d;
}

// a[k] for a lane-dependent k in [0, 8), by a tree of selects (no local memory).
__device__ __forceinline__ uint32_t pick8(const uint32_t (&a)[8], int k) {
    const bool b0 = k & 1, b1 = k & 2, b2 = k & 4;
    const uint32_t a01 = b0 ? a[1] : a[0], a23 = b0 ? a[3] : a[2], a45 = b0 ? a[5] : a[4], a67 = b0 ? a[7] : a[6];
    const uint32_t a03 = b1 ? a23 : a01, a47 = b1 ? a67 : a45;
    return b2 ? a47 : a03;
}

// Byte offset of 16-byte chunk c of row r in a 128-byte-swizzled operand tile.
__device__ __forceinline__ uint32_t sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// FLT: float descriptor pairs may occur (compiled out otherwise: the rerank
// state costs registers).
//
// Roles.  Warps 0-3 (the consumers, one thread per query of the tile): the
// query records, their windows' hulls, the u8 query rows widened to FP16,
// and per chunk the exact tests and the best two over their own columns.
// Warp 4 (the producer): the tile's windows as runs of boxes; per chunk the
// band's rows -- u8 rows gathered by the sorted records' indices (one row
// per lane per box) and widened to FP16 in place, binary rows gathered into
// a slot -- then (lane 0, the control thread) the records' bulk copies, the
// tcgen05.mma chain and its commits.  Rings, indexed by the running chunk
// number g of the CTA:
//   records, u8 norms, binary rows   kRS slots (g mod kRS); a slot is reused
//                                    once the consumers have finished its chunk
//   operand stages                   2 (g mod 2); reused once the chunk's MMA is done
//   accumulators                     kNA (g mod kNA); reused once the consumers
//                                    have read them
// so the producer runs up to kNA - 1 chunks ahead of the consumers and the
// consumers do not wait for each other's rows.
template <int CB, int CPS, bool FLT>
__global__ void __launch_bounds__(kBandThreads, CPS)
    band_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Launch L) {
    pdl_begin();
    using Shape = BandShape<CB, CPS, FLT>;
    using BandSmem = typename Shape::Smem;
    constexpr int kCB = Shape::kCB, kCN = Shape::kCN, kNA = Shape::kNA, kNB = Shape::kNB;
    constexpr uint32_t kTmemCols = Shape::kTmemCols;
    extern __shared__ uint8_t smraw[];
    // 1024-byte alignment by pointer arithmetic on the shared array, so that
    // accesses through S stay shared-memory accesses
    BandSmem &S = *reinterpret_cast<BandSmem *>(smraw + ((1024u - (tc::smem_addr(smraw) & 1023u)) & 1023u));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const bool ctl = tid == kTM;
    if (ctl) {
        for (int s = 0; s < kRS; s++) {
            tc::mbar_init(&S.fullR[s], 1);
            tc::mbar_init(&S.rows[s], 1);
            tc::mbar_init(&S.rfree[s], 4);
        }
        for (int s = 0; s < kNB; s++) {
            tc::mbar_init(&S.sfree[s], 1);
            tc::mbar_init(&S.fullB[s], 1);
        }
        for (int s = 0; s < kNA; s++) {
            tc::mbar_init(&S.done[s], 1);
            tc::mbar_init(&S.tfree[s], 4);
        }
        tc::mbar_init(&S.afull, kOperandArrivals);
        tc::mbar_init(&S.probe, 1);
        tc::fence_mbar_init();
        S.err = 0;
        S.gpair = -1;
        for (int w = 0; w < 4; w++) S.xn[w] = 0u;
        S.td = fetch_tile(L, atomicAdd(L.work, 1u));
        S.tdn = fetch_tile(L, atomicAdd(L.work, 1u));
        if (FLT) {
            tc::prefetch_tmap(&tmA);
            tc::prefetch_tmap(&tmB);
        }
    }
    if (warp == 4) {
        tc::tmem_alloc(&S.tmem, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = S.tmem;
    // a bounded wait; after any failure every later wait returns at once
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (S.err) return false;
        if (tc::mbar_wait(bar, parity)) return true;
        S.err = 1;
        atomicOr(L.status, kStTimeout);
        return false;
    };
    uint32_t seq = 0;                           // chunks of earlier tiles (the rings' running count)
    uint32_t nwin = 0, ncand = 0, nexact = 0;  // per-thread counts (counters on)
    // phases the control thread armed with copies or MMAs (records per slot,
    // float operand loads per stage, the query tile, the MMA chain): after a
    // failed wait, the CTA lets the last of each complete before it leaves
    uint32_t armR[kRS] = {}, armB[3] = {0u, 0u, 0u}, armA = 0u, lastD = 0u;
    bool anyD = false, txA = false;
    if (L.probe) {
        // the timeout check: a short wait on a barrier that nothing arrives
        // on, before any copy or MMA is issued, takes the error path below
        if (ctl && !tc::mbar_wait(&S.probe, 0u, 10000ull)) {
            S.err = 1;
            atomicOr(L.status, kStTimeout);
        }
        __syncthreads();
    }

    // the next tile's query record (u8 and binary pairs), copied at the end of
    // a tile into the operand stage 1 (idle by then) while the tile ends
    bool staged = false;
    uint32_t qi_next = 0;
    int64_t qoff_next = 0;
    for (;;) {
        const TileDesc td = S.td;
        if (td.pair < 0 || S.err) break;
        const int p = td.pair, mt = td.mt, kind = td.kind;
        const int64_t q_off = td.q_off, q_first = td.q_first;
        // binary pairs: Hamming distances by popcount, no operand rows; float
        // pairs: packed rows by TMA; u8 pairs: rows widened here
        const bool pop = kind == EGM_DESC_BIN;
        const bool flt = FLT && kind == EGM_DESC_F32_L2;
        const bool cvt = !pop && !flt;
        // ---- the tile's queries: records in sorted order (float pairs: with
        // norm and rounding error in the padding), else through the order
        QueryRec r;
        const bool qv = warp < 4 && tid < mt;
        uint32_t qi = 0;
        float qn = 0.0f, qerr = 0.0f;
        if (qv) {
            if (flt) {
                r = L.qsrt[q_first + tid];
                qi = r.pad[0];
                qn = __uint_as_float(r.pad[1]);
                qerr = __uint_as_float((uint32_t)r.pair);  // |q - q~|
            } else if (staged) {
                tc::cp_async_wait_all();
                qi = qi_next;
                const uint4 *sr = reinterpret_cast<const uint4 *>(S.B[1][0] + tid * sizeof(QueryRec));
                uint4 w[3] = {sr[0], sr[1], sr[2]};
                memcpy(&r, w, sizeof(QueryRec));
            } else {
                qi = L.qperm[q_first + tid];
                r = L.qrec[q_off + qi];
            }
        } else {
            r.A = r.B = r.C = r.key = r.aux0 = r.aux1 = r.E0 = r.E1 = 0.0f;
            r.flags = EGM_FLAG_DEGENERATE_LINE;
            r.pair = p;
            r.pad[0] = r.pad[1] = 0;
        }
        const float qs = flt && qv ? L.qscale[q_first + tid] : 1.0f;  // row scale of the FP8 pass
        if (ctl && !pop) {
            if (flt) {
                tc::mbar_arrive_expect_tx(&S.afull, 2 * kTM * 128);
                tc::tma_load_2d(S.A[0], &tmA, 0, (int32_t)q_first, &S.afull);
                tc::tma_load_2d(S.A[1], &tmA, 128, (int32_t)q_first, &S.afull);
            } else {
                tc::mbar_arrive(&S.afull);
            }
            armA++;
            txA = flt;
        }
        // a u8 query's bytes: staged in its thread's row of A[1] (128-byte
        // swizzle, so that the 32 rows of a warp spread over the banks),
        // widened once the windows are known (the copy's latency hides behind them)
        if (cvt && qv) {
            const uint8_t *qrow = L.pairs[p].desc1 + (int64_t)qi * 128;
#pragma unroll
            for (int k = 0; k < 8; k++) tc::cp_async16(S.A[1] + sw128(tid, k), qrow + 16 * k);
        }
        // a binary query's row, in the idle query-tile buffer (its thread's slot)
        uint4 *qbrow = reinterpret_cast<uint4 *>(S.A[0] + tid * kBinRowB);
        if (pop && qv) {
            const uint4 *qrow = reinterpret_cast<const uint4 *>(L.pairs[p].desc1 + (int64_t)qi * kBinRowB);
            qbrow[0] = __ldg(qrow);
            qbrow[1] = __ldg(qrow + 1);
        }
        // the pair's geometry and table entry (kept from the last tile of the pair)
        if (warp == 4 && p != S.gpair) {
            __syncwarp();
            copy16(&S.g, L.geom + p, (int)sizeof(PairGeom), lane);
            copy16(&S.pd, L.pairs + p, (int)sizeof(PairDesc), lane);
            if (lane == 0) S.gpair = p;
        }
        __syncthreads();
        const PairDesc &P = S.pd;
        const PairGeom &G = S.g;
        if (warp == 4) {
            const uint32_t nz = __ballot_sync(0xffffffffu, G.cnt[lane] > 0);
            if (nz & (1u << lane)) S.lv[__popc(nz & lt)] = lane;
            if (lane == 0) S.nlev = __popc(nz);
        }
        __syncthreads();
        const int nlev = S.nlev;
        // ---- each warp's hull of its queries' windows: the extremes of its
        // queries' keys and pad arguments, then one window per level (lane = level)
        if (warp < 4) {
            const bool use = qv && !(r.flags & EGM_FLAG_DEGENERATE_LINE);
            const bool ex = use && (r.flags & kQExactOnly);
            const bool kv = use && !ex;
            const float kmin = unsortable(__reduce_min_sync(0xffffffffu, sortable(kv ? r.key : INFINITY)));
            const float kmax = unsortable(__reduce_max_sync(0xffffffffu, sortable(kv ? r.key : -INFINITY)));
            const float kabs = unsortable(__reduce_max_sync(0xffffffffu, sortable(kv ? fabsf(r.key) : 0.0f)));
            const float a0hi = unsortable(__reduce_max_sync(0xffffffffu, sortable(kv ? r.aux0 : -INFINITY)));
            const float a0lo = unsortable(__reduce_min_sync(0xffffffffu, sortable(kv ? r.aux0 : INFINITY)));
            const float a1hi = unsortable(__reduce_max_sync(0xffffffffu, sortable(kv ? r.aux1 : -INFINITY)));
            const bool anyex = __any_sync(0xffffffffu, ex), anykv = __any_sync(0xffffffffu, kv);
            if (lane < nlev) {
                KeyWin w;
                w.kind = 0;
                w.lo = w.hi = 0.0f;
                if (anyex || anykv)
                    w = key_window_span(G, S.lv[lane], kmin, kmax, kabs, G.mode == kModeAngular ? a0hi : a0lo,
                                        a1hi, anyex);
                S.u.hull.wkind[warp][lane] = w.kind;
                S.u.hull.wlo[warp][lane] = w.lo;
                S.u.hull.whi[warp][lane] = w.hi;
            }
        }
        __syncthreads();
        // ---- windows as sorted positions: warps 0-3 their own (kept by the
        // lane of the level index: wr0, wr1), warp 4 the tile's
        uint2 wr0 = make_uint2(0u, 0u), wr1 = wr0;
        {
            const int li = lane;
            KeyWin w;
            w.kind = 0;
            w.lo = w.hi = 0.0f;
            if (li < nlev) {
                if (warp < 4) {
                    w.kind = S.u.hull.wkind[warp][li];
                    w.lo = S.u.hull.wlo[warp][li];
                    w.hi = S.u.hull.whi[warp][li];
                } else {
                    float lo = INFINITY, hi = -INFINITY;
                    for (int q = 0; q < 4; q++) {
                        const int kq = S.u.hull.wkind[q][li];
                        if (kq == 1) w.kind = 1;
                        if (kq == 2) {
                            if (w.kind == 0) w.kind = 2;
                            lo = fminf(lo, S.u.hull.wlo[q][li]);
                            hi = fmaxf(hi, S.u.hull.whi[q][li]);
                        }
                    }
                    w.lo = lo;
                    w.hi = hi;
                }
            }
            const int lvl = li < nlev ? S.lv[li] : kLevels;
            const WinKeys wk = win_buckets(G, lvl, w);
            uint32_t a = 0, b = 0;
            if (wk.kind >= 2) {
                const uint32_t *T = L.tab + P.t_off + G.tab[lvl];
                a = __ldg(T + wk.ta);
                b = __ldg(T + wk.tb);
            }
            const Window wn = window_ranges(wk, a, b);
            if (warp < 4) {
                if (li < nlev) {
                    wr0 = make_uint2(wn.b0, wn.len0);
                    wr1 = make_uint2(wn.b1, wn.len1);
                }
            } else {
                const bool h0 = li < nlev && wn.len0 > 0, h1 = li < nlev && wn.len1 > 0;
                const uint32_t m0 = __ballot_sync(0xffffffffu, h0), m1 = __ballot_sync(0xffffffffu, h1);
                const int base = __popc(m0 & lt) + __popc(m1 & lt);
                const uint32_t nb0 = h0 ? (wn.len0 + kBoxR - 1) / kBoxR : 0u;
                const uint32_t nb1 = h1 ? (wn.len1 + kBoxR - 1) / kBoxR : 0u;
                const uint32_t tot = nb0 + nb1;
                uint32_t incl = tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += x;
                }
                const uint32_t excl = incl - tot;
                if (h0) {
                    Piece pc;
                    pc.start = wn.b0;
                    pc.len = wn.len0;
                    pc.box0 = excl;
                    pc.li = li;
                    S.pc[base] = pc;
                }
                if (h1) {
                    Piece pc;
                    pc.start = wn.b1;
                    pc.len = wn.len1;
                    pc.box0 = excl + nb0;
                    pc.li = li;
                    S.pc[base + (h0 ? 1 : 0)] = pc;
                }
                if (lane == 31) {
                    S.npc = __popc(m0) + __popc(m1);
                    S.nbox = (int)incl;
                }
            }
        }
        // the hull arrays' last generic accesses before the record stages they
        // share are written by bulk copies again
        tc::fence_proxy_async();
        __syncthreads();
        const int nbox = S.nbox;
        const int nchunk = (nbox + kCB - 1) / kCB;
        // the next tile's query order entries, loaded while this tile runs
        staged = false;
        {
            const TileDesc &tn = S.tdn;
            if (warp < 4 && tn.pair >= 0 && !(FLT && tn.kind == EGM_DESC_F32_L2) && tid < tn.mt) {
                qi_next = L.qperm[tn.q_first + tid];
                qoff_next = tn.q_off;
                staged = true;
            }
        }

        if (warp == 4) {
            // ---- producer
            BoxCursor curR, curB;
            // records (and float norms) of chunk c into slot g mod kRS (control
            // thread; the slot's previous chunk is finished)
            auto issueR = [&](int c) {
                const uint32_t g = seq + (uint32_t)c, s = g % kRS;
                const int nb = min(kCB, nbox - c * kCB);
                tc::mbar_arrive_expect_tx(&S.fullR[s], (uint32_t)nb * (kBoxR * 16) * (flt ? 2u : 1u));
                armR[s]++;
                for (int bb = 0; bb < nb; bb++) {
                    uint32_t pos, len;
                    int li;
                    curR.next(S, pos, len, li);
                    const int64_t row = P.r_off + pos;
                    tc::bulk_load(&S.u.io.rec[s][bb * kBoxR], L.rec + row, kBoxR * 16, &S.fullR[s]);
                    if (flt) tc::bulk_load(&S.u.io.rn[FLT ? s : 0][bb][0], L.rnorm + row, kBoxR * 16, &S.fullR[s]);
                }
            };
            // float rows of chunk c by TMA into operand stage g mod 2, once the
            // MMA of chunk g - 2 is done (control thread)
            auto issueB = [&](int c) {
                const uint32_t g = seq + (uint32_t)c, st = g % kNB;
                if (g >= (uint32_t)kNB && !wait(&S.sfree[st], ((g - kNB) / kNB) & 1u)) return;
                const int nb = min(kCB, nbox - c * kCB);
                tc::mbar_arrive_expect_tx(&S.fullB[st], (uint32_t)nb * (2 * kBoxR * 128));
                armB[st]++;
                for (int bb = 0; bb < nb; bb++) {
                    uint32_t pos, len;
                    int li;
                    curB.next(S, pos, len, li);
                    const int32_t row = (int32_t)(P.r_off + pos);
                    tc::tma_load_2d(S.B[st][0] + bb * kBoxR * 128, &tmB, 0, row, &S.fullB[st]);
                    tc::tma_load_2d(S.B[st][1] + bb * kBoxR * 128, &tmB, 128, row, &S.fullB[st]);
                }
            };
            // u8 and binary rows of chunk c, one row per lane and box, by the
            // indices in its records: u8 bytes into K half 1 of operand stage
            // g mod 2 (128-byte swizzle), once the MMA of chunk g - 2 is done;
            // binary rows into slot g mod kRS of B[0][0] (free: its records'
            // slot was).  Returns the boxes whose row this lane copied.
            // Records are copied in chunk order as far ahead as their slots allow,
            // without waiting (test_wait), and waited for only at the tile end
            // (the consumers wait for them anyway).
            int nextR = 0;
            auto pollR = [&](int upto, bool block) {
                while (nextR < nchunk && nextR <= upto) {
                    const uint32_t g = seq + (uint32_t)nextR, s = g % kRS;
                    if (g >= (uint32_t)kRS) {
                        const uint32_t par = ((g - kRS) / kRS) & 1u;
                        if (block ? !wait(&S.rfree[s], par) : !tc::mbar_test_wait(&S.rfree[s], par)) break;
                    }
                    issueR(nextR++);
                }
            };
            // the row indices of chunk c, lane = row of each box (all ones: none)
            BoxCursor curJ;
            auto jload = [&](int c, uint32_t (&jj)[kCB]) {
                const int nb = c < nchunk ? min(kCB, nbox - c * kCB) : 0;
#pragma unroll
                for (int bb = 0; bb < kCB; bb++) {
                    jj[bb] = ~0u;
                    if (bb < nb) {
                        uint32_t pos, len;
                        int li;
                        curJ.next(S, pos, len, li);
                        if ((uint32_t)lane < len) jj[bb] = __float_as_uint(__ldg(&L.rec[P.r_off + pos + lane].w));
                    }
                }
            };
            auto gather = [&](int c, const uint32_t (&jj)[kCB]) -> uint32_t {
                const uint32_t g = seq + (uint32_t)c, s = g % kRS, st = g % kNB;
                // the slot's previous chunk tested (binary rows, u8 norms) and the
                // operand stage's previous MMA done (u8 bytes)
                bool ok = g < (uint32_t)kRS || wait(&S.rfree[s], ((g - kRS) / kRS) & 1u);
                if (cvt && g >= (uint32_t)kNB) ok = wait(&S.sfree[st], ((g - kNB) / kNB) & 1u) && ok;
                const int nb = min(kCB, nbox - c * kCB);
                uint32_t gv = 0u;
#pragma unroll
                for (int bb = 0; bb < kCB; bb++) {
                    if (bb >= nb) break;
                    const uint32_t j = jj[bb];
                    if (!ok || j >= (uint32_t)P.n) continue;  // no row (j never exceeds n otherwise)
                    const int R = bb * kBoxR + lane;
                    if (cvt) {
                        const uint8_t *src = P.desc2 + (int64_t)j * 128;
#pragma unroll
                        for (int k = 0; k < 8; k++) tc::cp_async16(S.B[st][1] + sw128(R, k), src + 16 * k);
                        gv |= 1u << bb;
                    } else {
                        uint8_t *dst = S.B[0][0] + ((int)s * kCN + R) * kBinRowB;
                        tc::cp_async16(dst, P.desc2 + (int64_t)j * kBinRowB);
                        tc::cp_async16(dst + 16, P.desc2 + (int64_t)j * kBinRowB + 16);
                    }
                }
                tc::cp_async_commit();
                return gv;
            };
            // u8 rows of chunk c widened in place (each lane its own rows:
            // K half 0 from staged chunks 0-3, then half 1 over the staged
            // bytes from chunks 4-7) and their norms into slot g mod kRS
            auto widen_rows = [&](int c, uint32_t gv) {
                const uint32_t g = seq + (uint32_t)c, s = g % kRS, st = g % kNB;
                const int nb = min(kCB, nbox - c * kCB);
#pragma unroll
                for (int bb = 0; bb < kCB; bb++) {
                    if (bb >= nb) break;
                    const int R = bb * kBoxR + lane;
                    const bool have = (gv >> bb) & 1u;
                    uint32_t nrm = 0;
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        uint4 w[4];
#pragma unroll
                        for (int k = 0; k < 4; k++)
                            w[k] = have ? *reinterpret_cast<const uint4 *>(S.B[st][1] + sw128(R, 4 * h + k))
                                        : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            uint4 o0, o1;
                            widen16(w[k], o0, o1, nrm);
                            *reinterpret_cast<uint4 *>(S.B[st][h] + sw128(R, 2 * k)) = o0;
                            *reinterpret_cast<uint4 *>(S.B[st][h] + sw128(R, 2 * k + 1)) = o1;
                        }
                    }
                    S.u.io.n8[s][R] = (float)nrm;
                }
            };
            // E4M3 operands: float rows of the FP8 pass
            const bool e4m3 = flt && L.fp8;
            // the gathers in chunk order: chunk k's row indices load two gathers
            // ahead.  Two operand stages: chunk c + 1's rows are gathered before
            // chunk c is widened; three: chunk c + 2's after chunk c's MMA (its
            // stage is chunk c - 1's, whose MMA is an iteration old by then)
            uint32_t j1[kCB], j2[kCB];
            auto next_gather = [&](int k) -> uint32_t {
                const uint32_t gvk = gather(k, j1);
#pragma unroll
                for (int bb = 0; bb < kCB; bb++) j1[bb] = j2[bb];
                jload(k + 2, j2);
                return gvk;
            };
            if (!flt) {
                jload(0, j1);
                jload(1, j2);
            }
            if (ctl) {
                pollR(1, true);
                if (flt && nchunk > 0) issueB(0);
            }
            __syncwarp();
            uint32_t gv = 0u, gvn = 0u;  // boxes copied by this lane: chunk c, chunk c + 1
            if (nchunk > 0 && !flt) {
                gv = next_gather(0);
                if (kNB == 3 && nchunk > 1) gvn = next_gather(1);
            }
            for (int c = 0; c < nchunk; c++) {
                const uint32_t g = seq + (uint32_t)c, s = g % kRS, st = g % kNB, as = g % kNA;
                const bool more = c + 1 < nchunk;
                // two stages: the next chunk's rows in flight while this one is widened
                if (kNB == 2 && !flt && more) gvn = next_gather(c + 1);
                if (!flt) {
                    // this chunk's copies landed (chunk c + 1's may still be in flight)
                    if (more) tc::cp_async_wait_group<1>();
                    else tc::cp_async_wait_group<0>();
                    if (cvt) widen_rows(c, gv);
                    tc::fence_proxy_async();
                }
                __syncwarp();
                if (ctl) {
                    // the chunk's norms and binary rows are visible to the consumers
                    tc::mbar_arrive(&S.rows[s]);
                    if (flt && more) issueB(c + 1);
                    bool ok = true;
                    if (g >= (uint32_t)kNA) ok = wait(&S.tfree[as], ((g - kNA) / kNA) & 1u);
                    if (flt) ok = wait(&S.fullB[st], (armB[st] - 1u) & 1u) && ok;
                    if (c == 0 && !pop) ok = wait(&S.afull, (armA - 1u) & 1u) && ok;
                    if (ok) {
                        if (pop) {
                            // no product: the accumulator and the stage are free at once
                            tc::mbar_arrive(&S.done[as]);
                            tc::mbar_arrive(&S.sfree[st]);
                        } else {
                            tc::tc_fence_after();
                            const int nb = min(kCB, nbox - c * kCB);
                            const uint32_t idesc = e4m3  ? tc::idesc_e4m3(kTM, nb * kBoxR)
                                                   : flt ? tc::idesc_bf16(kTM, nb * kBoxR)
                                                         : tc::idesc_f16(kTM, nb * kBoxR);
                            const uint32_t dcol = tmem + as * kCN;
#pragma unroll
                            for (int k = 0; k < 8; k++) {
                                const int h = k >> 2, kk = k & 3;
                                const uint64_t ad = tc::sdesc_sw128(tc::smem_addr(S.A[h]) + 32 * kk);
                                const uint64_t bd = tc::sdesc_sw128(tc::smem_addr(S.B[st][h]) + 32 * kk);
                                if (e4m3) tc::mma_e4m3(dcol, ad, bd, idesc, k > 0);
                                else tc::mma_f16(dcol, ad, bd, idesc, k > 0);
                            }
                            tc::mma_commit(&S.done[as]);
                            tc::mma_commit(&S.sfree[st]);
                            anyD = true;
                            lastD = g;
                        }
                    }
                    // records ahead, after the MMA, as far as their slots are free
                    pollR(c + 3, false);
                }
                __syncwarp();
                uint32_t gvnn = 0u;
                if (kNB == 3 && !flt && c + 2 < nchunk) gvnn = next_gather(c + 2);
                gv = gvn;
                gvn = gvnn;
            }
            if (ctl) {
                pollR(nchunk, true);
                // the query tile's load completes before its buffer is reused
                if (nchunk == 0 && !pop) wait(&S.afull, (armA - 1u) & 1u);
                // the tile after the next one, while the consumers finish
                S.tdnn = fetch_tile(L, atomicAdd(L.work, 1u));
            }
        }

        // ---- consumers: the query tile's operand rows (u8: widened here), then
        // the tests and best two over each warp's own columns
        unsigned long long b1 = ~0ull, b2 = ~0ull;
        const bool isf = flt;
        FBuf fb;
        fb.init();
        if (warp < 4) {
            if (!pop) {
                if (cvt) {
                    tc::cp_async_wait_all();
                    // own row only: K half 0 from staged chunks 0-3, then half 1
                    // (over the staged bytes) from chunks 4-7
                    uint32_t nq = 0;
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        uint4 w[4];
#pragma unroll
                        for (int k = 0; k < 4; k++)
                            w[k] = qv ? *reinterpret_cast<const uint4 *>(S.A[1] + sw128(tid, 4 * h + k))
                                      : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            uint4 o0, o1;
                            widen16(w[k], o0, o1, nq);
                            *reinterpret_cast<uint4 *>(S.A[h] + sw128(tid, 2 * k)) = o0;
                            *reinterpret_cast<uint4 *>(S.A[h] + sw128(tid, 2 * k + 1)) = o1;
                        }
                    }
                    qn = (float)nq;
                    tc::fence_proxy_async();
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.afull);
            }
            if (nchunk > 0) {
                BoxCursor cur;
                const bool exact_only = (r.flags & kQExactOnly) != 0;
                const bool live = qv && !(r.flags & EGM_FLAG_DEGENERATE_LINE);
                const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
                // The pre-test bound of the plain kernel, 9.6e-7 S + 1.2e-7 eps + E1 (|x| + |y| + 2 eps)
                // + E0 + 1e-9 with S = |A x| + |B y| + |C|, taken with |A|, |B| <= 1 (the line is
                // normalised): bound = k1 (|x| + |y|) + ke eps + k0, never smaller.
                const float k1 = 9.6e-7f * 1.00001f + r.E1;
                const float ke = 1.2e-7f + 2.0f * r.E1;
                const float k0 = fmaf(9.6e-7f, fabsf(r.C), r.E0 + 1e-9f);
                for (int c = 0; c < nchunk; c++) {
                    const uint32_t g = seq + (uint32_t)c, rs = g % kRS, as = g % kNA;
                    // the accumulator, the chunk's norms and binary rows, its records
                    const bool ok = wait(&S.done[as], (g / kNA) & 1u) && wait(&S.rows[rs], (g / kRS) & 1u) &&
                                    wait(&S.fullR[rs], (g / kRS) & 1u);
                    tc::tc_fence_after();
                    const int nb = min(kCB, nbox - c * kCB);
                    for (int bb = 0; bb < nb; bb++) {
                        uint32_t pos, len;
                        int li;
                        cur.next(S, pos, len, li);
                        if (!ok) continue;
                        // columns of this box inside the warp's own windows
                        const uint2 w0 = make_uint2(__shfl_sync(0xffffffffu, wr0.x, li),
                                                    __shfl_sync(0xffffffffu, wr0.y, li));
                        const uint2 w1 = make_uint2(__shfl_sync(0xffffffffu, wr1.x, li),
                                                    __shfl_sync(0xffffffffu, wr1.y, li));
                        const int x0 = (int)max(pos, w0.x) - (int)pos;
                        const int x1 = (int)min(pos + len, w0.x + w0.y) - (int)pos;
                        const int y0 = (int)max(pos, w1.x) - (int)pos;
                        const int y1 = (int)min(pos + len, w1.x + w1.y) - (int)pos;
                        if (x1 <= x0 && y1 <= y0) continue;
                        const float4 *rnb = &S.u.io.rn[FLT ? rs : 0][bb][0];
                        const float *n8b = &S.u.io.n8[rs][bb * kBoxR];
                        const float4 *recb = &S.u.io.rec[rs][bb * kBoxR];
                        const uint8_t *binb = S.B[0][0] + ((int)rs * kCN + bb * kBoxR) * kBinRowB;
                        const uint32_t tb = tmem + lanebase + as * kCN + bb * kBoxR;
                        // the box's columns inside the warp's windows, as a bit mask
                        auto span = [](int a, int b) {
                            a = max(a, 0);
                            b = min(b, kBoxR);
                            return b <= a ? 0u : (b - a >= 32 ? ~0u : ((1u << (b - a)) - 1u) << a);
                        };
                        const uint32_t inbox = live ? (span(x0, x1) | span(y0, y1)) : 0u;
    #pragma unroll 1
                        for (int g = 0; g < kBoxR; g += kGroup) {
                            if (!__any_sync(0xffffffffu, (inbox >> g) & 0xffu)) continue;
                            // the group's records, loaded together with its accumulators
                            float4 rcs[kGroup];
#pragma unroll
                            for (int k = 0; k < kGroup; k++) rcs[k] = recb[g + k];
                            uint32_t v[kGroup];
                            if (!pop) {
                                tc::tmem_ld8(tb + g, v);
                                tc::tmem_wait_ld();
                            }
                            // membership of all columns first, branch-free (independent
                            // work for the scheduler); then the few candidates
                            const uint32_t gm = (inbox >> g) & 0xffu;
                            uint32_t cm = 0, um = 0;  // FP32 sure members; members or inconclusive
#pragma unroll
                            for (int k = 0; k < kGroup; k++) {
                                const float x = rcs[k].x, y = rcs[k].y, e = rcs[k].z;
                                const float d = fabsf(fmaf(r.A, x, fmaf(r.B, y, r.C)));
                                const float bound = fmaf(k1, fabsf(x) + fabsf(y), fmaf(ke, e, k0));
                                cm |= (uint32_t)(d <= e - bound) << k;
                                um |= (uint32_t)(d <= e + bound) << k;
                            }
                            if (exact_only) {
                                cm = 0u;
                                um = 0xffu;
                            }
                            cm &= gm;
                            uint32_t exm = um & ~cm & gm;  // left to the FP64 expression
                            nwin += __popc(gm);
                            // FP32 inconclusive: the brute-force FP64 expression decides.
                            // Float rows at once; u8 and binary rows with their
                            // distance key formed now (the accumulator and the rows
                            // are gone by then) and the test deferred to the tile end,
                            // where the warp's lanes run the deferred tests together
                            for (uint32_t m = exm; m; m &= m - 1u) {
                                const int k = __ffs(m) - 1;
                                nexact++;
                                const uint32_t jk = __float_as_uint(recb[g + k].w);
                                if (isf) {
                                    if (exact_pair(P, qi, jk)) cm |= 1u << k;
                                    continue;
                                }
                                uint32_t dh;
                                if (pop) {
                                    const uint4 *rb = reinterpret_cast<const uint4 *>(binb + (g + k) * kBinRowB);
                                    const uint4 r0 = rb[0], r1 = rb[1], q0 = qbrow[0], q1 = qbrow[1];
                                    dh = __popc(q0.x ^ r0.x) + __popc(q0.y ^ r0.y) + __popc(q0.z ^ r0.z) +
                                         __popc(q0.w ^ r0.w) + __popc(q1.x ^ r1.x) + __popc(q1.y ^ r1.y) +
                                         __popc(q1.z ^ r1.z) + __popc(q1.w ^ r1.w);
                                } else {
                                    dh = __float_as_uint(fmaf(-2.0f, __uint_as_float(pick8(v, k)), qn + n8b[g + k]));
                                }
                                const uint32_t slot = atomicAdd(&S.xn[warp], 1u);
                                if (slot < (uint32_t)kDeferCap) {
                                    S.xq[warp][slot] = make_uint4(dh, jk, (uint32_t)lane, 0u);
                                } else if (exact_pair(P, qi, jk)) {
                                    ncand++;
                                    top2(((unsigned long long)dh << 32) | jk, b1, b2);
                                }
                            }
                            if (pop) {
                                // Hamming distance of the binary rows by popcount
                                for (; cm; cm &= cm - 1u) {
                                    const int k = __ffs(cm) - 1;
                                    const uint4 *rb = reinterpret_cast<const uint4 *>(binb + (g + k) * kBinRowB);
                                    const uint4 r0 = rb[0], r1 = rb[1], q0 = qbrow[0], q1 = qbrow[1];
                                    const uint32_t h = __popc(q0.x ^ r0.x) + __popc(q0.y ^ r0.y) + __popc(q0.z ^ r0.z) +
                                                       __popc(q0.w ^ r0.w) + __popc(q1.x ^ r1.x) + __popc(q1.y ^ r1.y) +
                                                       __popc(q1.z ^ r1.z) + __popc(q1.w ^ r1.w);
                                    ncand++;
                                    top2(((unsigned long long)h << 32) | __float_as_uint(recb[g + k].w), b1, b2);
                                }
                            }
                            if (cvt && __any_sync(0xffffffffu, cm)) {
                                // the group's distances first, branch-free (integers below
                                // 2^24: exact in FP32, compared by their bit patterns);
                                // then the candidates pick theirs by a select tree
                                const float4 na = *reinterpret_cast<const float4 *>(n8b + g);
                                const float4 nb4 = *reinterpret_cast<const float4 *>(n8b + g + 4);
                                const float nk[kGroup] = {na.x, na.y, na.z, na.w, nb4.x, nb4.y, nb4.z, nb4.w};
                                uint32_t dk[kGroup], jv[kGroup];
#pragma unroll
                                for (int k = 0; k < kGroup; k++) {
                                    dk[k] = __float_as_uint(fmaf(-2.0f, __uint_as_float(v[k]), qn + nk[k]));
                                    jv[k] = __float_as_uint(rcs[k].w);
                                }
                                // a candidate farther than the second best so far cannot enter
                                ncand += __popc(cm);
                                const uint32_t d2 = (uint32_t)(b2 >> 32);
                                uint32_t near = 0u;
#pragma unroll
                                for (int k = 0; k < kGroup; k++) near |= (uint32_t)(dk[k] <= d2) << k;
                                for (cm &= near; cm; cm &= cm - 1u) {
                                    const int k = __ffs(cm) - 1;
                                    top2(((unsigned long long)pick8(dk, k) << 32) | pick8(jv, k), b1, b2);
                                }
                            }
                            for (; cm; cm &= cm - 1u) {
                                // float rows
                                const int k = __ffs(cm) - 1;
                                uint32_t jv[kGroup];
#pragma unroll
                                for (int t = 0; t < kGroup; t++) jv[t] = __float_as_uint(rcs[t].w);
                                const uint32_t vk = pick8(v, k), jk = pick8(jv, k);
                                ncand++;
                                // the accumulator holds the product of the scaled rows (scales 1
                                // except in the FP8 pass)
                                const float4 rk = rnb[g + k];
                                const float dist = qn + rk.x - 2.0f * ((qs * rk.z) * __uint_as_float(vk));
                                // distance of the BF16-rounded rows, bracketed around the FP32
                                // distance the rerank will compute
                                float lo, hi;
                                float_bounds(dist, qn, rk.x, qerr, rk.y, lo, hi);
                                fb.insert(lo, hi, jk);
                            }
                        }
                    }
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        tc::mbar_arrive(&S.tfree[as]);
                        tc::mbar_arrive(&S.rfree[rs]);
                    }
                }
                if (!isf) {
                    // the deferred FP64 tests of the warp, one per lane, then the
                    // members into their owners' best two
                    __syncwarp();
                    const uint32_t n = min(S.xn[warp], (uint32_t)kDeferCap);
                    if (n > 0) {
                        uint4 e = make_uint4(0u, 0u, (uint32_t)lane, 0u);
                        if ((uint32_t)lane < n) e = S.xq[warp][lane];
                        const uint32_t qo = __shfl_sync(0xffffffffu, qi, (int)e.z);
                        const bool mem = (uint32_t)lane < n && exact_pair_inline(P, qo, e.y);
                        for (uint32_t bal = __ballot_sync(0xffffffffu, mem); bal; bal &= bal - 1u) {
                            const int src = __ffs(bal) - 1;
                            const uint32_t owner = __shfl_sync(0xffffffffu, e.z, src);
                            const uint32_t kh = __shfl_sync(0xffffffffu, e.x, src);
                            const uint32_t kj = __shfl_sync(0xffffffffu, e.y, src);
                            if ((uint32_t)lane == owner) {
                                ncand++;
                                top2(((unsigned long long)kh << 32) | kj, b1, b2);
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0) S.xn[warp] = 0u;
                    __syncwarp();
                }
                if (isf) {
                    // FP32 rerank, one query of the warp at a time, the lanes over the
                    // dimensions: the candidates that can be among the best two, or
                    // (buffer overflow) every reference in the warp's windows
                    const bool live = qv && !(r.flags & EGM_FLAG_DEGENERATE_LINE);
                    const bool complete = fb.complete();
                    const bool exact_only = (r.flags & kQExactOnly) != 0;
                    for (int q = 0; q < 32; q++) {
                        if (!__shfl_sync(0xffffffffu, (int)live, q)) continue;
                        const uint32_t qiq = __shfl_sync(0xffffffffu, qi, q);
                        const float4 qv4 = __ldg(reinterpret_cast<const float4 *>(P.desc1 + (int64_t)qiq * 512) + lane);
                        unsigned long long k1 = ~0ull, k2 = ~0ull;
                        if (__shfl_sync(0xffffffffu, (int)complete, q)) {
                            const float U2q = __shfl_sync(0xffffffffu, fb.U2, q);
#pragma unroll
                            for (int t = 0; t < kFBuf; t++) {
                                const float Lt = __shfl_sync(0xffffffffu, fb.L[t], q);
                                const uint32_t jt = __shfl_sync(0xffffffffu, fb.J[t], q);
                                if (Lt <= U2q) {
                                    const float d = coop_dist(qv4, P.desc2 + (int64_t)jt * 512, lane);
                                    top2(((unsigned long long)__float_as_uint(d) << 32) | jt, k1, k2);
                                }
                            }
                        } else {
                            const float qA = __shfl_sync(0xffffffffu, r.A, q), qB = __shfl_sync(0xffffffffu, r.B, q);
                            const float qC = __shfl_sync(0xffffffffu, r.C, q);
                            const float qE0 = __shfl_sync(0xffffffffu, r.E0, q);
                            const float qE1 = __shfl_sync(0xffffffffu, r.E1, q);
                            const bool qex = __shfl_sync(0xffffffffu, (int)exact_only, q) != 0;
                            for (int li = 0; li < nlev; li++)
                                for (int h = 0; h < 2; h++) {
                                    const uint2 wh = h ? wr1 : wr0;
                                    const uint2 w = make_uint2(__shfl_sync(0xffffffffu, wh.x, li),
                                                               __shfl_sync(0xffffffffu, wh.y, li));
                                    for (uint32_t b0 = 0; b0 < w.y; b0 += 32) {
                                        const bool valid = b0 + (uint32_t)lane < w.y;
                                        uint32_t j = 0;
                                        int m = 0;
                                        if (valid) {
                                            const float4 rc = L.rec[P.r_off + w.x + b0 + lane];
                                            j = __float_as_uint(rc.w);
                                            m = qex ? 2 : member32(qA, qB, qC, qE0, qE1, rc);
                                            if (m == 2) m = exact_pair(P, qiq, j) ? 1 : 0;
                                        }
                                        for (uint32_t bal = __ballot_sync(0xffffffffu, m == 1); bal; bal &= bal - 1u) {
                                            const uint32_t jt = __shfl_sync(0xffffffffu, j, __ffs(bal) - 1);
                                            const float d = coop_dist(qv4, P.desc2 + (int64_t)jt * 512, lane);
                                            top2(((unsigned long long)__float_as_uint(d) << 32) | jt, k1, k2);
                                        }
                                    }
                                }
                        }
                        if (lane == q) {
                            b1 = k1;
                            b2 = k2;
                        }
                    }
                }
            }
        }
        // no gathered copy may still be landing when the tile's memory is reused
        tc::cp_async_wait_all();
        seq += (uint32_t)nchunk;
        if (cvt) {
            // u8 keys hold the distance's FP32 bits: the integer distance, as elsewhere
            auto as_int = [](unsigned long long b) {
                return b == ~0ull ? b
                                  : ((unsigned long long)(uint32_t)__uint_as_float((uint32_t)(b >> 32)) << 32) |
                                        (b & 0xffffffffull);
            };
            b1 = as_int(b1);
            b2 = as_int(b2);
        }
        if (qv) store_match(L, q_off + qi, P, r.flags, b1, b2);
        if (staged) {
            // every MMA of this tile is done and stage 1 holds no binary rows
            const uint8_t *src = reinterpret_cast<const uint8_t *>(L.qrec + qoff_next + qi_next);
            uint8_t *dst = S.B[1][0] + tid * sizeof(QueryRec);
            tc::cp_async16(dst, src);
            tc::cp_async16(dst + 16, src + 16);
            tc::cp_async16(dst + 32, src + 32);
        }
        // generic accesses of this tile (query rows, binary rows, widened
        // rows) before the next tile's copies into the same memory
        tc::fence_proxy_async();
        if (ctl) {
            S.td = S.tdn;
            S.tdn = S.tdnn;
        }
        __syncthreads();
    }
    tc::cp_async_wait_all();
    if (L.counters && warp < 4) {
        const uint32_t a = __reduce_add_sync(0xffffffffu, nwin);
        const uint32_t b = __reduce_add_sync(0xffffffffu, ncand);
        const uint32_t c = __reduce_add_sync(0xffffffffu, nexact);
        if (lane == 0) {
            atomicAdd(L.counters + 2, (unsigned long long)a);
            atomicAdd(L.counters + 3, (unsigned long long)b);
            atomicAdd(L.counters + 4, (unsigned long long)c);
        }
    }
    if (ctl && S.err) {
        // A wait gave up.  Before the CTA's shared memory and TMEM are
        // released, every copy and MMA it issued must have landed: wait
        // (bounded) for the last phase armed on each barrier that carries
        // copies, and for the commit of the last MMA chain (a commit covers
        // every earlier MMA of the thread).  A barrier is re-armed only
        // after its previous phase was waited for, so at most that last
        // phase is outstanding.
        for (int s = 0; s < kRS; s++)
            if (armR[s]) tc::mbar_wait(&S.fullR[s], (armR[s] - 1u) & 1u);
        for (int st = 0; st < kNB; st++)
            if (armB[st]) tc::mbar_wait(&S.fullB[st], (armB[st] - 1u) & 1u);
        if (anyD) tc::mbar_wait(&S.done[lastD % kNA], (lastD / kNA) & 1u);
        if (armA && txA) tc::mbar_wait(&S.afull, (armA - 1u) & 1u);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 4) tc::tmem_dealloc(tmem, kTmemCols);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

// Rows of 256 bytes, boxes of 128 bytes x `box_rows` rows, 128-byte swizzle.
cudaError_t make_tmap(CUtensorMap *m, const void *base, int64_t rows, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)kRowB, (cuuint64_t)(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)kRowB};
    cuuint32_t box[2] = {128u, box_rows};
    cuuint32_t es[2] = {1u, 1u};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

bool band_supported(int kind, int dim) {
    return (kind == EGM_DESC_U8_L2 && dim == 128) || (kind == EGM_DESC_BIN && dim == 256) ||
           (kind == EGM_DESC_F32_L2 && dim == 128);
}

int band_row_bytes() { return kRowB; }
int band_tile_queries() { return kTM; }

cudaError_t launch_query_sort(const Launch &L, cudaStream_t s) {
    if (L.nq == 0) return cudaSuccess;
    // plain launches here and for the pack kernel: both follow a cross-stream
    // event wait, which must order them in full
    query_sort_kernel<<<L.npairs, kQSortThreads, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_pack(const Launch &L, cudaStream_t s) {
    const int64_t rows = L.nr + L.nq;
    if (rows == 0 || !(L.kinds & (1u << EGM_DESC_F32_L2))) return cudaSuccess;
    int64_t blocks = (rows * 8 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (L.fp8 && (L.kinds & (1u << EGM_DESC_F32_L2))) pack_kernel<true><<<(int)blocks, 256, 0, s>>>(L);
    else pack_kernel<false><<<(int)blocks, 256, 0, s>>>(L);
    return cudaGetLastError();
}

template <int CB, int CPS, bool FLT>
cudaError_t launch_band_shape(const Launch &L, int sms, const CUtensorMap &tA, const CUtensorMap &tB,
                              bool zero_work, bool pdl, cudaStream_t s) {
    const int smem = (int)BandShape<CB, CPS, FLT>::kDynSmem;
    int64_t grid = L.ntiles;
    if (grid > CPS * (int64_t)sms) grid = CPS * (int64_t)sms;
    cudaError_t e;
    if (zero_work && (e = cudaMemsetAsync(L.work, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(band_kernel<CB, CPS, FLT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (pdl)
        return launch_pdl(band_kernel<CB, CPS, FLT>, dim3((unsigned)grid), dim3(kBandThreads), (size_t)smem, s, tA,
                          tB, L);
    band_kernel<CB, CPS, FLT><<<(unsigned)grid, kBandThreads, (size_t)smem, s>>>(tA, tB, L);
    return cudaGetLastError();
}

int band_shapes() { return 7; }

cudaError_t launch_band(const Launch &L, int sms, int shape, cudaStream_t s, bool zero_work) {
    if (L.ntiles == 0) return cudaSuccess;
    // Packed operand rows (and the tensor maps over them) exist for float
    // pairs only; otherwise the maps cover the minimal buffers and are never
    // used.  The pack kernel runs for float pairs only, so the band kernel
    // follows it as a dependent launch, or else follows the join of the
    // query-sort stream in full.
    const bool flt = (L.kinds & (1u << EGM_DESC_F32_L2)) != 0;
    CUtensorMap tA, tB;
    cudaError_t e = make_tmap(&tA, L.descA, flt ? L.nq : kTM, kTM);
    if (e != cudaSuccess) return e;
    if ((e = make_tmap(&tB, L.descB, flt ? L.nr : kTM, kBoxR)) != cudaSuccess) return e;
    if (flt) return launch_band_shape<2, 2, true>(L, sms, tA, tB, zero_work, true, s);
    switch (shape) {
        case 0: return launch_band_shape<4, 2, false>(L, sms, tA, tB, zero_work, zero_work, s);
        case 1: return launch_band_shape<2, 3, false>(L, sms, tA, tB, zero_work, zero_work, s);
        case 2: return launch_band_shape<1, 4, false>(L, sms, tA, tB, zero_work, zero_work, s);
        case 3: return launch_band_shape<1, 3, false>(L, sms, tA, tB, zero_work, zero_work, s);
        case 4: return launch_band_shape<2, 2, false>(L, sms, tA, tB, zero_work, zero_work, s);
        case 5: return launch_band_shape<4, 1, false>(L, sms, tA, tB, zero_work, zero_work, s);
        case 6: return launch_band_shape<1, 2, false>(L, sms, tA, tB, zero_work, zero_work, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace egm
