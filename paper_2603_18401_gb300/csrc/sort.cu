// Ordering of the reference keypoints by (level, angle bucket).
//
// This replaces the paper's centred segment tree (Sec. 4.4, "Segment Tree
// Structure"): once the keypoints of each angular-radius level are ordered by
// angle, a query's angle window is a contiguous run of them, found through a
// per-level bucket table (bucket -> first position).
//
// Keys are 27 bits: level (5) | quantised angle (22).  The tables resolve at
// most 16 bits of the angle, about two buckets per member of a level, so a
// counting sort by (level, bucket) is all the order the windows need (the
// bucket kernels below).
//
// A stable LSD block radix sort (ballot-based warp multi-split over tiles of
// 16384 elements; 7-bit digits) orders candidate rows of the CSR output that
// are longer than a warp sorts.
#include <cooperative_groups.h>

#include "egm_internal.cuh"

namespace cg = cooperative_groups;

namespace egm {

namespace {

constexpr int kSortThreads = 1024;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItems = 16;
constexpr int kTile = kSortThreads * kItems;     // 16384
constexpr int kWarpSpan = 32 * kItems;           // 512 elements per warp
constexpr int kRBits = 7;
constexpr int kBins = 1 << kRBits;

struct SortSmem {
    uint32_t whist[kSortWarps * kBins];  // [warp][digit]
    uint32_t dbase[kBins];               // first position of each digit in the segment
    uint32_t run[kBins];                 // elements of each digit in earlier tiles
    uint32_t ttot[kBins];                // elements of each digit in this tile
    uint32_t skey[kTile];
    uint32_t sval[kTile];
};

__device__ __forceinline__ uint32_t digit_of(uint32_t key, int shift) {
    return shift < 32 ? (key >> shift) & (kBins - 1) : 0u;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Per-warp stable ranks of this tile's items and per-(warp, digit) counts,
// followed by the exclusive scan of each digit's counts over the warps.  The
// lanes holding the same digit are found with one ballot per digit bit.
// Ranks are below 512 (a warp's share of a tile), so two share a register.
__device__ __forceinline__ uint32_t rank_at(const uint32_t (&rank)[kItems / 2], int k) {
    return (rank[k >> 1] >> ((k & 1) * 16)) & 0xffffu;
}

__device__ __forceinline__ void rank_tile(SortSmem &S, const uint32_t (&key)[kItems], uint32_t (&rank)[kItems / 2],
                                          int shift, int warp, int lane) {
    uint32_t *wh = S.whist + warp * kBins;
    for (int d = lane; d < kBins; d += 32) wh[d] = 0u;
    __syncwarp();
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < kItems; k++) {
        const uint32_t dg = digit_of(key[k], shift);
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < kRBits; b++) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (dg >> b) & 1u);
            peers &= ((dg >> b) & 1u) ? bal : ~bal;
        }
        const uint32_t before = wh[dg];
        const uint32_t rk = before + __popc(peers & lt);
        if (k & 1) rank[k >> 1] |= rk << 16; else rank[k >> 1] = rk;
        __syncwarp();
        if ((peers & lt) == 0u) wh[dg] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < kBins) {
        uint32_t acc = 0;
#pragma unroll 8
        for (int w = 0; w < kSortWarps; w++) {
            uint32_t *c = S.whist + w * kBins + threadIdx.x;  // stride kBins: no bank conflicts
            const uint32_t v = *c;
            *c = acc;
            acc += v;
        }
        S.ttot[threadIdx.x] = acc;
    }
    __syncthreads();
}

// Exclusive scan of S.ttot into S.dbase by warp 0 (4 digits per lane).
__device__ __forceinline__ void digit_base_from(SortSmem &S, const uint32_t *tot, int warp, int lane) {
    if (warp == 0) {
        uint32_t v[4], s = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) { v[q] = tot[lane * 4 + q]; s += v[q]; }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        uint32_t acc = incl - s;
#pragma unroll
        for (int q = 0; q < 4; q++) { S.dbase[lane * 4 + q] = acc; acc += v[q]; }
    }
    __syncthreads();
}

// Stable sort of n keys (and values, when iv != nullptr) by one thread block,
// on the digits at bit first_shift + 7 p for p < passes.  Long segments
// ping-pong between alt and out so that the last pass lands in out; in == out
// is allowed only with an even number of passes.
__device__ void block_radix_sort(SortSmem &S, const uint32_t *ik, const uint32_t *iv, uint32_t *ak, uint32_t *av,
                                 uint32_t *ok, uint32_t *ov, int n, int first_shift, int passes) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool has_vals = iv != nullptr;
    uint32_t key[kItems], val[kItems], rank[kItems / 2];
    if (n <= 0) return;
    if (n <= kTile) {
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            const int idx = warp * kWarpSpan + k * 32 + lane;
            key[k] = idx < n ? ik[idx] : 0xffffffffu;
            val[k] = (idx < n && has_vals) ? iv[idx] : 0u;
        }
        __syncthreads();  // every read of `in` is done before `out` (possibly the same) is written
        for (int pass = 0; pass < passes; pass++) {
            const int shift = first_shift + pass * kRBits;
            rank_tile(S, key, rank, shift, warp, lane);
            digit_base_from(S, S.ttot, warp, lane);
#pragma unroll
            for (int k = 0; k < kItems; k++) {
                const uint32_t dg = digit_of(key[k], shift);
                const uint32_t pos = S.dbase[dg] + S.whist[warp * kBins + dg] + rank_at(rank, k);
                S.skey[pos] = key[k];
                S.sval[pos] = val[k];
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kItems; k++) {
                const int idx = warp * kWarpSpan + k * 32 + lane;
                key[k] = S.skey[idx];
                val[k] = S.sval[idx];
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            const int idx = warp * kWarpSpan + k * 32 + lane;
            if (idx < n) {
                ok[idx] = key[k];
                if (has_vals) ov[idx] = val[k];
            }
        }
        __syncthreads();
        return;
    }

    const uint32_t *sk = ik;
    const uint32_t *sv = iv;
    const int ntiles = (n + kTile - 1) / kTile;
    for (int pass = 0; pass < passes; pass++) {
        const int shift = first_shift + pass * kRBits;
        const bool to_out = ((passes - 1 - pass) & 1) == 0;
        uint32_t *dk = to_out ? ok : ak;
        uint32_t *dv = to_out ? ov : av;
        if (threadIdx.x < kBins) { S.ttot[threadIdx.x] = 0u; S.run[threadIdx.x] = 0u; }
        __syncthreads();
        for (int i0 = 0; i0 < n; i0 += kSortThreads) {
            const int i = i0 + threadIdx.x;
            if (i < n) atomicAdd(&S.ttot[digit_of(sk[i], shift)], 1u);
        }
        __syncthreads();
        digit_base_from(S, S.ttot, warp, lane);
        for (int t = 0; t < ntiles; t++) {
            const int t0 = t * kTile;
#pragma unroll
            for (int k = 0; k < kItems; k++) {
                const int idx = t0 + warp * kWarpSpan + k * 32 + lane;
                key[k] = idx < n ? sk[idx] : 0xffffffffu;
                val[k] = (idx < n && has_vals) ? sv[idx] : 0u;
            }
            rank_tile(S, key, rank, shift, warp, lane);
#pragma unroll
            for (int k = 0; k < kItems; k++) {
                const int idx = t0 + warp * kWarpSpan + k * 32 + lane;
                if (idx < n) {
                    const uint32_t dg = digit_of(key[k], shift);
                    const uint32_t pos = S.dbase[dg] + S.run[dg] + S.whist[warp * kBins + dg] + rank_at(rank, k);
                    dk[pos] = key[k];
                    if (has_vals) dv[pos] = val[k];
                }
            }
            __syncthreads();
            if (threadIdx.x < kBins) S.run[threadIdx.x] += S.ttot[threadIdx.x];
            __syncthreads();
        }
        sk = dk;
        sv = dv;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Bucket sort of the references: one counting pass per pair.
//   (the prep kernel zeroes the tables and lays out every pair's levels)
//   bucket_count_kernel   per reference: one atomic add on its bucket
//   bucket_scan_kernel    per pair: one exclusive scan over the concatenated
//                         per-level tables, which yields every level's table
//                         at once (the first position of each bucket; in each
//                         level's extra last entry, the level's end), and a
//                         copy as fill cursors; then every reference takes
//                         the next position of its bucket and moves its FP32
//                         record (x - cx, y - cy, eps, index), written by the
//                         prep kernel, there.
// The order within a bucket follows the atomics and is not fixed; everything
// downstream depends only on bucket order (ties between candidates are broken
// by index).

__device__ __forceinline__ uint32_t bucket_slot(const PairGeom &G, uint32_t key) {
    const int lv = (int)(key >> kQBits);
    return G.tab[lv] + ((key & kQMax) >> (kQBits - G.bits[lv]));
}

__global__ void __launch_bounds__(256) bucket_count_kernel(Launch L) {
    pdl_begin();
    __shared__ int64_t offs[kSmemPairs + 1];
    __shared__ uint32_t s_tab[kLevels], s_start[kLevels + 1];
    __shared__ int32_t s_bits[kLevels];
    const bool one = L.inl_use != 0;  // one pair: every reference is pair 0
    const bool cached = one || load_offsets(offs, L.r_offs, L.npairs);
    if (one && threadIdx.x < 32) {
        // a single pair's level layout from the final level counts (the prep
        // kernel leaves it to this kernel); block 0 publishes it for the
        // kernels after this one
        const int lane = threadIdx.x;
        level_layout_lane(L.geom[0].cnt[lane], s_start, s_bits, s_tab, kMaxBucketBits, lane);
        if (blockIdx.x == 0) {
            PairGeom &G = L.geom[0];
            G.start[lane] = s_start[lane];
            G.bits[lane] = s_bits[lane];
            G.tab[lane] = s_tab[lane];
            if (lane == kLevels - 1) G.start[kLevels] = s_start[kLevels];
        }
    }
    __syncthreads();
    for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < L.nr; g0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = g0 + threadIdx.x;
        if (one) {
            if (g < L.nr) {
                const uint32_t key = L.key_a[g];
                const int lv = (int)(key >> kQBits);
                atomicAdd(L.tab + L.inl.t_off + s_tab[lv] + ((key & kQMax) >> (kQBits - s_bits[lv])), 1u);
            }
            continue;
        }
        // the reference's pair (the warp is converged here; every row is a reference)
        int p = 0;
        if (cached) {
            if (g0 + (threadIdx.x & ~31) < L.nr) p = warp_pair(offs, offs, L.npairs, L.nr, g);
        } else if (g < L.nr) {
            p = pair_of(L.r_offs, L.npairs, g);
        }
        if (g < L.nr) atomicAdd(L.tab + L.pairs[p].t_off + bucket_slot(L.geom[p], L.key_a[g]), 1u);
    }
}

// The scan and the placement of one pair run on a thread-block cluster: its
// warps hold rows of 128 table entries (a 16-byte vector per lane) in
// registers, so a pass over the table is one round trip to memory; the
// blocks' totals are exchanged through distributed shared memory.  A call
// of one pair takes a cluster of 16 blocks of 512 threads (the placement's
// atomics and stores spread over more SMs: the nine-pair config-2 step runs
// 0.377 instead of 0.397 ms); a batch 8 blocks of 256 per pair (the larger
// clusters took its sort stage from 0.118 to 0.262 ms).  kScanRound: rows a
// warp keeps in registers per round; kPre: references a thread loads ahead;
// kMinCtas: resident blocks per SM the register budget is held to (a batch
// runs its pairs' clusters in waves, which more resident clusters shorten).
template <int kScanCtas, int kScanThreads, int kScanRound, int kPre, int kMinCtas>
__global__ void __cluster_dims__(kScanCtas, 1, 1) __launch_bounds__(kScanThreads, kMinCtas)
    bucket_scan_kernel(Launch L) {
    constexpr int kScanWarps = kScanThreads / 32;
    pdl_begin();
    __shared__ __align__(16) PairGeom G;
    __shared__ uint32_t wtot[kScanWarps];
    __shared__ uint32_t ctot;     // this block's total, read by the higher-ranked blocks
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p = blockIdx.x / kScanCtas;
    const PairView P = pair_view(L, p);
    if (tid < (int)(sizeof(PairGeom) / 16))
        reinterpret_cast<uint4 *>(&G)[tid] = reinterpret_cast<const uint4 *>(L.geom + p)[tid];
    __syncthreads();
    const uint32_t used = G.tab[kLevels - 1] + (1u << G.bits[kLevels - 1]) + 1u;
    const uint32_t used4 = (used + 3u) & ~3u;  // the table's capacity leaves room for the padding
    uint4 *T4 = reinterpret_cast<uint4 *>(L.tab + P.t_off);
    uint4 *C4 = reinterpret_cast<uint4 *>(L.curs + P.t_off);
    // warp gw of the cluster owns rows [gw R, gw R + R) of 128 entries
    const uint32_t rows = (used4 + 127u) / 128u;
    const uint32_t nw = kScanCtas * kScanWarps, gw = (uint32_t)(rank * kScanWarps + warp);
    const uint32_t R = (rows + nw - 1) / nw, r0 = gw * R, r1 = min(rows, r0 + R);
    auto load_row = [&](uint32_t r) {
        const uint32_t i = r * 32u + (uint32_t)lane;  // uint4 index
        return i * 4u < used4 ? T4[i] : make_uint4(0, 0, 0, 0);
    };
    // this thread's first references, loaded now so that the loads overlap the scan
    const int64_t b = P.r_off;
    const int stride = kScanCtas * kScanThreads;
    uint32_t key[kPre];
    float4 rv[kPre];
    auto load_refs = [&](int e0) {
#pragma unroll
        for (int k = 0; k < kPre; k++) {
            const int e = e0 + k * stride;
            key[k] = 0xffffffffu;
            if (e < P.n) {
                key[k] = L.key_a[b + e];
                rv[k] = L.rtmp[b + e];
            }
        }
    };
    const int first = rank * kScanThreads + tid;
    load_refs(first);
    // pass 1: this warp's total (rows kept in registers when they fit one round)
    uint4 v[kScanRound];
    uint32_t sum = 0;
    for (uint32_t r = r0; r < r1; r += kScanRound) {
#pragma unroll
        for (int k = 0; k < kScanRound; k++) v[k] = r + k < r1 ? load_row(r + k) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < kScanRound; k++) sum += v[k].x + v[k].y + v[k].z + v[k].w;
    }
    sum = __reduce_add_sync(0xffffffffu, sum);
    if (lane == 0) wtot[warp] = sum;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kScanWarps ? wtot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kScanWarps) wtot[lane] = wi - w;
        if (lane == 31) ctot = wi;
    }
    cluster.sync();  // every block total published
    // the lower-ranked blocks' totals, read in parallel (lane c reads block c)
    uint32_t lower = lane < rank ? *cluster.map_shared_rank(&ctot, lane) : 0u;
    lower = __reduce_add_sync(0xffffffffu, lower);
    uint32_t carry = wtot[warp] + lower;
    // pass 2: exclusive values: the table (first position of each bucket) and the cursors
    const bool one_round = r1 <= r0 + kScanRound;
    for (uint32_t r = r0; r < r1; r += kScanRound) {
        if (!one_round) {
#pragma unroll
            for (int k = 0; k < kScanRound; k++) v[k] = r + k < r1 ? load_row(r + k) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int k = 0; k < kScanRound; k++) {
            if (r + k >= r1) break;
            const uint32_t ls = v[k].x + v[k].y + v[k].z + v[k].w;
            uint32_t incl = ls;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t e0 = carry + incl - ls;
            const uint4 out = make_uint4(e0, e0 + v[k].x, e0 + v[k].x + v[k].y, e0 + v[k].x + v[k].y + v[k].z);
            const uint32_t i = (r + k) * 32u + (uint32_t)lane;
            if (i * 4u < used4) {
                T4[i] = out;
                C4[i] = out;
            }
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    cluster.sync();  // every cursor in place (cluster-scope ordering of the global writes)
    // placement: the pair's references into their buckets
    for (int e0 = first; e0 < P.n; e0 += stride * kPre) {
        if (e0 != first) load_refs(e0);
#pragma unroll
        for (int k = 0; k < kPre; k++) {
            if (key[k] == 0xffffffffu) continue;
            const uint32_t pos = atomicAdd(L.curs + P.t_off + bucket_slot(G, key[k]), 1u);
            L.rec[b + pos] = rv[k];
        }
    }
    cluster.sync();  // no block leaves while another may still read its shared memory
}

// Candidate rows longer than a warp sorts: one block sorts them one after the
// other (ascending reference index), with key_c as the ping-pong buffer.
__global__ void __launch_bounds__(kSortThreads, 1) long_row_sort_kernel(Launch L, const uint32_t *list,
                                                                        const uint32_t *count) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &S = *reinterpret_cast<SortSmem *>(smem_raw);
    const uint32_t nl = *count;
    for (uint32_t k = 0; k < nl; k++) {
        const int64_t row = list[k];
        const int64_t a = L.cand_offsets[row], e = L.cand_offsets[row + 1];
        const int len = (int)(e - a);
        uint32_t *rk = reinterpret_cast<uint32_t *>(L.cand_idx + a);
        const int passes = L.nr <= (1 << 28) ? 4 : 6;  // indices < n <= nr
        block_radix_sort(S, rk, nullptr, L.key_c, nullptr, rk, nullptr, len, 0, passes);
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_sort(const Launch &L, cudaStream_t s) {
    if (L.nr == 0) return cudaSuccess;
    int64_t blocks = (L.nr + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    cudaError_t e = launch_pdl(bucket_count_kernel, dim3((unsigned)blocks), dim3(256), 0, s, L);
    if (e != cudaSuccess) return e;
    if (L.npairs == 1) {
        e = cudaFuncSetAttribute(bucket_scan_kernel<16, 512, 8, 8, 1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        return launch_pdl(bucket_scan_kernel<16, 512, 8, 8, 1>, dim3(16), dim3(512), 0, s, L);
    }
    return launch_pdl(bucket_scan_kernel<8, 256, 4, 4, 4>, dim3(L.npairs * 8), dim3(256), 0, s, L);
}

cudaError_t launch_long_row_sort(const Launch &L, const uint32_t *list, const uint32_t *count, cudaStream_t s) {
    const int smem = (int)sizeof(SortSmem);
    cudaError_t e = cudaFuncSetAttribute(long_row_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    long_row_sort_kernel<<<1, kSortThreads, smem, s>>>(L, list, count);
    return cudaGetLastError();
}

}  // namespace egm
