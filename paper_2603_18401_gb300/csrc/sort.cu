// Device LSD radix sort of the reference keys, one thread block per pair.
//
// This replaces the paper's centred segment tree (Sec. 4.4, "Segment Tree
// Structure"): once the keypoints of each angular-radius level are sorted by
// angle, a query's angle window is a contiguous range of the sorted array.
//
// Keys are 27 bits: level (5) | quantised angle (22); values are the
// keypoints' local indices.  The bucket tables that replace the tree resolve
// at most 16 bits of the angle, so the sort orders the keys by bits 6..26
// (level and the top 16 angle bits) in three stable passes of 7-bit digits;
// the full key stays in the array for the exact window filter.  Within a
// tile of 16384 elements every warp owns 512 consecutive elements in striped
// order (item k of lane l is element 32 k + l); ranking items in k order with
// a ballot-based warp multi-split keeps the sort stable.
// A segment that fits one tile stays in registers and shared memory for all
// passes; longer segments ping-pong through global scratch tile by tile.
//
// The block also derives, from the level counts of the prep kernel, each
// level's first sorted position, bucket-table size and table offset.
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
constexpr int kFirstShift = 6;                                               // bits below are not needed
constexpr int kPasses = (kKeyBits - kFirstShift + kRBits - 1) / kRBits;  // 3

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

__global__ void __launch_bounds__(kSortThreads, 1) sort_kernel(Launch L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &S = *reinterpret_cast<SortSmem *>(smem_raw);
    const int p = blockIdx.x;
    const PairDesc &P = L.pairs[p];
    PairGeom &G = L.geom[p];

    if (P.n <= kClusterMaxN) return;  // sorted by the cluster kernel
    if (threadIdx.x == 0) level_layout(G.cnt, G.start, G.bits, G.tab, kQBits - kFirstShift);
    const int64_t b = P.r_off;
    block_radix_sort(S, L.key_a + b, L.val_a + b, L.key_c + b, L.val_c + b, L.key_b + b, L.val_b + b, P.n,
                     kFirstShift, kPasses);
}

// ---------------------------------------------------------------------------
// Cluster sort: the eight blocks of a thread-block cluster sort one pair.
// Block r owns sorted positions [r*chunk, (r+1)*chunk).  Per pass every block
// ranks its elements (ballot multi-split per warp), publishes its 128 digit
// totals in shared memory, reads all blocks' totals through distributed
// shared memory to place its elements, and stores each element straight into
// the shared memory of the block that owns its new position.  After the last
// pass the blocks write the sorted keys, the FP32 records and the bucket
// tables (the work of post_sort_kernel) for their positions.
constexpr int kCWarps = kClusterThreads / 32;
constexpr int kCChunk = kClusterThreads * kClusterItems;

struct ClusterSmem {
    uint32_t rkey[kCChunk];
    uint32_t rval[kCChunk];
    uint32_t whist[kCWarps * kBins];
    uint32_t hist[kBins];      // this block's digit totals, read by the whole cluster
    uint32_t tot[kBins];
    uint32_t base[kBins];
    uint32_t start[kLevels + 1];
    int32_t bits[kLevels];
    uint32_t tab[kLevels];
};

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads)
    cluster_sort_kernel(Launch L) {
    __shared__ __align__(16) ClusterSmem S;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int p = blockIdx.x / kClusterCtas;
    const PairDesc &P = L.pairs[p];
    PairGeom &G = L.geom[p];
    const int n = P.n;
    if (n <= 0 || n > kClusterMaxN) return;  // the same for every block of the cluster
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int items = (n + kClusterCtas * kClusterThreads - 1) / (kClusterCtas * kClusterThreads);
    const int chunk = items * kClusterThreads;
    const int wspan = items * 32;
    const uint32_t lt = lanemask_lt();
    if (threadIdx.x == 0) {
        level_layout(G.cnt, S.start, S.bits, S.tab, kQBits - kFirstShift);
        if (rank == 0) {
            for (int l = 0; l < kLevels; l++) {
                G.start[l] = S.start[l];
                G.bits[l] = S.bits[l];
                G.tab[l] = S.tab[l];
            }
            G.start[kLevels] = S.start[kLevels];
        }
    }
    const int64_t b = P.r_off;
    uint32_t key[kClusterItems], val[kClusterItems], rk[kClusterItems / 2];
#pragma unroll
    for (int k = 0; k < kClusterItems; k++) {
        key[k] = 0xffffffffu;
        val[k] = 0u;
        if (k < items) {
            const int e = rank * chunk + warp * wspan + k * 32 + lane;
            if (e < n) {
                key[k] = L.key_a[b + e];
                val[k] = L.val_a[b + e];
            }
        }
    }
    for (int pass = 0; pass < kPasses; pass++) {
        const int shift = kFirstShift + pass * kRBits;
        if (pass > 0) {
#pragma unroll
            for (int k = 0; k < kClusterItems; k++)
                if (k < items) {
                    const int e = warp * wspan + k * 32 + lane;
                    key[k] = S.rkey[e];
                    val[k] = S.rval[e];
                }
        }
        uint32_t *wh = S.whist + warp * kBins;
        for (int d = lane; d < kBins; d += 32) wh[d] = 0u;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kClusterItems; k++) {
            if (k < items) {
                const uint32_t dg = digit_of(key[k], shift);
                uint32_t peers = 0xffffffffu;
#pragma unroll
                for (int bit = 0; bit < kRBits; bit++) {
                    const uint32_t bal = __ballot_sync(0xffffffffu, (dg >> bit) & 1u);
                    peers &= ((dg >> bit) & 1u) ? bal : ~bal;
                }
                const uint32_t before = wh[dg];
                const uint32_t r = before + __popc(peers & lt);
                if (k & 1) rk[k >> 1] |= r << 16; else rk[k >> 1] = r;
                __syncwarp();
                if ((peers & lt) == 0u) wh[dg] = before + __popc(peers);
                __syncwarp();
            }
        }
        __syncthreads();
        if (threadIdx.x < kBins) {
            uint32_t acc = 0;
#pragma unroll
            for (int w = 0; w < kCWarps; w++) {
                uint32_t *c = S.whist + w * kBins + threadIdx.x;
                const uint32_t v = *c;
                *c = acc;
                acc += v;
            }
            S.hist[threadIdx.x] = acc;
        }
        cluster.sync();  // all totals published; every block has read its receive buffer
        if (threadIdx.x < kBins) {
            uint32_t tot = 0, pre = 0;
            for (int c = 0; c < kClusterCtas; c++) {
                const uint32_t v = cluster.map_shared_rank(S.hist, c)[threadIdx.x];
                tot += v;
                if (c < rank) pre += v;
            }
            S.tot[threadIdx.x] = tot;
            S.base[threadIdx.x] = pre;
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t v[4], sum = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) { v[q] = S.tot[lane * 4 + q]; sum += v[q]; }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            uint32_t acc = incl - sum;
#pragma unroll
            for (int q = 0; q < 4; q++) { S.base[lane * 4 + q] += acc; acc += v[q]; }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kClusterItems; k++) {
            if (k < items) {
                const uint32_t dg = digit_of(key[k], shift);
                const uint32_t r = (rk[k >> 1] >> ((k & 1) * 16)) & 0xffffu;
                const uint32_t pos = S.base[dg] + wh[dg] + r;
                const int dest = (int)(pos / (uint32_t)chunk);
                const uint32_t off = pos - (uint32_t)dest * (uint32_t)chunk;
                cluster.map_shared_rank(S.rkey, dest)[off] = key[k];
                cluster.map_shared_rank(S.rval, dest)[off] = val[k];
            }
        }
        cluster.sync();  // every element has landed in its owner's buffer
    }

    // sorted keys, FP32 records and bucket tables for this block's positions
    const PairGeom &Gc = G;
    const double cx = Gc.cx, cy = Gc.cy;
    for (int i = threadIdx.x; i < chunk; i += kClusterThreads) {
        const int pos = rank * chunk + i;
        if (pos >= n) break;
        const uint32_t kk = S.rkey[i];
        const uint32_t j = S.rval[i];
        L.key_b[b + pos] = kk;
        L.val_b[b + pos] = j;
        const double x = P.xy2[2 * (int64_t)j], y = P.xy2[2 * (int64_t)j + 1];
        const double eps = P.eps2 ? P.eps2[j] : P.eps_scalar;
        L.rec[b + pos] = make_float4((float)(x - cx), (float)(y - cy), (float)eps, __uint_as_float(j));
        const int lv = (int)(kk >> kQBits);
        const uint32_t s0 = S.start[lv], e0 = S.start[lv + 1];
        const int sh = kQBits - S.bits[lv];
        uint32_t *T = L.tab + P.t_off + S.tab[lv];
        const int64_t bk = (int64_t)((kk & kQMax) >> sh);
        int64_t bp = -1;
        if ((uint32_t)pos != s0) {
            const uint32_t prev = i > 0 ? S.rkey[i - 1] : cluster.map_shared_rank(S.rkey, rank - 1)[chunk - 1];
            bp = (int64_t)((prev & kQMax) >> sh);
        }
        for (int64_t bb = bp + 1; bb <= bk; bb++) T[bb] = (uint32_t)pos;
        if ((uint32_t)pos == e0 - 1) {
            const int64_t nb = (int64_t)1 << S.bits[lv];
            for (int64_t bb = bk + 1; bb <= nb; bb++) T[bb] = e0;
        }
    }
    cluster.sync();  // keep this block's shared memory alive for its neighbour's reads
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

cudaError_t launch_sort(const Launch &L, int max_n, cudaStream_t s) {
    cluster_sort_kernel<<<L.npairs * kClusterCtas, kClusterThreads, 0, s>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || max_n <= kClusterMaxN) return e;
    const int smem = (int)sizeof(SortSmem);
    e = cudaFuncSetAttribute(sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    sort_kernel<<<L.npairs, kSortThreads, smem, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_long_row_sort(const Launch &L, const uint32_t *list, const uint32_t *count, cudaStream_t s) {
    const int smem = (int)sizeof(SortSmem);
    cudaError_t e = cudaFuncSetAttribute(long_row_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    long_row_sort_kernel<<<1, kSortThreads, smem, s>>>(L, list, count);
    return cudaGetLastError();
}

}  // namespace egm
