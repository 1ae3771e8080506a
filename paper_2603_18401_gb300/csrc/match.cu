// After matching: the mutual (cross-check) test and the compact match list.
//
//   mutual_kernel   rows [0, m) are image-1 queries matched into image 2,
//                   rows [m, m + n) image-2 queries matched into image 1 (the
//                   same pair with the roles swapped and F transposed, Sec. 3);
//                   a match i -> j is mutual when j's best is i.  The flag
//                   EGM_FLAG_MUTUAL is added to both rows.
//   compact kernels the (query, best) pairs of the rows whose flags contain a
//                   required mask, in ascending query order: per-block counts,
//                   one block's scan of them, then the writes.
#include "egm_internal.cuh"

namespace egm {

namespace {

__global__ void mutual_kernel(const int32_t *best, uint8_t *flags, int64_t m, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m + n) return;
    const int32_t b = best[t];
    bool mutual = false;
    if (t < m) mutual = b >= 0 && b < n && best[m + b] == (int32_t)t;
    else mutual = b >= 0 && b < m && best[b] == (int32_t)(t - m);
    if (mutual) flags[t] |= (uint8_t)EGM_FLAG_MUTUAL;
}

constexpr int kCompactThreads = 256;
constexpr int kCompactItems = 8;
constexpr int kCompactTile = kCompactThreads * kCompactItems;

__device__ __forceinline__ bool keep(const uint8_t *flags, int64_t i, int64_t m, uint32_t require) {
    return i < m && (flags[i] & require) == require;
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *wsum, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kCompactThreads / 32 ? wsum[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += x;
        }
        if (lane < kCompactThreads / 32) wsum[lane] = wi - w;
        if (lane == 31) wsum[kCompactThreads / 32] = wi;
    }
    __syncthreads();
    total = wsum[kCompactThreads / 32];
    const uint32_t r = wsum[warp] + incl - v;
    __syncthreads();
    return r;
}

// per tile of kCompactTile rows: the number kept
__global__ void __launch_bounds__(kCompactThreads) compact_count_kernel(const uint8_t *flags, int64_t m,
                                                                        uint32_t require, uint32_t *tile_count) {
    __shared__ uint32_t wsum[kCompactThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kCompactTile;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kCompactItems; k++) c += keep(flags, base + (int64_t)k * kCompactThreads + threadIdx.x, m, require);
    uint32_t total;
    block_exclusive_scan(c, wsum, total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = total;
}

// exclusive scan of the tile counts (one block, any number of tiles)
__global__ void __launch_bounds__(kCompactThreads) compact_scan_kernel(uint32_t *tile_count, int64_t tiles,
                                                                       int64_t *count) {
    __shared__ uint32_t wsum[kCompactThreads / 32 + 1];
    uint32_t carry = 0;
    for (int64_t t0 = 0; t0 < tiles; t0 += kCompactThreads) {
        const int64_t t = t0 + threadIdx.x;
        const uint32_t v = t < tiles ? tile_count[t] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, wsum, total);
        if (t < tiles) tile_count[t] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *count = carry;
}

__global__ void __launch_bounds__(kCompactThreads) compact_write_kernel(const uint8_t *flags, const int32_t *best,
                                                                        int64_t m, uint32_t require,
                                                                        const uint32_t *tile_off, int32_t *qi,
                                                                        int32_t *rj) {
    __shared__ uint32_t wsum[kCompactThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kCompactTile;
    // thread t owns rows base + t * kCompactItems + k: ascending order within the tile
    bool kp[kCompactItems];
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kCompactItems; k++) {
        kp[k] = keep(flags, base + (int64_t)threadIdx.x * kCompactItems + k, m, require);
        c += kp[k];
    }
    uint32_t total;
    uint32_t pos = tile_off[blockIdx.x] + block_exclusive_scan(c, wsum, total);
#pragma unroll
    for (int k = 0; k < kCompactItems; k++)
        if (kp[k]) {
            const int64_t i = base + (int64_t)threadIdx.x * kCompactItems + k;
            qi[pos] = (int32_t)i;
            rj[pos] = best[i];
            pos++;
        }
}

}  // namespace

// F^T of a row-major 3 x 3 matrix (the reverse direction of a pair, Sec. 3).
__global__ void transpose3_kernel(const double *F, double *Ft) {
    const int k = threadIdx.x;
    if (k < 9) Ft[3 * (k % 3) + k / 3] = F[k];
}

cudaError_t launch_transpose3(const double *F, double *Ft, cudaStream_t s) {
    transpose3_kernel<<<1, 32, 0, s>>>(F, Ft);
    return cudaGetLastError();
}

cudaError_t launch_mutual(const int32_t *best, uint8_t *flags, int64_t m, int64_t n, cudaStream_t s) {
    if (m + n == 0) return cudaSuccess;
    mutual_kernel<<<(int)((m + n + 255) / 256), 256, 0, s>>>(best, flags, m, n);
    return cudaGetLastError();
}

int64_t compact_tiles(int64_t m) { return (m + kCompactTile - 1) / kCompactTile; }

cudaError_t launch_compact(const uint8_t *flags, const int32_t *best, int64_t m, uint32_t require,
                           uint32_t *tile_count, int32_t *qi, int32_t *rj, int64_t *count, cudaStream_t s) {
    const int64_t tiles = compact_tiles(m);
    if (tiles == 0) return cudaMemsetAsync(count, 0, sizeof(int64_t), s);
    compact_count_kernel<<<(int)tiles, kCompactThreads, 0, s>>>(flags, m, require, tile_count);
    compact_scan_kernel<<<1, kCompactThreads, 0, s>>>(tile_count, tiles, count);
    compact_write_kernel<<<(int)tiles, kCompactThreads, 0, s>>>(flags, best, m, require, tile_count, qi, rj);
    return cudaGetLastError();
}

}  // namespace egm
