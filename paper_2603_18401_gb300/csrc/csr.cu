// Candidate sets in CSR form (Eq. 4: C_i for every query, ascending index).
//
//   scan_*           exclusive prefix sum of the per-query candidate counts
//                    into cand_offsets (three launches: tile sums, a scan of
//                    the tile sums, tile scans); the last one checks the
//                    caller's capacity.
//   row_sort_kernel  one warp per row: bitonic sort in shared memory for rows
//                    of up to 1024 entries; longer rows are listed for the
//                    block radix sort (launch_long_row_sort).
#include "egm_internal.cuh"

namespace egm {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *warp_sums, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_sums[lane] = wi - w;
        if (lane == 31) warp_sums[32] = wi;
    }
    __syncthreads();
    const int64_t r = warp_sums[warp] + incl - v;
    total = warp_sums[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(Launch L) {
    pdl_begin();
    __shared__ int64_t ws[33];
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t i = t0 + (int64_t)threadIdx.x * kScanItems + k;
        if (i < L.nq) s += L.qcount[i];
    }
    int64_t total;
    block_excl_scan(s, ws, total);
    if (threadIdx.x == 0) L.scan_tmp[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(Launch L, int nblocks, uint32_t *long_count) {
    pdl_begin();
    __shared__ int64_t ws[33];
    if (threadIdx.x == 0) *long_count = 0u;
    int64_t carry = 0;
    for (int b0 = 0; b0 < nblocks; b0 += kScanThreads) {
        const int b = b0 + threadIdx.x;
        const int64_t v = b < nblocks ? L.scan_tmp[b] : 0;
        int64_t total;
        const int64_t ex = block_excl_scan(v, ws, total);
        if (b < nblocks) L.scan_tmp[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        L.scan_tmp[nblocks] = carry;
        L.cand_offsets[L.nq] = carry;
        *L.cand_total = carry;
        if (carry > L.cand_capacity) atomicOr(L.status, kStCapacity);
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_final_kernel(Launch L) {
    pdl_begin();
    __shared__ int64_t ws[33];
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t i = t0 + (int64_t)threadIdx.x * kScanItems + k;
        v[k] = i < L.nq ? L.qcount[i] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t ex = block_excl_scan(s, ws, total) + L.scan_tmp[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t i = t0 + (int64_t)threadIdx.x * kScanItems + k;
        if (i < L.nq) L.cand_offsets[i] = ex;
        ex += v[k];
    }
}

constexpr int kRowWarps = 8;
constexpr int kRowMax = 1024;

__global__ void __launch_bounds__(kRowWarps * 32) row_sort_kernel(Launch L, uint32_t *long_list,
                                                                  uint32_t *long_count) {
    pdl_begin();
    __shared__ uint32_t buf_all[kRowWarps][kRowMax];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *buf = buf_all[warp];
    if (L.cand_offsets[L.nq] > L.cand_capacity) return;  // rows were not written
    for (int64_t row = (int64_t)blockIdx.x * kRowWarps + warp; row < L.nq; row += (int64_t)gridDim.x * kRowWarps) {
        const int64_t a = L.cand_offsets[row];
        const int len = (int)(L.cand_offsets[row + 1] - a);
        if (len <= 1) continue;
        if (len > kRowMax) {
            if (lane == 0) long_list[atomicAdd(long_count, 1u)] = (uint32_t)row;
            continue;
        }
        int P = 32;
        while (P < len) P <<= 1;
        uint32_t *rk = reinterpret_cast<uint32_t *>(L.cand_idx + a);
        for (int i = lane; i < P; i += 32) buf[i] = i < len ? rk[i] : 0xffffffffu;
        __syncwarp();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < P; i += 32) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const uint32_t x = buf[i], y = buf[ixj];
                        const bool up = (i & k) == 0;
                        if (up ? x > y : x < y) { buf[i] = y; buf[ixj] = x; }
                    }
                }
                __syncwarp();
            }
        }
        for (int i = lane; i < len; i += 32) rk[i] = buf[i];
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_csr_offsets(const Launch &L, uint32_t *long_count, cudaStream_t s) {
    const int nb = (int)((L.nq + kScanTile - 1) / kScanTile);
    if (nb > 0) scan_partials_kernel<<<nb, kScanThreads, 0, s>>>(L);
    scan_top_kernel<<<1, kScanThreads, 0, s>>>(L, nb, long_count);
    if (nb > 0) scan_final_kernel<<<nb, kScanThreads, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_csr_row_sort(const Launch &L, uint32_t *long_list, uint32_t *long_count, cudaStream_t s) {
    if (L.nq > 0) {
        int64_t blocks = (L.nq + kRowWarps - 1) / kRowWarps;
        if (blocks > 152 * 16) blocks = 152 * 16;
        row_sort_kernel<<<(int)blocks, kRowWarps * 32, 0, s>>>(L, long_list, long_count);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_long_row_sort(L, long_list, long_count, s);
}

}  // namespace egm
