// Grid-based motion statistics (GMS) filter of a pair's matches: the filter
// the paper applies to its guided matches by default, with the neighbour
// threshold 6 (Sec. 5.1; Sec. 4.3 names GMS as suited to guided matching).
// GMS is from Bian et al. (CVPR 2017):
//
//   cells      image 1: floor(x * G / W1 + s) for a grid shift s in {0, 1/2}
//              (clamped to 0 .. G), image 2: floor(x * G / W2) (0 .. G - 1);
//              FP64 with one rounding per operation
//   motion     M[c][d] = matches from image-1 cell c to image-2 cell d,
//              N[c] = matches in c; d*(c) = argmax_d M[c][d] (lowest d on ties)
//   score      S(c) = sum over the 3 x 3 offsets o of M[c + o][d*(c) + o]
//   keep       d == d*(c) and S(c) > alpha * sqrt(sum_o N[c + o] / 9),
//              the union over the four shifts
//
// gms_cells_kernel: one block per shift.  Counting sort of the matches by
// image-1 cell (shared-memory counts, the image-2 cells placed in global
// scratch), then a warp per cell: a shared-memory histogram over image-2
// cells gives d*, and counts in the neighbour cells' lists give S.  The
// decision of each cell (d* or -1) goes to a table per shift.
// gms_flag_kernel: one thread per row sets or clears EGM_FLAG_GMS.
#include "egm_internal.cuh"

namespace egm {

namespace {

constexpr int kGmsThreads = 1024;
constexpr int kGmsWarps = kGmsThreads / 32;
constexpr int kGmsSmemBudget = 160 * 1024;

__device__ __forceinline__ int gms_cell(double v, int G, double size, double shift, int top) {
    const double t = __dadd_rn(__ddiv_rn(__dmul_rn(v, (double)G), size), shift);
    const double f = floor(t);
    if (!(f > 0.0)) return 0;  // also NaN
    return f >= (double)top ? top : (int)f;
}

__device__ __forceinline__ double shift_x(int s) { return (s & 1) ? 0.5 : 0.0; }
__device__ __forceinline__ double shift_y(int s) { return (s & 2) ? 0.5 : 0.0; }

struct GmsArgs {
    const double *xy1, *xy2;
    const int32_t *best;
    const uint8_t *flags;
    int64_t m, n;
    uint32_t require;
    double w1, h1, w2, h2;
    int G;
    double alpha;
};

__device__ __forceinline__ bool gms_input(const GmsArgs &a, int64_t i, int32_t &j) {
    j = a.best[i];
    return j >= 0 && j < a.n && (a.flags[i] & a.require) == a.require;
}

__device__ __forceinline__ int cell1(const GmsArgs &a, int64_t i, int s) {
    const int G1 = a.G + 1;
    const int cx = gms_cell(a.xy1[2 * i], a.G, a.w1, shift_x(s), a.G);
    const int cy = gms_cell(a.xy1[2 * i + 1], a.G, a.h1, shift_y(s), a.G);
    return cy * G1 + cx;
}

__device__ __forceinline__ int cell2(const GmsArgs &a, int32_t j) {
    const int dx = gms_cell(a.xy2[2 * (int64_t)j], a.G, a.w2, 0.0, a.G - 1);
    const int dy = gms_cell(a.xy2[2 * (int64_t)j + 1], a.G, a.h2, 0.0, a.G - 1);
    return dy * a.G + dx;
}

// dynamic shared memory: count, start, cursor, dstar [(G + 1)^2] int32, then
// the histograms of `hw` warps, G^2 uint32 each
__global__ void __launch_bounds__(kGmsThreads) gms_cells_kernel(GmsArgs a, int hw, uint16_t *dsorted,
                                                                 int32_t *decision) {
    extern __shared__ int32_t gsm[];
    const int G = a.G, G1 = G + 1, C1 = G1 * G1, C2 = G * G;
    const int s = blockIdx.x;
    int32_t *count = gsm, *start = gsm + C1, *cursor = gsm + 2 * C1, *dstar = gsm + 3 * C1;
    uint32_t *hist = reinterpret_cast<uint32_t *>(gsm + 4 * C1);
    uint16_t *ds = dsorted + (int64_t)s * a.m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (int k = threadIdx.x; k < C1; k += kGmsThreads) count[k] = 0, cursor[k] = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < a.m; i += kGmsThreads) {
        int32_t j;
        if (gms_input(a, i, j)) atomicAdd(&count[cell1(a, i, s)], 1);
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the counts
        int carry = 0;
        for (int b = 0; b < C1; b += 32) {
            const int v = b + lane < C1 ? count[b + lane] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += x;
            }
            if (b + lane < C1) start[b + lane] = carry + incl - v;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < a.m; i += kGmsThreads) {
        int32_t j;
        if (!gms_input(a, i, j)) continue;
        const int c = cell1(a, i, s);
        ds[start[c] + atomicAdd(&cursor[c], 1)] = (uint16_t)cell2(a, j);
    }
    __syncthreads();

    // d*(c): the most frequent image-2 cell of c's list
    if (warp < hw) {
        uint32_t *h = hist + (size_t)warp * C2;
        for (int c = warp; c < C1; c += hw) {
            const int len = count[c];
            if (len == 0) {
                if (lane == 0) dstar[c] = -1;
                continue;
            }
            for (int b = lane; b < C2; b += 32) h[b] = 0u;
            __syncwarp();
            const uint16_t *lst = ds + start[c];
            for (int k = lane; k < len; k += 32) atomicAdd(&h[lst[k]], 1u);
            __syncwarp();
            uint32_t bc = 0;
            int bb = C2;
            for (int b = lane; b < C2; b += 32) {
                const uint32_t v = h[b];
                if (v > bc) bc = v, bb = b;  // ascending b: the first maximum of this lane
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
                const int ob = __shfl_xor_sync(0xffffffffu, bb, o);
                if (oc > bc || (oc == bc && ob < bb)) bc = oc, bb = ob;
            }
            if (lane == 0) dstar[c] = bb;
            __syncwarp();
        }
    }
    __syncthreads();

    // S(c) and the threshold
    for (int c = warp; c < C1; c += kGmsWarps) {
        const int d = dstar[c];
        int32_t res = -1;
        if (d >= 0) {
            const int cx = c % G1, cy = c / G1, dx = d % G, dy = d / G;
            uint32_t S = 0;
            int64_t total = 0;
            for (int o = 0; o < 9; o++) {
                const int ox = o % 3 - 1, oy = o / 3 - 1;
                const int ax = cx + ox, ay = cy + oy;
                if (ax < 0 || ax >= G1 || ay < 0 || ay >= G1) continue;
                const int ac = ay * G1 + ax;
                total += count[ac];
                const int bx = dx + ox, by = dy + oy;
                if (bx < 0 || bx >= G || by < 0 || by >= G) continue;
                const uint16_t target = (uint16_t)(by * G + bx);
                const uint16_t *lst = ds + start[ac];
                uint32_t k0 = 0;
                for (int k = lane; k < count[ac]; k += 32) k0 += lst[k] == target;
                S += __reduce_add_sync(0xffffffffu, k0);
            }
            const double thr = __dmul_rn(a.alpha, __dsqrt_rn(__ddiv_rn((double)total, 9.0)));
            if ((double)S > thr) res = d;
        }
        if (lane == 0) decision[(int64_t)s * C1 + c] = res;
    }
}

__global__ void gms_flag_kernel(GmsArgs a, const int32_t *decision, uint8_t *flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    const int C1 = (a.G + 1) * (a.G + 1);
    int32_t j;
    bool keep = false;
    if (gms_input(a, i, j)) {
        const int d = cell2(a, j);
#pragma unroll
        for (int s = 0; s < 4; s++) keep |= decision[s * C1 + cell1(a, i, s)] == d;
    }
    const uint8_t f = a.flags[i];
    flags[i] = (uint8_t)((f & ~EGM_FLAG_GMS) | (keep ? EGM_FLAG_GMS : 0));
}

}  // namespace

size_t gms_scratch_bytes(int64_t m, int grid) {
    const size_t ds = ((size_t)4 * (size_t)m * sizeof(uint16_t) + 255) & ~(size_t)255;
    return ds + (size_t)4 * (grid + 1) * (grid + 1) * sizeof(int32_t);
}

cudaError_t launch_gms(const double *xy1, int64_t m, const double *xy2, int64_t n, const int32_t *best,
                       uint8_t *flags, double w1, double h1, double w2, double h2, uint32_t require, int grid,
                       double alpha, void *scratch, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    GmsArgs a{xy1, xy2, best, flags, m, n, require, w1, h1, w2, h2, grid, alpha};
    const int C1 = (grid + 1) * (grid + 1), C2 = grid * grid;
    const size_t fixed = (size_t)4 * C1 * sizeof(int32_t);
    const int hw = (int)std::min<size_t>(kGmsWarps, (kGmsSmemBudget - fixed) / ((size_t)C2 * sizeof(uint32_t)));
    const size_t smem = fixed + (size_t)hw * C2 * sizeof(uint32_t);
    uint16_t *ds = static_cast<uint16_t *>(scratch);
    int32_t *decision = reinterpret_cast<int32_t *>(static_cast<char *>(scratch) +
                                                    (((size_t)4 * (size_t)m * sizeof(uint16_t) + 255) & ~(size_t)255));
    cudaError_t e = cudaFuncSetAttribute(gms_cells_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gms_cells_kernel<<<4, kGmsThreads, smem, st>>>(a, hw, ds, decision);
    gms_flag_kernel<<<(int)((m + 255) / 256), 256, 0, st>>>(a, decision, flags);
    return cudaGetLastError();
}

}  // namespace egm
