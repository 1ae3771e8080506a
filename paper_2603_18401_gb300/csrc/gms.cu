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
// gms_prep_kernel: one thread per row; the image-1 cell under each shift and
// the image-2 cell, each coordinate divided once (x * G / W, then + 1/2 for
// the shifted grids: the same operations, in the same order, as the cell
// formula), packed as 16-bit cell numbers.
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

constexpr uint16_t kNoCell = 0xFFFF;

__device__ __forceinline__ int clamp_cell(double t, int top) {
    const double f = floor(t);
    if (!(f > 0.0)) return 0;  // also NaN
    return f >= (double)top ? top : (int)f;
}

// x * G / size, rounded as written
__device__ __forceinline__ double grid_coord(double v, int G, double size) {
    return __ddiv_rn(__dmul_rn(v, (double)G), size);
}

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

// c1[i] = image-1 cell under shifts 0..3 (x shift = bit 0, y shift = bit 1),
// c2[i] = image-2 cell, kNoCell where row i is not an input match
__global__ void gms_prep_kernel(GmsArgs a, ushort4 *c1, uint16_t *c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    const int32_t j = a.best[i];
    const bool in = j >= 0 && j < a.n && (a.flags[i] & a.require) == a.require;
    if (!in) {
        c1[i] = make_ushort4(kNoCell, kNoCell, kNoCell, kNoCell);
        c2[i] = kNoCell;
        return;
    }
    const int G = a.G, G1 = G + 1;
    const double tx = grid_coord(a.xy1[2 * i], G, a.w1), ty = grid_coord(a.xy1[2 * i + 1], G, a.h1);
    const int x0 = clamp_cell(tx, G), x1 = clamp_cell(__dadd_rn(tx, 0.5), G);
    const int y0 = clamp_cell(ty, G), y1 = clamp_cell(__dadd_rn(ty, 0.5), G);
    c1[i] = make_ushort4((uint16_t)(y0 * G1 + x0), (uint16_t)(y0 * G1 + x1), (uint16_t)(y1 * G1 + x0),
                         (uint16_t)(y1 * G1 + x1));
    const int dx = clamp_cell(grid_coord(a.xy2[2 * (int64_t)j], G, a.w2), G - 1);
    const int dy = clamp_cell(grid_coord(a.xy2[2 * (int64_t)j + 1], G, a.h2), G - 1);
    c2[i] = (uint16_t)(dy * G + dx);
}

__device__ __forceinline__ uint16_t shift_cell(const ushort4 &v, int s) {
    return s == 0 ? v.x : s == 1 ? v.y : s == 2 ? v.z : v.w;
}

// dynamic shared memory: count, start, cursor, dstar [(G + 1)^2] int32, then
// the histograms of `hw` warps, G^2 uint32 each
__global__ void __launch_bounds__(kGmsThreads) gms_cells_kernel(int64_t m, int G, double alpha, int hw,
                                                                 const ushort4 *c1, const uint16_t *c2,
                                                                 uint16_t *dsorted, int32_t *decision) {
    extern __shared__ int32_t gsm[];
    const int G1 = G + 1, C1 = G1 * G1, C2 = G * G;
    const int s = blockIdx.x;
    int32_t *count = gsm, *start = gsm + C1, *cursor = gsm + 2 * C1, *dstar = gsm + 3 * C1;
    uint32_t *hist = reinterpret_cast<uint32_t *>(gsm + 4 * C1);
    uint16_t *ds = dsorted + (int64_t)s * m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (int k = threadIdx.x; k < C1; k += kGmsThreads) count[k] = 0, cursor[k] = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < m; i += kGmsThreads) {
        const uint16_t c = shift_cell(c1[i], s);
        if (c != kNoCell) atomicAdd(&count[c], 1);
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
    for (int64_t i = threadIdx.x; i < m; i += kGmsThreads) {
        const uint16_t c = shift_cell(c1[i], s);
        if (c != kNoCell) ds[start[c] + atomicAdd(&cursor[c], 1)] = c2[i];
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
            const double thr = __dmul_rn(alpha, __dsqrt_rn(__ddiv_rn((double)total, 9.0)));
            if ((double)S > thr) res = d;
        }
        if (lane == 0) decision[(int64_t)s * C1 + c] = res;
    }
}

__global__ void gms_flag_kernel(int64_t m, int G, const ushort4 *c1, const uint16_t *c2, const int32_t *decision,
                                uint8_t *flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int C1 = (G + 1) * (G + 1);
    const uint16_t d = c2[i];
    bool keep = false;
    if (d != kNoCell) {
        const ushort4 c = c1[i];
        keep = decision[c.x] == d || decision[C1 + c.y] == d || decision[2 * C1 + c.z] == d ||
               decision[3 * C1 + c.w] == d;
    }
    const uint8_t f = flags[i];
    flags[i] = (uint8_t)((f & ~EGM_FLAG_GMS) | (keep ? EGM_FLAG_GMS : 0));
}

}  // namespace

// scratch: sorted lists 4 m x 16 bit | decisions 4 (G + 1)^2 x 32 bit |
// image-1 cells m x 64 bit | image-2 cells m x 16 bit
namespace {
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
}

size_t gms_scratch_bytes(int64_t m, int grid) {
    return align256((size_t)4 * m * sizeof(uint16_t)) + align256((size_t)4 * (grid + 1) * (grid + 1) * sizeof(int32_t)) +
           align256((size_t)m * sizeof(ushort4)) + align256((size_t)m * sizeof(uint16_t));
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
    char *p = static_cast<char *>(scratch);
    uint16_t *ds = reinterpret_cast<uint16_t *>(p);
    p += align256((size_t)4 * m * sizeof(uint16_t));
    int32_t *decision = reinterpret_cast<int32_t *>(p);
    p += align256((size_t)4 * C1 * sizeof(int32_t));
    ushort4 *c1 = reinterpret_cast<ushort4 *>(p);
    p += align256((size_t)m * sizeof(ushort4));
    uint16_t *c2 = reinterpret_cast<uint16_t *>(p);
    cudaError_t e = cudaFuncSetAttribute(gms_cells_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((m + 255) / 256);
    gms_prep_kernel<<<blocks, 256, 0, st>>>(a, c1, c2);
    gms_cells_kernel<<<4, kGmsThreads, smem, st>>>(m, grid, alpha, hw, c1, c2, ds, decision);
    gms_flag_kernel<<<blocks, 256, 0, st>>>(m, grid, c1, c2, decision, flags);
    return cudaGetLastError();
}

}  // namespace egm
