// Grid-based motion statistics (GMS) filter of the matches of a batch of
// pairs (one pair: a batch of one): the filter
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
// Rows of all pairs are concatenated (pair p's rows start at row_off[p]).
// gms_prep_kernel: one thread per row; the image-1 cell under each shift and
// the image-2 cell, each coordinate divided once (x * G / W, then + 1/2 for
// the shifted grids: the same operations, in the same order, as the cell
// formula), packed as 16-bit cell numbers.
// gms_cells_kernel: one block per (pair, shift).  Counting sort of the matches by
// image-1 cell (shared-memory counts, the image-2 cells placed in global
// scratch), then a warp per cell: a shared-memory histogram over image-2
// cells gives d*, and counts in the neighbour cells' lists give S.  The
// decision of each cell (d* or -1) goes to a table per pair and shift.
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
    const GmsPair *pairs;
    const int64_t *row_offs;  // npairs + 1
    int32_t npairs;
    int64_t rows;
    uint32_t require;
    int G;
    double alpha;
};

__device__ __forceinline__ int gms_pair_of(const GmsArgs &a, const int64_t *s_offs, bool cached, int64_t i) {
    return cached ? pair_of_shared(s_offs, a.npairs, i) : pair_of(a.row_offs, a.npairs, i);
}

// c1[i] = image-1 cell under shifts 0..3 (x shift = bit 0, y shift = bit 1),
// c2[i] = image-2 cell, kNoCell where row i is not an input match
__global__ void __launch_bounds__(256) gms_prep_kernel(GmsArgs a, ushort4 *c1, uint16_t *c2) {
    __shared__ int64_t s_offs[kSmemPairs + 1];
    const bool cached = load_offsets(s_offs, a.row_offs, a.npairs);
    __syncthreads();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.rows;
         g += (int64_t)gridDim.x * blockDim.x) {
        const GmsPair &P = a.pairs[gms_pair_of(a, s_offs, cached, g)];
        const int64_t i = g - P.row_off;
        const int32_t j = P.best[i];
        const bool in = j >= 0 && j < P.n && (P.flags[i] & a.require) == a.require;
        if (!in) {
            c1[g] = make_ushort4(kNoCell, kNoCell, kNoCell, kNoCell);
            c2[g] = kNoCell;
            continue;
        }
        const int G = a.G, G1 = G + 1;
        const double tx = grid_coord(P.xy1[2 * i], G, P.w1), ty = grid_coord(P.xy1[2 * i + 1], G, P.h1);
        const int x0 = clamp_cell(tx, G), x1 = clamp_cell(__dadd_rn(tx, 0.5), G);
        const int y0 = clamp_cell(ty, G), y1 = clamp_cell(__dadd_rn(ty, 0.5), G);
        c1[g] = make_ushort4((uint16_t)(y0 * G1 + x0), (uint16_t)(y0 * G1 + x1), (uint16_t)(y1 * G1 + x0),
                             (uint16_t)(y1 * G1 + x1));
        const int dx = clamp_cell(grid_coord(P.xy2[2 * (int64_t)j], G, P.w2), G - 1);
        const int dy = clamp_cell(grid_coord(P.xy2[2 * (int64_t)j + 1], G, P.h2), G - 1);
        c2[g] = (uint16_t)(dy * G + dx);
    }
}

__device__ __forceinline__ uint16_t shift_cell(const ushort4 &v, int s) {
    return s == 0 ? v.x : s == 1 ? v.y : s == 2 ? v.z : v.w;
}

// dynamic shared memory: count, start, cursor, dstar [(G + 1)^2] int32, then
// the histograms of `hw` warps, G^2 uint32 each.  Block b: pair b / 4, shift b % 4.
__global__ void __launch_bounds__(kGmsThreads, 1) gms_cells_kernel(GmsArgs a, int hw, const ushort4 *c1g,
                                                                 const uint16_t *c2g, uint16_t *dsorted,
                                                                 int32_t *decision) {
    extern __shared__ int32_t gsm[];
    const int G = a.G, G1 = G + 1, C1 = G1 * G1, C2 = G * G;
    const int p = blockIdx.x >> 2, s = blockIdx.x & 3;
    const int64_t m = a.pairs[p].m, roff = a.pairs[p].row_off;
    const ushort4 *c1 = c1g + roff;
    const uint16_t *c2 = c2g + roff;
    int32_t *count = gsm, *start = gsm + C1, *cursor = gsm + 2 * C1, *dstar = gsm + 3 * C1;
    uint32_t *hist = reinterpret_cast<uint32_t *>(gsm + 4 * C1);
    uint16_t *ds = dsorted + 4 * roff + (int64_t)s * m;
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
    int32_t *dec = decision + (int64_t)blockIdx.x * C1;
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
        if (lane == 0) dec[c] = res;
    }
}

__global__ void __launch_bounds__(256) gms_flag_kernel(GmsArgs a, const ushort4 *c1, const uint16_t *c2,
                                                        const int32_t *decision) {
    __shared__ int64_t s_offs[kSmemPairs + 1];
    const bool cached = load_offsets(s_offs, a.row_offs, a.npairs);
    __syncthreads();
    const int C1 = (a.G + 1) * (a.G + 1);
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.rows;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int p = gms_pair_of(a, s_offs, cached, g);
        const GmsPair &P = a.pairs[p];
        const int64_t i = g - P.row_off;
        const uint16_t d = c2[g];
        bool keep = false;
        if (d != kNoCell) {
            const ushort4 c = c1[g];
            const int32_t *dec = decision + (int64_t)p * 4 * C1;
            keep = dec[c.x] == d || dec[C1 + c.y] == d || dec[2 * C1 + c.z] == d || dec[3 * C1 + c.w] == d;
        }
        const uint8_t f = P.flags[i];
        P.flags[i] = (uint8_t)((f & ~EGM_FLAG_GMS) | (keep ? EGM_FLAG_GMS : 0));
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// scratch: pair table | row offsets | sorted lists 4 rows x 16 bit |
// decisions 4 npairs (G + 1)^2 x 32 bit | image-1 cells rows x 64 bit |
// image-2 cells rows x 16 bit
GmsLayout gms_layout(int npairs, int64_t rows, int grid) {
    GmsLayout l;
    l.table = 0;
    l.offs = align256(sizeof(GmsPair) * (size_t)npairs);
    l.ds = l.offs + align256(sizeof(int64_t) * (size_t)(npairs + 1));
    l.dec = l.ds + align256((size_t)4 * (size_t)rows * sizeof(uint16_t));
    l.c1 = l.dec + align256((size_t)4 * npairs * (grid + 1) * (grid + 1) * sizeof(int32_t));
    l.c2 = l.c1 + align256((size_t)rows * sizeof(ushort4));
    l.total = l.c2 + align256((size_t)rows * sizeof(uint16_t));
    return l;
}

cudaError_t launch_gms(void *scratch, const GmsLayout &l, int npairs, int64_t rows, uint32_t require, int grid,
                       double alpha, cudaStream_t st) {
    if (rows == 0 || npairs == 0) return cudaSuccess;
    char *b = static_cast<char *>(scratch);
    GmsArgs a{reinterpret_cast<const GmsPair *>(b + l.table), reinterpret_cast<const int64_t *>(b + l.offs),
              npairs, rows, require, grid, alpha};
    const int C1 = (grid + 1) * (grid + 1), C2 = grid * grid;
    const size_t fixed = (size_t)4 * C1 * sizeof(int32_t);
    const int hw = (int)std::min<size_t>(kGmsWarps, (kGmsSmemBudget - fixed) / ((size_t)C2 * sizeof(uint32_t)));
    const size_t smem = fixed + (size_t)hw * C2 * sizeof(uint32_t);
    uint16_t *ds = reinterpret_cast<uint16_t *>(b + l.ds);
    int32_t *dec = reinterpret_cast<int32_t *>(b + l.dec);
    ushort4 *c1 = reinterpret_cast<ushort4 *>(b + l.c1);
    uint16_t *c2 = reinterpret_cast<uint16_t *>(b + l.c2);
    cudaError_t e = cudaFuncSetAttribute(gms_cells_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (rows + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    gms_prep_kernel<<<(int)blocks, 256, 0, st>>>(a, c1, c2);
    gms_cells_kernel<<<4 * npairs, kGmsThreads, smem, st>>>(a, hw, c1, c2, ds, dec);
    gms_flag_kernel<<<(int)blocks, 256, 0, st>>>(a, c1, c2, dec);
    return cudaGetLastError();
}

}  // namespace egm
