// egm_match_pair_static: the one-pair matching call with no allocation at all.
//
// Some callers cannot allocate device memory: code that runs while another
// component owns the device allocator (a framework with its own memory pool
// and a fixed budget), real-time loops that must not stall in cudaMalloc or
// cudaFree (both may synchronise the whole device), and plug-ins that are
// handed a stream but no context of their own.  This entry point serves them.
// It creates no egm_ctx and calls no cudaMalloc, cudaFree, cudaMallocHost or
// other allocating routine: every scratch buffer of the pipeline lives in one
// file-scope __device__ array of fixed size, and the caller passes inputs and
// outputs as with egm_match_pair.
//
// The array is a module global: every GPU that loads libegm.so holds it until
// the process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.
#include <mutex>
#include <string.h>

#include "egm_internal.cuh"

using namespace egm;

namespace {

constexpr int64_t kStaticMaxKeypoints = 16384;  // per image (m and n)

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the scratch array (offsets in bytes).
constexpr int64_t M = kStaticMaxKeypoints, N = kStaticMaxKeypoints;
constexpr size_t kOffPairs = 0;
constexpr size_t kOffGeom = align256(kOffPairs + sizeof(PairDesc));
constexpr size_t kOffOffs = align256(kOffGeom + sizeof(PairGeom));
constexpr size_t kOffKeys = align256(kOffOffs + 4 * sizeof(int64_t));
constexpr size_t kOffRec = align256(kOffKeys + 6 * sizeof(uint32_t) * N);
constexpr size_t kOffRtmp = align256(kOffRec + sizeof(float4) * N);
constexpr size_t kOffTab = align256(kOffRtmp + sizeof(float4) * N);
constexpr int64_t kTabCap = 4 * N + 2 * kLevels + 32;
constexpr size_t kOffCurs = align256(kOffTab + sizeof(uint32_t) * kTabCap);
constexpr size_t kOffQrec = align256(kOffCurs + sizeof(uint32_t) * kTabCap);
constexpr size_t kOffQcount = align256(kOffQrec + sizeof(QueryRec) * M);
constexpr size_t kOffScan = align256(kOffQcount + sizeof(int64_t) * (M + 1));
constexpr size_t kOffLong = align256(kOffScan + sizeof(int64_t) * (M / 8192 + 2));
constexpr size_t kOffBlk = align256(kOffLong + sizeof(uint32_t) * (M + 1));
constexpr size_t kOffSmall = align256(kOffBlk + sizeof(int32_t) * (M / kStabQB + 2));
constexpr size_t kScratchBytes = align256(kOffSmall + 256);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices];
std::mutex g_setup_mutex;

// Device address of g_scratch on the current device (looked up once).
cudaError_t scratch_address(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

int row_bytes_static(int kind, int dim) {
    return kind == EGM_DESC_U8_L2 ? dim : kind == EGM_DESC_F32_L2 ? 4 * dim : kind == EGM_DESC_BIN ? dim / 8 : -1;
}

bool aligned16_static(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

egm_status status_from(uint32_t st) {
    if (st & kStNan) return EGM_ERR_NAN;
    if (st & kStDegenerateF) return EGM_ERR_DEGENERATE_F;
    if (st & kStArg) return EGM_ERR_ARG;
    if (st & kStCapacity) return EGM_ERR_CAPACITY;
    if (st & kStTimeout) return EGM_ERR_TIMEOUT;
    return EGM_OK;
}

}  // namespace

#define EGM_STATIC_TRY(x)                                                         \
    do {                                                                          \
        cudaError_t e_ = (x);                                                     \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? EGM_ERR_NOMEM : EGM_ERR_CUDA; \
    } while (0)

extern "C" egm_status egm_match_pair_static(const egm_pair *P, const egm_out *out, const egm_params *params,
                                            void *stream) {
    if (!P || !out) return EGM_ERR_ARG;
    // the same argument rules as egm_match_pair
    if (P->m < 0 || P->n < 0 || !P->F || P->width <= 0 || P->height <= 0) return EGM_ERR_ARG;
    if ((P->m > 0 && !P->xy1) || (P->n > 0 && !P->xy2)) return EGM_ERR_ARG;
    if (P->m > kStaticMaxKeypoints || P->n > kStaticMaxKeypoints) return EGM_ERR_CAPACITY;
    if (!P->eps2) {
        if (P->eps_scalar != P->eps_scalar || P->eps_scalar == INFINITY) return EGM_ERR_NAN;
        if (!(P->eps_scalar > 0.0)) return EGM_ERR_ARG;
    }
    const bool desc = P->desc1 != nullptr || P->desc2 != nullptr;
    int rb = 0;
    if (desc) {
        if ((!P->desc1 && P->m > 0) || (!P->desc2 && P->n > 0)) return EGM_ERR_ARG;
        if (P->kind == EGM_DESC_BIN && (P->dim <= 0 || P->dim % 128 != 0)) return EGM_ERR_ARG;
        rb = row_bytes_static(P->kind, P->dim);
        if (rb <= 0 || rb % 16 != 0 || rb > 2048) return EGM_ERR_ARG;
        if (!aligned16_static(P->desc1) || !aligned16_static(P->desc2)) return EGM_ERR_ARG;
    }
    const bool csr = out->cand_offsets != nullptr;
    if (csr && (!out->cand_total || out->cand_capacity < 0 || (out->cand_capacity > 0 && !out->cand_idx)))
        return EGM_ERR_ARG;
    if (!csr && !desc) return EGM_ERR_ARG;
    int32_t rn = 4, rd = 5;
    if (params) {
        if (params->ratio_num <= 0 || params->ratio_den <= 0 || params->ratio_num > 1000000 ||
            params->ratio_den > 1000000)
            return EGM_ERR_ARG;
        rn = params->ratio_num;
        rd = params->ratio_den;
    }

    int device = 0;
    EGM_STATIC_TRY(cudaGetDevice(&device));
    unsigned char *base = nullptr;
    EGM_STATIC_TRY(scratch_address(device, &base));
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // The pair travels in the launch parameters: the geometry kernel writes
    // the pair table and offsets into the array for the later kernels, so the
    // call copies nothing from host memory.
    PairDesc pd;
    memset(&pd, 0, sizeof(pd));
    pd.xy1 = P->xy1;
    pd.xy2 = P->xy2;
    pd.F = P->F;
    pd.eps2 = P->eps2;
    pd.desc1 = static_cast<const uint8_t *>(P->desc1);
    pd.desc2 = static_cast<const uint8_t *>(P->desc2);
    pd.eps_scalar = P->eps_scalar;
    pd.m = P->m;
    pd.n = P->n;
    pd.kind = desc ? P->kind : EGM_DESC_U8_L2;
    pd.dim = P->dim;
    pd.row_bytes = rb;
    pd.width = P->width;
    pd.height = P->height;
    // bucket-table entries this pair needs (the prep kernel zeroes them all)
    pd.t_cap = 4 * (int64_t)P->n + 2 * kLevels + 32;
    // the array keeps the previous call's contents: clear the status word and counters
    EGM_STATIC_TRY(cudaMemsetAsync(base + kOffSmall, 0, 256, st));

    Launch L;
    memset(&L, 0, sizeof(L));
    L.pairs = reinterpret_cast<const PairDesc *>(base + kOffPairs);
    L.geom = reinterpret_cast<PairGeom *>(base + kOffGeom);
    L.npairs = 1;
    L.nq = P->m;
    L.nr = P->n;
    L.q_offs = reinterpret_cast<const int64_t *>(base + kOffOffs);
    L.r_offs = reinterpret_cast<const int64_t *>(base + kOffOffs) + 2;
    uint32_t *k = reinterpret_cast<uint32_t *>(base + kOffKeys);
    const size_t nr = (size_t)(P->n > 0 ? P->n : 1);
    L.key_a = k;
    L.val_a = k + nr;
    L.key_b = k + 2 * nr;
    L.val_b = k + 3 * nr;
    L.key_c = k + 4 * nr;
    L.val_c = k + 5 * nr;
    L.rec = reinterpret_cast<float4 *>(base + kOffRec);
    L.rtmp = reinterpret_cast<float4 *>(base + kOffRtmp);
    L.tab = reinterpret_cast<uint32_t *>(base + kOffTab);
    L.ntab = pd.t_cap;
    L.curs = reinterpret_cast<uint32_t *>(base + kOffCurs);
    L.prep_done = reinterpret_cast<uint32_t *>(base + kOffSmall) + 40;
    L.qrec = reinterpret_cast<QueryRec *>(base + kOffQrec);
    L.status = reinterpret_cast<uint32_t *>(base + kOffSmall);
    L.counters = nullptr;
    L.qcount = reinterpret_cast<int64_t *>(base + kOffQcount);
    L.scan_tmp = reinterpret_cast<int64_t *>(base + kOffScan);
    L.blkpair = reinterpret_cast<int32_t *>(base + kOffBlk);
    L.ratio_num = rn;
    L.ratio_den = rd;
    L.max_n = P->n;
    L.kind = pd.kind;
    L.inl_use = 1;
    L.inl = pd;
    L.best = out->best;
    L.second = out->second;
    L.best_d = out->best_d;
    L.second_d = out->second_d;
    L.flags = out->flags;
    L.cand_offsets = out->cand_offsets;
    L.cand_idx = out->cand_idx;
    L.cand_capacity = out->cand_capacity;
    L.cand_total = out->cand_total;

    EGM_STATIC_TRY(launch_geometry(L, st));
    EGM_STATIC_TRY(launch_prep(L, st));
    EGM_STATIC_TRY(launch_sort(L, st));
    if (csr) {
        uint32_t *long_list = reinterpret_cast<uint32_t *>(base + kOffLong);
        uint32_t *long_count = reinterpret_cast<uint32_t *>(base + kOffSmall) + 16;
        EGM_STATIC_TRY(launch_stab(L, 1, st));
        EGM_STATIC_TRY(launch_csr_offsets(L, long_count, st));
        EGM_STATIC_TRY(launch_stab(L, 2, st));
        EGM_STATIC_TRY(launch_csr_row_sort(L, long_list, long_count, st));
    } else {
        EGM_STATIC_TRY(launch_stab(L, 0, st));
    }
    uint32_t status = 0;
    EGM_STATIC_TRY(cudaMemcpyAsync(&status, base + kOffSmall, sizeof(status), cudaMemcpyDeviceToHost, st));
    EGM_STATIC_TRY(cudaStreamSynchronize(st));
    return status_from(status);
}
