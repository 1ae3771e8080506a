// C ABI of libegm: context, scratch memory, argument checks and the launch
// sequence of the matching pipeline (declarations and conventions in egm.h).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "egm_internal.cuh"

namespace egm {
// The learned-tolerance network's forward pass with layers 2 and 3 on the
// tensor cores (mlp.cu); a timed-out MMA wait sets kStTimeout in *err
// (device); samples without a finite output get `fallback` in eps.  With pre
// (the pre-activations a1..a3, [layer][unit][sample]) the training pass runs
// instead: pre and z (the output before the softplus) are written, eps is
// not.
cudaError_t launch_mlp_forward_tc(const float *params, const float *feat, int64_t n, double *eps, uint32_t *err,
                                  double fallback, int sms, cudaStream_t s, float *pre = nullptr, float *z = nullptr);
}  // namespace egm

using namespace egm;

namespace {

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

cudaError_t grow(DevBuf &b, size_t need) {
    if (need <= b.bytes) return cudaSuccess;
    if (b.ptr) {
        cudaError_t e = cudaFree(b.ptr);
        if (e != cudaSuccess) return e;
        b.ptr = nullptr;
        b.bytes = 0;
    }
    size_t alloc = need + need / 4 + 4096;
    cudaError_t e = cudaMalloc(&b.ptr, alloc);
    if (e != cudaSuccess) return e;
    b.bytes = alloc;
    return cudaSuccess;
}

template <typename T>
T *as(DevBuf &b) { return reinterpret_cast<T *>(b.ptr); }

// Device scratch of one pipeline instance (a context, or a captured graph).
struct Scratch {
    DevBuf pairs, geom, offs, keys, rec, rtmp, tab, curs, qrec, qcount, scan, longlist, small, counters, blkpair, band;
    // the pair table, offsets and geometry are double-buffered: call k uses
    // half k mod 2, so that its geometry kernel can write while call k - 1's
    // last kernel still reads the other half
    int parity = 0;
    void release() {
        DevBuf *b[] = {&pairs, &geom, &offs, &keys, &rec, &rtmp, &tab, &curs, &qrec, &qcount, &scan, &longlist, &small,
                       &counters, &blkpair, &band};
        for (DevBuf *x : b) {
            if (x->ptr) cudaFree(x->ptr);
            x->ptr = nullptr;
            x->bytes = 0;
        }
    }
};

}  // namespace

// One regime's timings and choice (the tuner's cache entry).
struct TuneEntry {
    int32_t form = EGM_FORM_PLAIN;  // the faster form
    int32_t shape = 0;              // the fastest band tile shape
    float ms_plain = 0.0f, ms_band = 0.0f;
};

struct egm_ctx {
    int device = 0;
    int sms = 1;       // streaming multiprocessors of the device
    cudaStream_t stream = nullptr;
    egm_params params;
    bool counters_on = false;
    egm_stats last{};
    Scratch sc;
    DevBuf stage;  // host-path staging of inputs and outputs
    DevBuf compact;  // tile counts of egm_compact_matches
    DevBuf ft;       // egm_match_mutual_pair: F^T of the reverse direction
    DevBuf gms;      // egm_gms: pair table, matches sorted by cell, decisions per grid shift
    void *gms_host = nullptr;        // pinned staging of the GMS pair table
    size_t gms_host_bytes = 0;
    cudaEvent_t gms_host_ev = nullptr;
    // pinned host memory for the pair table and the status word
    // pinned staging slots of the pair-table uploads, used round-robin: the
    // host waits only when a slot's previous upload is still in flight
    static constexpr int kSlots = 8;
    void *h_table[kSlots] = {};
    size_t h_table_bytes[kSlots] = {};
    cudaEvent_t slot_ev[kSlots] = {};
    bool slot_pending[kSlots] = {};
    int slot = 0;
    uint32_t *h_status = nullptr;
    unsigned long long *h_counters = nullptr;
    // per-stage timing: kStages + 1 events per timed call
    bool timing_on = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<size_t> ev_calls;   // first event of each timed call
    std::vector<bool> ev_band;      // whether that call ran the banded form
    egm_timing tsum{};
    // the banded form sorts the queries on a second stream, beside the reference sort
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // egm_match_batch_host: input and output copies run on their own streams,
    // ordered against the matching by one event per pair and direction
    cudaStream_t copy = nullptr, copy_out = nullptr;
    cudaEvent_t copy_start = nullptr, out_done = nullptr;
    std::vector<cudaEvent_t> in_ev, done_ev;
    // the tuner's choice per call regime (regime_key)
    std::map<uint64_t, TuneEntry> tuned;
};

namespace {
constexpr int kStages = 6;  // geometry, prep, sort, post_sort, stab, csr
}

namespace {

egm_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return EGM_OK;
    if (e == cudaErrorMemoryAllocation) return EGM_ERR_NOMEM;
    return EGM_ERR_CUDA;
}

egm_status from_bits(uint32_t st) {
    if (st & kStNan) return EGM_ERR_NAN;
    if (st & kStDegenerateF) return EGM_ERR_DEGENERATE_F;
    if (st & kStArg) return EGM_ERR_ARG;
    if (st & kStCapacity) return EGM_ERR_CAPACITY;
    if (st & kStTimeout) return EGM_ERR_TIMEOUT;
    return EGM_OK;
}

#define EGM_TRY(x)                                   \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return from_cuda(e_); \
    } while (0)

int row_bytes_of(int kind, int dim) {
    switch (kind) {
        case EGM_DESC_U8_L2: return dim;
        case EGM_DESC_F32_L2: return 4 * dim;
        case EGM_DESC_BIN: return dim / 8;
        default: return -1;
    }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Descriptors are requested when either array is given.
bool has_desc(const egm_pair *P) { return P->desc1 != nullptr || P->desc2 != nullptr; }

egm_status check_pair(const egm_pair *P) {
    if (!P) return EGM_ERR_ARG;
    if (P->m < 0 || P->n < 0) return EGM_ERR_ARG;
    if (P->m > 0 && !P->xy1) return EGM_ERR_ARG;
    if (P->n > 0 && !P->xy2) return EGM_ERR_ARG;
    if (!P->F) return EGM_ERR_ARG;
    if (P->width <= 0 || P->height <= 0) return EGM_ERR_ARG;
    if (!P->eps2) {
        if (P->eps_scalar != P->eps_scalar || P->eps_scalar == INFINITY) return EGM_ERR_NAN;
        if (!(P->eps_scalar > 0.0)) return EGM_ERR_ARG;
    }
    if (has_desc(P)) {
        // a descriptor array may be NULL only when it has no rows
        if ((!P->desc1 && P->m > 0) || (!P->desc2 && P->n > 0)) return EGM_ERR_ARG;
        if (P->kind == EGM_DESC_BIN && (P->dim <= 0 || P->dim % 128 != 0)) return EGM_ERR_ARG;
        const int rb = row_bytes_of(P->kind, P->dim);
        if (rb <= 0 || rb % 16 != 0 || rb > 2048) return EGM_ERR_ARG;
        if (!aligned16(P->desc1) || !aligned16(P->desc2)) return EGM_ERR_ARG;
    }
    return EGM_OK;
}

struct Plan {
    std::vector<PairDesc> pd;
    std::vector<int64_t> offs;      // query, reference and tile offsets: 3 x (npairs + 1), then the
                                    // tile order (int32, packed two per entry)
    std::vector<int64_t> qoffs, roffs;
    int64_t nq = 0, nr = 0, ntab = 0, ntiles = 0;
    int max_n = 0;
    bool band_ok = false;           // every pair fits the banded form
    bool has_float = false;         // some pair has float descriptors
    bool dense_u8 = false;          // every pair u8 with a scalar tolerance and >= 32 estimated candidates per query
    double kbar_q = 0.0;            // sum over pairs of (estimated candidates per query) x (queries)
    bool eps_vec = false;           // some pair has per-keypoint tolerances (density unknown on the host)
    uint32_t kinds = 0;             // descriptor kinds present (bit k: kind k)
};

egm_status make_plan(const egm_pair *pairs, int npairs, Plan &pl) {
    pl.pd.resize(npairs);
    pl.qoffs.resize(npairs + 1);
    pl.roffs.resize(npairs + 1);
    for (int p = 0; p < npairs; p++) {
        egm_status s = check_pair(pairs + p);
        if (s != EGM_OK) return s;
        const egm_pair &A = pairs[p];
        PairDesc &D = pl.pd[p];
        memset(&D, 0, sizeof(D));
        D.xy1 = A.xy1;
        D.xy2 = A.xy2;
        D.F = A.F;
        D.eps2 = A.eps2;
        D.desc1 = static_cast<const uint8_t *>(A.desc1);
        D.desc2 = static_cast<const uint8_t *>(A.desc2);
        D.eps_scalar = A.eps_scalar;
        D.m = A.m;
        D.n = A.n;
        D.kind = has_desc(&A) ? A.kind : EGM_DESC_U8_L2;
        D.dim = A.dim;
        D.row_bytes = has_desc(&A) ? row_bytes_of(A.kind, A.dim) : 0;
        D.width = A.width;
        D.height = A.height;
        D.q_off = pl.nq;
        D.r_off = pl.nr;
        D.t_off = pl.ntab;
        D.t_cap = 4 * (int64_t)A.n + 2 * kLevels + 32;
        pl.qoffs[p] = pl.nq;
        pl.roffs[p] = pl.nr;
        pl.nq += A.m;
        pl.nr += A.n;
        pl.ntab += D.t_cap;
        pl.max_n = std::max(pl.max_n, A.n);
    }
    pl.qoffs[npairs] = pl.nq;
    pl.roffs[npairs] = pl.nr;
    pl.offs.resize(3 * (size_t)(npairs + 1));
    const int tm = band_tile_queries();
    pl.band_ok = true;
    // candidates per query of a pair, estimated as the expected count within
    // eps of a line crossing the image: 2 eps (n / (W H)) L, with the mean
    // chord L taken as 0.8 of the diagonal
    pl.dense_u8 = npairs > 0;
    for (int p = 0; p < npairs; p++) {
        const egm_pair &A = pairs[p];
        const double W = A.width, H = A.height;
        const double kbar = 2.0 * A.eps_scalar * (double)A.n / (W * H) * 0.8 * std::sqrt(W * W + H * H);
        pl.dense_u8 = pl.dense_u8 && has_desc(&A) && A.kind == EGM_DESC_U8_L2 && !A.eps2 && kbar >= 32.0;
        pl.kbar_q += A.eps2 ? 0.0 : kbar * (double)A.m;
        pl.eps_vec = pl.eps_vec || A.eps2 != nullptr;
        if (has_desc(&A)) pl.kinds |= 1u << (A.kind & 7);
    }
    for (int p = 0; p <= npairs; p++) {
        pl.offs[p] = pl.qoffs[p];
        pl.offs[(npairs + 1) + p] = pl.roffs[p];
        pl.offs[2 * (npairs + 1) + p] = pl.ntiles;
        if (p < npairs) {
            pl.ntiles += (pairs[p].m + tm - 1) / tm;
            pl.band_ok = pl.band_ok && has_desc(pairs + p) && band_supported(pairs[p].kind, pairs[p].dim);
            pl.has_float = pl.has_float || (has_desc(pairs + p) && pairs[p].kind == EGM_DESC_F32_L2);
        }
    }
    // Tiles are handed out costliest first (longest-processing-time order): a
    // tile's band holds about tm * n / m references plus its windows.
    std::vector<int> order(npairs);
    for (int p = 0; p < npairs; p++) order[p] = p;
    auto cost = [&](int p) { return (double)tm * pairs[p].n / std::max(pairs[p].m, 1) + 64.0; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    // one int64 entry per tile: the tile (low 32 bits) and its pair (high)
    const size_t base = pl.offs.size();
    pl.offs.resize(base + (size_t)pl.ntiles, 0);
    int64_t k = 0;
    for (int p : order)
        for (int64_t t = pl.offs[2 * (npairs + 1) + p]; t < pl.offs[2 * (npairs + 1) + p + 1]; t++)
            pl.offs[base + k++] = (int64_t)(uint32_t)t | ((int64_t)p << 32);
    return EGM_OK;
}

// int64 entries of the offsets upload for a batch of npairs pairs and nq queries.
size_t offs_entries(int npairs, int64_t nq) {
    return 3 * (size_t)(npairs + 1) + (size_t)(nq / band_tile_queries() + npairs + 2) + 1;
}

// The banded form runs when every pair fits it, no candidate lists are asked
// for, and it is requested -- or left to the library and either the call has
// more than two tiles per SM or its u8 pairs are dense (about 32 or more
// candidates per query).  With few tiles of sparse pairs every CTA of the
// band kernel takes one latency-bound tile and the plain form (no query
// sort, no packing) finishes first; with many tiles the banded form's
// throughput wins, and on dense pairs its tensor-core distances beat one
// CUDA-core distance per candidate.
egm_status choose_band(const Plan &pl, const egm_params &prm, bool csr, int sms, bool &band) {
    band = pl.band_ok && !csr &&
           (prm.form == EGM_FORM_BANDED ||
            (prm.form == EGM_FORM_AUTO && (pl.ntiles > 2 * (int64_t)sms || pl.dense_u8)));
    if (prm.form == EGM_FORM_BANDED && !band) return EGM_ERR_UNIMPLEMENTED;
    return EGM_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Banded-form scratch: query permutation and buckets; with float pairs
// (`packed`) also the sorted query records, the packed operand rows and
// their norms (padded for the aligned 16-byte bulk copies that read past a
// pair's last row).
// Without float pairs the operand buffers keep one tile of rows, which the
// band kernel's (unused) tensor maps cover.
struct BandLayout {
    size_t qperm, descA, descB, qbkt, qsrt, qscale, rnorm, total;
    BandLayout(int64_t nq, int64_t nr, bool packed) {
        const size_t rb = (size_t)band_row_bytes();
        const int64_t ta = packed ? nq : band_tile_queries(), tb = packed ? nr : band_tile_queries();
        qperm = 0;
        descA = qperm + align256(sizeof(uint32_t) * (size_t)std::max<int64_t>(nq, 1));
        descB = descA + align256(rb * (size_t)std::max<int64_t>(ta, 1));
        qbkt = descB + align256(rb * (size_t)std::max<int64_t>(tb, 1));
        qsrt = qbkt + align256(sizeof(uint16_t) * (size_t)std::max<int64_t>(nq, 1));
        qscale = qsrt + align256(sizeof(QueryRec) * (size_t)std::max<int64_t>(packed ? nq : 1, 1));
        rnorm = qscale + align256(sizeof(float) * (size_t)std::max<int64_t>(packed ? nq : 1, 1));
        // 64 rows of padding: bulk copies of a 32-row box may run past the last row
        total = rnorm + align256(sizeof(float4) * (size_t)((packed ? nr : 0) + 64));
    }
};

cudaError_t reserve(Scratch &c_, int64_t nq, int64_t nr, int64_t ntab, int npairs, bool band, bool packed) {
    Scratch *c = &c_;
    cudaError_t e;
    if (band && (e = grow(c->band, BandLayout(nq, nr, packed).total)) != cudaSuccess) return e;
    if ((e = grow(c->pairs, 2 * sizeof(PairDesc) * (size_t)std::max(npairs, 1) + 512)) != cudaSuccess) return e;
    if ((e = grow(c->geom, 2 * sizeof(PairGeom) * (size_t)std::max(npairs, 1) + 512)) != cudaSuccess) return e;
    if ((e = grow(c->offs, 2 * sizeof(int64_t) * offs_entries(npairs, nq) + 512)) != cudaSuccess) return e;
    if ((e = grow(c->keys, sizeof(uint32_t) * 6 * (size_t)std::max<int64_t>(nr, 1))) != cudaSuccess) return e;
    // 32 records of padding: bulk copies of a 32-row box may run past the last row
    if ((e = grow(c->rec, sizeof(float4) * (size_t)(nr + 32))) != cudaSuccess) return e;
    if ((e = grow(c->rtmp, sizeof(float4) * (size_t)std::max<int64_t>(nr, 1))) != cudaSuccess) return e;
    if ((e = grow(c->tab, sizeof(uint32_t) * (size_t)std::max<int64_t>(ntab, 1))) != cudaSuccess) return e;
    if ((e = grow(c->curs, sizeof(uint32_t) * (size_t)std::max<int64_t>(ntab, 1))) != cudaSuccess) return e;
    if ((e = grow(c->qrec, sizeof(QueryRec) * (size_t)std::max<int64_t>(nq, 1))) != cudaSuccess) return e;
    if ((e = grow(c->qcount, sizeof(int64_t) * (size_t)(nq + 1))) != cudaSuccess) return e;
    if ((e = grow(c->scan, sizeof(int64_t) * (size_t)(nq / 8192 + 2))) != cudaSuccess) return e;
    if ((e = grow(c->longlist, sizeof(uint32_t) * (size_t)(nq + 1))) != cudaSuccess) return e;
    if ((e = grow(c->blkpair, sizeof(int32_t) * (size_t)(nq / kStabQB + 2))) != cudaSuccess) return e;
    if ((e = grow(c->small, 256)) != cudaSuccess) return e;
    if ((e = grow(c->counters, 8 * sizeof(unsigned long long))) != cudaSuccess) return e;
    return cudaSuccess;
}

// Half `parity` of a double-buffered scratch buffer (halves of half its
// capacity, 256-byte aligned: the same split for every call while the buffer
// does not grow).
template <class T>
T *half_of(DevBuf &b, int parity) {
    return reinterpret_cast<T *>(static_cast<char *>(b.ptr) + (parity ? (b.bytes / 2) & ~(size_t)255 : 0));
}

Launch make_launch(Scratch &sc, bool counters_on, const egm_params &prm, const Plan &pl, int npairs,
                   const egm_out *out, bool band = false) {
    Scratch *c = &sc;
    Launch L;
    memset(&L, 0, sizeof(L));
    L.pairs = half_of<PairDesc>(c->pairs, c->parity);
    L.geom = half_of<PairGeom>(c->geom, c->parity);
    L.npairs = npairs;
    L.nq = pl.nq;
    L.nr = pl.nr;
    int64_t *offs = half_of<int64_t>(c->offs, c->parity);
    L.q_offs = offs;
    L.r_offs = offs + (npairs + 1);
    uint32_t *k = as<uint32_t>(c->keys);
    const size_t nr = (size_t)std::max<int64_t>(pl.nr, 1);
    L.key_a = k;
    L.val_a = k + nr;
    L.key_b = k + 2 * nr;
    L.val_b = k + 3 * nr;
    L.key_c = k + 4 * nr;
    L.val_c = k + 5 * nr;
    L.rec = as<float4>(c->rec);
    L.rtmp = as<float4>(c->rtmp);
    L.tab = as<uint32_t>(c->tab);
    L.ntab = pl.ntab;
    L.curs = as<uint32_t>(c->curs);
    L.prep_done = as<uint32_t>(c->small) + 40;
    L.qrec = as<QueryRec>(c->qrec);
    L.status = as<uint32_t>(c->small);
    L.counters = counters_on ? as<unsigned long long>(c->counters) : nullptr;
    L.qcount = as<int64_t>(c->qcount);
    L.scan_tmp = as<int64_t>(c->scan);
    L.blkpair = as<int32_t>(c->blkpair);
    L.ratio_num = prm.ratio_num;
    L.ratio_den = prm.ratio_den;
    if (npairs == 1) {
        L.inl_use = 1;
        L.inl = pl.pd[0];
    }
    L.max_n = pl.max_n;
    if (band) {
        const BandLayout bl(pl.nq, pl.nr, pl.has_float);
        unsigned char *b = static_cast<unsigned char *>(c->band.ptr);
        L.qperm = reinterpret_cast<uint32_t *>(b + bl.qperm);
        L.descA = b + bl.descA;
        L.descB = b + bl.descB;
        L.qbkt = reinterpret_cast<uint16_t *>(b + bl.qbkt);
        L.qsrt = reinterpret_cast<QueryRec *>(b + bl.qsrt);
        L.rnorm = reinterpret_cast<float4 *>(b + bl.rnorm);
        L.qscale = reinterpret_cast<float *>(b + bl.qscale);
        L.fp8 = prm.float_pass == EGM_FLOAT_PASS_FP8;
        L.probe = prm.timeout_check;
        L.tile_offs = offs + 2 * (npairs + 1);
        L.tile_seq = reinterpret_cast<const int2 *>(offs + 3 * (npairs + 1));
        L.work = as<uint32_t>(c->small) + 32;
        L.ntiles = pl.ntiles;
    }
    L.kind = pl.pd.empty() ? -1 : pl.pd[0].kind;
    for (const PairDesc &d : pl.pd) {
        if (d.kind != L.kind) L.kind = -1;
        if (d.row_bytes > 0) L.kinds |= 1u << d.kind;
    }
    if (out) {
        L.best = out->best;
        L.second = out->second;
        L.best_d = out->best_d;
        L.second_d = out->second_d;
        L.flags = out->flags;
        L.cand_offsets = out->cand_offsets;
        L.cand_idx = out->cand_idx;
        L.cand_capacity = out->cand_capacity;
        L.cand_total = out->cand_total;
    }
    return L;
}

// Upload the pair table and offsets through a pinned staging slot.  The
// device copy is ordered on the stream after the previous call's kernels; the
// host reuses a slot only once its previous upload has been consumed.
cudaError_t upload_plan(egm_ctx *c, const Plan &pl, int npairs) {
    const size_t tb = sizeof(PairDesc) * npairs, ob = sizeof(int64_t) * pl.offs.size();
    const int k = c->slot;
    c->slot = (k + 1) % egm_ctx::kSlots;
    cudaError_t e;
    if (!c->slot_ev[k] && (e = cudaEventCreateWithFlags(&c->slot_ev[k], cudaEventDisableTiming)) != cudaSuccess)
        return e;
    if (c->slot_pending[k]) {
        if ((e = cudaEventSynchronize(c->slot_ev[k])) != cudaSuccess) return e;
        c->slot_pending[k] = false;
    }
    if (tb + ob > c->h_table_bytes[k]) {
        if (c->h_table[k]) cudaFreeHost(c->h_table[k]);
        c->h_table[k] = nullptr;
        const size_t want = (tb + ob) * 2 + 4096;
        if ((e = cudaMallocHost(&c->h_table[k], want)) != cudaSuccess) {
            c->h_table_bytes[k] = 0;
            return e;
        }
        c->h_table_bytes[k] = want;
    }
    unsigned char *h = static_cast<unsigned char *>(c->h_table[k]);
    memcpy(h, pl.pd.data(), tb);
    memcpy(h + tb, pl.offs.data(), ob);
    if ((e = cudaMemcpyAsync(half_of<PairDesc>(c->sc.pairs, c->sc.parity), h, tb, cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(half_of<int64_t>(c->sc.offs, c->sc.parity), h + tb, ob, cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
        return e;
    if ((e = cudaEventRecord(c->slot_ev[k], c->stream)) != cudaSuccess) return e;
    c->slot_pending[k] = true;
    return cudaSuccess;
}

// Records the boundary event before stage `k` (k == kStages: end of call).
cudaError_t mark(egm_ctx *c, size_t base, int k) {
    if (!c->timing_on) return cudaSuccess;
    const size_t idx = base + (size_t)k;
    while (c->ev_pool.size() <= idx) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        c->ev_pool.push_back(e);
    }
    return cudaEventRecord(c->ev_pool[idx], c->stream);
}

egm_status finish(egm_ctx *c, bool sync) {
    if (!sync) return EGM_OK;
    return egm_sync(c);
}

// The kernel sequence of one match call.  `tc` receives stage events when
// per-stage timing is on (NULL: no events, e.g. while capturing a graph).
// A second stream and its fork / join events (created on first use).
cudaError_t ensure_side(egm_ctx *c) {
    cudaError_t e = cudaSuccess;
    if (!c->side) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->fork_ev) e = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess && !c->join_ev) e = cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming);
    return e;
}

// `shape`: the band kernel's tile shape; negative stops before the band
// kernel (the tuner then runs it once per shape).
cudaError_t enqueue_pipeline(const Launch &L, Scratch &sc, bool csr, int max_n, cudaStream_t st, egm_ctx *tc,
                             bool band, int sms, egm_ctx *sidec, int shape) {
    size_t tb = 0;
    if (tc && tc->timing_on) {
        tb = tc->ev_used;
        tc->ev_calls.push_back(tb);
        tc->ev_band.push_back(band);
        tc->ev_used += kStages + 1;
    } else {
        tc = nullptr;
    }
    cudaError_t e;
#define EGM_Q(x)                           \
    do {                                   \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    if (tc) EGM_Q(mark(tc, tb, 0));
    EGM_Q(launch_geometry(L, st));
    if (tc) EGM_Q(mark(tc, tb, 1));
    if (band) {
        // the queries' preparation and order run beside the references'
        // preparation and sort (the band kernel reads no per-pair query
        // statistics)
        EGM_Q(cudaEventRecord(sidec->fork_ev, st));
        EGM_Q(cudaStreamWaitEvent(sidec->side, sidec->fork_ev, 0));
        EGM_Q(launch_prep(L, sidec->side, 2));
        EGM_Q(launch_query_sort(L, sidec->side));
        EGM_Q(cudaEventRecord(sidec->join_ev, sidec->side));
        EGM_Q(launch_prep(L, st, 1));
    } else {
        EGM_Q(launch_prep(L, st, 0));
    }
    if (tc) EGM_Q(mark(tc, tb, 2));
    EGM_Q(launch_sort(L, st));
    if (band) EGM_Q(cudaStreamWaitEvent(st, sidec->join_ev, 0));
    if (tc) EGM_Q(mark(tc, tb, 3));
    if (band) EGM_Q(launch_pack(L, st));  // float pairs only
    if (tc) EGM_Q(mark(tc, tb, 4));
    if (band) {
        if (shape >= 0) EGM_Q(launch_band(L, sms, shape, st, false));
        if (tc) EGM_Q(mark(tc, tb, 5));
    } else if (csr) {
        uint32_t *long_list = as<uint32_t>(sc.longlist);
        uint32_t *long_count = as<uint32_t>(sc.small) + 16;
        EGM_Q(launch_stab(L, 1, st));
        if (tc) EGM_Q(mark(tc, tb, 5));
        EGM_Q(launch_csr_offsets(L, long_count, st));
        EGM_Q(launch_stab(L, 2, st));
        EGM_Q(launch_csr_row_sort(L, long_list, long_count, st));
    } else {
        EGM_Q(launch_stab(L, 0, st));
        if (tc) EGM_Q(mark(tc, tb, 5));
    }
    if (tc) EGM_Q(mark(tc, tb, 6));
#undef EGM_Q
    return cudaSuccess;
}

int tile_class(int64_t ntiles) {
    int k = 0;
    while (ntiles > 1) {
        ntiles >>= 1;
        k++;
    }
    return k;
}

// A call's regime, what the fastest form and band tile shape depend on:
// the number of 128-query tiles (log2), one or several pairs, the
// descriptor kinds present, and the expected candidates per query (log2 of
// 1 + the estimate; 15 when some tolerance is per keypoint and therefore
// unknown on the host).
uint64_t regime_key(const Plan &pl, int npairs) {
    int dens = 15;
    if (!pl.eps_vec) {
        const double kb = pl.kbar_q / (double)std::max<int64_t>(pl.nq, 1);
        dens = 0;
        while (dens < 14 && (double)(2 << dens) <= kb + 1.0) dens++;
    }
    return (uint64_t)std::min(tile_class(pl.ntiles), 63) | ((uint64_t)(npairs == 1) << 6) |
           ((uint64_t)(pl.kinds & 7u) << 8) | ((uint64_t)dens << 12);
}

// Times the whole pipeline of the call in one configuration (form and band
// tile shape) on the call's own inputs and outputs: one warm-up run, then
// the median of three, each waited for, so that the runs do not overlap.
// Every configuration computes the same exact results.
cudaError_t time_config(egm_ctx *c, Scratch &sc, const Plan &pl, int npairs, const egm_out *out, bool band,
                        int shape, float &ms) {
    const Launch L = make_launch(sc, false, c->params, pl, npairs, out, band);
    cudaStream_t st = c->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float t[3] = {0.0f, 0.0f, 0.0f};
    for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = enqueue_pipeline(L, sc, false, pl.max_n, st, nullptr, band, c->sms, c, shape);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float x = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
        if (rep > 0) t[rep - 1] = x;
    }
    std::sort(t, t + 3);
    ms = t[1];
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

// The configuration of a call.  Forced choices (plain form, candidate lists,
// a forced shape) need no timing; with params.tune == 0 the heuristic of
// choose_band picks the form, and the shape is (4 boxes, 2 CTAs per SM) up
// to two tiles per SM, else (1 box, 4 CTAs); otherwise the regime's entry
// in the tuner's cache decides, and `tune` asks the caller to time the
// candidates first (the regime has none yet).
egm_status choose_config(const egm_ctx *c, const Plan &pl, int npairs, bool csr, bool &band, int &shape,
                         bool &tune) {
    const egm_params &prm = c->params;
    band = false;
    shape = 0;
    tune = false;
    const bool can_band = pl.band_ok && !csr;
    if (prm.form == EGM_FORM_BANDED && !can_band) return EGM_ERR_UNIMPLEMENTED;
    if (!can_band || prm.form == EGM_FORM_PLAIN) return EGM_OK;
    const int forced = pl.has_float ? 0 : prm.band_tile > 0 ? prm.band_tile - 1 : -1;
    if (!prm.tune) {
        egm_status s = choose_band(pl, prm, csr, c->sms, band);
        if (s != EGM_OK) return s;
        shape = forced >= 0 ? forced : pl.ntiles <= 2 * (int64_t)c->sms ? 0 : 2;
        return EGM_OK;
    }
    const auto it = c->tuned.find(regime_key(pl, npairs));
    if (it == c->tuned.end()) {
        tune = true;
        return EGM_OK;
    }
    band = prm.form == EGM_FORM_BANDED || it->second.form == EGM_FORM_BANDED;
    shape = forced >= 0 ? forced : it->second.shape;
    return EGM_OK;
}

// Times every candidate configuration of the call (the plain form and each
// band tile shape) and records the regime's fastest; band, shape receive
// the configuration the call then runs (a forced form or shape is kept).
egm_status tune_regime(egm_ctx *c, Scratch &sc, const Plan &pl, int npairs, const egm_out *out, bool &band,
                       int &shape) {
    TuneEntry t;
    EGM_TRY(time_config(c, sc, pl, npairs, out, false, 0, t.ms_plain));
    t.ms_band = INFINITY;
    t.shape = 0;
    const int nshape = pl.has_float ? 1 : band_shapes();
    for (int k = 0; k < nshape; k++) {
        float ms = 0.0f;
        EGM_TRY(time_config(c, sc, pl, npairs, out, true, k, ms));
        if (ms < t.ms_band) {
            t.ms_band = ms;
            t.shape = k;
        }
    }
    t.form = t.ms_band < t.ms_plain ? EGM_FORM_BANDED : EGM_FORM_PLAIN;
    c->tuned[regime_key(pl, npairs)] = t;
    const egm_params &prm = c->params;
    band = prm.form == EGM_FORM_BANDED || t.form == EGM_FORM_BANDED;
    shape = pl.has_float ? 0 : prm.band_tile > 0 ? prm.band_tile - 1 : t.shape;
    return EGM_OK;
}

egm_status check_out(const egm_pair *pairs, int npairs, const egm_out *out) {
    const bool csr = out->cand_offsets != nullptr;
    if (csr && (!out->cand_total || out->cand_capacity < 0 || (out->cand_capacity > 0 && !out->cand_idx)))
        return EGM_ERR_ARG;
    bool any_desc = false;
    for (int p = 0; p < npairs; p++) any_desc |= has_desc(pairs + p);
    if (!csr && !any_desc) return EGM_ERR_ARG;  // nothing to compute
    return EGM_OK;
}

egm_status run_batch(egm_ctx *c, const egm_pair *pairs, int npairs, const egm_out *out, bool sync) {
    if (!c || npairs < 0 || (npairs > 0 && !pairs) || !out) return EGM_ERR_ARG;
    if (npairs == 0) return EGM_OK;
    Plan pl;
    egm_status s = make_plan(pairs, npairs, pl);
    if (s != EGM_OK) return s;
    if ((s = check_out(pairs, npairs, out)) != EGM_OK) return s;
    const bool csr = out->cand_offsets != nullptr;
    bool band = false, tune = false;
    int shape = 0;
    if ((s = choose_config(c, pl, npairs, csr, band, shape, tune)) != EGM_OK) return s;
    EGM_TRY(cudaSetDevice(c->device));
    if (band || tune) EGM_TRY(ensure_side(c));
    EGM_TRY(reserve(c->sc, pl.nq, pl.nr, pl.ntab, npairs, band || tune, pl.has_float));
    c->sc.parity ^= 1;
    if (npairs > 1) EGM_TRY(upload_plan(c, pl, npairs));  // one pair: the plan rides in the launch
    cudaStream_t st = c->stream;
    if (sync) EGM_TRY(cudaMemsetAsync(as<uint32_t>(c->sc.small), 0, sizeof(uint32_t), st));
    // a regime met for the first time: every configuration is timed on this call's data
    if (tune && (s = tune_regime(c, c->sc, pl, npairs, out, band, shape)) != EGM_OK) return s;
    Launch L = make_launch(c->sc, c->counters_on, c->params, pl, npairs, out, band);
    if (c->counters_on) EGM_TRY(cudaMemsetAsync(c->sc.counters.ptr, 0, 8 * sizeof(unsigned long long), st));
    EGM_TRY(enqueue_pipeline(L, c->sc, csr, pl.max_n, st, c, band, c->sms, c, shape));
    c->last.queries = pl.nq;
    c->last.refs = pl.nr;
    return finish(c, sync);
}

}  // namespace

extern "C" {

void egm_default_params(egm_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->ratio_num = 4;
    p->ratio_den = 5;
    p->sync = 1;
    p->form = EGM_FORM_AUTO;
    p->tune = 1;
}

egm_status egm_create(egm_ctx **out, int device, void *stream) {
    if (!out) return EGM_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return EGM_ERR_CUDA;
    egm_ctx *c = new (std::nothrow) egm_ctx();
    if (!c) return EGM_ERR_NOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    egm_default_params(&c->params);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_status, 64);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_counters, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = grow(c->sc.small, 256);
    if (e == cudaSuccess) e = cudaMemset(c->sc.small.ptr, 0, 256);
    if (e != cudaSuccess) {
        egm_destroy(c);
        return from_cuda(e);
    }
    *out = c;
    return EGM_OK;
}

egm_status egm_destroy(egm_ctx *c) {
    if (!c) return EGM_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->copy) {
        cudaStreamSynchronize(c->copy);
        cudaStreamDestroy(c->copy);
    }
    if (c->copy_out) {
        cudaStreamSynchronize(c->copy_out);
        cudaStreamDestroy(c->copy_out);
    }
    if (c->copy_start) cudaEventDestroy(c->copy_start);
    if (c->out_done) cudaEventDestroy(c->out_done);
    for (cudaEvent_t e : c->in_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->done_ev) cudaEventDestroy(e);
    c->sc.release();
    if (c->stage.ptr) cudaFree(c->stage.ptr);
    if (c->compact.ptr) cudaFree(c->compact.ptr);
    if (c->ft.ptr) cudaFree(c->ft.ptr);
    if (c->gms.ptr) cudaFree(c->gms.ptr);
    if (c->gms_host) cudaFreeHost(c->gms_host);
    if (c->gms_host_ev) cudaEventDestroy(c->gms_host_ev);
    for (int k = 0; k < egm_ctx::kSlots; k++) {
        if (c->h_table[k]) cudaFreeHost(c->h_table[k]);
        if (c->slot_ev[k]) cudaEventDestroy(c->slot_ev[k]);
    }
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_counters) cudaFreeHost(c->h_counters);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
    return EGM_OK;
}

egm_status egm_set_stream(egm_ctx *c, void *stream) {
    if (!c) return EGM_ERR_ARG;
    c->stream = static_cast<cudaStream_t>(stream);
    return EGM_OK;
}

egm_status egm_set_params(egm_ctx *c, const egm_params *p) {
    if (!c || !p) return EGM_ERR_ARG;
    if (p->ratio_num <= 0 || p->ratio_den <= 0 || p->ratio_num > 1000000 || p->ratio_den > 1000000)
        return EGM_ERR_ARG;
    if (p->form < EGM_FORM_AUTO || p->form > EGM_FORM_BANDED) return EGM_ERR_ARG;
    if (p->band_tile < 0 || p->band_tile > band_shapes()) return EGM_ERR_ARG;
    if (p->float_pass != EGM_FLOAT_PASS_BF16 && p->float_pass != EGM_FLOAT_PASS_FP8) return EGM_ERR_ARG;
    if (p->timeout_check != 0 && p->timeout_check != 1) return EGM_ERR_ARG;
    if (p->tune != 0 && p->tune != 1) return EGM_ERR_ARG;
    c->params = *p;
    return EGM_OK;
}

egm_status egm_get_params(egm_ctx *c, egm_params *p) {
    if (!c || !p) return EGM_ERR_ARG;
    *p = c->params;
    return EGM_OK;
}

egm_status egm_reserve(egm_ctx *c, int64_t queries, int64_t refs, int32_t pairs) {
    if (!c || queries < 0 || refs < 0 || pairs < 0) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(c->device));
    const int64_t ntab = 4 * refs + (int64_t)std::max(pairs, 1) * (2 * kLevels + 32);
    EGM_TRY(reserve(c->sc, queries, refs, ntab, std::max(pairs, 1), true, true));
    return EGM_OK;
}

egm_status egm_tuner_export(egm_ctx *c, void *buf, int64_t capacity, int64_t *size) {
    if (!c || !size || capacity < 0) return EGM_ERR_ARG;
    const int64_t need = 16 + 24 * (int64_t)c->tuned.size();
    *size = need;
    if (!buf) return EGM_OK;
    if (capacity < need) return EGM_ERR_CAPACITY;
    unsigned char *o = static_cast<unsigned char *>(buf);
    const uint32_t head[4] = {0x544d4745u /* "EGMT" */, 1u, (uint32_t)c->tuned.size(), (uint32_t)c->sms};
    memcpy(o, head, 16);
    o += 16;
    for (const auto &kv : c->tuned) {
        const uint64_t key = kv.first;
        const int32_t fs[2] = {kv.second.form, kv.second.shape};
        const float ms[2] = {kv.second.ms_plain, kv.second.ms_band};
        memcpy(o, &key, 8);
        memcpy(o + 8, fs, 8);
        memcpy(o + 16, ms, 8);
        o += 24;
    }
    return EGM_OK;
}

egm_status egm_tuner_import(egm_ctx *c, const void *buf, int64_t size) {
    if (!c || !buf || size < 16) return EGM_ERR_ARG;
    const unsigned char *in = static_cast<const unsigned char *>(buf);
    uint32_t head[4];
    memcpy(head, in, 16);
    if (head[0] != 0x544d4745u || head[1] != 1u || size != 16 + 24 * (int64_t)head[2]) return EGM_ERR_ARG;
    std::map<uint64_t, TuneEntry> t;
    for (uint32_t k = 0; k < head[2]; k++) {
        const unsigned char *e = in + 16 + 24 * (size_t)k;
        uint64_t key;
        int32_t fs[2];
        float ms[2];
        memcpy(&key, e, 8);
        memcpy(fs, e + 8, 8);
        memcpy(ms, e + 16, 8);
        if ((fs[0] != EGM_FORM_PLAIN && fs[0] != EGM_FORM_BANDED) || fs[1] < 0 || fs[1] >= band_shapes())
            return EGM_ERR_ARG;
        TuneEntry x;
        x.form = fs[0];
        x.shape = fs[1];
        x.ms_plain = ms[0];
        x.ms_band = ms[1];
        t[key] = x;
    }
    c->tuned.swap(t);
    return EGM_OK;
}

egm_status egm_sync(egm_ctx *c) {
    if (!c) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(c->device));
    EGM_TRY(cudaMemcpyAsync(c->h_status, c->sc.small.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    if (c->counters_on)
        EGM_TRY(cudaMemcpyAsync(c->h_counters, c->sc.counters.ptr, 8 * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, c->stream));
    EGM_TRY(cudaStreamSynchronize(c->stream));
    const uint32_t st = *c->h_status;
    if (st) EGM_TRY(cudaMemsetAsync(c->sc.small.ptr, 0, sizeof(uint32_t), c->stream));
    if (c->counters_on) {
        c->last.window_refs = (int64_t)c->h_counters[2];
        c->last.candidates = (int64_t)c->h_counters[3];
        c->last.fp64_rechecks = (int64_t)c->h_counters[4];
    }
    return from_bits(st);
}

egm_status egm_match_batch(egm_ctx *c, const egm_pair *pairs, int32_t npairs, const egm_out *out) {
    if (!c) return EGM_ERR_ARG;
    return run_batch(c, pairs, npairs, out, c->params.sync != 0);
}

egm_status egm_match_pair(egm_ctx *c, const egm_pair *pair, const egm_out *out) {
    if (!c) return EGM_ERR_ARG;
    return run_batch(c, pair, 1, out, c->params.sync != 0);
}

egm_status egm_match_pair_host(egm_ctx *c, const egm_pair *hp, const egm_out *ho) {
    if (!c || !hp || !ho) return EGM_ERR_ARG;
    egm_status s = check_pair(hp);
    if (s != EGM_OK) return s;
    const int64_t m = hp->m, n = hp->n;
    const int rb = has_desc(hp) ? row_bytes_of(hp->kind, hp->dim) : 0;
    const bool csr = ho->cand_offsets != nullptr;
    if (csr && (!ho->cand_total || ho->cand_capacity < 0 || (ho->cand_capacity > 0 && !ho->cand_idx)))
        return EGM_ERR_ARG;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    const size_t o_xy1 = off; off += al(16 * m);
    const size_t o_xy2 = off; off += al(16 * n);
    const size_t o_F = off; off += al(72);
    const size_t o_eps = off; off += al(hp->eps2 ? 8 * n : 0);
    const size_t o_d1 = off; off += al((size_t)rb * m);
    const size_t o_d2 = off; off += al((size_t)rb * n);
    const size_t o_best = off; off += al(4 * m);
    const size_t o_second = off; off += al(4 * m);
    const size_t o_bd = off; off += al(4 * m);
    const size_t o_sd = off; off += al(4 * m);
    const size_t o_fl = off; off += al(m);
    const size_t o_co = off; off += al(csr ? 8 * (m + 1) : 0);
    const size_t o_ct = off; off += al(csr ? 8 : 0);
    const size_t o_ci = off; off += al(csr ? 4 * (size_t)ho->cand_capacity : 0);
    EGM_TRY(cudaSetDevice(c->device));
    EGM_TRY(grow(c->stage, off));
    unsigned char *d = static_cast<unsigned char *>(c->stage.ptr);
    cudaStream_t st = c->stream;
    const cudaMemcpyKind H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
    if (m) EGM_TRY(cudaMemcpyAsync(d + o_xy1, hp->xy1, 16 * m, H2D, st));
    if (n) EGM_TRY(cudaMemcpyAsync(d + o_xy2, hp->xy2, 16 * n, H2D, st));
    EGM_TRY(cudaMemcpyAsync(d + o_F, hp->F, 72, H2D, st));
    if (hp->eps2 && n) EGM_TRY(cudaMemcpyAsync(d + o_eps, hp->eps2, 8 * n, H2D, st));
    if (rb && m) EGM_TRY(cudaMemcpyAsync(d + o_d1, hp->desc1, (size_t)rb * m, H2D, st));
    if (rb && n) EGM_TRY(cudaMemcpyAsync(d + o_d2, hp->desc2, (size_t)rb * n, H2D, st));
    egm_pair dp = *hp;
    dp.xy1 = reinterpret_cast<const double *>(d + o_xy1);
    dp.xy2 = reinterpret_cast<const double *>(d + o_xy2);
    dp.F = reinterpret_cast<const double *>(d + o_F);
    dp.eps2 = hp->eps2 ? reinterpret_cast<const double *>(d + o_eps) : nullptr;
    dp.desc1 = rb ? d + o_d1 : nullptr;
    dp.desc2 = rb ? d + o_d2 : nullptr;
    egm_out dout;
    memset(&dout, 0, sizeof(dout));
    dout.best = ho->best ? reinterpret_cast<int32_t *>(d + o_best) : nullptr;
    dout.second = ho->second ? reinterpret_cast<int32_t *>(d + o_second) : nullptr;
    dout.best_d = ho->best_d ? reinterpret_cast<float *>(d + o_bd) : nullptr;
    dout.second_d = ho->second_d ? reinterpret_cast<float *>(d + o_sd) : nullptr;
    dout.flags = ho->flags ? d + o_fl : nullptr;
    if (csr) {
        dout.cand_offsets = reinterpret_cast<int64_t *>(d + o_co);
        dout.cand_total = reinterpret_cast<int64_t *>(d + o_ct);
        dout.cand_idx = reinterpret_cast<int32_t *>(d + o_ci);
        dout.cand_capacity = ho->cand_capacity;
    }
    EGM_TRY(cudaMemsetAsync(c->sc.small.ptr, 0, sizeof(uint32_t), st));
    s = run_batch(c, &dp, 1, &dout, false);
    if (s != EGM_OK) return s;
    if (ho->best) EGM_TRY(cudaMemcpyAsync(ho->best, dout.best, 4 * m, D2H, st));
    if (ho->second) EGM_TRY(cudaMemcpyAsync(ho->second, dout.second, 4 * m, D2H, st));
    if (ho->best_d) EGM_TRY(cudaMemcpyAsync(ho->best_d, dout.best_d, 4 * m, D2H, st));
    if (ho->second_d) EGM_TRY(cudaMemcpyAsync(ho->second_d, dout.second_d, 4 * m, D2H, st));
    if (ho->flags) EGM_TRY(cudaMemcpyAsync(ho->flags, dout.flags, m, D2H, st));
    if (csr) {
        EGM_TRY(cudaMemcpyAsync(ho->cand_offsets, dout.cand_offsets, 8 * (m + 1), D2H, st));
        EGM_TRY(cudaMemcpyAsync(ho->cand_total, dout.cand_total, 8, D2H, st));
    }
    s = egm_sync(c);
    if (s != EGM_OK) return s;
    if (csr) {
        const int64_t tot = *ho->cand_total;
        if (tot > 0 && tot <= ho->cand_capacity) {
            EGM_TRY(cudaMemcpyAsync(ho->cand_idx, dout.cand_idx, 4 * (size_t)tot, D2H, st));
            EGM_TRY(cudaStreamSynchronize(st));
        }
    }
    return EGM_OK;
}

egm_status egm_match_batch_host(egm_ctx *c, const egm_pair *hp, int32_t npairs, const egm_out *ho) {
    if (!c || npairs < 0 || (npairs > 0 && (!hp || !ho))) return EGM_ERR_ARG;
    if (npairs == 0) return EGM_OK;
    struct Off {
        size_t xy1, xy2, F, eps, d1, d2, best, second, bd, sd, fl;
    };
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    std::vector<Off> offs((size_t)npairs);
    size_t off = 0;
    for (int k = 0; k < npairs; k++) {
        egm_status s = check_pair(hp + k);
        if (s != EGM_OK) return s;
        if (ho[k].cand_offsets || !has_desc(hp + k)) return EGM_ERR_ARG;
        const int64_t m = hp[k].m, n = hp[k].n;
        const size_t rb = (size_t)row_bytes_of(hp[k].kind, hp[k].dim);
        Off &o = offs[(size_t)k];
        o.xy1 = off; off += al(16 * (size_t)m);
        o.xy2 = off; off += al(16 * (size_t)n);
        o.F = off; off += al(72);
        o.eps = off; off += al(hp[k].eps2 ? 8 * (size_t)n : 0);
        o.d1 = off; off += al(rb * (size_t)m);
        o.d2 = off; off += al(rb * (size_t)n);
        o.best = off; off += al(4 * (size_t)m);
        o.second = off; off += al(4 * (size_t)m);
        o.bd = off; off += al(4 * (size_t)m);
        o.sd = off; off += al(4 * (size_t)m);
        o.fl = off; off += al((size_t)m);
    }
    EGM_TRY(cudaSetDevice(c->device));
    EGM_TRY(grow(c->stage, off));
    if (!c->copy) EGM_TRY(cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking));
    if (!c->copy_out) EGM_TRY(cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking));
    if (!c->copy_start) EGM_TRY(cudaEventCreateWithFlags(&c->copy_start, cudaEventDisableTiming));
    if (!c->out_done) EGM_TRY(cudaEventCreateWithFlags(&c->out_done, cudaEventDisableTiming));
    while ((int)c->in_ev.size() < npairs) {
        cudaEvent_t e, f;
        EGM_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->in_ev.push_back(e);
        EGM_TRY(cudaEventCreateWithFlags(&f, cudaEventDisableTiming));
        c->done_ev.push_back(f);
    }
    unsigned char *d = static_cast<unsigned char *>(c->stage.ptr);
    cudaStream_t st = c->stream, cs = c->copy, co = c->copy_out;
    const cudaMemcpyKind H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
    // the copies start once the context's stream is done with the staging buffer
    EGM_TRY(cudaEventRecord(c->copy_start, st));
    EGM_TRY(cudaStreamWaitEvent(cs, c->copy_start, 0));
    EGM_TRY(cudaMemsetAsync(c->sc.small.ptr, 0, sizeof(uint32_t), st));
    // on a failure after copies were queued, wait for them: they read the caller's buffers
    auto fail = [&](egm_status s) {
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(st);
        cudaStreamSynchronize(co);
        return s;
    };
    for (int k = 0; k < npairs; k++) {
        const egm_pair &P = hp[k];
        const Off &o = offs[(size_t)k];
        const size_t rb = (size_t)row_bytes_of(P.kind, P.dim);
        cudaError_t e = cudaSuccess;
        if (P.m) e = cudaMemcpyAsync(d + o.xy1, P.xy1, 16 * (size_t)P.m, H2D, cs);
        if (e == cudaSuccess && P.n) e = cudaMemcpyAsync(d + o.xy2, P.xy2, 16 * (size_t)P.n, H2D, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d + o.F, P.F, 72, H2D, cs);
        if (e == cudaSuccess && P.eps2 && P.n) e = cudaMemcpyAsync(d + o.eps, P.eps2, 8 * (size_t)P.n, H2D, cs);
        if (e == cudaSuccess && P.m) e = cudaMemcpyAsync(d + o.d1, P.desc1, rb * (size_t)P.m, H2D, cs);
        if (e == cudaSuccess && P.n) e = cudaMemcpyAsync(d + o.d2, P.desc2, rb * (size_t)P.n, H2D, cs);
        if (e == cudaSuccess) e = cudaEventRecord(c->in_ev[(size_t)k], cs);
        if (e != cudaSuccess) return fail(from_cuda(e));
    }
    int covered = -1;  // the inputs of pairs 0 .. covered are on the device for the matching stream
    for (int k = 0; k < npairs; k++) {
        const egm_pair &P = hp[k];
        const egm_out &O = ho[k];
        const Off &o = offs[(size_t)k];
        const size_t m = (size_t)P.m;
        egm_pair dp = P;
        dp.xy1 = reinterpret_cast<const double *>(d + o.xy1);
        dp.xy2 = reinterpret_cast<const double *>(d + o.xy2);
        dp.F = reinterpret_cast<const double *>(d + o.F);
        dp.eps2 = P.eps2 ? reinterpret_cast<const double *>(d + o.eps) : nullptr;
        dp.desc1 = d + o.d1;
        dp.desc2 = d + o.d2;
        egm_out dout;
        memset(&dout, 0, sizeof(dout));
        dout.best = O.best ? reinterpret_cast<int32_t *>(d + o.best) : nullptr;
        dout.second = O.second ? reinterpret_cast<int32_t *>(d + o.second) : nullptr;
        dout.best_d = O.best_d ? reinterpret_cast<float *>(d + o.bd) : nullptr;
        dout.second_d = O.second_d ? reinterpret_cast<float *>(d + o.sd) : nullptr;
        dout.flags = O.flags ? d + o.fl : nullptr;
        // The matching of pair k needs pair k's inputs.  The copy stream runs
        // in order, so the event of a later pair covers every earlier one:
        // waiting at pairs 0, 1, 2, 4, 7, ... for the inputs of pairs up to
        // about 1.5 k keeps most consecutive pairs' kernels chained (an event
        // wait ends a chain of dependent launches) while the uploads, faster
        // than the matching, stay ahead.
        cudaError_t e = cudaSuccess;
        if (k > covered) {
            covered = std::min(npairs - 1, k + k / 2);
            e = cudaStreamWaitEvent(st, c->in_ev[(size_t)covered], 0);
        }
        if (e != cudaSuccess) return fail(from_cuda(e));
        egm_status s = run_batch(c, &dp, 1, &dout, false);
        if (s != EGM_OK) return fail(s);
        // the outputs go back on the output stream, off the matching's path
        e = cudaEventRecord(c->done_ev[(size_t)k], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(co, c->done_ev[(size_t)k], 0);
        if (e == cudaSuccess && O.best) e = cudaMemcpyAsync(O.best, dout.best, 4 * m, D2H, co);
        if (e == cudaSuccess && O.second) e = cudaMemcpyAsync(O.second, dout.second, 4 * m, D2H, co);
        if (e == cudaSuccess && O.best_d) e = cudaMemcpyAsync(O.best_d, dout.best_d, 4 * m, D2H, co);
        if (e == cudaSuccess && O.second_d) e = cudaMemcpyAsync(O.second_d, dout.second_d, 4 * m, D2H, co);
        if (e == cudaSuccess && O.flags) e = cudaMemcpyAsync(O.flags, dout.flags, m, D2H, co);
        if (e != cudaSuccess) return fail(from_cuda(e));
    }
    // the context's stream waits for the last output copy, then the status
    cudaError_t e = cudaEventRecord(c->out_done, co);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->out_done, 0);
    if (e != cudaSuccess) return fail(from_cuda(e));
    return egm_sync(c);
}

egm_status egm_match_mutual(egm_ctx *c, const egm_pair *fwd, const egm_pair *rev, const egm_out *out) {
    if (!c || !fwd || !rev || !out || !out->best || !out->flags || out->cand_offsets) return EGM_ERR_ARG;
    if (rev->m != fwd->n || rev->n != fwd->m || rev->kind != fwd->kind || rev->dim != fwd->dim) return EGM_ERR_ARG;
    const egm_pair both[2] = {*fwd, *rev};
    EGM_TRY(cudaSetDevice(c->device));
    if (c->params.sync) EGM_TRY(cudaMemsetAsync(c->sc.small.ptr, 0, sizeof(uint32_t), c->stream));
    egm_status s = run_batch(c, both, 2, out, false);
    if (s != EGM_OK) return s;
    EGM_TRY(launch_mutual(out->best, out->flags, fwd->m, fwd->n, c->stream));
    return finish(c, c->params.sync != 0);
}

egm_status egm_match_mutual_pair(egm_ctx *c, const egm_pair *fwd, const double *eps1, double eps1_scalar,
                                 int32_t width1, int32_t height1, const egm_out *out) {
    if (!c || !fwd || !fwd->F || !out) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(c->device));
    EGM_TRY(grow(c->ft, 9 * sizeof(double)));
    // the reverse direction: image 2's keypoints query image 1's under F^T
    egm_pair rev = *fwd;
    rev.xy1 = fwd->xy2;
    rev.xy2 = fwd->xy1;
    rev.m = fwd->n;
    rev.n = fwd->m;
    rev.desc1 = fwd->desc2;
    rev.desc2 = fwd->desc1;
    rev.eps2 = eps1;
    rev.eps_scalar = eps1_scalar;
    rev.width = width1;
    rev.height = height1;
    rev.F = as<double>(c->ft);
    egm_status s = check_pair(&rev);
    if (s != EGM_OK) return s;
    EGM_TRY(launch_transpose3(fwd->F, as<double>(c->ft), c->stream));
    return egm_match_mutual(c, fwd, &rev, out);
}

egm_status egm_compact_matches(egm_ctx *c, const uint8_t *flags, const int32_t *best, int64_t m,
                               uint32_t require, int32_t *qi, int32_t *rj, int64_t *count) {
    if (!c || m < 0 || !count || (m > 0 && (!flags || !best || !qi || !rj))) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(c->device));
    EGM_TRY(grow(c->compact, sizeof(uint32_t) * (size_t)std::max<int64_t>(compact_tiles(m), 1)));
    EGM_TRY(launch_compact(flags, best, m, require, static_cast<uint32_t *>(c->compact.ptr), qi, rj, count,
                           c->stream));
    if (c->params.sync) EGM_TRY(cudaStreamSynchronize(c->stream));
    return EGM_OK;
}

namespace {

// GMS over a table of pairs: validation, upload of the table and row offsets
// (pinned staging, reused once its previous copy has finished), launch.
egm_status run_gms(egm_ctx *c, const egm_gms_pair *pairs, int32_t npairs, uint32_t require, int32_t grid,
                   double alpha) {
    if (!c || npairs < 0 || (npairs > 0 && !pairs) || grid < 1 || grid > 48 || !(alpha > 0.0) ||
        !(alpha < INFINITY))
        return EGM_ERR_ARG;
    std::vector<GmsPair> tab((size_t)npairs);
    std::vector<int64_t> offs((size_t)npairs + 1, 0);
    for (int k = 0; k < npairs; k++) {
        const egm_gms_pair &q = pairs[k];
        if (q.m < 0 || q.m > INT32_MAX || q.n < 0 || q.width1 <= 0 || q.height1 <= 0 || q.width2 <= 0 ||
            q.height2 <= 0)
            return EGM_ERR_ARG;
        if (q.m > 0 && (!q.xy1 || !q.best || !q.flags || (q.n > 0 && !q.xy2))) return EGM_ERR_ARG;
        tab[(size_t)k] = GmsPair{q.xy1, q.xy2, q.best, q.flags, q.m, q.n, offs[(size_t)k],
                                 (double)q.width1, (double)q.height1, (double)q.width2, (double)q.height2};
        offs[(size_t)k + 1] = offs[(size_t)k] + q.m;
    }
    const int64_t rows = offs[(size_t)npairs];
    if (rows > INT32_MAX) return EGM_ERR_ARG;
    if (rows == 0) return EGM_OK;
    EGM_TRY(cudaSetDevice(c->device));
    const GmsLayout l = gms_layout(npairs, rows, grid);
    EGM_TRY(grow(c->gms, l.total));
    const size_t tb = sizeof(GmsPair) * (size_t)npairs, ob = sizeof(int64_t) * offs.size();
    if (c->gms_host_ev) EGM_TRY(cudaEventSynchronize(c->gms_host_ev));  // the staging's previous copy
    else EGM_TRY(cudaEventCreateWithFlags(&c->gms_host_ev, cudaEventDisableTiming));
    if (tb + ob > c->gms_host_bytes) {
        if (c->gms_host) cudaFreeHost(c->gms_host);
        c->gms_host = nullptr;
        c->gms_host_bytes = 0;
        EGM_TRY(cudaMallocHost(&c->gms_host, 2 * (tb + ob) + 4096));
        c->gms_host_bytes = 2 * (tb + ob) + 4096;
    }
    unsigned char *h = static_cast<unsigned char *>(c->gms_host);
    memcpy(h, tab.data(), tb);
    memcpy(h + tb, offs.data(), ob);
    unsigned char *d = static_cast<unsigned char *>(c->gms.ptr);
    EGM_TRY(cudaMemcpyAsync(d + l.table, h, tb, cudaMemcpyHostToDevice, c->stream));
    EGM_TRY(cudaMemcpyAsync(d + l.offs, h + tb, ob, cudaMemcpyHostToDevice, c->stream));
    EGM_TRY(cudaEventRecord(c->gms_host_ev, c->stream));
    EGM_TRY(launch_gms(c->gms.ptr, l, npairs, rows, require, grid, alpha, c->stream));
    if (c->params.sync) EGM_TRY(cudaStreamSynchronize(c->stream));
    return EGM_OK;
}

}  // namespace

egm_status egm_gms(egm_ctx *c, const double *xy1, int64_t m, const double *xy2, int64_t n, const int32_t *best,
                   uint8_t *flags, int32_t width1, int32_t height1, int32_t width2, int32_t height2,
                   uint32_t require, int32_t grid, double alpha) {
    const egm_gms_pair q{xy1, xy2, best, flags, m, n, width1, height1, width2, height2};
    return run_gms(c, &q, 1, require, grid, alpha);
}

egm_status egm_gms_batch(egm_ctx *c, const egm_gms_pair *pairs, int32_t npairs, uint32_t require, int32_t grid,
                         double alpha) {
    return run_gms(c, pairs, npairs, require, grid, alpha);
}

egm_status egm_intervals(egm_ctx *c, const egm_pair *pair, double *theta, double *delta, double *e3,
                         int32_t *mode) {
    if (!c || !pair) return EGM_ERR_ARG;
    egm_pair p = *pair;
    p.desc1 = p.desc2 = nullptr;
    Plan pl;
    egm_status s = make_plan(&p, 1, pl);
    if (s != EGM_OK) return s;
    EGM_TRY(cudaSetDevice(c->device));
    EGM_TRY(reserve(c->sc, pl.nq, pl.nr, pl.ntab, 1, false, false));
    c->sc.parity ^= 1;
    EGM_TRY(upload_plan(c, pl, 1));
    Launch L = make_launch(c->sc, false, c->params, pl, 1, nullptr);
    if (c->params.sync) EGM_TRY(cudaMemsetAsync(L.status, 0, sizeof(uint32_t), c->stream));
    EGM_TRY(launch_geometry(L, c->stream));
    EGM_TRY(launch_intervals(L, theta, delta, e3, mode, c->stream));
    return finish(c, c->params.sync != 0);
}

}  // extern "C"

struct egm_graph {
    egm_ctx *ctx = nullptr;
    Scratch sc;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

egm_status egm_graph_create(egm_ctx *c, const egm_pair *pairs, int32_t npairs, const egm_out *out,
                            egm_graph **graph) {
    if (!c || !graph || !out || npairs <= 0 || !pairs) return EGM_ERR_ARG;
    *graph = nullptr;
    Plan pl;
    egm_status s = make_plan(pairs, npairs, pl);
    if (s != EGM_OK) return s;
    if ((s = check_out(pairs, npairs, out)) != EGM_OK) return s;
    const bool csr = out->cand_offsets != nullptr;
    bool band = false, tune = false;
    int shape = 0;
    if ((s = choose_config(c, pl, npairs, csr, band, shape, tune)) != EGM_OK) return s;
    EGM_TRY(cudaSetDevice(c->device));
    egm_graph *g = new (std::nothrow) egm_graph();
    if (!g) return EGM_ERR_NOMEM;
    g->ctx = c;
    cudaError_t e = band || tune ? ensure_side(c) : cudaSuccess;
    if (e == cudaSuccess) e = reserve(g->sc, pl.nq, pl.nr, pl.ntab, npairs, band || tune, pl.has_float);
    const size_t ob = sizeof(int64_t) * pl.offs.size();
    std::vector<unsigned char> h(sizeof(PairDesc) * npairs + ob);
    memcpy(h.data(), pl.pd.data(), sizeof(PairDesc) * npairs);
    memcpy(h.data() + sizeof(PairDesc) * npairs, pl.offs.data(), ob);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(g->sc.pairs.ptr, h.data(), sizeof(PairDesc) * npairs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->sc.offs.ptr, h.data() + sizeof(PairDesc) * npairs, ob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(g->sc.small.ptr, 0, 256);
    if (e == cudaSuccess && tune) {
        // tune on the graph's own scratch before capturing
        s = tune_regime(c, g->sc, pl, npairs, out, band, shape);
        if (s != EGM_OK) {
            cudaStreamSynchronize(c->stream);
            egm_graph_destroy(g);
            return s;
        }
    }
    cudaStream_t cs = nullptr;
    cudaGraph_t gr = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        const Launch L = make_launch(g->sc, false, c->params, pl, npairs, out, band);
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = cudaMemsetAsync(L.status, 0, sizeof(uint32_t), cs);
            if (e2 == cudaSuccess) e2 = enqueue_pipeline(L, g->sc, csr, pl.max_n, cs, nullptr, band, c->sms, c, shape);
            e = cudaStreamEndCapture(cs, &gr);
            if (e == cudaSuccess) e = e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        egm_graph_destroy(g);
        return from_cuda(e);
    }
    *graph = g;
    return EGM_OK;
}

egm_status egm_graph_launch(egm_graph *g) {
    if (!g || !g->exec) return EGM_ERR_ARG;
    egm_ctx *c = g->ctx;
    EGM_TRY(cudaSetDevice(c->device));
    EGM_TRY(cudaGraphLaunch(g->exec, c->stream));
    if (!c->params.sync) return EGM_OK;
    EGM_TRY(cudaMemcpyAsync(c->h_status, g->sc.small.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    EGM_TRY(cudaStreamSynchronize(c->stream));
    return from_bits(*c->h_status);
}

egm_status egm_graph_destroy(egm_graph *g) {
    if (!g) return EGM_OK;
    cudaSetDevice(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->sc.release();
    delete g;
    return EGM_OK;
}

}  // extern "C"

struct egm_mlp {
    egm_ctx *ctx = nullptr;
    DevBuf params, m, v, grad, pre, z, loss, err;
    int64_t step = 0;
    double fallback = 2.0;   // tolerance (px) of samples without a finite network output
};

namespace {
// Waits for the stream and reports (and clears) a tensor-core wait that gave
// up in a training forward pass since the last report.
egm_status take_training_error(egm_mlp *m) {
    cudaStream_t st = m->ctx->stream;
    uint32_t bits = 0;
    EGM_TRY(cudaMemcpyAsync(&bits, as<uint32_t>(m->err) + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    EGM_TRY(cudaStreamSynchronize(st));
    if (bits == 0) return EGM_OK;
    EGM_TRY(cudaMemsetAsync(as<uint32_t>(m->err) + 1, 0, sizeof(uint32_t), st));
    EGM_TRY(cudaStreamSynchronize(st));
    return from_bits(bits);
}
}  // namespace

extern "C" {

egm_status egm_mlp_create(egm_ctx *c, const float *params, egm_mlp **out) {
    if (!c || !params || !out) return EGM_ERR_ARG;
    *out = nullptr;
    if (mlp_param_count() != EGM_MLP_PARAMS) return EGM_ERR_UNIMPLEMENTED;
    EGM_TRY(cudaSetDevice(c->device));
    egm_mlp *m = new (std::nothrow) egm_mlp();
    if (!m) return EGM_ERR_NOMEM;
    m->ctx = c;
    const size_t pb = sizeof(float) * EGM_MLP_PARAMS;
    cudaError_t e = grow(m->params, pb);
    if (e == cudaSuccess) e = grow(m->m, pb);
    if (e == cudaSuccess) e = grow(m->v, pb);
    if (e == cudaSuccess) e = grow(m->grad, pb);
    if (e == cudaSuccess) e = grow(m->loss, 64);
    if (e == cudaSuccess) e = grow(m->err, 16);  // word 0: inference; word 1: training
    if (e == cudaSuccess) e = cudaMemset(m->err.ptr, 0, 16);
    if (e == cudaSuccess) e = cudaMemcpy(m->params.ptr, params, pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m.ptr, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(m->v.ptr, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(m->grad.ptr, 0, pb);
    if (e != cudaSuccess) {
        egm_mlp_destroy(m);
        return from_cuda(e);
    }
    *out = m;
    return EGM_OK;
}

egm_status egm_mlp_destroy(egm_mlp *m) {
    if (!m) return EGM_OK;
    cudaSetDevice(m->ctx->device);
    cudaStreamSynchronize(m->ctx->stream);
    DevBuf *b[] = {&m->params, &m->m, &m->v, &m->grad, &m->pre, &m->z, &m->loss, &m->err};
    for (DevBuf *x : b)
        if (x->ptr) cudaFree(x->ptr);
    delete m;
    return EGM_OK;
}

egm_status egm_mlp_get_state(egm_mlp *m, float *params, float *am, float *av, int64_t *step) {
    if (!m) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(m->ctx->device));
    EGM_TRY(cudaStreamSynchronize(m->ctx->stream));
    const size_t pb = sizeof(float) * EGM_MLP_PARAMS;
    if (params) EGM_TRY(cudaMemcpy(params, m->params.ptr, pb, cudaMemcpyDeviceToHost));
    if (am) EGM_TRY(cudaMemcpy(am, m->m.ptr, pb, cudaMemcpyDeviceToHost));
    if (av) EGM_TRY(cudaMemcpy(av, m->v.ptr, pb, cudaMemcpyDeviceToHost));
    if (step) *step = m->step;
    return take_training_error(m);
}

egm_status egm_mlp_set_state(egm_mlp *m, const float *params, const float *am, const float *av, int64_t step) {
    if (!m || step < 0) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(m->ctx->device));
    EGM_TRY(cudaStreamSynchronize(m->ctx->stream));
    const size_t pb = sizeof(float) * EGM_MLP_PARAMS;
    if (params) EGM_TRY(cudaMemcpy(m->params.ptr, params, pb, cudaMemcpyHostToDevice));
    if (am) EGM_TRY(cudaMemcpy(m->m.ptr, am, pb, cudaMemcpyHostToDevice));
    if (av) EGM_TRY(cudaMemcpy(m->v.ptr, av, pb, cudaMemcpyHostToDevice));
    m->step = step;
    return EGM_OK;
}

egm_status egm_mlp_set_fallback(egm_mlp *m, double eps_px) {
    if (!m || !(eps_px > 0.0) || !(eps_px < INFINITY)) return EGM_ERR_ARG;
    m->fallback = eps_px;
    return EGM_OK;
}

egm_status egm_mlp_infer(egm_mlp *m, const float *feat, int64_t n, double *eps) {
    if (!m || n < 0 || (n > 0 && (!feat || !eps))) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(m->ctx->device));
    if (n == 0) return EGM_OK;
    cudaStream_t st = m->ctx->stream;
    EGM_TRY(cudaMemsetAsync(m->err.ptr, 0, sizeof(uint32_t), st));
    EGM_TRY(launch_mlp_forward_tc(as<float>(m->params), feat, n, eps, as<uint32_t>(m->err), m->fallback,
                                  m->ctx->sms, st));
    uint32_t bits = 0;
    EGM_TRY(cudaMemcpyAsync(&bits, m->err.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    EGM_TRY(cudaStreamSynchronize(st));
    return from_bits(bits);
}

namespace {
egm_status mlp_backprop(egm_mlp *m, const float *feat, const float *resid, int64_t n, float q) {
    cudaStream_t st = m->ctx->stream;
    EGM_TRY(grow(m->pre, sizeof(float) * 3 * 64 * (size_t)n));
    EGM_TRY(grow(m->z, sizeof(float) * (size_t)n));
    EGM_TRY(cudaMemsetAsync(m->grad.ptr, 0, sizeof(float) * EGM_MLP_PARAMS, st));
    EGM_TRY(cudaMemsetAsync(m->loss.ptr, 0, sizeof(float), st));
    // the forward pass on the tensor cores; a timed-out wait is recorded in
    // the training word of the error flags (reported by egm_mlp_grad and
    // egm_mlp_get_state)
    EGM_TRY(launch_mlp_forward_tc(as<float>(m->params), feat, n, nullptr, as<uint32_t>(m->err) + 1, m->fallback,
                                  m->ctx->sms, st, as<float>(m->pre), as<float>(m->z)));
    EGM_TRY(launch_mlp_backward(as<float>(m->params), feat, resid, n, q, as<float>(m->pre), as<float>(m->z),
                                as<float>(m->grad), as<float>(m->loss), st));
    return EGM_OK;
}
}  // namespace

egm_status egm_mlp_grad(egm_mlp *m, const float *feat, const float *resid, int64_t n, float q, float *grad,
                        float *loss) {
    if (!m || n <= 0 || !feat || !resid || !(q > 0.0f && q < 1.0f)) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(m->ctx->device));
    egm_status s = mlp_backprop(m, feat, resid, n, q);
    if (s != EGM_OK) return s;
    cudaStream_t st = m->ctx->stream;
    if (grad) EGM_TRY(cudaMemcpyAsync(grad, m->grad.ptr, sizeof(float) * EGM_MLP_PARAMS, cudaMemcpyDeviceToDevice, st));
    if (loss) EGM_TRY(cudaMemcpyAsync(loss, m->loss.ptr, sizeof(float), cudaMemcpyDeviceToDevice, st));
    return take_training_error(m);
}

egm_status egm_mlp_train_step(egm_mlp *m, const float *feat, const float *resid, int64_t n, float lr, float q,
                              float *loss) {
    if (!m || n <= 0 || !feat || !resid || !(q > 0.0f && q < 1.0f) || !(lr > 0.0f)) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(m->ctx->device));
    egm_status s = mlp_backprop(m, feat, resid, n, q);
    if (s != EGM_OK) return s;
    cudaStream_t st = m->ctx->stream;
    if (loss) EGM_TRY(cudaMemcpyAsync(loss, m->loss.ptr, sizeof(float), cudaMemcpyDeviceToDevice, st));
    m->step += 1;
    EGM_TRY(launch_adam(as<float>(m->params), as<float>(m->grad), as<float>(m->m), as<float>(m->v), lr, m->step, st));
    return EGM_OK;
}

egm_status egm_pair_residuals(egm_ctx *c, const egm_pair *pair, const int32_t *qi, const int32_t *rj, int64_t k,
                              double *dist) {
    if (!c || !pair || k < 0 || (k > 0 && (!qi || !rj || !dist || !pair->xy1 || !pair->xy2 || !pair->F)))
        return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(c->device));
    EGM_TRY(launch_residuals(pair->xy1, pair->xy2, pair->F, pair->m, pair->n, qi, rj, k, dist, c->stream));
    if (c->params.sync) EGM_TRY(cudaStreamSynchronize(c->stream));
    return EGM_OK;
}

egm_status egm_set_timing(egm_ctx *c, int32_t enable) {
    if (!c) return EGM_ERR_ARG;
    c->timing_on = enable != 0;
    c->ev_used = 0;
    c->ev_calls.clear();
    c->ev_band.clear();
    memset(&c->tsum, 0, sizeof(c->tsum));
    return EGM_OK;
}

egm_status egm_get_timing(egm_ctx *c, egm_timing *t) {
    if (!c || !t) return EGM_ERR_ARG;
    EGM_TRY(cudaSetDevice(c->device));
    EGM_TRY(cudaStreamSynchronize(c->stream));
    for (size_t q = 0; q < c->ev_calls.size(); q++) {
        const size_t b = c->ev_calls[q];
        float ms[kStages];
        for (int k = 0; k < kStages; k++)
            EGM_TRY(cudaEventElapsedTime(&ms[k], c->ev_pool[b + k], c->ev_pool[b + k + 1]));
        c->tsum.geometry_ms += ms[0];
        c->tsum.prep_ms += ms[1];
        c->tsum.sort_ms += ms[2];
        c->tsum.post_sort_ms += ms[3];
        c->tsum.stab_ms += ms[4];
        c->tsum.csr_ms += ms[5];
        c->tsum.calls += 1;
        c->tsum.banded_calls += c->ev_band[q] ? 1 : 0;
    }
    c->ev_calls.clear();
    c->ev_band.clear();
    c->ev_used = 0;
    *t = c->tsum;
    return EGM_OK;
}

egm_status egm_set_counters(egm_ctx *c, int32_t enable) {
    if (!c) return EGM_ERR_ARG;
    c->counters_on = enable != 0;
    return EGM_OK;
}

egm_status egm_get_stats(egm_ctx *c, egm_stats *s) {
    if (!c || !s) return EGM_ERR_ARG;
    egm_status st = egm_sync(c);
    *s = c->last;
    return st;
}

const char *egm_status_string(egm_status s) {
    switch (s) {
        case EGM_OK: return "ok";
        case EGM_ERR_ARG: return "invalid argument";
        case EGM_ERR_CUDA: return "CUDA runtime error";
        case EGM_ERR_NOMEM: return "out of device memory";
        case EGM_ERR_CAPACITY: return "candidate capacity too small";
        case EGM_ERR_DEGENERATE_F: return "degenerate fundamental matrix (rank < 2)";
        case EGM_ERR_NAN: return "NaN or Inf in the inputs";
        case EGM_ERR_TIMEOUT: return "bounded device wait timed out";
        case EGM_ERR_UNIMPLEMENTED: return "not implemented";
    }
    return "unknown status";
}

int32_t egm_version(void) { return EGM_VERSION; }

}  // extern "C"
