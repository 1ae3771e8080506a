// Learned per-keypoint tolerance: a 5 -> 64 -> 64 -> 64 -> 1 network.
//
// The paper names per-point tolerances as a promising direction (Sec. 6)
// without a model.  Network, features, target and loss here are this
// library's reading:
//   u   = (ln s, orientation / 2 pi, ln response, x / W, y / H)
//   h_l = GELU(W_l h_{l-1} + b_l), l = 1..3, GELU(x) = x Phi(x)
//   eps = softplus(W4 h3 + b4) + 0.25 px
//   loss: pinball loss at quantile q of the residual r (the distance of the
//   true match from its epipolar line, Eq. 3) against eps.
// Weights are kept in FP32 (the Adam master copy) and rounded to BF16 when a
// kernel loads them; every sum is FP32 (the tensor-core layers take each FP32
// activation as the sum of two BF16 parts, the rest is FP32 arithmetic).
//
//   mlp_forward_tc_kernel  inference and the training forward pass (which
//                        also writes the pre-activations and the output):
//                        one thread per sample, layer 1 and GELU on the CUDA
//                        cores, layers 2 and 3 on the tensor cores
//                        (tcgen05.mma, M = 128 samples, N = 64 units, K = 64)
//   mlp_backward_kernel  persistent blocks taking tiles of 64 samples: deltas
//                        layer by layer, the weight gradients in 4 x 4 register
//                        tiles and the other sums split over all threads, kept
//                        over the block's tiles and added to the global
//                        gradient with atomics once
//   adam_kernel          the Adam update, one thread per parameter
//   residual_kernel      FP64 distances of given (query, reference) pairs,
//                        in the brute force's exact evaluation order
#include <cuda_bf16.h>
#include <math.h>

#include "egm_internal.cuh"
#include "tc.cuh"

namespace egm {

namespace {

constexpr int kH = 64;
constexpr int kIn = 5;
constexpr int kP = kH * kIn + kH + 2 * (kH * kH + kH) + kH + 1;  // 8769
// offsets in the flat layout W1, b1, W2, b2, W3, b3, W4, b4 (rows = outputs)
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * kH, oW4 = ob3 + kH, ob4 = oW4 + kH;
static_assert(ob4 + 1 == kP, "layout");
constexpr float kEpsFloor = 0.25f;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}
__device__ __forceinline__ float softplus(float z) { return z > 20.0f ? z : log1pf(expf(z)); }
__device__ __forceinline__ float sigmoid(float z) { return 1.0f / (1.0f + expf(-z)); }

__device__ __forceinline__ void load_weights(float *w, const float *params) {
    for (int k = threadIdx.x; k < kP; k += blockDim.x) w[k] = bf16r(params[k]);
}

__device__ __forceinline__ void features(const float *feat, int64_t s, float *u) {
    const float *f = feat + 5 * s;
    u[0] = logf(f[0]);
    u[1] = f[1] * 0.15915494309189535f;
    u[2] = logf(f[2]);
    u[3] = f[3];
    u[4] = f[4];
}

constexpr int kWPad = (kP + 3) & ~3;  // weights, then the activation buffer (16-byte aligned)
static_assert(oW2 % 4 == 0 && oW3 % 4 == 0 && oW4 % 4 == 0, "float4 weight rows");

// ------------------------------------------------------------ tensor-core forward
// Layers 2 and 3 (the two 64 x 64 products, 96 % of the network's multiply-adds) as
// tcgen05.mma with FP32 accumulators in TMEM: A = the tile's 128 activation
// rows, B = the layer's weight rows (already BF16), both K-major rows of 64
// BF16 values (128 bytes) in the 128-byte swizzle layout.  A layer's FP32
// activations h are split into hi = bf16(h) and lo = bf16(h - hi); both
// products accumulate, so the operand carries h to about 2^-17 relative and
// the result stays within FP32-level error of the CUDA-core kernel.  Layer 1
// (5 inputs), layer 4 (one output), the biases and GELU run on the CUDA
// cores; one thread per sample, which is also the sample's TMEM lane.
constexpr int kTT = 128;            // samples per tile (MMA M, TMEM lanes)
constexpr uint32_t kTmemMlp = 64;   // accumulator columns (N)

struct __align__(1024) MlpTcSmem {
    uint8_t Ahi[kTT * 128];         // activation rows, hi part (1024-byte swizzle atoms)
    uint8_t Alo[kTT * 128];         //   and lo part
    uint8_t W2[kH * 128];           // weight rows [unit][input] of layers 2 and 3
    uint8_t W3[kH * 128];
    float w1[kH * kIn], b1[kH], b2[kH], b3[kH], w4[kH], b4;
    uint64_t bar;                   // MMA completion
    uint32_t tmem;
};

// Byte offset of the 16-byte chunk c (0..7) of row r in a tile of 128-byte
// rows with the 128-byte swizzle: the chunk index is XORed with the row's
// position in its 8-row atom, as the tensor cores read it.
__device__ __forceinline__ uint32_t sw128_off(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ uint32_t bf16x2(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// Row r of the hi and lo activation tiles from h[0..63].
__device__ __forceinline__ void store_split(MlpTcSmem &S, int r, const float (&h)[kH]) {
#pragma unroll
    for (int c = 0; c < 8; c++) {
        float hi[8], lo[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            hi[k] = bf16r(h[8 * c + k]);
            lo[k] = h[8 * c + k] - hi[k];  // exact
        }
        *reinterpret_cast<uint4 *>(S.Ahi + sw128_off(r, c)) =
            make_uint4(bf16x2(hi[0], hi[1]), bf16x2(hi[2], hi[3]), bf16x2(hi[4], hi[5]), bf16x2(hi[6], hi[7]));
        *reinterpret_cast<uint4 *>(S.Alo + sw128_off(r, c)) =
            make_uint4(bf16x2(lo[0], lo[1]), bf16x2(lo[2], lo[3]), bf16x2(lo[4], lo[5]), bf16x2(lo[6], lo[7]));
    }
}

// Persistent: each block takes tiles of 128 samples in turn.  Every wait on
// the MMA barrier is bounded; a timeout sets the timeout bit in *err and the
// block issues no more MMAs.  A sample whose output is not a finite
// tolerance (non-finite features, or a block whose MMA wait gave up) gets the
// fixed tolerance `fallback` instead.  kTrain: the training forward pass,
// which writes the pre-activations and outputs instead of eps (a separate
// instance: the stores cost the inference instance registers).
template <bool kTrain>
__global__ void __launch_bounds__(kTT, 4) mlp_forward_tc_kernel(const float *params, const float *feat, int64_t n,
                                                                double *eps, uint32_t *err, double fallback,
                                                                float *pre, float *zout) {
    extern __shared__ uint8_t smraw[];
    MlpTcSmem &S = *reinterpret_cast<MlpTcSmem *>(smraw + ((1024u - (tc::smem_addr(smraw) & 1023u)) & 1023u));
    const int t = threadIdx.x, warp = t >> 5;
    // the weights: BF16 tiles of W2 and W3 (one 16-byte chunk per step), FP32 copies of the rest
    for (int i = t; i < 2 * kH * 8; i += kTT) {
        const int l = i / (kH * 8), r = (i / 8) % kH, c = i % 8;
        const float *src = params + (l == 0 ? oW2 : oW3) + r * kH + 8 * c;
        *reinterpret_cast<uint4 *>((l == 0 ? S.W2 : S.W3) + sw128_off(r, c)) =
            make_uint4(bf16x2(src[0], src[1]), bf16x2(src[2], src[3]), bf16x2(src[4], src[5]), bf16x2(src[6], src[7]));
    }
    for (int i = t; i < kH * kIn; i += kTT) S.w1[i] = bf16r(params[oW1 + i]);
    if (t < kH) {
        S.b1[t] = bf16r(params[ob1 + t]);
        S.b2[t] = bf16r(params[ob2 + t]);
        S.b3[t] = bf16r(params[ob3 + t]);
        S.w4[t] = bf16r(params[oW4 + t]);
    }
    if (t == 0) {
        S.b4 = bf16r(params[ob4]);
        tc::mbar_init(&S.bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, kTmemMlp);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async();  // the weight tiles' generic writes, before the MMAs read them
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    constexpr uint32_t idesc = tc::idesc_bf16(kTT, kH);
    const int64_t ntiles = (n + kTT - 1) / kTT;
    // A failed wait ends the block's MMAs; every decision about it is uniform
    // where it must be (the warp for TMEM loads, the block for barriers), and
    // no thread leaves the loops early.
    bool failed = false;
    uint32_t mma_commits = 0;  // phases of S.bar armed (the same count in every thread)
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t s = tile * kTT + t;
        const bool valid = s < n;
        float u[kIn] = {0, 0, 0, 0, 0};
        if (valid) features(feat, s, u);
        float h[kH];
#pragma unroll
        for (int k = 0; k < kH; k++) {
            float a = S.b1[k];
#pragma unroll
            for (int j = 0; j < kIn; j++) a = fmaf(S.w1[k * kIn + j], u[j], a);
            if (kTrain && valid) pre[k * n + s] = a;
            h[k] = gelu(a);
        }
        store_split(S, t, h);
#pragma unroll 1
        for (int l = 0; l < 2; l++) {
            // every row written and the previous accumulator read before the MMAs
            tc::fence_proxy_async();
            tc::tc_fence_before();
            failed = __syncthreads_or(failed) != 0;
            if (!failed) {
                if (t == 0) {
                    tc::tc_fence_after();
                    const uint8_t *W = l == 0 ? S.W2 : S.W3;
#pragma unroll
                    for (int kk = 0; kk < 4; kk++)
                        tc::mma_f16(tmem, tc::sdesc_sw128(tc::smem_addr(S.Ahi) + 32 * kk),
                                     tc::sdesc_sw128(tc::smem_addr(W) + 32 * kk), idesc, kk > 0);
#pragma unroll
                    for (int kk = 0; kk < 4; kk++)
                        tc::mma_f16(tmem, tc::sdesc_sw128(tc::smem_addr(S.Alo) + 32 * kk),
                                     tc::sdesc_sw128(tc::smem_addr(W) + 32 * kk), idesc, 1);
                    tc::mma_commit(&S.bar);
                }
                mma_commits++;
                // two commits per tile: the layer's phase parity is l
                const bool done = tc::mbar_wait(&S.bar, (uint32_t)l);
                failed = __any_sync(0xffffffffu, !done);
                if (failed && (t & 31) == 0) atomicOr(err, kStTimeout);
            }
            if (!failed) {
                tc::tc_fence_after();
                const float *b = l == 0 ? S.b2 : S.b3;
#pragma unroll
                for (int half = 0; half < 2; half++) {
                    uint32_t v[32];
                    tc::tmem_ld32(tmem + lane_base + 32 * half, v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 32; k++) {
                        const float a = __uint_as_float(v[k]) + b[32 * half + k];
                        if (kTrain && valid) pre[((1 + l) * kH + 32 * half + k) * n + s] = a;
                        h[32 * half + k] = gelu(a);
                    }
                }
                if (l == 0) store_split(S, t, h);
            }
        }
        float z = S.b4;
#pragma unroll
        for (int j = 0; j < kH; j++) z = fmaf(S.w4[j], h[j], z);
        if (valid && !kTrain) {
            const float e = softplus(z) + kEpsFloor;
            eps[s] = (failed || !isfinite(e)) ? fallback : (double)e;
        }
        if (valid && kTrain) zout[s] = z;
    }
    // after a failed wait the MMAs of the last commit may still run: wait for
    // that commit's phase (bounded) before the TMEM is released
    if (failed && t == 0) tc::mbar_wait(&S.bar, (uint32_t)(mma_commits - 1) & 1u);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemMlp);
}

constexpr int kBB = 64;        // backward samples per block
constexpr int kRS = kH + 4;    // padded row stride of the [sample][unit] buffers (16-byte rows)

// Persistent blocks of 256 threads, each taking tiles of kBB samples in turn;
// per tile the activations, their GELU slopes and the deltas are stored
// sample-major in shared memory, so that
//   weight gradients  dW[k][j] = sum_c D[c][k] H[c][j]: a thread accumulates a
//                     4 x 4 tile from two float4 loads per sample;
//   deltas below      E[c][j] = (sum_k W[k][j] D[c][k]) gelu'(a[c][j]): a
//                     thread accumulates a 4 x 4 (sample x unit) tile from
//                     eight float4 loads per four k.
// A thread keeps its gradient tiles in registers over all of its block's
// tiles; the block adds them to the global gradient with atomics once, at
// the end.  Every sum within a tile runs over samples, or over k, in
// ascending order.
__global__ void __launch_bounds__(256, 2) mlp_backward_kernel(const float *params, const float *feat,
                                                              const float *resid, int64_t n, float q,
                                                              const float *pre, const float *zin, float *grad,
                                                              float *loss) {
    extern __shared__ float sm[];
    float *w = sm;                   // kP
    float *Hs = w + kWPad;           // activations of the layer below  [sample][unit]
    float *Gs = Hs + kBB * kRS;      // their GELU slopes               [sample][unit]
    float *D0 = Gs + kBB * kRS;      // deltas of the current layer     [sample][unit]
    float *E0 = D0 + kBB * kRS;      // deltas of the layer below       [sample][unit]
    float *dz = E0 + kBB * kRS;      // [sample]
    float *red = dz + kBB;           // loss partials of the warps
    load_weights(w, params);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int kt = t >> 4, jt = t & 15;  // this thread's 4 x 4 tile of a 64 x 64 gradient
    // the sums over a tile's samples of the other gradients: unit u, samples
    // [16 sq, 16 sq + 16) (every thread; the four quarters meet in the atomics)
    const int u = t & (kH - 1), sq = t >> 6, c0 = 16 * sq;
    static_assert(kH == 64 && kBB == 64, "four sample quarters of 16 per unit");
    float acc3[4][4], acc2[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc3[i][j] = acc2[i][j] = 0.0f;
    // W4 and the biases (unit u), b4 (threads 0-3), and five (W1 entry, quarter)
    // pairs: pair k = t + 256 k is entry k % 320 over quarter k / 320
    constexpr int kW1 = kH * kIn, kW1Per = 4 * kW1 / 256;
    static_assert(4 * kW1 % 256 == 0, "W1's (entry, quarter) pairs fill the threads");
    float gw4 = 0.0f, gb4 = 0.0f, gb3 = 0.0f, gb2 = 0.0f, gb1 = 0.0f, gw1[kW1Per];
#pragma unroll
    for (int k = 0; k < kW1Per; k++) gw1[k] = 0.0f;
    float lsum = 0.0f;
    __syncthreads();
    const int64_t ntiles = (n + kBB - 1) / kBB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t s0 = tile * kBB;
        const int nb = (int)min((int64_t)kBB, n - s0);
        float *Ds = D0, *Es = E0;
        // output layer: dL/dz and the loss
        if (t < kBB) {
            float d = 0.0f;
            if (t < nb) {
                const int64_t s = s0 + t;
                const float z = zin[s];
                const float e = softplus(z) + kEpsFloor;
                const float r = resid[s];
                const float diff = r - e;
                lsum += fmaxf(q * diff, (q - 1.0f) * diff);
                const float de = r > e ? -q : (r < e ? 1.0f - q : 0.0f);
                d = de / (float)n * sigmoid(z);
            }
            dz[t] = d;
        }
        __syncthreads();
        // h3 and delta3 = dz W4 gelu'(a3): sample c = t mod 64, the four runs of
        // four units 4 (t / 64 + 4 r) ..; the 16 pre-activations loaded together,
        // each run stored as one float4 (a warp's 32 samples then fall on
        // distinct banks)
        {
            const int c = t & (kBB - 1), gq = t >> 6;
            float a[16];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int j = 0; j < 4; j++)
                    a[4 * r + j] = c < nb ? pre[(2 * kH + 4 * (gq + 4 * r) + j) * n + s0 + c] : 0.0f;
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int k0 = 4 * (gq + 4 * r);
                float h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                if (c < nb) {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        h[j] = gelu(a[4 * r + j]);
                        d[j] = dz[c] * w[oW4 + k0 + j] * gelu_grad(a[4 * r + j]);
                    }
                }
                *reinterpret_cast<float4 *>(Hs + c * kRS + k0) = make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4 *>(Ds + c * kRS + k0) = make_float4(d[0], d[1], d[2], d[3]);
            }
        }
        __syncthreads();
        // W4, b4 (rows past the tile's samples are zero)
#pragma unroll 4
        for (int c = c0; c < c0 + 16; c++) gw4 = fmaf(dz[c], Hs[c * kRS + u], gw4);
        if (t < 4)
#pragma unroll 4
            for (int c = 16 * t; c < 16 * t + 16; c++) gb4 += dz[c];
        __syncthreads();
        // layers 3 and 2: weights of layer L map H (below) to D (current)
#pragma unroll
        for (int L = 3; L >= 2; L--) {
            const float *W = w + (L == 3 ? oW3 : oW2);
            float (&acc)[4][4] = L == 3 ? acc3 : acc2;
            // activations of the layer below and their slopes (as above)
            {
                const int c = t & (kBB - 1), gq = t >> 6;
                float a[16];
#pragma unroll
                for (int r = 0; r < 4; r++)
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        a[4 * r + j] = c < nb ? pre[((L - 2) * kH + 4 * (gq + 4 * r) + j) * n + s0 + c] : 0.0f;
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int k0 = 4 * (gq + 4 * r);
                    float h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, gg[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    if (c < nb) {
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            h[j] = gelu(a[4 * r + j]);
                            gg[j] = gelu_grad(a[4 * r + j]);
                        }
                    }
                    *reinterpret_cast<float4 *>(Hs + c * kRS + k0) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4 *>(Gs + c * kRS + k0) = make_float4(gg[0], gg[1], gg[2], gg[3]);
                }
            }
            __syncthreads();
            // weight gradients of layer L: the thread's 4 x 4 tile (rows 4 kt.., columns 4 jt..)
            for (int c = 0; c < nb; c++) {
                const float4 d4 = *reinterpret_cast<const float4 *>(Ds + c * kRS + 4 * kt);
                const float4 h4 = *reinterpret_cast<const float4 *>(Hs + c * kRS + 4 * jt);
                const float dv[4] = {d4.x, d4.y, d4.z, d4.w}, hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fmaf(dv[i], hv[j], acc[i][j]);
            }
            {
                float g = 0.0f;
#pragma unroll 4
                for (int c = c0; c < c0 + 16; c++) g += Ds[c * kRS + u];
                if (L == 3) gb3 += g;
                else gb2 += g;
            }
            // deltas of the layer below: E[c][j] = (sum_k W[k][j] D[c][k]) gelu'(a[c][j]),
            // a 4 x 4 tile (samples 4 ct.., units 4 jt..) per thread and step
            for (int tl = t; tl < (kH / 4) * (kBB / 4); tl += blockDim.x) {
                const int jt2 = tl & 15, ct = tl >> 4;
                float e[4][4];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) e[i][j] = 0.0f;
                for (int k = 0; k < kH; k += 4) {
                    float4 wr[4], dr[4];
#pragma unroll
                    for (int i = 0; i < 4; i++) wr[i] = *reinterpret_cast<const float4 *>(W + (k + i) * kH + 4 * jt2);
#pragma unroll
                    for (int cc = 0; cc < 4; cc++)
                        dr[cc] = *reinterpret_cast<const float4 *>(Ds + (4 * ct + cc) * kRS + k);
#pragma unroll
                    for (int cc = 0; cc < 4; cc++) {
                        const float dv[4] = {dr[cc].x, dr[cc].y, dr[cc].z, dr[cc].w};
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const float wv[4] = {j == 0 ? wr[0].x : j == 1 ? wr[0].y : j == 2 ? wr[0].z : wr[0].w,
                                                 j == 0 ? wr[1].x : j == 1 ? wr[1].y : j == 2 ? wr[1].z : wr[1].w,
                                                 j == 0 ? wr[2].x : j == 1 ? wr[2].y : j == 2 ? wr[2].z : wr[2].w,
                                                 j == 0 ? wr[3].x : j == 1 ? wr[3].y : j == 2 ? wr[3].z : wr[3].w};
#pragma unroll
                            for (int i = 0; i < 4; i++) e[cc][j] = fmaf(wv[i], dv[i], e[cc][j]);
                        }
                    }
                }
#pragma unroll
                for (int cc = 0; cc < 4; cc++) {
                    const int c = 4 * ct + cc;
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        Es[c * kRS + 4 * jt2 + j] = c < nb ? e[cc][j] * Gs[c * kRS + 4 * jt2 + j] : 0.0f;
                }
            }
            __syncthreads();
            float *tmp = Ds;
            Ds = Es;
            Es = tmp;
        }
        // layer 1: inputs are the features (sample-major in Hs, kIn columns)
        for (int c = t; c < kBB; c += blockDim.x) {
            float u[kIn] = {0, 0, 0, 0, 0};
            if (c < nb) features(feat, s0 + c, u);
#pragma unroll
            for (int j = 0; j < kIn; j++) Hs[c * kRS + j] = u[j];
        }
        __syncthreads();
        // W1: the thread's (entry, quarter) pairs; b1
#pragma unroll
        for (int k = 0; k < kW1Per; k++) {
            const int pk = t + 256 * k, e = pk % kW1, cq = 16 * (pk / kW1);
            const float *dr = Ds + e / kIn, *hr = Hs + e % kIn;
            float g = 0.0f;
#pragma unroll 4
            for (int c = cq; c < cq + 16; c++) g = fmaf(dr[c * kRS], hr[c * kRS], g);
            gw1[k] += g;
        }
        {
            float g = 0.0f;
#pragma unroll 4
            for (int c = c0; c < c0 + 16; c++) g += Ds[c * kRS + u];
            gb1 += g;
        }
        __syncthreads();  // the tile's buffers are read before the next tile writes them
    }
    // the block's gradients and loss, once
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            atomicAdd(grad + oW3 + (4 * kt + i) * kH + 4 * jt + j, acc3[i][j]);
            atomicAdd(grad + oW2 + (4 * kt + i) * kH + 4 * jt + j, acc2[i][j]);
        }
    atomicAdd(grad + oW4 + u, gw4);
    atomicAdd(grad + ob3 + u, gb3);
    atomicAdd(grad + ob2 + u, gb2);
    atomicAdd(grad + ob1 + u, gb1);
    if (t < 4) atomicAdd(grad + ob4, gb4);
#pragma unroll
    for (int k = 0; k < kW1Per; k++) atomicAdd(grad + oW1 + (t + 256 * k) % kW1, gw1[k]);
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) red[warp] = lsum;
    __syncthreads();
    if (t == 0 && loss) {
        float v = 0.0f;
        for (int k = 0; k < 8; k++) v += red[k];
        atomicAdd(loss, v / (float)n);
    }
}

__global__ void adam_kernel(float *p, float *g, float *m, float *v, int np, float lr, float b1, float b2, float e,
                            float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + e);
    g[i] = 0.0f;
}

__global__ void residual_kernel(const double *xy1, const double *xy2, const double *F, int64_t m, int64_t n,
                                const int32_t *qi, const int32_t *rj, int64_t k, double *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= k) return;
    const int32_t i = qi[t], j = rj[t];
    if (i < 0 || i >= m || j < 0 || j >= n) {   // an index out of range gives NaN
        out[t] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    double a, b, c;
    exact_line(F, xy1[2 * (int64_t)i], xy1[2 * (int64_t)i + 1], a, b, c);
    const double N = exact_norm(a, b);
    const double num = fabs(__dadd_rn(__dadd_rn(__dmul_rn(a, xy2[2 * (int64_t)j]), __dmul_rn(b, xy2[2 * (int64_t)j + 1])), c));
    out[t] = N > 0.0 ? __ddiv_rn(num, N) : INFINITY;
}

}  // namespace

int mlp_param_count() { return kP; }

size_t mlp_backward_smem() { return sizeof(float) * (kWPad + 4 * kBB * kRS + kBB + 8); }

cudaError_t launch_mlp_forward_tc(const float *params, const float *feat, int64_t n, double *eps, uint32_t *err,
                                  double fallback, int sms, cudaStream_t s, float *pre, float *z) {
    if (n <= 0) return cudaSuccess;
    const int smem = (int)sizeof(MlpTcSmem) + 1024;
    const bool train = pre != nullptr;
    cudaError_t e = train ? cudaFuncSetAttribute(mlp_forward_tc_kernel<true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                          : cudaFuncSetAttribute(mlp_forward_tc_kernel<false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + kTT - 1) / kTT;
    const int grid = (int)std::min<int64_t>(tiles, 4 * (int64_t)sms);
    if (train) mlp_forward_tc_kernel<true><<<grid, kTT, smem, s>>>(params, feat, n, eps, err, fallback, pre, z);
    else mlp_forward_tc_kernel<false><<<grid, kTT, smem, s>>>(params, feat, n, eps, err, fallback, pre, z);
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float *params, const float *feat, const float *resid, int64_t n, float q,
                                const float *pre, const float *z, float *grad, float *loss, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int smem = (int)mlp_backward_smem();
    cudaError_t e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // two persistent blocks per SM (the kernel's bound), at most one per tile
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t tiles = (n + kBB - 1) / kBB;
    const int grid = (int)std::min<int64_t>(tiles, 2 * (int64_t)sms);
    mlp_backward_kernel<<<grid, 256, smem, s>>>(params, feat, resid, n, q, pre, z, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, float *g, float *m, float *v, float lr, int64_t step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<(kP + 255) / 256, 256, 0, s>>>(p, g, m, v, kP, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_residuals(const double *xy1, const double *xy2, const double *F, int64_t m, int64_t n,
                             const int32_t *qi, const int32_t *rj, int64_t k, double *out, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    residual_kernel<<<(int)((k + 255) / 256), 256, 0, s>>>(xy1, xy2, F, m, n, qi, rj, k, out);
    return cudaGetLastError();
}

}  // namespace egm
