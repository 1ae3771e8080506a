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
// kernel loads them; every product and sum is FP32.
//
//   mlp_forward_kernel   one thread per sample, 128 samples per block, the
//                        weights and the block's activations in shared
//                        memory (activations column-major: no bank conflicts
//                        while every thread reads the same weight)
//   mlp_backward_kernel  64 samples per block: deltas layer by layer, then the
//                        block's weight gradients with one thread per weight
//                        element summing over the samples, added to the global
//                        gradient with atomics
//   adam_kernel          the Adam update, one thread per parameter
//   residual_kernel      FP64 distances of given (query, reference) pairs,
//                        in the brute force's exact evaluation order
#include <cuda_bf16.h>
#include <math.h>

#include "egm_internal.cuh"

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

constexpr int kFB = 128;  // forward samples per block

// eps (double) and, for training, pre-activations a1..a3 stored [layer][unit][sample].
__global__ void __launch_bounds__(kFB) mlp_forward_kernel(const float *params, const float *feat, int64_t n,
                                                          double *eps, float *pre, float *zout) {
    extern __shared__ float sm[];
    float *w = sm;                  // kP
    float *ha = w + kP + 3;         // kH x kFB
    float *hb = ha + kH * kFB;      // kH x kFB
    load_weights(w, params);
    __syncthreads();
    const int t = threadIdx.x;
    const int64_t s = (int64_t)blockIdx.x * kFB + t;
    const bool valid = s < n;
    float u[kIn] = {0, 0, 0, 0, 0};
    if (valid) features(feat, s, u);
    // layer 1
    for (int k = 0; k < kH; k++) {
        float a = w[ob1 + k];
#pragma unroll
        for (int j = 0; j < kIn; j++) a = fmaf(w[oW1 + k * kIn + j], u[j], a);
        if (valid && pre) pre[(0 * kH + k) * n + s] = a;
        ha[k * kFB + t] = gelu(a);
    }
    // layers 2 and 3
    float *hin = ha, *hout = hb;
    for (int l = 0; l < 2; l++) {
        const float *W = w + (l == 0 ? oW2 : oW3);
        const float *b = w + (l == 0 ? ob2 : ob3);
        for (int k = 0; k < kH; k++) {
            float a = b[k];
#pragma unroll 8
            for (int j = 0; j < kH; j++) a = fmaf(W[k * kH + j], hin[j * kFB + t], a);
            if (valid && pre) pre[((1 + l) * kH + k) * n + s] = a;
            hout[k * kFB + t] = gelu(a);
        }
        float *tmp = hin;
        hin = hout;
        hout = tmp;
    }
    float z = w[ob4];
#pragma unroll 8
    for (int j = 0; j < kH; j++) z = fmaf(w[oW4 + j], hin[j * kFB + t], z);
    if (valid) {
        if (eps) eps[s] = (double)(softplus(z) + kEpsFloor);
        if (zout) zout[s] = z;
    }
}

constexpr int kBB = 64;        // backward samples per block
constexpr int kBS = kBB + 1;   // padded row stride of the [unit][sample] buffers

__global__ void __launch_bounds__(256) mlp_backward_kernel(const float *params, const float *feat,
                                                           const float *resid, int64_t n, float q, const float *pre,
                                                           const float *zin, float *grad, float *loss) {
    extern __shared__ float sm[];
    float *w = sm;                   // kP
    float *H = w + kP + 3;           // activations of the layer below  [unit][sample]
    float *D = H + kH * kBS;         // deltas of the current layer     [unit][sample]
    float *E = D + kH * kBS;         // deltas of the layer below
    float *dz = E + kH * kBS;        // [sample]
    float *red = dz + kBB;           // loss partials
    load_weights(w, params);
    const int t = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * kBB;
    const int nb = (int)min((int64_t)kBB, n - s0);
    __syncthreads();
    // output layer: dL/dz and the loss
    float lsum = 0.0f;
    if (t < kBB) {
        float d = 0.0f;
        if (t < nb) {
            const int64_t s = s0 + t;
            const float z = zin[s];
            const float e = softplus(z) + kEpsFloor;
            const float r = resid[s];
            const float diff = r - e;
            lsum = fmaxf(q * diff, (q - 1.0f) * diff);
            const float de = r > e ? -q : (r < e ? 1.0f - q : 0.0f);
            d = de / (float)n * sigmoid(z);
        }
        dz[t] = d;
    }
    __syncthreads();
    // h3 and delta3 = dz W4 gelu'(a3)
    for (int i = t; i < kH * kBB; i += blockDim.x) {
        const int k = i / kBB, c = i % kBB;
        float h = 0.0f, d = 0.0f;
        if (c < nb) {
            const float a = pre[(2 * kH + k) * n + s0 + c];
            h = gelu(a);
            d = dz[c] * w[oW4 + k] * gelu_grad(a);
        }
        H[k * kBS + c] = h;
        D[k * kBS + c] = d;
    }
    if (t < 32) {
        float v = lsum;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (t == 0) red[0] = v;
    } else if (t < 64) {
        float v = lsum;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (t == 32) red[1] = v;
    }
    __syncthreads();
    if (t == 0 && loss) atomicAdd(loss, (red[0] + red[1]) / (float)n);
    // W4, b4
    if (t < kH) {
        float g = 0.0f;
        for (int c = 0; c < nb; c++) g = fmaf(dz[c], H[t * kBS + c], g);
        atomicAdd(grad + oW4 + t, g);
    } else if (t == kH) {
        float g = 0.0f;
        for (int c = 0; c < nb; c++) g += dz[c];
        atomicAdd(grad + ob4, g);
    }
    __syncthreads();
    // layers 3 and 2: weights of layer L map H (below) to D (current)
    for (int L = 3; L >= 2; L--) {
        const float *W = w + (L == 3 ? oW3 : oW2);
        const int oW = L == 3 ? oW3 : oW2, ob = L == 3 ? ob3 : ob2;
        // activations of the layer below
        for (int i = t; i < kH * kBB; i += blockDim.x) {
            const int k = i / kBB, c = i % kBB;
            H[k * kBS + c] = c < nb ? gelu(pre[((L - 2) * kH + k) * n + s0 + c]) : 0.0f;
        }
        __syncthreads();
        // weight gradients of layer L: one thread per (row, column) group
        for (int i = t; i < kH * kH; i += blockDim.x) {
            const int k = i / kH, j = i % kH;
            float g = 0.0f;
            for (int c = 0; c < nb; c++) g = fmaf(D[k * kBS + c], H[j * kBS + c], g);
            atomicAdd(grad + oW + i, g);
        }
        if (t < kH) {
            float g = 0.0f;
            for (int c = 0; c < nb; c++) g += D[t * kBS + c];
            atomicAdd(grad + ob + t, g);
        }
        // deltas of the layer below: E = (W^T D) * gelu'(a_{L-1})
        for (int i = t; i < kH * kBB; i += blockDim.x) {
            const int j = i / kBB, c = i % kBB;
            float a = 0.0f;
            for (int k = 0; k < kH; k++) a = fmaf(W[k * kH + j], D[k * kBS + c], a);
            E[j * kBS + c] = c < nb ? a * gelu_grad(pre[((L - 2) * kH + j) * n + s0 + c]) : 0.0f;
        }
        __syncthreads();
        float *tmp = D;
        D = E;
        E = tmp;
    }
    // layer 1: inputs are the features
    for (int i = t; i < kIn * kBB; i += blockDim.x) {
        const int j = i / kBB, c = i % kBB;
        float u[kIn] = {0, 0, 0, 0, 0};
        if (c < nb) features(feat, s0 + c, u);
        H[j * kBS + c] = u[j];
    }
    __syncthreads();
    for (int i = t; i < kH * kIn; i += blockDim.x) {
        const int k = i / kIn, j = i % kIn;
        float g = 0.0f;
        for (int c = 0; c < nb; c++) g = fmaf(D[k * kBS + c], H[j * kBS + c], g);
        atomicAdd(grad + oW1 + i, g);
    }
    if (t < kH) {
        float g = 0.0f;
        for (int c = 0; c < nb; c++) g += D[t * kBS + c];
        atomicAdd(grad + ob1 + t, g);
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

size_t mlp_forward_smem() { return sizeof(float) * (kP + 3 + 2 * kH * kFB); }
size_t mlp_backward_smem() { return sizeof(float) * (kP + 3 + 3 * kH * kBS + kBB + 8); }

cudaError_t launch_mlp_forward(const float *params, const float *feat, int64_t n, double *eps, float *pre, float *z,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int smem = (int)mlp_forward_smem();
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    mlp_forward_kernel<<<(int)((n + kFB - 1) / kFB), kFB, smem, s>>>(params, feat, n, eps, pre, z);
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float *params, const float *feat, const float *resid, int64_t n, float q,
                                const float *pre, const float *z, float *grad, float *loss, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int smem = (int)mlp_backward_smem();
    cudaError_t e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    mlp_backward_kernel<<<(int)((n + kBB - 1) / kBB), 256, smem, s>>>(params, feat, resid, n, q, pre, z, grad, loss);
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
