// Hit-ranking MLP (12 -> 64 ReLU -> 1): bfloat16 conversion, forward, gradient
// of the mean binary cross-entropy, Adam.  FP32 arithmetic with bfloat16-rounded
// weights.  The batch reduction of the gradient is done in a fixed order
// (per-chunk compensated sums, then the chunk partials in order), so results do
// not depend on how blocks are scheduled.
#include <cuda_runtime.h>

#include <algorithm>

#include "mkf_internal.h"

namespace {

constexpr int kIn = MKF_MLP_IN;
constexpr int kHid = MKF_MLP_HIDDEN;
constexpr int kP = MKF_MLP_PARAMS;
constexpr int kOffB1 = kIn * kHid;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid;
constexpr int kChunk = 256;  // samples per reduction chunk

// float -> bfloat16 bits, round to nearest, ties to even (NaN kept quiet)
__device__ __forceinline__ uint16_t to_bf16(float f) {
    const uint32_t u = __float_as_uint(f);
    if ((u & 0x7fffffffu) > 0x7f800000u) return static_cast<uint16_t>((u >> 16) | 0x40u);
    const uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
    return static_cast<uint16_t>(r >> 16);
}

__device__ __forceinline__ float from_bf16(uint16_t b) { return __uint_as_float(static_cast<uint32_t>(b) << 16); }

__global__ void to_bf16_kernel(const float *w, uint16_t *o, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = to_bf16(w[i]);
}

__device__ __forceinline__ void load_weights(const uint16_t *wb, float *ws) {
    for (int i = threadIdx.x; i < kP; i += blockDim.x) ws[i] = from_bf16(wb[i]);
    __syncthreads();
}

__global__ void __launch_bounds__(128) forward_kernel(const uint16_t *wb, const float *feat, int n, float *logit) {
    __shared__ float ws[kP];
    load_weights(wb, ws);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) x[k] = feat[(int64_t)s * kIn + k];
    float z = ws[kOffB2];
    for (int j = 0; j < kHid; ++j) {
        float a = ws[kOffB1 + j];
#pragma unroll
        for (int k = 0; k < kIn; ++k) a = fmaf(ws[j * kIn + k], x[k], a);
        z = fmaf(ws[kOffW2 + j], fmaxf(a, 0.f), z);
    }
    logit[s] = z;
}

// Per sample: forward, d(loss)/d(logit) = (sigmoid(z) - y) / n, the hidden
// activations H and the pre-activation gradient dA, and the sample's loss.
__global__ void __launch_bounds__(128) sample_grad_kernel(const uint16_t *wb, const float *feat, const float *label,
                                                          int n, float *H, float *dA, float *g, float *ls) {
    __shared__ float ws[kP];
    load_weights(wb, ws);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) x[k] = feat[(int64_t)s * kIn + k];
    float z = ws[kOffB2];
    for (int j = 0; j < kHid; ++j) {
        float a = ws[kOffB1 + j];
#pragma unroll
        for (int k = 0; k < kIn; ++k) a = fmaf(ws[j * kIn + k], x[k], a);
        const float h = fmaxf(a, 0.f);
        H[(int64_t)s * kHid + j] = h;
        dA[(int64_t)s * kHid + j] = a > 0.f ? 1.f : 0.f;  // ReLU mask, scaled below
        z = fmaf(ws[kOffW2 + j], h, z);
    }
    const float y = label[s];
    const float e = expf(-fabsf(z));
    const float sig = z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
    const float gs = (sig - y) / static_cast<float>(n);
    g[s] = gs;
    ls[s] = fmaxf(z, 0.f) - z * y + log1pf(e);
    for (int j = 0; j < kHid; ++j) dA[(int64_t)s * kHid + j] *= gs * ws[kOffW2 + j];
}

// Partial sums over one chunk of samples for every parameter (+ the loss),
// compensated (Kahan) summation in sample order.
__global__ void __launch_bounds__(128) chunk_reduce_kernel(const float *feat, const float *H, const float *dA,
                                                           const float *g, const float *ls, int n, float *part) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;  // parameter index, kP = the loss
    if (p > kP) return;
    const int s0 = blockIdx.y * kChunk, s1 = min(n, s0 + kChunk);
    float sum = 0.f, comp = 0.f;
    for (int s = s0; s < s1; ++s) {
        float t;
        if (p < kOffB1) {
            const int j = p / kIn, k = p - j * kIn;
            t = dA[(int64_t)s * kHid + j] * feat[(int64_t)s * kIn + k];
        } else if (p < kOffW2) {
            t = dA[(int64_t)s * kHid + (p - kOffB1)];
        } else if (p < kOffB2) {
            t = g[s] * H[(int64_t)s * kHid + (p - kOffW2)];
        } else if (p == kOffB2) {
            t = g[s];
        } else {
            t = ls[s];
        }
        const float yv = t - comp;
        const float tt = sum + yv;
        comp = (tt - sum) - yv;
        sum = tt;
    }
    part[(int64_t)blockIdx.y * (kP + 1) + p] = sum;
}

// Sum the chunk partials in chunk order; optionally apply Adam.
__global__ void __launch_bounds__(128) finish_kernel(const float *part, int nchunks, int n, float *grad, float *loss,
                                                     float *w, float *m, float *v, int t, mkf_adam hp, uint16_t *wb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kP) return;
    float sum = 0.f, comp = 0.f;
    for (int c = 0; c < nchunks; ++c) {
        const float yv = part[(int64_t)c * (kP + 1) + p] - comp;
        const float tt = sum + yv;
        comp = (tt - sum) - yv;
        sum = tt;
    }
    if (p == kP) {
        if (loss) *loss = sum / static_cast<float>(n);
        return;
    }
    if (grad) grad[p] = sum;
    if (w) {
        const float mm = hp.beta1 * m[p] + (1.f - hp.beta1) * sum;
        const float vv = hp.beta2 * v[p] + (1.f - hp.beta2) * sum * sum;
        m[p] = mm;
        v[p] = vv;
        const float mh = mm / (1.f - powf(hp.beta1, static_cast<float>(t)));
        const float vh = vv / (1.f - powf(hp.beta2, static_cast<float>(t)));
        const float nw = w[p] - hp.lr * mh / (sqrtf(vh) + hp.eps);
        w[p] = nw;
        wb[p] = to_bf16(nw);
    }
}

mkf_status run_grad(mkf_ctx *ctx, const uint16_t *wb, const float *feat, const float *label, int n, float *grad,
                    float *loss, float *w, float *m, float *v, int t, const mkf_adam *hp, uint16_t *wb_out) {
    const int nchunks = (n + kChunk - 1) / kChunk;
    const size_t floats = (size_t)n * kHid * 2 + (size_t)n * 2 + (size_t)nchunks * (kP + 1);
    void *scratch = nullptr;
    mkf_status st = mkf_scratch(ctx, floats * sizeof(float), &scratch);
    if (st != MKF_OK) return st;
    float *H = static_cast<float *>(scratch);
    float *dA = H + (size_t)n * kHid;
    float *g = dA + (size_t)n * kHid;
    float *ls = g + n;
    float *part = ls + n;
    cudaStream_t s = ctx->stream;
    sample_grad_kernel<<<(n + 127) / 128, 128, 0, s>>>(wb, feat, label, n, H, dA, g, ls);
    MKF_CUDA_TRY(cudaGetLastError());
    dim3 grid((kP + 1 + 127) / 128, nchunks);
    chunk_reduce_kernel<<<grid, 128, 0, s>>>(feat, H, dA, g, ls, n, part);
    MKF_CUDA_TRY(cudaGetLastError());
    mkf_adam h = hp ? *hp : mkf_adam{0.f, 0.f, 0.f, 0.f};
    finish_kernel<<<(kP + 1 + 127) / 128, 128, 0, s>>>(part, nchunks, n, grad, loss, w, m, v, t, h, wb_out);
    MKF_CUDA_TRY(cudaGetLastError());
    return MKF_OK;
}

}  // namespace

extern "C" mkf_status mkf_mlp_to_bf16(mkf_ctx *ctx, const float *w, uint16_t *w_bf16, int32_t n) {
    if (!ctx || n < 0 || (n > 0 && (!w || !w_bf16))) return MKF_ERR_ARG;
    if (n == 0) return MKF_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    to_bf16_kernel<<<(n + 255) / 256, 256, 0, ctx->stream>>>(w, w_bf16, n);
    MKF_CUDA_TRY(cudaGetLastError());
    return MKF_OK;
}

extern "C" mkf_status mkf_mlp_forward(mkf_ctx *ctx, const uint16_t *w_bf16, const float *feat, int32_t n,
                                      float *logit) {
    if (!ctx || !w_bf16 || n < 0 || (n > 0 && (!feat || !logit))) return MKF_ERR_ARG;
    if (n == 0) return MKF_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    forward_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(w_bf16, feat, n, logit);
    MKF_CUDA_TRY(cudaGetLastError());
    return MKF_OK;
}

extern "C" mkf_status mkf_mlp_grad(mkf_ctx *ctx, const uint16_t *w_bf16, const float *feat, const float *label,
                                   int32_t n, float *grad, float *loss) {
    if (!ctx || !w_bf16 || !feat || !label || !grad || n < 1) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    return run_grad(ctx, w_bf16, feat, label, n, grad, loss, nullptr, nullptr, nullptr, 0, nullptr, nullptr);
}

extern "C" mkf_status mkf_mlp_train_step(mkf_ctx *ctx, const float *feat, const float *label, int32_t n, float *w,
                                         float *m, float *v, int32_t t, const mkf_adam *hp, uint16_t *w_bf16,
                                         float *loss) {
    if (!ctx || !feat || !label || !w || !m || !v || !hp || !w_bf16 || n < 1 || t < 1) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    // bfloat16 copy of the current masters for the forward pass
    to_bf16_kernel<<<(MKF_MLP_PARAMS + 255) / 256, 256, 0, ctx->stream>>>(w, w_bf16, MKF_MLP_PARAMS);
    MKF_CUDA_TRY(cudaGetLastError());
    return run_grad(ctx, w_bf16, feat, label, n, nullptr, loss, w, m, v, t, hp, w_bf16);
}
