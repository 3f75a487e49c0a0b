// FP32 throughput probe: the denominator of the finder's and the fit's
// roofline.  The paper has no counterpart (it reports no roofline); the
// Kalman-filter kernels are bound by the FP32 pipe, whose peak the driver's
// measured peaks do not include.
//
// Every thread runs kChains independent dependent-FMA chains x <- x * a + b for
// `iters` rounds.  With 8 chains per thread and 8 warps per scheduler the FMA
// latency is covered, so the SMs issue one FP32 FMA per lane per cycle.
#include <cuda_runtime.h>

#include "mkf_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) fma_chains_kernel(int32_t iters, float a, float b, float *out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = static_cast<float>(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // a result that depends on every chain keeps the compiler from removing them
    if (s == 1.2345f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" mkf_status mkf_fp32_probe(mkf_ctx *ctx, int32_t iters, float *out, double *flops) {
    if (!ctx || iters < 1 || !out || !flops) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    const int blocks = ctx->num_sms * kBlocksPerSm;
    // a = 1 - 2^-20 and b = 2^-20 keep every chain in [0, 1): no overflow, no denormals
    fma_chains_kernel<<<blocks, kThreads, 0, ctx->stream>>>(iters, 0.99999904632568359375f,
                                                           9.5367431640625e-7f, out);
    MKF_CUDA_TRY(cudaGetLastError());
    *flops = 2.0 * kChains * 16.0 * static_cast<double>(iters) * blocks * kThreads;
    return MKF_OK;
}
