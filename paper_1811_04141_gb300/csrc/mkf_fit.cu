// Track fit along fixed hit lists: one thread per track, state and covariance in
// registers for the whole hit list (Sec. 1: Kalman-filter fitting), and the
// backward fit, the same filter through the hits in reverse order.
#include <cuda_runtime.h>

#include "mkf_internal.h"

namespace {

using namespace mkf;

struct FitArgs {
    Geom G;
    const float *X, *Y, *Z;
    const int32_t *hit_layer;
    int32_t n_hits;
    const int32_t *hit_idx;
    int32_t max_hits, n;
    const float *seed_par, *seed_cov;
    float inflate;  // backward fit: factor on the starting covariance
    float *out_par, *out_cov, *chi2;
    int32_t *ndf;
    uint32_t *status;
    mkf_fault *fault;
};

__device__ __forceinline__ void record_fault(mkf_fault *f, int code, int where) {
    if (atomicCAS(&f->code, 0, code) == 0) f->where = where;
}

// The helix traversed the other way: the same curve with the momentum turned
// around, p -> (x, y, z, -q/pT, phi + pi, pi - theta) with pi as a float pair,
// and C -> F C F with F = diag(1, 1, 1, -1, 1, -1) (the covariances between
// {q/pT, theta} and the other parameters change sign).
__device__ __forceinline__ void reverse_state(float p[6], Lo &lo, float C[21]) {
    constexpr float kPiHi = 3.14159274101257324219f;  // float(pi)
    constexpr float kPiLo = -8.74227765734758e-8f;    // pi - float(pi)
    p[3] = -p[3];
    df_add(p[4], lo.phi, kPiHi);
    df_add(p[4], lo.phi, kPiLo);
    df_wrap_pi(p[4], lo.phi);
    p[5] = (kPiHi - p[5]) + kPiLo;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j)
            if ((i == 3 || i == 5) != (j == 3 || j == 5)) C[sym(i, j)] = -C[sym(i, j)];
}

// kBackward: hits in reverse order from the given state at the last hit, turned
// around and inflated; the result at the first hit is turned back.  kPhys: 0
// uniform field without material; 1 material effects compiled in (selected
// when any layer has material); 2 the parameterised field (Runge-Kutta
// propagation) with the material effects.
template <bool kBackward, int kPhys>
__global__ void __launch_bounds__(128, kPhys == 2 ? 4 : 8) fit_kernel(const __grid_constant__ FitArgs A) {
    constexpr bool kMaterial = kPhys >= 1, kParamField = kPhys == 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.n) return;
    const Geom &G = A.G;
    float p[6], C[21];
    Lo lo{0.f, 0.f, 0.f, 0.f};
    uint32_t st = 0;
    float chi2 = 0.f;
    int used = 0;

    // first three valid hits (seed) and validity of all indices
    int first[3] = {-1, -1, -1}, nfirst = 0;
    for (int k = 0; k < A.max_hits; ++k) {
        int h = A.hit_idx[(int64_t)k * A.n + t];
        if (h < 0) continue;
        if (h >= A.n_hits) {
            record_fault(A.fault, kFaultBadHitIndex, t);
            continue;
        }
        if (nfirst < 3) first[nfirst++] = h;
    }
    bool ok = nfirst >= 3;
    if (ok) {
        int l0 = A.hit_layer[first[0]];
        if (l0 < 0 || l0 >= G.n_layers) {
            record_fault(A.fault, kFaultBadLayer, first[0]);
            ok = false;
        } else if (A.seed_par) {
#pragma unroll
            for (int i = 0; i < 6; ++i) p[i] = A.seed_par[(int64_t)i * A.n + t];
#pragma unroll
            for (int k = 0; k < 21; ++k) C[k] = A.seed_cov[(int64_t)k * A.n + t];
            if (kBackward) {
                reverse_state(p, lo, C);
#pragma unroll
                for (int k = 0; k < 21; ++k) C[k] *= A.inflate;
            }
        } else {
            float h1[3], h2[3], h3[3], eta;
            h1[0] = A.X[first[0]]; h1[1] = A.Y[first[0]]; h1[2] = A.Z[first[0]];
            h2[0] = A.X[first[1]]; h2[1] = A.Y[first[1]]; h2[2] = A.Z[first[1]];
            h3[0] = A.X[first[2]]; h3[1] = A.Y[first[2]]; h3[2] = A.Z[first[2]];
            // the parameterised field at the middle hit sets the curvature scale
            const float kbs = kParamField ? G.kb * bz_factor(G.alpha, h2[0], h2[1], h2[2]) : G.kb;
            ok = seed_state(G.L[l0], kbs, h1, h2, h3, p, C, eta);
        }
    }
    if (!ok) st |= MKF_ST_BADSEED;

    if (ok) {
        bool firsthit = true;
        for (int kk = 0; kk < A.max_hits; ++kk) {
            const int k = kBackward ? A.max_hits - 1 - kk : kk;
            const int h = A.hit_idx[(int64_t)k * A.n + t];
            if (h < 0 || h >= A.n_hits) continue;
            const int l = A.hit_layer[h];
            if (l < 0 || l >= G.n_layers) {
                record_fault(A.fault, kFaultBadLayer, h);
                continue;
            }
            const LayerDesc &Ld = G.L[l];
            const float xh = A.X[h], yh = A.Y[h], zh = A.Z[h];
            if (!firsthit) {
                float sphi, cphi;
                sincos_pair(p[4], lo.phi, sphi, cphi);
                const float cot = cot_of(p[5]);
                // path estimate from the helix in the local axial field
                const float kbl = kParamField ? G.kb * bz_factor(G.alpha, p[0], p[1], p[2]) : G.kb;
                float s;
                if (!path_to_layer(Ld, kbl, p, lo, sphi, cphi, cot, s)) {
                    st |= MKF_ST_UNREACHABLE;
                    continue;
                }
                if (kParamField)
                    propagate_field(Ld, G.kb, G.alpha, p, lo, C, sphi, cphi, -p[3] * kbl, s);
                else
                    propagate_transport(Ld, G.kb, p, lo, C, sphi, cphi, cot, s);
                if (!kBackward && kMaterial) {
                    float mx0, mk;
                    material_at(G, Ld, p, mx0, mk);
                    add_scattering(Ld.kind, mx0, p, C);
                    apply_eloss(Ld.kind, mx0, mk, p, C, 1.f);
                }
            }
            firsthit = false;
            const Frame f = frame_of(p);
            Innov I;
            if (innovation(Ld.kind, Ld.su2, Ld.sv2, f, C, I)) {
                float u, v;
                const float zr = Ld.kind == 0 ? zh : sqrtf(fmaf(xh, xh, yh * yh));
                residual(Ld.kind, Ld.rz, p, lo, f, xh, yh, zr, u, v);
                chi2 += chi2_of(I, u, v);
                kf_apply(I, u, v, p, lo, C);
                ++used;
            } else {
                st |= MKF_ST_BADS;
            }
            // reversed in time a layer's material follows its hit (at every hit,
            // the last one included): the energy lost there is gained back, then
            // the scattering noise is added
            if (kBackward && kMaterial) {
                float mx0, mk;
                material_at(G, Ld, p, mx0, mk);
                apply_eloss(Ld.kind, mx0, mk, p, C, -1.f);
                add_scattering(Ld.kind, mx0, p, C);
            }
        }
        if (kBackward) reverse_state(p, lo, C);
        if (!finite_state(p) || !isfinite(chi2)) st |= MKF_ST_NONFINITE;
    }
    const float nanv = __int_as_float(0x7fc00000);
    p[0] += lo.x;
    p[1] += lo.y;
    p[2] += lo.z;
    p[4] += lo.phi;
#pragma unroll
    for (int i = 0; i < 6; ++i) A.out_par[(int64_t)i * A.n + t] = ok ? p[i] : nanv;
#pragma unroll
    for (int k = 0; k < 21; ++k) A.out_cov[(int64_t)k * A.n + t] = ok ? C[k] : nanv;
    A.chi2[t] = chi2;
    A.ndf[t] = 2 * used - (G.kb != 0.f ? 5 : 4);
    A.status[t] = st;
}

}  // namespace

static mkf_status launch_fit(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits,
                             const int32_t *hit_idx, int32_t max_hits, int32_t n, const float *seed_par,
                             const float *seed_cov, float inflate, bool backward, float *out_par, float *out_cov,
                             float *chi2, int32_t *ndf, uint32_t *status) {
    if (!ctx) return MKF_ERR_ARG;
    if (!ctx->has_geom) return MKF_ERR_GEOMETRY;
    if (n < 0 || n_hits < 0 || max_hits < 1) return MKF_ERR_ARG;
    if (max_hits > MKF_MAX_LAYERS) return MKF_ERR_CAPACITY;
    if (n_hits > MKF_MAX_HITS) return MKF_ERR_CAPACITY;
    if ((seed_par == nullptr) != (seed_cov == nullptr)) return MKF_ERR_ARG;
    if (backward && !(inflate >= 1.f && inflate < 3.0e38f)) return MKF_ERR_ARG;
    if (n == 0) return MKF_OK;
    if (!xyz || !hit_layer || !hit_idx || !out_par || !out_cov || !chi2 || !ndf || !status) return MKF_ERR_ARG;
    if (backward && !seed_par) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    FitArgs A;
    A.G = ctx->geom;
    A.X = xyz;
    A.Y = xyz + n_hits;
    A.Z = xyz + 2 * (int64_t)n_hits;
    A.hit_layer = hit_layer;
    A.n_hits = n_hits;
    A.hit_idx = hit_idx;
    A.max_hits = max_hits;
    A.n = n;
    A.seed_par = seed_par;
    A.seed_cov = seed_cov;
    A.inflate = inflate;
    A.out_par = out_par;
    A.out_cov = out_cov;
    A.chi2 = chi2;
    A.ndf = ndf;
    A.status = status;
    A.fault = ctx->fault;
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    switch (mkf_phys_variant(ctx->geom) + (backward ? 3 : 0)) {
        case 0: fit_kernel<false, 0><<<blocks, threads, 0, ctx->stream>>>(A); break;
        case 1: fit_kernel<false, 1><<<blocks, threads, 0, ctx->stream>>>(A); break;
        case 2: fit_kernel<false, 2><<<blocks, threads, 0, ctx->stream>>>(A); break;
        case 3: fit_kernel<true, 0><<<blocks, threads, 0, ctx->stream>>>(A); break;
        case 4: fit_kernel<true, 1><<<blocks, threads, 0, ctx->stream>>>(A); break;
        default: fit_kernel<true, 2><<<blocks, threads, 0, ctx->stream>>>(A); break;
    }
    MKF_CUDA_TRY(cudaGetLastError());
    return MKF_OK;
}

extern "C" mkf_status mkf_fit(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits,
                              const int32_t *hit_idx, int32_t max_hits, int32_t n, const float *seed_par,
                              const float *seed_cov, float *out_par, float *out_cov, float *chi2, int32_t *ndf,
                              uint32_t *status) {
    return launch_fit(ctx, xyz, hit_layer, n_hits, hit_idx, max_hits, n, seed_par, seed_cov, 1.f, false, out_par,
                      out_cov, chi2, ndf, status);
}

extern "C" mkf_status mkf_fit_backward(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits,
                                       const int32_t *hit_idx, int32_t max_hits, int32_t n, const float *last_par,
                                       const float *last_cov, float inflate, float *out_par, float *out_cov,
                                       float *chi2, int32_t *ndf, uint32_t *status) {
    return launch_fit(ctx, xyz, hit_layer, n_hits, hit_idx, max_hits, n, last_par, last_cov, inflate, true, out_par,
                      out_cov, chi2, ndf, status);
}
