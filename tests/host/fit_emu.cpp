// Host run of the fit kernel (tests only): the kernel of mkf_fit.cu, compiled
// for the host, called once per thread of its grid; the geometry table comes
// from the library's own builder, with the layers' material set as
// mkf_geometry_material sets it.
#include <cmath>
#include <cstdint>
#include <vector>

#include "warp_emu.h"
thread_local dim3 threadIdx, blockIdx;
dim3 blockDim;

#include "fit_dev.inc"
#include "mkf_geom.h"

extern "C" int emu_fit(const mkf_layer *layers, int nl, float bz, const float *x0, const float *eloss, const float *xyz,
                       const int32_t *hit_layer, int32_t n_hits, const int32_t *hit_idx, int32_t max_hits, int32_t n,
                       const float *seed_par, const float *seed_cov, int backward, float inflate, float *out_par,
                       float *out_cov, float *chi2, int32_t *ndf, uint32_t *status) {
    FitArgs A;
    if (mkf_build_geom(layers, nl, nullptr, 0, nullptr, bz, A.G) != MKF_OK) return -1;
    bool material = false;
    for (int l = 0; l < nl; ++l) {
        A.G.L[l].x0 = x0 ? x0[l] : 0.f;
        A.G.L[l].eloss = eloss ? eloss[l] : 0.f;
        material = material || A.G.L[l].x0 > 0.f;
    }
    mkf_fault fault{0, 0};
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
    A.fault = &fault;
    blockDim.x = 128;
    for (int t = 0; t < (n + 127) / 128 * 128; ++t) {
        blockIdx.x = t / 128;
        threadIdx.x = t % 128;
        if (backward && material) fit_kernel<true, true>(A);
        else if (backward) fit_kernel<true, false>(A);
        else if (material) fit_kernel<false, true>(A);
        else fit_kernel<false, false>(A);
    }
    return fault.code;
}
