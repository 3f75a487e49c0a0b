// Host run of the fit kernel (tests only): the kernel of mkf_fit.cu, compiled
// for the host, called once per thread of its grid; the geometry table comes
// from the library's own builder, with the layers' material and the field set
// as mkf_geometry_material and mkf_geometry_field set them.
#include <cmath>
#include <cstdint>
#include <vector>

#include "warp_emu.h"
thread_local dim3 threadIdx, blockIdx;
dim3 blockDim;

#include "fit_dev.inc"
#include "mkf_geom.h"

extern "C" int emu_fit(const mkf_layer *layers, int nl, float bz, const float *x0, const float *eloss, int field_kind,
                       float alpha, int map_nr, int map_nz, float map_rmax, float map_zmin,
                       float map_zmax, const float *map_x0, const float *map_eloss, const float *xyz,
                       const int32_t *hit_layer, int32_t n_hits, const int32_t *hit_idx, int32_t max_hits, int32_t n,
                       const float *seed_par, const float *seed_cov, int backward, float inflate, float *out_par,
                       float *out_cov, float *chi2, int32_t *ndf, uint32_t *status) {
    FitArgs A;
    if (mkf_build_geom(layers, nl, nullptr, 0, nullptr, bz, A.G) != MKF_OK) return -1;
    for (int l = 0; l < nl; ++l) {
        A.G.L[l].x0 = x0 ? x0[l] : 0.f;
        A.G.L[l].eloss = eloss ? eloss[l] : 0.f;
    }
    A.G.field_kind = field_kind;
    A.G.alpha = field_kind ? alpha : 0.f;
    std::vector<float2> mapv;
    if (map_nr > 0) {  // as mkf_geometry_material_map sets it
        mapv.resize(static_cast<size_t>(map_nr) * map_nz);
        for (size_t i = 0; i < mapv.size(); ++i) mapv[i] = make_float2(map_x0[i], map_eloss ? map_eloss[i] : 0.f);
        A.G.mat_map = mapv.data();
        A.G.map_nr = map_nr;
        A.G.map_nz = map_nz;
        A.G.map_rinv = static_cast<float>(map_nr) / map_rmax;
        A.G.map_zmin = map_zmin;
        A.G.map_zinv = static_cast<float>(map_nz) / (map_zmax - map_zmin);
    }
    const int phys = mkf_phys_variant(A.G);
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
        switch (phys + (backward ? 3 : 0)) {
            case 0: fit_kernel<false, 0>(A); break;
            case 1: fit_kernel<false, 1>(A); break;
            case 2: fit_kernel<false, 2>(A); break;
            case 3: fit_kernel<true, 0>(A); break;
            case 4: fit_kernel<true, 1>(A); break;
            default: fit_kernel<true, 2>(A); break;
        }
    }
    return fault.code;
}

// The smoother kernel of mkf_fit.cu run thread by thread (geometry, material,
// map and field as emu_fit).
extern "C" int emu_smooth(const mkf_layer *layers, int nl, float bz, const float *x0, const float *eloss,
                          int field_kind, float alpha, int map_nr, int map_nz, float map_rmax, float map_zmin,
                          float map_zmax, const float *map_x0, const float *map_eloss, const float *xyz,
                          const int32_t *hit_layer, int32_t n_hits, const int32_t *hit_idx, int32_t max_hits, int32_t n,
                          float inflate, float *sm_par, float *sm_cov, float *chi2, int32_t *ndf, uint32_t *status) {
    FitArgs A;
    if (mkf_build_geom(layers, nl, nullptr, 0, nullptr, bz, A.G) != MKF_OK) return -1;
    for (int l = 0; l < nl; ++l) {
        A.G.L[l].x0 = x0 ? x0[l] : 0.f;
        A.G.L[l].eloss = eloss ? eloss[l] : 0.f;
    }
    A.G.field_kind = field_kind;
    A.G.alpha = field_kind ? alpha : 0.f;
    std::vector<float2> mapv;
    if (map_nr > 0) {
        mapv.resize(static_cast<size_t>(map_nr) * map_nz);
        for (size_t i = 0; i < mapv.size(); ++i) mapv[i] = make_float2(map_x0[i], map_eloss ? map_eloss[i] : 0.f);
        A.G.mat_map = mapv.data();
        A.G.map_nr = map_nr;
        A.G.map_nz = map_nz;
        A.G.map_rinv = static_cast<float>(map_nr) / map_rmax;
        A.G.map_zmin = map_zmin;
        A.G.map_zinv = static_cast<float>(map_nz) / (map_zmax - map_zmin);
    }
    const int phys = mkf_phys_variant(A.G);
    mkf_fault fault{0, 0};
    A.X = xyz;
    A.Y = xyz + n_hits;
    A.Z = xyz + 2 * (int64_t)n_hits;
    A.hit_layer = hit_layer;
    A.n_hits = n_hits;
    A.hit_idx = hit_idx;
    A.max_hits = max_hits;
    A.n = n;
    A.seed_par = nullptr;
    A.seed_cov = nullptr;
    A.inflate = inflate;
    A.out_par = nullptr;
    A.out_cov = nullptr;
    A.sm_par = sm_par;
    A.sm_cov = sm_cov;
    A.chi2 = chi2;
    A.ndf = ndf;
    A.status = status;
    A.fault = &fault;
    blockDim.x = 128;
    for (int t = 0; t < (n + 127) / 128 * 128; ++t) {
        blockIdx.x = t / 128;
        threadIdx.x = t % 128;
        if (phys == 0) smooth_kernel<0>(A);
        else if (phys == 1) smooth_kernel<1>(A);
        else smooth_kernel<2>(A);
    }
    return fault.code;
}

// The smoother's weighted mean of two estimates on a surface (combine5), for
// unit tests of its arithmetic.
extern "C" int emu_combine5(int kind, float rz, const float *pf, const float *Cf, const float *pb, const float *Cb,
                            float *ps, float *Cs) {
    return combine5(kind, rz, pf, Cf, pb, Cb, ps, Cs) ? 1 : 0;
}
