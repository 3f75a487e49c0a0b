// Host-side construction of the device geometry table (layer descriptors,
// bin layout, radius- and z-sorted layer lists, tracking regions) from the
// public layer and plan descriptions; no CUDA calls.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "mkf.h"
#include "mkf_math.cuh"

inline mkf_status mkf_build_geom(const mkf_layer *layers, int32_t n_layers, const mkf_plan *plans, int32_t n_plans,
                                 const float *region_eta_edges, float bz_tesla, mkf::Geom &G) {
    if (!layers || n_layers < 1) return MKF_ERR_ARG;
    if (n_layers > MKF_MAX_LAYERS) return MKF_ERR_CAPACITY;
    if (n_plans < 0) return MKF_ERR_ARG;
    if (n_plans > MKF_MAX_REGIONS) return MKF_ERR_CAPACITY;
    if (n_plans > 0 && !plans) return MKF_ERR_ARG;
    if (n_plans > 1 && !region_eta_edges) return MKF_ERR_ARG;
    if (!std::isfinite(bz_tesla)) return MKF_ERR_GEOMETRY;
    std::memset(&G, 0, sizeof(G));
    G.n_layers = n_layers;
    G.kb = mkf::kField * bz_tesla;
    G.field_kind = 0;  // the parameterised field comes from mkf_geometry_field
    G.alpha = 0.f;
    G.mat_map = nullptr;  // the r-z material map comes from mkf_geometry_material_map
    G.map_nr = G.map_nz = 0;
    G.map_rinv = G.map_zmin = G.map_zinv = 0.f;
    int64_t base = 0;
    for (int l = 0; l < n_layers; ++l) {
        const mkf_layer &s = layers[l];
        mkf::LayerDesc &d = G.L[l];
        if (s.kind != 0 && s.kind != 1) return MKF_ERR_GEOMETRY;
        if (!(std::isfinite(s.r_or_z) && std::isfinite(s.lo) && std::isfinite(s.hi) && s.hi > s.lo)) return MKF_ERR_GEOMETRY;
        if (s.kind == 0 && !(s.r_or_z > 0.f)) return MKF_ERR_GEOMETRY;
        if (s.kind == 1 && !(s.r_or_z != 0.f && s.lo >= 0.f)) return MKF_ERR_GEOMETRY;
        if (!(s.sigma_u > 0.f && s.sigma_v > 0.f && std::isfinite(s.sigma_u) && std::isfinite(s.sigma_v)))
            return MKF_ERR_GEOMETRY;
        if (s.n_phi_bins < 1 || s.n_phi_bins > 4096 || s.n_zr_bins < 1 || s.n_zr_bins > 4096) return MKF_ERR_GEOMETRY;
        d.kind = s.kind;
        d.rz = s.r_or_z;
        d.lo = s.lo;
        d.hi = s.hi;
        d.su2 = s.sigma_u * s.sigma_u;
        d.sv2 = s.sigma_v * s.sigma_v;
        float sig = 10.f * std::max(s.sigma_u, s.sigma_v);
        d.seed_sig2 = sig * sig;
        d.nphi = s.n_phi_bins;
        d.nzr = s.n_zr_bins;
        d.bin_base = static_cast<int>(base);
        d.phi_scale = static_cast<float>(s.n_phi_bins / (2.0 * M_PI));
        d.zr_scale = static_cast<float>(s.n_zr_bins / (static_cast<double>(s.hi) - s.lo));
        d.x0 = 0.f;  // material comes from mkf_geometry_material
        d.eloss = 0.f;
        base += static_cast<int64_t>(s.n_phi_bins) * s.n_zr_bins;
        if (base > (int64_t(1) << 26)) return MKF_ERR_CAPACITY;
    }
    G.bins_per_event = static_cast<int>(base);
    // sorted cylinder and disk lists
    int cyl[MKF_MAX_LAYERS], dsk[MKF_MAX_LAYERS], nc = 0, nd = 0;
    for (int l = 0; l < n_layers; ++l) {
        if (layers[l].kind == 0) cyl[nc++] = l;
        else dsk[nd++] = l;
    }
    std::stable_sort(cyl, cyl + nc, [&](int a, int b) { return layers[a].r_or_z < layers[b].r_or_z; });
    std::stable_sort(dsk, dsk + nd, [&](int a, int b) { return layers[a].r_or_z < layers[b].r_or_z; });
    G.n_cyl = nc;
    G.n_dsk = nd;
    for (int l = 0; l < MKF_MAX_LAYERS; ++l) G.cyl_pos[l] = G.dsk_pos[l] = -1;
    for (int i = 0; i < nc; ++i) {
        G.cyl[i] = static_cast<int8_t>(cyl[i]);
        G.cyl_pos[cyl[i]] = static_cast<int8_t>(i);
    }
    for (int i = 0; i < nd; ++i) {
        G.dsk[i] = static_cast<int8_t>(dsk[i]);
        G.dsk_pos[dsk[i]] = static_cast<int8_t>(i);
    }
    for (int i = nc - 1; i >= 0; --i) {
        const float hi = layers[cyl[i]].hi, lo = layers[cyl[i]].lo;
        G.cyl_hi_beyond[i] = (i == nc - 1) ? hi : std::max(hi, G.cyl_hi_beyond[i + 1]);
        G.cyl_lo_beyond[i] = (i == nc - 1) ? lo : std::min(lo, G.cyl_lo_beyond[i + 1]);
    }
    // regions
    unsigned long long all = n_layers == 64 ? ~0ull : ((1ull << n_layers) - 1ull);
    if (n_plans == 0) {
        G.n_regions = 1;
        G.mask[0] = all;
    } else {
        G.n_regions = n_plans;
        for (int r = 0; r < n_plans; ++r) {
            if (plans[r].n_layers < 0 || (plans[r].n_layers > 0 && !plans[r].layer_ids)) return MKF_ERR_ARG;
            unsigned long long m = 0;
            for (int k = 0; k < plans[r].n_layers; ++k) {
                int id = plans[r].layer_ids[k];
                if (id < 0 || id >= n_layers) return MKF_ERR_GEOMETRY;
                m |= 1ull << id;
            }
            G.mask[r] = m;
        }
        for (int r = 0; r + 1 < n_plans; ++r) {
            if (!std::isfinite(region_eta_edges[r])) return MKF_ERR_GEOMETRY;
            if (r > 0 && !(region_eta_edges[r] > region_eta_edges[r - 1])) return MKF_ERR_GEOMETRY;
            G.edges[r] = region_eta_edges[r];
        }
    }
    return MKF_OK;
}
