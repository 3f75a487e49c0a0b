// libmkf: context, geometry, status strings, synchronisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "mkf_internal.h"

extern "C" const char *mkf_status_string(mkf_status s) {
    switch (s) {
        case MKF_OK: return "ok";
        case MKF_ERR_ARG: return "invalid argument";
        case MKF_ERR_GEOMETRY: return "invalid or missing geometry";
        case MKF_ERR_CAPACITY: return "size exceeds a library maximum";
        case MKF_ERR_CUDA: return "CUDA runtime error";
        case MKF_ERR_DEVICE_CHECK: return "invalid device input detected by a kernel";
        default: return "unknown status";
    }
}

extern "C" mkf_status mkf_create(mkf_ctx **out, int32_t cuda_device, void *cuda_stream) {
    if (!out) return MKF_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return MKF_ERR_CUDA;
    if (cuda_device < 0 || cuda_device >= ndev) return MKF_ERR_ARG;
    DeviceGuard g(cuda_device);
    if (!g.ok) return MKF_ERR_CUDA;
    mkf_ctx *c = new (std::nothrow) mkf_ctx;
    if (!c) return MKF_ERR_CUDA;
    std::memset(c, 0, sizeof(*c));
    c->device = cuda_device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMalloc(&c->fault, sizeof(mkf_fault)) != cudaSuccess) {
        delete c;
        return MKF_ERR_CUDA;
    }
    if (cudaMemset(c->fault, 0, sizeof(mkf_fault)) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, cuda_device) != cudaSuccess) {
        cudaFree(c->fault);
        delete c;
        return MKF_ERR_CUDA;
    }
    *out = c;
    return MKF_OK;
}

extern "C" void mkf_destroy(mkf_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->fault);
    if (ctx->scratch) cudaFree(ctx->scratch);
    delete ctx;
}

extern "C" mkf_status mkf_set_stream(mkf_ctx *ctx, void *cuda_stream) {
    if (!ctx) return MKF_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return MKF_OK;
}

extern "C" mkf_status mkf_sync(mkf_ctx *ctx) {
    if (!ctx) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    mkf_fault f;
    MKF_CUDA_TRY(cudaMemcpyAsync(&f, ctx->fault, sizeof(f), cudaMemcpyDeviceToHost, ctx->stream));
    MKF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    MKF_CUDA_TRY(cudaGetLastError());
    if (f.code != 0) {
        MKF_CUDA_TRY(cudaMemsetAsync(ctx->fault, 0, sizeof(mkf_fault), ctx->stream));
        MKF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        return MKF_ERR_DEVICE_CHECK;
    }
    return MKF_OK;
}

mkf_status mkf_scratch(mkf_ctx *ctx, size_t bytes, void **out) {
    if (bytes > ctx->scratch_bytes) {
        if (ctx->scratch) {
            MKF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            MKF_CUDA_TRY(cudaFree(ctx->scratch));
            ctx->scratch = nullptr;
            ctx->scratch_bytes = 0;
        }
        size_t b = std::max<size_t>(bytes, 1 << 20);
        MKF_CUDA_TRY(cudaMalloc(&ctx->scratch, b));
        ctx->scratch_bytes = b;
    }
    *out = ctx->scratch;
    return MKF_OK;
}

extern "C" mkf_status mkf_geometry_load(mkf_ctx *ctx, const mkf_layer *layers, int32_t n_layers, const mkf_plan *plans,
                                        int32_t n_plans, const float *region_eta_edges, float bz_tesla) {
    if (!ctx || !layers) return MKF_ERR_ARG;
    if (n_layers < 1) return MKF_ERR_ARG;
    if (n_layers > MKF_MAX_LAYERS) return MKF_ERR_CAPACITY;
    if (n_plans < 0) return MKF_ERR_ARG;
    if (n_plans > MKF_MAX_REGIONS) return MKF_ERR_CAPACITY;
    if (n_plans > 0 && !plans) return MKF_ERR_ARG;
    if (n_plans > 1 && !region_eta_edges) return MKF_ERR_ARG;
    if (!std::isfinite(bz_tesla)) return MKF_ERR_GEOMETRY;
    mkf::Geom G;
    std::memset(&G, 0, sizeof(G));
    G.n_layers = n_layers;
    G.kb = mkf::kField * bz_tesla;
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
    ctx->geom = G;
    ctx->has_geom = 1;
    ctx->geom_version++;
    return MKF_OK;
}
