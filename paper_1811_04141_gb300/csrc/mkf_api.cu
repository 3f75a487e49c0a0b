// libmkf: context, geometry, status strings, synchronisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "mkf_geom.h"
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
    if (ctx->mat_map) cudaFree(ctx->mat_map);
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
    if (!ctx) return MKF_ERR_ARG;
    mkf::Geom G;  // the table builder checks every argument
    const mkf_status st = mkf_build_geom(layers, n_layers, plans, n_plans, region_eta_edges, bz_tesla, G);
    if (st != MKF_OK) return st;
    ctx->geom = G;
    ctx->has_geom = 1;
    ctx->geom_version++;
    return MKF_OK;
}

extern "C" mkf_status mkf_geometry_material(mkf_ctx *ctx, const float *x0, const float *eloss, int32_t n_layers) {
    if (!ctx) return MKF_ERR_ARG;
    if (!ctx->has_geom) return MKF_ERR_GEOMETRY;
    if (!x0 || n_layers != ctx->geom.n_layers) return MKF_ERR_ARG;
    for (int l = 0; l < n_layers; ++l) {
        if (!(x0[l] >= 0.f && x0[l] < 1.0e3f)) return MKF_ERR_GEOMETRY;
        if (eloss && !(eloss[l] >= 0.f && eloss[l] < 1.0e3f)) return MKF_ERR_GEOMETRY;
    }
    for (int l = 0; l < n_layers; ++l) {
        ctx->geom.L[l].x0 = x0[l];
        ctx->geom.L[l].eloss = eloss ? eloss[l] : 0.f;
    }
    return MKF_OK;
}

extern "C" mkf_status mkf_geometry_field(mkf_ctx *ctx, int32_t kind, float alpha) {
    if (!ctx) return MKF_ERR_ARG;
    if (kind != 0 && kind != 1) return MKF_ERR_ARG;
    if (!(fabsf(alpha) < 1.0e-2f)) return MKF_ERR_ARG;
    if (!ctx->has_geom) return MKF_ERR_GEOMETRY;
    ctx->geom.field_kind = kind;
    ctx->geom.alpha = kind == 1 ? alpha : 0.f;
    return MKF_OK;
}

extern "C" mkf_status mkf_geometry_material_map(mkf_ctx *ctx, int32_t nr, int32_t nz, float r_max, float z_min,
                                                float z_max, const float *x0, const float *eloss) {
    if (!ctx) return MKF_ERR_ARG;
    if (!ctx->has_geom) return MKF_ERR_GEOMETRY;
    if (nr == 0 && nz == 0) {  // back to the layers' own material
        ctx->geom.mat_map = nullptr;
        ctx->geom.map_nr = ctx->geom.map_nz = 0;
        return MKF_OK;
    }
    if (nr < 1 || nz < 1 || nr > 4096 || nz > 4096 || static_cast<int64_t>(nr) * nz > (1 << 20)) return MKF_ERR_ARG;
    if (!x0 || !(r_max > 0.f && r_max < 1.0e6f) || !(z_max > z_min) || !(z_min > -1.0e6f && z_max < 1.0e6f))
        return MKF_ERR_ARG;
    const size_t cells = static_cast<size_t>(nr) * nz;
    std::vector<float2> h(cells);
    for (size_t i = 0; i < cells; ++i) {
        if (!(x0[i] >= 0.f && x0[i] < 1.0e3f)) return MKF_ERR_GEOMETRY;
        if (eloss && !(eloss[i] >= 0.f && eloss[i] < 1.0e3f)) return MKF_ERR_GEOMETRY;
        h[i] = make_float2(x0[i], eloss ? eloss[i] : 0.f);
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    if (cells > ctx->mat_map_cells) {
        if (ctx->mat_map) {
            MKF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            MKF_CUDA_TRY(cudaFree(ctx->mat_map));
            ctx->mat_map = nullptr;
            ctx->mat_map_cells = 0;
        }
        MKF_CUDA_TRY(cudaMalloc(&ctx->mat_map, cells * sizeof(float2)));
        ctx->mat_map_cells = cells;
    }
    // kernels queued before this call may still read the previous map
    MKF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    MKF_CUDA_TRY(cudaMemcpy(ctx->mat_map, h.data(), cells * sizeof(float2), cudaMemcpyHostToDevice));
    ctx->geom.mat_map = ctx->mat_map;
    ctx->geom.map_nr = nr;
    ctx->geom.map_nz = nz;
    ctx->geom.map_rinv = static_cast<float>(nr) / r_max;
    ctx->geom.map_zmin = z_min;
    ctx->geom.map_zinv = static_cast<float>(nz) / (z_max - z_min);
    return MKF_OK;
}
