// Host-side internals of libmkf: context, bin store, error plumbing.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "mkf.h"
#include "mkf_math.cuh"

// Device fault record written by kernels (bounds and input checks); read and
// cleared by mkf_sync.
struct mkf_fault {
    int code;   // 0 = none, else a kernel-specific code
    int where;  // index of the offending element
};

enum : int {
    kFaultBadLayer = 1,       // hit with a layer id outside the geometry
    kFaultBadEvent = 2,       // hit outside the event offsets
    kFaultBadSeedHit = 3,     // seed hit index out of range
    kFaultHistOverflow = 4,   // candidate history longer than reserved
    kFaultBadHitIndex = 5,    // fit hit index out of range
    kFaultBadSeedList = 6,    // finder seed-list entry out of range
};

struct mkf_ctx {
    int device;
    cudaStream_t stream;
    int has_geom;
    uint32_t geom_version;
    mkf::Geom geom;
    mkf_fault *fault;  // device, one record
    // reusable scratch owned by the context
    void *scratch;
    size_t scratch_bytes;
    int num_sms;
    int find_smem_attr;  // dynamic shared memory the find kernel is configured for
    // cached occupancy per finder variant: (plain, learned) x (uniform field,
    // material, parameterised field) x (beam width at run time, 1, 10)
    int find_occ_threads[18], find_occ_smem[18], find_occ_blocks[18];
    // r-z material map in device memory (geom.mat_map points here when loaded)
    float2 *mat_map;
    size_t mat_map_cells;
};

struct mkf_hitbins {
    int device;
    uint32_t geom_version;
    int32_t n_hits, n_events;
    int64_t n_bins;
    // capacities
    int64_t cap_hits, cap_bins;
    float4 *rec;        // [n_hits] binned hits: x, y, z-or-r, original index (int bits)
    int32_t *inv;       // [n_hits] original index -> binned position
    uint8_t *layer;     // [n_hits] layer of each original hit
    float *zhit;        // [n_hits] z of each original hit (seeds on disks need it)
    int32_t *key;       // [n_hits] bin of each original hit (-1 if dropped)
    int32_t *offsets;   // [n_bins + 1] CSR offsets of the bins
    int32_t *counts;    // [n_bins] scratch histogram
    int64_t zero_bins;  // counts[0, zero_bins) hold zero between calls
    int32_t *blocksums; // scan scratch
    int64_t cap_blocks;
    int ordered;        // hits within each bin in ascending original index
};

#define MKF_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return MKF_ERR_CUDA;         \
    } while (0)

// Make the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Context scratch of at least `bytes` (grown with cudaMalloc, never shrunk).
mkf_status mkf_scratch(mkf_ctx *ctx, size_t bytes, void **out);

// Physics variant of the kernels for a geometry: 2 parameterised field (with
// the material effects compiled in), 1 material in some layer, 0 neither.
inline int mkf_phys_variant(const mkf::Geom &G) {
    if (G.field_kind == 1) return 2;
    if (G.mat_map) return 1;
    for (int l = 0; l < G.n_layers; ++l)
        if (G.L[l].x0 > 0.f) return 1;
    return 0;
}

// Exclusive scan of counts [n] into offsets [n + 1] (offsets[n] = the total),
// enqueued on `s`; tilesums is scratch of mkf_scan_tilesums(n) ints.
int64_t mkf_scan_tilesums(int64_t n);
mkf_status mkf_run_scan(cudaStream_t s, const int32_t *counts, int64_t n, int32_t *tilesums, int32_t *offsets);
