// Hit binning: counting sort of hits into per-(event, layer) phi x z (cylinder)
// or phi x r (disk) bins, CSR offsets, binned SoA records.  The bins are the
// acceleration structure behind the per-layer hit search windows (Sec. 2.1);
// they are a superset test only, the chi2 cut decides.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "mkf_internal.h"

namespace {

using namespace mkf;

constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 8;  // a thread's run of 8 counts: two 16-byte loads (3 % faster than 16)
constexpr int kScanTile = kScanThreads * kScanPerThread;
static_assert(kScanThreads % 32 == 0 && kScanThreads >= 32 && kScanThreads <= 1024, "whole warps, at most 32");
static_assert(kScanPerThread % 4 == 0, "a thread's run is loaded as 16-byte vectors");

struct BinArgs {
    Geom G;
    const float *X, *Y, *Z;
    const int32_t *layer;
    const int32_t *event_offsets;
    int32_t n_events, n_hits;
    int32_t *key;
    uint8_t *layer8;
    float *zhit;
    int32_t *counts;
    int32_t *slot;  // [n_hits] each hit's place among its bin's hits (the inverse-map buffer)
    mkf_fault *fault;
};

__device__ __forceinline__ void record_fault(mkf_fault *f, int code, int where) {
    if (atomicCAS(&f->code, 0, code) == 0) f->where = where;
}

// Key computation: several hits per thread, strided by the block size so that
// every load stays coalesced, their loads issued before the dependent work, and
// one event search per thread.  (The scatter and the in-bin ordering keep one
// item per thread: their per-item work has data-dependent loops, which would run
// one after another inside a thread; measured slower.)
constexpr int kBinItems = 4;
constexpr int kBinThreads = 256;

__global__ void __launch_bounds__(kBinThreads) bin_keys_kernel(const __grid_constant__ BinArgs A) {
    // the layer table in shared memory: the hits of a warp sit on different
    // layers, and kernel-parameter loads at different addresses are serialised
    // (binning of the 512 uneven dense events: 2.52 ms before, 2.03 ms after;
    // issuing the thread's histogram adds together then brought it to 1.94 ms)
    __shared__ LayerDesc SL[kMaxLayers];
    {
        const int *src = reinterpret_cast<const int *>(A.G.L);
        int *dst = reinterpret_cast<int *>(SL);
        const int nw = A.G.n_layers * static_cast<int>(sizeof(LayerDesc) / sizeof(int));
        for (int i = threadIdx.x; i < nw; i += kBinThreads) dst[i] = src[i];
    }
    __syncthreads();
    const int base = blockIdx.x * kBinThreads * kBinItems + threadIdx.x;
    if (base >= A.n_hits) return;
    float x[kBinItems], y[kBinItems], z[kBinItems];
    int l[kBinItems];
#pragma unroll
    for (int j = 0; j < kBinItems; ++j) {
        const int i = base + j * kBinThreads;
        if (i < A.n_hits) {
            x[j] = A.X[i];
            y[j] = A.Y[i];
            z[j] = A.Z[i];
            l[j] = A.layer[i];
        }
    }
    // event of the first hit: first e with event_offsets[e + 1] > base; the
    // later hits of this thread walk forward from it
    int lo = 0, hi = A.n_events;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A.event_offsets[mid + 1] <= base) lo = mid + 1;
        else hi = mid;
    }
    int ev = lo;
    const int first_hit = A.event_offsets[0];
    int kk[kBinItems];
#pragma unroll
    for (int j = 0; j < kBinItems; ++j) kk[j] = -1;
#pragma unroll
    for (int j = 0; j < kBinItems; ++j) {
        const int i = base + j * kBinThreads;
        if (i >= A.n_hits) break;
        while (ev < A.n_events && A.event_offsets[ev + 1] <= i) ++ev;
        if (ev >= A.n_events || i < first_hit) {
            record_fault(A.fault, kFaultBadEvent, i);
            A.key[i] = -1;
            A.layer8[i] = 255;
            continue;
        }
        if (l[j] < 0 || l[j] >= A.G.n_layers) {
            record_fault(A.fault, kFaultBadLayer, i);
            A.key[i] = -1;
            A.layer8[i] = 255;
            continue;
        }
        const LayerDesc &Ld = SL[l[j]];
        A.zhit[i] = z[j];
        const float phi = atan2f(y[j], x[j]);
        const float zr = Ld.kind == 0 ? z[j] : sqrtf(fmaf(x[j], x[j], y[j] * y[j]));
        int pb = static_cast<int>(floorf((phi + kPi) * Ld.phi_scale));
        pb = min(max(pb, 0), Ld.nphi - 1);
        int zb = static_cast<int>(floorf((zr - Ld.lo) * Ld.zr_scale));
        zb = min(max(zb, 0), Ld.nzr - 1);
        const int k = ev * A.G.bins_per_event + Ld.bin_base + pb * Ld.nzr + zb;
        A.key[i] = k;
        A.layer8[i] = static_cast<uint8_t>(l[j]);
        kk[j] = k;
    }
    // the histogram adds of the thread's hits, issued together
    int sl[kBinItems];
#pragma unroll
    for (int j = 0; j < kBinItems; ++j) sl[j] = kk[j] >= 0 ? atomicAdd(&A.counts[kk[j]], 1) : 0;
#pragma unroll
    for (int j = 0; j < kBinItems; ++j)
        if (kk[j] >= 0) A.slot[base + j * kBinThreads] = sl[j];
}

// Block-wide exclusive scan of kScanTile elements; returns the block total.
__device__ int block_scan_tile(const int32_t *in, int64_t n, int64_t base, int vals[kScanPerThread]) {
    __shared__ int warp_tot[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t first = base + (int64_t)tid * kScanPerThread;
    int v[kScanPerThread];
    if (first + kScanPerThread <= n && (reinterpret_cast<uintptr_t>(in + first) & 15) == 0) {
        const int4 *q = reinterpret_cast<const int4 *>(in + first);
#pragma unroll
        for (int k = 0; k < kScanPerThread / 4; ++k) {
            const int4 w = q[k];
            v[4 * k] = w.x;
            v[4 * k + 1] = w.y;
            v[4 * k + 2] = w.z;
            v[4 * k + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanPerThread; ++k) v[k] = first + k < n ? in[first + k] : 0;
    }
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        vals[k] = s;
        s += v[k];
    }
    int incl = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int o = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += o;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive
    }
    __syncthreads();
    const int excl = warp_tot[wid] + incl - s;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) vals[k] += excl;
    __shared__ int total;
    if (tid == kScanThreads - 1) total = excl + s;
    __syncthreads();
    int t = total;
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const int32_t *counts, int64_t n, int32_t *blocksums) {
    int vals[kScanPerThread];
    int t = block_scan_tile(counts, n, (int64_t)blockIdx.x * kScanTile, vals);
    if (threadIdx.x == 0) blocksums[blockIdx.x] = t;
}

// Offsets of one tile: the tile's exclusive scan plus the sum of the tile
// totals before it (summed by the block itself, so no pass over the totals is
// needed); the last tile also writes the grand total offsets[n].  zero_counts:
// the block clears the counts it has read, leaving the histogram ready for the
// next call.
__global__ void __launch_bounds__(kScanThreads) scan_write_kernel(int32_t *counts, int64_t n, const int32_t *tilesums,
                                                                int64_t nblk, int32_t *offsets, bool zero_counts) {
    __shared__ int red[kScanThreads / 32];
    __shared__ int add_s;
    int part = 0;
    for (int64_t b = threadIdx.x; b < (int64_t)blockIdx.x; b += kScanThreads) part += tilesums[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) add_s = v;
    }
    __syncthreads();
    const int add = add_s;
    int vals[kScanPerThread];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int total = block_scan_tile(counts, n, base, vals);
    const int64_t first = base + (int64_t)threadIdx.x * kScanPerThread;
    if (first + kScanPerThread <= n && (reinterpret_cast<uintptr_t>(offsets + first) & 15) == 0 &&
        (reinterpret_cast<uintptr_t>(counts + first) & 15) == 0) {
        int4 *q = reinterpret_cast<int4 *>(offsets + first);
#pragma unroll
        for (int k = 0; k < kScanPerThread / 4; ++k)
            q[k] = make_int4(vals[4 * k] + add, vals[4 * k + 1] + add, vals[4 * k + 2] + add, vals[4 * k + 3] + add);
        if (zero_counts) {
            int4 *c = reinterpret_cast<int4 *>(counts + first);
#pragma unroll
            for (int k = 0; k < kScanPerThread / 4; ++k) c[k] = make_int4(0, 0, 0, 0);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanPerThread; ++k)
            if (first + k < n) {
                offsets[first + k] = vals[k] + add;
                if (zero_counts) counts[first + k] = 0;
            }
    }
    if (blockIdx.x == nblk - 1 && threadIdx.x == 0) offsets[n] = add + total;
}

__global__ void __launch_bounds__(kBinThreads) scatter_kernel(const float *X, const float *Y, const float *Z,
                                                              const int32_t *key, const uint8_t *layer8, int32_t n_hits,
                                                              unsigned long long disk_mask, const int32_t *offsets,
                                                              float4 *rec, int32_t *inv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_hits) return;
    const int k = key[i];
    if (k < 0) {
        inv[i] = -1;
        return;
    }
    // the key pass left the hit's place among its bin's hits in inv[i]; places
    // were handed out in arrival order, which follows the original index for
    // most bins (warps run roughly in order), so the in-bin ordering pass
    // usually finds a bin already in order
    const int pos = offsets[k] + inv[i];
    const float x = X[i], y = Y[i], z = Z[i];
    const float zr = ((disk_mask >> layer8[i]) & 1ull) == 0 ? z : sqrtf(fmaf(x, x, y * y));
    rec[pos] = make_float4(x, y, zr, __int_as_float(i));
    inv[i] = pos;
}

// Order the hits of each bin by original index (the scatter's atomics leave
// arrival order), one thread per bin, insertion sort in place; bins with fewer
// than two hits, or already in order, are left as the scatter mapped them.  (Staging a
// block's bins in shared memory, or a sorting network in registers, measured
// slower: most bins hold zero or one hit.)
constexpr int kSortBins = 256;

__global__ void __launch_bounds__(kSortBins) bin_sort_kernel(const int32_t *offsets, int64_t n_bins, float4 *rec,
                                                             int32_t *inv) {
    const int64_t b = (int64_t)blockIdx.x * kSortBins + threadIdx.x;
    if (b >= n_bins) return;
    const int s = offsets[b], e = offsets[b + 1];
    if (e - s < 2) return;
    bool sorted = true;
    for (int i = s + 1; i < e && sorted; ++i) sorted = __float_as_int(rec[i - 1].w) < __float_as_int(rec[i].w);
    if (sorted) return;
    for (int i = s + 1; i < e; ++i) {
        const float4 v = rec[i];
        const int key = __float_as_int(v.w);
        int j = i - 1;
        while (j >= s && __float_as_int(rec[j].w) > key) {
            rec[j + 1] = rec[j];
            --j;
        }
        rec[j + 1] = v;
    }
    for (int i = s; i < e; ++i) inv[__float_as_int(rec[i].w)] = i;
}

mkf_status grow(mkf_hitbins *b, int64_t n_hits, int64_t n_bins) {
    if (n_hits > b->cap_hits) {
        cudaFree(b->rec);
        cudaFree(b->inv);
        cudaFree(b->layer);
        cudaFree(b->key);
        cudaFree(b->zhit);
        b->zhit = nullptr;
        b->rec = nullptr;
        b->inv = b->key = nullptr;
        b->layer = nullptr;
        b->cap_hits = 0;
        int64_t c = std::max<int64_t>(n_hits, 1024);
        MKF_CUDA_TRY(cudaMalloc(&b->rec, c * sizeof(float4)));
        MKF_CUDA_TRY(cudaMalloc(&b->inv, c * sizeof(int32_t)));
        MKF_CUDA_TRY(cudaMalloc(&b->key, c * sizeof(int32_t)));
        MKF_CUDA_TRY(cudaMalloc(&b->layer, c * sizeof(uint8_t)));
        MKF_CUDA_TRY(cudaMalloc(&b->zhit, c * sizeof(float)));
        b->cap_hits = c;
    }
    const int64_t nblk = (n_bins + kScanTile - 1) / kScanTile;
    if (n_bins > b->cap_bins || nblk > b->cap_blocks) {
        cudaFree(b->offsets);
        cudaFree(b->counts);
        cudaFree(b->blocksums);
        b->offsets = b->counts = b->blocksums = nullptr;
        b->cap_bins = b->cap_blocks = 0;
        b->zero_bins = 0;
        int64_t c = std::max<int64_t>(n_bins, 1024);
        int64_t cb = std::max<int64_t>((c + kScanTile - 1) / kScanTile, 1);
        MKF_CUDA_TRY(cudaMalloc(&b->offsets, (c + 1) * sizeof(int32_t)));
        MKF_CUDA_TRY(cudaMalloc(&b->counts, c * sizeof(int32_t)));
        MKF_CUDA_TRY(cudaMalloc(&b->blocksums, cb * sizeof(int32_t)));
        b->cap_bins = c;
        b->cap_blocks = cb;
    }
    return MKF_OK;
}

// The binning pipeline on given buffers: keys, histogram and each hit's place
// in its bin; exclusive scan (which clears the histogram again); scatter; and
// (order_bins) the in-bin ordering by original index.  counts [n_bins] must be
// zero on entry and is zero on exit; tilesums [ceil(n_bins / kScanTile)] is
// scan scratch; inv carries the places from the key pass to the scatter.
mkf_status run_binning(mkf_ctx *ctx, const float *xyz, const int32_t *layer, const int32_t *event_offsets,
                       int32_t n_events, int32_t n_hits, int64_t n_bins, int32_t *counts, int32_t *tilesums,
                       int32_t *key, uint8_t *layer8, float *zhit, int32_t *offsets, float4 *rec, int32_t *inv,
                       bool order_bins) {
    cudaStream_t s = ctx->stream;
    if (n_hits > 0) {
        BinArgs A;
        A.G = ctx->geom;
        A.X = xyz;
        A.Y = xyz + n_hits;
        A.Z = xyz + 2 * (int64_t)n_hits;
        A.layer = layer;
        A.event_offsets = event_offsets;
        A.n_events = n_events;
        A.n_hits = n_hits;
        A.key = key;
        A.layer8 = layer8;
        A.zhit = zhit;
        A.counts = counts;
        A.slot = inv;
        A.fault = ctx->fault;
        bin_keys_kernel<<<(n_hits + kBinThreads * kBinItems - 1) / (kBinThreads * kBinItems), kBinThreads, 0, s>>>(A);
        MKF_CUDA_TRY(cudaGetLastError());
    }
    const int64_t nblk = (n_bins + kScanTile - 1) / kScanTile;
    scan_tiles_kernel<<<(unsigned)nblk, kScanThreads, 0, s>>>(counts, n_bins, tilesums);
    MKF_CUDA_TRY(cudaGetLastError());
    scan_write_kernel<<<(unsigned)nblk, kScanThreads, 0, s>>>(counts, n_bins, tilesums, nblk, offsets, true);
    MKF_CUDA_TRY(cudaGetLastError());
    if (n_hits > 0) {
        unsigned long long disk_mask = 0;
        for (int l = 0; l < ctx->geom.n_layers; ++l)
            if (ctx->geom.L[l].kind == 1) disk_mask |= 1ull << l;
        scatter_kernel<<<(n_hits + kBinThreads - 1) / kBinThreads, kBinThreads, 0, s>>>(xyz, xyz + n_hits, xyz + 2 * (int64_t)n_hits, key, layer8,
                                                           n_hits, disk_mask, offsets, rec, inv);
        MKF_CUDA_TRY(cudaGetLastError());
        if (order_bins) {
            bin_sort_kernel<<<(unsigned)((n_bins + kSortBins - 1) / kSortBins), kSortBins, 0, s>>>(offsets, n_bins, rec,
                                                                                                   inv);
            MKF_CUDA_TRY(cudaGetLastError());
        }
    }
    return MKF_OK;
}


}  // namespace

int64_t mkf_scan_tilesums(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

mkf_status mkf_run_scan(cudaStream_t s, const int32_t *counts, int64_t n, int32_t *tilesums, int32_t *offsets) {
    const int64_t nblk = mkf_scan_tilesums(n);
    if (nblk == 0) {
        MKF_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int32_t), s));
        return MKF_OK;
    }
    scan_tiles_kernel<<<(unsigned)nblk, kScanThreads, 0, s>>>(counts, n, tilesums);
    MKF_CUDA_TRY(cudaGetLastError());
    // the counts stay as they are (the caller hands out places from them)
    scan_write_kernel<<<(unsigned)nblk, kScanThreads, 0, s>>>(const_cast<int32_t *>(counts), n, tilesums, nblk, offsets,
                                                              false);
    MKF_CUDA_TRY(cudaGetLastError());
    return MKF_OK;
}

extern "C" void mkf_hitbins_free(mkf_hitbins *b) {
    if (!b) return;
    DeviceGuard g(b->device);
    cudaFree(b->rec);
    cudaFree(b->inv);
    cudaFree(b->layer);
    cudaFree(b->key);
    cudaFree(b->zhit);
    cudaFree(b->offsets);
    cudaFree(b->counts);
    cudaFree(b->blocksums);
    delete b;
}

extern "C" mkf_status mkf_hitbins_info(const mkf_hitbins *b, int32_t *n_hits, int32_t *n_events, int64_t *n_bins) {
    if (!b) return MKF_ERR_ARG;
    if (n_hits) *n_hits = b->n_hits;
    if (n_events) *n_events = b->n_events;
    if (n_bins) *n_bins = b->n_bins;
    return MKF_OK;
}

extern "C" mkf_status mkf_hitbins_export(mkf_ctx *ctx, const mkf_hitbins *b, float *rec, int32_t *inv,
                                         int32_t *offsets) {
    if (!ctx || !b || b->device != ctx->device) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    cudaStream_t s = ctx->stream;
    if ((rec || inv) && !b->ordered) {
        // put each bin into ascending original index, in place (the store's
        // contents stay the same set; later calls see the ordered layout)
        mkf_hitbins *m = const_cast<mkf_hitbins *>(b);
        bin_sort_kernel<<<(unsigned)((b->n_bins + kSortBins - 1) / kSortBins), kSortBins, 0, s>>>(m->offsets, m->n_bins,
                                                                                                  m->rec, m->inv);
        MKF_CUDA_TRY(cudaGetLastError());
        m->ordered = 1;
    }
    if (rec && b->n_hits)
        MKF_CUDA_TRY(cudaMemcpyAsync(rec, b->rec, sizeof(float4) * b->n_hits, cudaMemcpyDeviceToDevice, s));
    if (inv && b->n_hits)
        MKF_CUDA_TRY(cudaMemcpyAsync(inv, b->inv, sizeof(int32_t) * b->n_hits, cudaMemcpyDeviceToDevice, s));
    if (offsets)
        MKF_CUDA_TRY(cudaMemcpyAsync(offsets, b->offsets, sizeof(int32_t) * (b->n_bins + 1), cudaMemcpyDeviceToDevice, s));
    return MKF_OK;
}

extern "C" mkf_status mkf_hits_bin(mkf_ctx *ctx, const float *xyz, const int32_t *layer, const int32_t *event_offsets,
                                   int32_t n_events, int32_t n_hits, mkf_hitbins **inout) {
    if (!ctx || !inout) return MKF_ERR_ARG;
    if (!ctx->has_geom) return MKF_ERR_GEOMETRY;
    if (n_events < 1 || n_hits < 0) return MKF_ERR_ARG;
    if (n_hits > MKF_MAX_HITS) return MKF_ERR_CAPACITY;
    if (n_hits > 0 && (!xyz || !layer)) return MKF_ERR_ARG;
    if (!event_offsets) return MKF_ERR_ARG;
    const int64_t n_bins = (int64_t)n_events * ctx->geom.bins_per_event;
    if (n_bins >= (int64_t(1) << 31) - 1) return MKF_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    mkf_hitbins *b = *inout;
    bool fresh = false;
    if (!b) {
        b = new mkf_hitbins();
        b->device = ctx->device;
        fresh = true;
    } else if (b->device != ctx->device) {
        return MKF_ERR_ARG;
    }
    mkf_status st = grow(b, n_hits, n_bins);
    if (st != MKF_OK) {
        if (fresh) mkf_hitbins_free(b);
        return st;
    }
    b->geom_version = ctx->geom_version;
    b->n_hits = n_hits;
    b->n_events = n_events;
    b->n_bins = n_bins;
    cudaStream_t s = ctx->stream;
    // every binning leaves the histogram zero (the scan clears what it reads),
    // so it is set here only when this call's bins reach beyond the part known
    // to be zero (a new allocation, or a call that failed before its scan)
    const int64_t zero_before = std::max<int64_t>(b->zero_bins, 0);
    b->zero_bins = 0;  // until the scan has been enqueued
    if (n_bins > zero_before)
        MKF_CUDA_TRY(cudaMemsetAsync(b->counts, 0, n_bins * sizeof(int32_t), s));
    // the finder does not depend on the order of hits within a bin, so the store
    // keeps arrival order; mkf_hitbins_export orders it when asked for the layout
    st = run_binning(ctx, xyz, layer, event_offsets, n_events, n_hits, n_bins, b->counts, b->blocksums, b->key,
                     b->layer, b->zhit, b->offsets, b->rec, b->inv, false);
    if (st != MKF_OK) return st;
    b->zero_bins = std::max(zero_before, n_bins);
    b->ordered = n_hits == 0;
    *inout = b;
    return MKF_OK;
}

// ---------------------------------------------------------------------------
// Binning without allocation: working memory in one file-scope device array.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr int64_t kStaticHits = MKF_STATIC_MAX_HITS;
constexpr int64_t kStaticBins = MKF_STATIC_MAX_BINS;
constexpr int64_t kStaticBlocks = (kStaticBins + kScanTile - 1) / kScanTile;
constexpr size_t kOffCounts = 0;
constexpr size_t kOffBlocks = align256(kOffCounts + sizeof(int32_t) * kStaticBins);
constexpr size_t kOffKey = align256(kOffBlocks + sizeof(int32_t) * kStaticBlocks);
constexpr size_t kOffZ = align256(kOffKey + sizeof(int32_t) * kStaticHits);
constexpr size_t kOffLayer = align256(kOffZ + sizeof(float) * kStaticHits);
constexpr size_t kStaticBytes = align256(kOffLayer + sizeof(uint8_t) * kStaticHits);

// Reserved on a device when the module holding this file's kernels is loaded
// there: at library load, or under CUDA's lazy module loading (the default) at
// the first call of mkf_hits_bin or mkf_hits_bin_static on that device.  In
// host code this name is only a stand-in: the device address comes from
// cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_bin_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Device address of g_bin_scratch on `device` (which must be current).
mkf_status static_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return MKF_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_bin_scratch) != cudaSuccess || !ptr) return MKF_ERR_CUDA;
        g_scratch_addr[device] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_addr[device];
    return MKF_OK;
}

}  // namespace

extern "C" mkf_status mkf_hits_bin_static(mkf_ctx *ctx, const float *xyz, const int32_t *layer,
                                          const int32_t *event_offsets, int32_t n_events, int32_t n_hits, float *rec,
                                          int32_t *inv, int32_t *offsets) {
    if (!ctx) return MKF_ERR_ARG;
    if (!ctx->has_geom) return MKF_ERR_GEOMETRY;
    if (n_events < 1 || n_hits < 0) return MKF_ERR_ARG;
    if (!event_offsets || !offsets) return MKF_ERR_ARG;
    if (n_hits > 0 && (!xyz || !layer || !rec || !inv)) return MKF_ERR_ARG;
    // rec is written as float4 records: a buffer that does not start on a
    // 16-byte boundary is rejected here instead of faulting in the kernel
    if (n_hits > 0 && (reinterpret_cast<uintptr_t>(rec) & 15u) != 0) return MKF_ERR_ARG;
    const int64_t n_bins = (int64_t)n_events * ctx->geom.bins_per_event;
    if (n_hits > kStaticHits || n_bins > kStaticBins) return MKF_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    unsigned char *base = nullptr;
    mkf_status st = static_scratch(ctx->device, &base);
    if (st != MKF_OK) return st;
    int32_t *counts = reinterpret_cast<int32_t *>(base + kOffCounts);
    int32_t *blocksums = reinterpret_cast<int32_t *>(base + kOffBlocks);
    int32_t *key = reinterpret_cast<int32_t *>(base + kOffKey);
    float *zhit = reinterpret_cast<float *>(base + kOffZ);
    uint8_t *layer8 = base + kOffLayer;
    float4 *rec4 = reinterpret_cast<float4 *>(rec);
    cudaStream_t s = ctx->stream;
    // the histogram starts at zero on every call (the array keeps the last call's contents)
    MKF_CUDA_TRY(cudaMemsetAsync(counts, 0, n_bins * sizeof(int32_t), s));
    return run_binning(ctx, xyz, layer, event_offsets, n_events, n_hits, n_bins, counts, blocksums, key, layer8, zhit,
                       offsets, rec4, inv, true);
}
