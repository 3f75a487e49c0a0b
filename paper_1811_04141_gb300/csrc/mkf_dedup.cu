// Seed cleaning before finding and duplicate-track removal after it (Sec. 2.2:
// repeated seeds of one particle are removed using the identity of their hits
// and their fitted pT, eta and phi; Sec. 3: duplicate tracks from several seeds
// per particle are to be removed after finding).
//
// Both are decisions over the graph of items (seeds or tracks) that share hits.
// The graph is built as an inverse index, hit -> items using it (a count pass,
// the binning's exclusive scan, a fill pass), after which one thread per item
// walks its hits and the items listed on them.  An item is dropped when a
// duplicate that ranks above it exists, whether or not that one is dropped
// itself, so no decision waits on another and the result does not depend on
// the order of the threads.
#include <cuda_runtime.h>

#include "mkf_internal.h"

namespace {

constexpr int kThreads = 256;

// A hit of item i's list at row k that is valid and not listed earlier in the
// same list (lists are sets).
__device__ __forceinline__ bool first_listing(const int32_t *lists, int32_t k, int32_t n, int32_t i, int32_t h,
                                              int32_t n_hits) {
    if (h < 0 || h >= n_hits) return false;
    for (int32_t r = 0; r < k; ++r)
        if (lists[(int64_t)r * n + i] == h) return false;
    return true;
}

__global__ void __launch_bounds__(kThreads) count_kernel(const int32_t *lists, int32_t rows, int32_t n,
                                                         int32_t n_hits, int32_t *cnt) {
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= (int64_t)rows * n) return;
    const int32_t k = static_cast<int32_t>(t / n), i = static_cast<int32_t>(t - (int64_t)k * n);
    const int32_t h = lists[t];
    if (first_listing(lists, k, n, i, h, n_hits)) atomicAdd(&cnt[h], 1);
}

// Slots are handed out per hit with the counters running back to zero, so the
// counters are ready for the next call.
__global__ void __launch_bounds__(kThreads) fill_kernel(const int32_t *lists, int32_t rows, int32_t n, int32_t n_hits,
                                                        const int32_t *off, int32_t *cnt, int32_t *items) {
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= (int64_t)rows * n) return;
    const int32_t k = static_cast<int32_t>(t / n), i = static_cast<int32_t>(t - (int64_t)k * n);
    const int32_t h = lists[t];
    if (!first_listing(lists, k, n, i, h, n_hits)) return;
    items[off[h + 1] - atomicSub(&cnt[h], 1)] = i;
}

// eta of a polar angle, in double (both sides of a threshold test see the same
// value up to the last bit of a double).
__device__ __forceinline__ double eta_of(float theta) { return -log(tan(0.5 * static_cast<double>(theta))); }

__device__ __forceinline__ double wrapped_abs(double a) {
    constexpr double kPiD = 3.14159265358979323846;
    a = fmod(a + kPiD, 2.0 * kPiD);
    if (a < 0.0) a += 2.0 * kPiD;
    return fabs(a - kPiD);
}

// Seeds: drop i when a seed u < i shares a hit with it and their fitted q/pT,
// eta and phi agree within the tolerances (differences in double on the given
// float parameters).
__global__ void __launch_bounds__(kThreads) seeds_decide_kernel(const int32_t *seed_hits, int32_t n, int32_t n_hits,
                                                                const float *par, double max_dqpt, double max_deta,
                                                                double max_dphi, const int32_t *off,
                                                                const int32_t *items, int32_t *keep) {
    const int32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const double w = par[3 * (int64_t)n + i], ph = par[4 * (int64_t)n + i];
    const double et = eta_of(par[5 * (int64_t)n + i]);
    bool k_ = true;
    for (int32_t r = 0; r < 3 && k_; ++r) {
        const int32_t h = seed_hits[(int64_t)r * n + i];
        if (!first_listing(seed_hits, r, n, i, h, n_hits)) continue;
        for (int32_t p = off[h]; p < off[h + 1]; ++p) {
            const int32_t u = items[p];
            if (u >= i) continue;
            const double wu = par[3 * (int64_t)n + u], phu = par[4 * (int64_t)n + u];
            const double etu = eta_of(par[5 * (int64_t)n + u]);
            if (fabs(w - wu) <= max_dqpt && fabs(et - etu) <= max_deta && wrapped_abs(ph - phu) <= max_dphi) {
                k_ = false;
                break;
            }
        }
    }
    keep[i] = k_ ? 1 : 0;
}

// Tracks: drop i when a better track u (more hits, then lower chi2, then lower
// index) shares at least max(1, min_frac x the shorter one's hit count) hits.
__global__ void __launch_bounds__(kThreads) tracks_decide_kernel(const int32_t *hit_idx, int32_t rows, int32_t n,
                                                                 int32_t n_hits, const int32_t *nh, const float *chi2,
                                                                 float min_frac, const int32_t *off,
                                                                 const int32_t *items, int32_t *keep) {
    const int32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const int32_t ni = nh[i];
    const float ci = chi2[i];
    bool k_ = true;
    for (int32_t r = 0; r < rows && k_; ++r) {
        const int32_t h = hit_idx[(int64_t)r * n + i];
        if (!first_listing(hit_idx, r, n, i, h, n_hits)) continue;
        for (int32_t p = off[h]; p < off[h + 1] && k_; ++p) {
            const int32_t u = items[p];
            if (u == i) continue;
            const int32_t nu = nh[u];
            const float cu = chi2[u];
            const bool better = nu > ni || (nu == ni && (cu < ci || (cu == ci && u < i)));
            if (!better) continue;
            // hits of i (as a set) that u also lists
            int32_t shared = 0;
            for (int32_t a = 0; a < rows; ++a) {
                const int32_t ha = hit_idx[(int64_t)a * n + i];
                if (!first_listing(hit_idx, a, n, i, ha, n_hits)) continue;
                for (int32_t b = 0; b < rows; ++b)
                    if (hit_idx[(int64_t)b * n + u] == ha) {
                        ++shared;
                        break;
                    }
            }
            const double need = fmax(1.0, static_cast<double>(min_frac) * min(ni, nu));
            if (shared >= need) k_ = false;
        }
    }
    keep[i] = k_ ? 1 : 0;
}

// Inverse index hit -> items of `lists` [rows][n]; scratch carved from the
// context: counters, offsets, scan sums, item slots.
mkf_status build_index(mkf_ctx *ctx, const int32_t *lists, int32_t rows, int32_t n, int32_t n_hits,
                       const int32_t **off_out, const int32_t **items_out) {
    const int64_t pairs = (int64_t)rows * n;
    const int64_t nts = mkf_scan_tilesums(n_hits);
    auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
    const int64_t b_cnt = up(4 * (int64_t)n_hits), b_off = up(4 * ((int64_t)n_hits + 1)), b_ts = up(4 * (nts + 1)),
                  b_items = up(4 * pairs);
    void *scr = nullptr;
    const mkf_status st = mkf_scratch(ctx, b_cnt + b_off + b_ts + b_items, &scr);
    if (st != MKF_OK) return st;
    char *c = static_cast<char *>(scr);
    int32_t *cnt = reinterpret_cast<int32_t *>(c);
    int32_t *off = reinterpret_cast<int32_t *>(c + b_cnt);
    int32_t *ts = reinterpret_cast<int32_t *>(c + b_cnt + b_off);
    int32_t *items = reinterpret_cast<int32_t *>(c + b_cnt + b_off + b_ts);
    cudaStream_t s = ctx->stream;
    MKF_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)n_hits, s));
    const unsigned blocks = static_cast<unsigned>((pairs + kThreads - 1) / kThreads);
    if (pairs > 0) {
        count_kernel<<<blocks, kThreads, 0, s>>>(lists, rows, n, n_hits, cnt);
        MKF_CUDA_TRY(cudaGetLastError());
    }
    const mkf_status ss = mkf_run_scan(s, cnt, n_hits, ts, off);
    if (ss != MKF_OK) return ss;
    if (pairs > 0) {
        fill_kernel<<<blocks, kThreads, 0, s>>>(lists, rows, n, n_hits, off, cnt, items);
        MKF_CUDA_TRY(cudaGetLastError());
    }
    *off_out = off;
    *items_out = items;
    return MKF_OK;
}

}  // namespace

extern "C" mkf_status mkf_seeds_clean(mkf_ctx *ctx, const int32_t *seed_hits, int32_t n_seeds, int32_t n_hits,
                                      const float *seed_par, float max_dqpt, float max_deta, float max_dphi,
                                      int32_t *keep) {
    if (!ctx) return MKF_ERR_ARG;
    if (n_seeds < 0 || n_hits < 0) return MKF_ERR_ARG;
    if (n_hits > MKF_MAX_HITS) return MKF_ERR_CAPACITY;
    if (!(max_dqpt >= 0.f) || !(max_deta >= 0.f) || !(max_dphi >= 0.f)) return MKF_ERR_ARG;
    if (n_seeds == 0) return MKF_OK;
    if (!seed_hits || !seed_par || !keep) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    const int32_t *off = nullptr, *items = nullptr;
    const mkf_status st = build_index(ctx, seed_hits, 3, n_seeds, n_hits, &off, &items);
    if (st != MKF_OK) return st;
    seeds_decide_kernel<<<(n_seeds + kThreads - 1) / kThreads, kThreads, 0, ctx->stream>>>(
        seed_hits, n_seeds, n_hits, seed_par, max_dqpt, max_deta, max_dphi, off, items, keep);
    MKF_CUDA_TRY(cudaGetLastError());
    return MKF_OK;
}

extern "C" mkf_status mkf_tracks_dedup(mkf_ctx *ctx, const int32_t *hit_idx, int32_t max_hits, int32_t n,
                                       int32_t n_hits, const int32_t *track_nhits, const float *chi2, float min_frac,
                                       int32_t *keep) {
    if (!ctx) return MKF_ERR_ARG;
    if (n < 0 || n_hits < 0 || max_hits < 1) return MKF_ERR_ARG;
    if (max_hits > MKF_MAX_LAYERS + 8) return MKF_ERR_CAPACITY;
    if (n_hits > MKF_MAX_HITS) return MKF_ERR_CAPACITY;
    if (!(min_frac >= 0.f && min_frac <= 1.f)) return MKF_ERR_ARG;
    if (n == 0) return MKF_OK;
    if (!hit_idx || !track_nhits || !chi2 || !keep) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    const int32_t *off = nullptr, *items = nullptr;
    const mkf_status st = build_index(ctx, hit_idx, max_hits, n, n_hits, &off, &items);
    if (st != MKF_OK) return st;
    tracks_decide_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, ctx->stream>>>(
        hit_idx, max_hits, n, n_hits, track_nhits, chi2, min_frac, off, items, keep);
    MKF_CUDA_TRY(cudaGetLastError());
    return MKF_OK;
}
