// Host run of the seed-cleaning and duplicate-removal kernels (tests only): the
// kernels of mkf_dedup.cu, compiled for the host, are called once per thread of
// their grids in order; the count / scan / fill / decide sequence of the
// library's driver is repeated here with a host exclusive scan.
#include <cmath>
#include <cstdint>
#include <vector>

#include "warp_emu.h"
inline int atomicSub(int *p, int v) { return __atomic_fetch_sub(p, v, __ATOMIC_SEQ_CST); }
using std::fabs;
using std::fmax;
using std::fmod;
using std::log;
using std::tan;
thread_local dim3 threadIdx, blockIdx;
dim3 blockDim;

#include "dedup_dev.inc"

namespace {

template <class F>
void launch(int64_t threads, F f) {
    blockDim.x = kThreads;
    for (int64_t t = 0; t < threads; ++t) {
        blockIdx.x = static_cast<unsigned>(t / kThreads);
        threadIdx.x = static_cast<unsigned>(t % kThreads);
        f();
    }
}

void build(const int32_t *lists, int32_t rows, int32_t n, int32_t n_hits, std::vector<int32_t> &off,
           std::vector<int32_t> &items) {
    std::vector<int32_t> cnt(n_hits > 0 ? n_hits : 1, 0);
    const int64_t pairs = (int64_t)rows * n;
    launch((pairs + kThreads - 1) / kThreads * kThreads, [&] { count_kernel(lists, rows, n, n_hits, cnt.data()); });
    off.assign((size_t)n_hits + 1, 0);
    for (int32_t h = 0; h < n_hits; ++h) off[h + 1] = off[h] + cnt[h];
    items.assign(pairs > 0 ? pairs : 1, -1);
    launch((pairs + kThreads - 1) / kThreads * kThreads,
           [&] { fill_kernel(lists, rows, n, n_hits, off.data(), cnt.data(), items.data()); });
}

}  // namespace

extern "C" void emu_seeds_clean(const int32_t *seed_hits, int32_t n, int32_t n_hits, const float *par, float dq,
                                float de, float dp, int32_t *keep) {
    std::vector<int32_t> off, items;
    build(seed_hits, 3, n, n_hits, off, items);
    launch((int64_t)(n + kThreads - 1) / kThreads * kThreads, [&] {
        seeds_decide_kernel(seed_hits, n, n_hits, par, dq, de, dp, off.data(), items.data(), keep);
    });
}

extern "C" void emu_tracks_dedup(const int32_t *hit_idx, int32_t rows, int32_t n, int32_t n_hits, const int32_t *nh,
                                 const float *chi2, float min_frac, int32_t *keep) {
    std::vector<int32_t> off, items;
    build(hit_idx, rows, n, n_hits, off, items);
    launch((int64_t)(n + kThreads - 1) / kThreads * kThreads, [&] {
        tracks_decide_kernel(hit_idx, rows, n, n_hits, nh, chi2, min_frac, off.data(), items.data(), keep);
    });
}
