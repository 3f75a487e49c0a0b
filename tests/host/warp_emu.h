// Warp emulation on the host (tests only): the 32 lanes of one warp run as 32
// threads; every warp intrinsic is a rendezvous of all 32 lanes, so lanes must
// reach the intrinsics in the same order, exactly as the hardware requires of
// full-mask intrinsics.  A lane left waiting for more than a few seconds means
// the kernel diverged at an intrinsic: the process reports it and exits.
#pragma once
#include <algorithm>
#include <chrono>
#include <cmath>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#define __device__
#define __host__
#define __forceinline__ inline
#define __global__
#define __launch_bounds__(...)
#define __grid_constant__
#define __align__(n) alignas(n)
#include "cuda_runtime.h"

struct dim3 { unsigned x = 0, y = 0, z = 0; };
extern thread_local dim3 threadIdx, blockIdx;
extern dim3 blockDim;
using std::isfinite;
using std::max;
using std::min;
inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
inline int __float_as_int(float f) { int i; std::memcpy(&i, &f, 4); return i; }
inline float __uint_as_float(uint32_t i) { float f; std::memcpy(&f, &i, 4); return f; }
inline uint32_t __float_as_uint(float f) { uint32_t i; std::memcpy(&i, &f, 4); return i; }
inline int __popc(unsigned v) { return __builtin_popcount(v); }
inline int __ffs(unsigned v) { return __builtin_ffs(static_cast<int>(v)); }
template <class T> T atomicAdd(T *p, T v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline int atomicCAS(int *p, int cmp, int v) {
    __atomic_compare_exchange_n(p, &cmp, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST);
    return cmp;
}
inline unsigned long long atomicMin(unsigned long long *p, unsigned long long v) {
    unsigned long long o = *p;
    while (v < o && !__atomic_compare_exchange_n(p, &o, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) {}
    return o;
}
inline unsigned long long atomicMax(unsigned long long *p, unsigned long long v) {
    unsigned long long o = *p;
    while (v > o && !__atomic_compare_exchange_n(p, &o, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) {}
    return o;
}

struct WarpEmu {
    std::atomic<int> arrived{0};
    std::atomic<unsigned long long> gen{0};
    uint64_t v[32];
    void sync() {
        const unsigned long long g = gen.load(std::memory_order_acquire);
        if (arrived.fetch_add(1, std::memory_order_acq_rel) == 31) {
            arrived.store(0, std::memory_order_relaxed);
            gen.fetch_add(1, std::memory_order_acq_rel);
            return;
        }
        const auto t0 = std::chrono::steady_clock::now();
        for (unsigned long spins = 0; gen.load(std::memory_order_acquire) == g; ++spins) {
            std::this_thread::yield();
            if ((spins & 0xFFFF) == 0xFFFF && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(20)) {
                std::fprintf(stderr, "warp emulation: lanes diverged at a warp intrinsic\n");
                std::fflush(stderr);
                std::_Exit(3);
            }
        }
    }
};
extern WarpEmu *g_warp;
extern unsigned char *g_smem;

inline uint64_t warp_exchange(uint64_t mine, int src) {
    g_warp->v[threadIdx.x & 31] = mine;
    g_warp->sync();
    const uint64_t r = g_warp->v[src & 31];
    g_warp->sync();
    return r;
}
template <class T> T __shfl_sync(unsigned, T v, int src) {
    uint64_t b = 0;
    std::memcpy(&b, &v, sizeof(T));
    b = warp_exchange(b, src);
    T o;
    std::memcpy(&o, &b, sizeof(T));
    return o;
}
template <class T> T __shfl_down_sync(unsigned m, T v, unsigned off) {
    const int l = threadIdx.x & 31;
    const int s = l + static_cast<int>(off);
    return __shfl_sync(m, v, s > 31 ? l : s);
}
template <class T> T __shfl_up_sync(unsigned m, T v, unsigned off) {
    const int l = threadIdx.x & 31;
    const int s = l - static_cast<int>(off);
    return __shfl_sync(m, v, s < 0 ? l : s);
}
inline unsigned __ballot_sync(unsigned, bool p) {
    g_warp->v[threadIdx.x & 31] = p ? 1 : 0;
    g_warp->sync();
    unsigned r = 0;
    for (int i = 0; i < 32; ++i)
        if (g_warp->v[i]) r |= 1u << i;
    g_warp->sync();
    return r;
}
inline bool __any_sync(unsigned m, bool p) { return __ballot_sync(m, p) != 0; }
inline void __syncwarp(unsigned = 0xffffffffu) { g_warp->sync(); }
inline void __syncthreads() { g_warp->sync(); }
