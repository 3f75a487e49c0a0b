// Host builds of the library's device headers (tests only): the CUDA
// qualifiers mapped away and the few CUDA types and intrinsics they name.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#define __device__
#define __host__
#define __forceinline__ inline
using std::isfinite;
using std::max;
using std::min;
struct float2 {
    float x, y;
};
static inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
static inline int __float_as_int(float f) { int i; std::memcpy(&i, &f, 4); return i; }
