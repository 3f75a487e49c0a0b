// Host build of the device math header (FP32, same expressions) for CPU tests
// of its self-contained helpers.  Only the qualifiers are mapped away.
#include <cmath>
#include <cstdint>
#include <cstring>
#define __device__
#define __host__
#define __forceinline__ inline
using std::isfinite;
static inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
static inline int __float_as_int(float f) { int i; std::memcpy(&i, &f, 4); return i; }
#include "mkf_math.cuh"

extern "C" void host_sincos_small(const float *x, float *s, float *c, int n) {
    for (int i = 0; i < n; ++i) mkf::sincos_small(x[i], s[i], c[i]);
}

extern "C" void host_sinc_and_deriv(const float *a, float *sn, float *dsn, int n) {
    for (int i = 0; i < n; ++i) {
        float sa = std::sin(a[i]), ca = std::cos(a[i]);
        mkf::sinc_and_deriv(a[i], sa, ca, sn[i], dsn[i]);
    }
}
