// Host build of the device math header (FP32, same expressions) for CPU tests
// of its self-contained helpers.  Only the qualifiers are mapped away.
#include "host_prelude.h"
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
