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

// ---- the square-root form of the seed-hit filter against the covariance form
using mkf::SqrtCov;
constexpr int kHostSq = 9;

static void load_sqrt(const float *S, int k, SqrtCov<kHostSq> &Q) {
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < kHostSq; ++j) Q.S[i][j] = S[i * kHostSq + j];
    Q.k = k;
}

// Seed state and prior from three hits: p [6] and C = S S^T [21].
extern "C" int host_seed_prior(int kind, float sig2, float kb, const float *h1, const float *h2, const float *h3,
                               float *p, float *C) {
    mkf::LayerDesc L{};
    L.kind = kind;
    L.seed_sig2 = sig2;
    SqrtCov<kHostSq> Q;
    float eta;
    if (!mkf::seed_state(L, kb, h1, h2, h3, p, Q, eta)) return 0;
    mkf::sqrt_to_cov(Q, C);
    return Q.k;
}

// One hit through the square root: S [6][9] (row-major) and p [6] updated in
// place with the residual (u, v) of a hit on a layer of `kind`; returns chi2.
extern "C" float host_sqrt_update(int kind, float su2, float sv2, float *S, float *p, float u, float v) {
    SqrtCov<kHostSq> Q;
    load_sqrt(S, kHostSq, Q);
    mkf::Lo lo{0.f, 0.f, 0.f, 0.f, 0.f};
    const mkf::Frame f = mkf::frame_of(p);
    const float chi2 = mkf::sqrt_update(kind, su2, sv2, f, u, v, p, lo, &Q);
    p[0] += lo.x;
    p[1] += lo.y;
    p[2] += lo.z;
    p[4] += lo.phi;
    p[5] += lo.th;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < kHostSq; ++j) S[i * kHostSq + j] = Q.S[i][j];
    return chi2;
}

// The move of state p0 onto layer (kind, rz) with C = S S^T transported as C
// (Cc) and as J S (Cs = S' S'^T); 0 if the layer is not reached.
extern "C" int host_transport_both(int kind, float rz, float kb, const float *p0, const float *S, float *Cc,
                                   float *Cs) {
    mkf::LayerDesc L{};
    L.kind = kind;
    L.rz = rz;
    SqrtCov<kHostSq> Q;
    load_sqrt(S, kHostSq, Q);
    float C[21];
    mkf::sqrt_to_cov(Q, C);
    float p1[6], p2[6];
    for (int i = 0; i < 6; ++i) p1[i] = p2[i] = p0[i];
    mkf::Lo lo1{0.f, 0.f, 0.f, 0.f, 0.f}, lo2{0.f, 0.f, 0.f, 0.f, 0.f};
    float sphi, cphi, s;
    mkf::sincos_pair(p0[4], 0.f, sphi, cphi);
    const float cot = mkf::cot_pair(p0[5], 0.f);
    if (!mkf::path_to_layer(L, kb, p1, lo1, sphi, cphi, cot, s)) return 0;
    mkf::propagate_transport(L, kb, p1, lo1, C, sphi, cphi, cot, s);
    mkf::propagate_transport(L, kb, p2, lo2, &Q, sphi, cphi, cot, s);
    for (int i = 0; i < 21; ++i) Cc[i] = C[i];
    mkf::sqrt_to_cov(Q, Cs);
    return 1;
}

// Scattering noise and energy loss at state p0 (thickness t X0, loss k) on C
// (Cc) and on S with k_used columns filled (Cs = S' S'^T).
extern "C" void host_material_both(int kind, float t, float k, const float *p0, const float *S, int k_used,
                                   float *Cc, float *Cs) {
    SqrtCov<kHostSq> Q;
    load_sqrt(S, k_used, Q);
    float C[21];
    mkf::sqrt_to_cov(Q, C);
    float p1[6], p2[6];
    for (int i = 0; i < 6; ++i) p1[i] = p2[i] = p0[i];
    mkf::add_scattering(kind, t, p1, C);
    mkf::apply_eloss(kind, t, k, p1, C, 1.f);
    mkf::add_scattering(kind, t, p2, &Q);
    mkf::apply_eloss(kind, t, k, p2, &Q, 1.f);
    for (int i = 0; i < 21; ++i) Cc[i] = C[i];
    mkf::sqrt_to_cov(Q, Cs);
}
