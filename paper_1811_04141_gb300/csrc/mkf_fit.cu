// Track fit along fixed hit lists: one thread per track, state and covariance in
// registers for the whole hit list (Sec. 1: Kalman-filter fitting), and the
// backward fit, the same filter through the hits in reverse order.
#include <cuda_runtime.h>

#include <type_traits>

#include "mkf_internal.h"

namespace {

using namespace mkf;

struct FitArgs {
    Geom G;
    const float *X, *Y, *Z;
    const int32_t *hit_layer;
    int32_t n_hits;
    const int32_t *hit_idx;
    int32_t max_hits, n;
    const float *seed_par, *seed_cov;
    float inflate;  // backward fit: factor on the starting covariance
    float *sm_par, *sm_cov;  // smoother: [max_hits][6][n], [max_hits][21][n]
    float *out_par, *out_cov, *chi2;
    int32_t *ndf;
    uint32_t *status;
    mkf_fault *fault;
};

__device__ __forceinline__ void record_fault(mkf_fault *f, int code, int where) {
    if (atomicCAS(&f->code, 0, code) == 0) f->where = where;
}

// The helix traversed the other way: the same curve with the momentum turned
// around, p -> (x, y, z, -q/pT, phi + pi, pi - theta) with pi as a float pair
// (phi and theta are pairs too),
// and C -> F C F with F = diag(1, 1, 1, -1, 1, -1) (the covariances between
// {q/pT, theta} and the other parameters change sign).
__device__ __forceinline__ void reverse_state(float p[6], Lo &lo, float C[21]) {
    constexpr float kPiHi = 3.14159274101257324219f;  // float(pi)
    constexpr float kPiLo = -8.74227765734758e-8f;    // pi - float(pi)
    p[3] = -p[3];
    df_add(p[4], lo.phi, kPiHi);
    df_add(p[4], lo.phi, kPiLo);
    df_wrap_pi(p[4], lo.phi);
    float th = kPiHi, thl = kPiLo;
    df_add(th, thl, -p[5]);
    df_add(th, thl, -lo.th);
    p[5] = th;
    lo.th = thl;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j)
            if ((i == 3 || i == 5) != (j == 3 || j == 5)) C[sym(i, j)] = -C[sym(i, j)];
}

// Move the state onto layer Ld (the helix or, for kPhys = 2, Runge-Kutta steps
// in the parameterised field); false if the layer is not reached.
template <int kPhys, class Cov>
__device__ __forceinline__ bool move_to(const Geom &G, const LayerDesc &Ld, float p[6], Lo &lo, Cov C) {
    float sphi, cphi;
    sincos_pair(p[4], lo.phi, sphi, cphi);
    const float cot = cot_pair(p[5], lo.th);
    const float kbl = kPhys == 2 ? G.kb * bz_factor(G.alpha, p[0], p[1], p[2]) : G.kb;
    float s;
    if (!path_to_layer(Ld, kbl, p, lo, sphi, cphi, cot, s)) return false;
    if (kPhys == 2)
        propagate_field(Ld, G.kb, G.alpha, p, lo, C, sphi, cphi, -p[3] * kbl, s);
    else
        propagate_transport(Ld, G.kb, p, lo, C, sphi, cphi, cot, s);
    return true;
}

// Kalman update with the hit (xh, yh, zh) on layer Ld; false if the residual
// covariance is not positive definite.
__device__ __forceinline__ bool update_with(const LayerDesc &Ld, float xh, float yh, float zh, float p[6], Lo &lo,
                                            float C[21], float &dchi2) {
    const Frame f = frame_of(p);
    Innov I;
    if (!innovation(Ld.kind, Ld.su2, Ld.sv2, f, C, I)) return false;
    float u, v;
    const float zr = Ld.kind == 0 ? zh : sqrtf(fmaf(xh, xh, yh * yh));
    residual(Ld.kind, Ld.rz, p, lo, f, xh, yh, zr, u, v);
    dchi2 = chi2_of(I, u, v);
    kf_apply_joseph(I, u, v, p, lo, C);
    return true;
}

// The same with the covariance as a square root (the seed hits).
template <int K>
__device__ __forceinline__ bool update_with(const LayerDesc &Ld, float xh, float yh, float zh, float p[6], Lo &lo,
                                            SqrtCov<K> *Q, float &dchi2) {
    const Frame f = frame_of(p);
    float u, v;
    const float zr = Ld.kind == 0 ? zh : sqrtf(fmaf(xh, xh, yh * yh));
    residual(Ld.kind, Ld.rz, p, lo, f, xh, yh, zr, u, v);
    dchi2 = sqrt_update(Ld.kind, Ld.su2, Ld.sv2, f, u, v, p, lo, Q);
    return true;
}

// kBackward: hits in reverse order from the given state at the last hit, turned
// around and inflated; the result at the first hit is turned back.  kPhys: 0
// uniform field without material; 1 material effects compiled in (selected
// when any layer has material); 2 the parameterised field (Runge-Kutta
// propagation) with the material effects.
template <bool kBackward, int kPhys>
__global__ void __launch_bounds__(128, kPhys == 2 ? 4 : 6) fit_kernel(const __grid_constant__ FitArgs A) {
    constexpr bool kMaterial = kPhys >= 1, kParamField = kPhys == 2;
    constexpr int kSq = kMaterial ? 9 : 5;  // square-root columns through the seed hits
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.n) return;
    const Geom &G = A.G;
    float p[6], C[21];
    SqrtCov<kSq> Q;
    Lo lo{0.f, 0.f, 0.f, 0.f, 0.f};
    uint32_t st = 0;
    float chi2 = 0.f;
    int used = 0;

    // first three valid hits (seed) and validity of all indices
    int first[3] = {-1, -1, -1}, nfirst = 0;
    for (int k = 0; k < A.max_hits; ++k) {
        int h = A.hit_idx[(int64_t)k * A.n + t];
        if (h < 0) continue;
        if (h >= A.n_hits) {
            record_fault(A.fault, kFaultBadHitIndex, t);
            continue;
        }
        if (nfirst < 3) first[nfirst++] = h;
    }
    bool ok = nfirst >= 3;
    if (ok) {
        int l0 = A.hit_layer[first[0]];
        if (l0 < 0 || l0 >= G.n_layers) {
            record_fault(A.fault, kFaultBadLayer, first[0]);
            ok = false;
        } else if (A.seed_par) {
#pragma unroll
            for (int i = 0; i < 6; ++i) p[i] = A.seed_par[(int64_t)i * A.n + t];
#pragma unroll
            for (int k = 0; k < 21; ++k) C[k] = A.seed_cov[(int64_t)k * A.n + t];
            if (kBackward) {
                reverse_state(p, lo, C);
#pragma unroll
                for (int k = 0; k < 21; ++k) C[k] *= A.inflate;
            }
        } else {
            float h1[3], h2[3], h3[3], eta;
            h1[0] = A.X[first[0]]; h1[1] = A.Y[first[0]]; h1[2] = A.Z[first[0]];
            h2[0] = A.X[first[1]]; h2[1] = A.Y[first[1]]; h2[2] = A.Z[first[1]];
            h3[0] = A.X[first[2]]; h3[1] = A.Y[first[2]]; h3[2] = A.Z[first[2]];
            // the parameterised field at the middle hit sets the curvature scale
            const float kbs = kParamField ? G.kb * bz_factor(G.alpha, h2[0], h2[1], h2[2]) : G.kb;
            ok = seed_state(G.L[l0], kbs, h1, h2, h3, p, Q, eta);
        }
    }
    if (!ok) st |= MKF_ST_BADSEED;

    if (ok) {
        bool firsthit = true;
        // one hit: onto its layer (after the first), material, update; Cx is
        // the covariance (float[21]) or, through the seed hits, its square root
        auto hit = [&](auto Cx, int h) {
            const int l = A.hit_layer[h];
            if (l < 0 || l >= G.n_layers) {
                record_fault(A.fault, kFaultBadLayer, h);
                return;
            }
            const LayerDesc &Ld = G.L[l];
            if (!firsthit) {
                if (!move_to<kPhys>(G, Ld, p, lo, Cx)) {
                    st |= MKF_ST_UNREACHABLE;
                    return;
                }
                if (!kBackward && kMaterial) {
                    float mx0, mk;
                    material_at(G, Ld, p, mx0, mk);
                    add_scattering(Ld.kind, mx0, p, Cx);
                    apply_eloss(Ld.kind, mx0, mk, p, Cx, 1.f);
                }
            }
            firsthit = false;
            float dchi2;
            if (update_with(Ld, A.X[h], A.Y[h], A.Z[h], p, lo, Cx, dchi2)) {
                chi2 += dchi2;
                ++used;
            } else {
                st |= MKF_ST_BADS;
            }
            // reversed in time a layer's material follows its hit (at every hit,
            // the last one included): the energy lost there is gained back, then
            // the scattering noise is added
            if (kBackward && kMaterial) {
                float mx0, mk;
                material_at(G, Ld, p, mx0, mk);
                apply_eloss(Ld.kind, mx0, mk, p, Cx, -1.f);
                add_scattering(Ld.kind, mx0, p, Cx);
            }
        };
        auto hit_at = [&](int kk) {
            const int k = kBackward ? A.max_hits - 1 - kk : kk;
            const int h = A.hit_idx[(int64_t)k * A.n + t];
            return h < 0 || h >= A.n_hits ? -1 : h;
        };
        int kk = 0;
        if constexpr (!kBackward) {
            if (!A.seed_par) {  // from the seed prior: the seed hits with the square root
                for (; kk < A.max_hits && used < 3; ++kk) {
                    const int h = hit_at(kk);
                    if (h >= 0) hit(&Q, h);
                }
                sqrt_to_cov(Q, C);
            }
        }
        for (; kk < A.max_hits; ++kk) {
            const int h = hit_at(kk);
            if (h >= 0) hit(C, h);
        }
        if (kBackward) reverse_state(p, lo, C);
        if (!finite_state(p) || !isfinite(chi2)) st |= MKF_ST_NONFINITE;
    }
    const float nanv = __int_as_float(0x7fc00000);
    p[0] += lo.x;
    p[1] += lo.y;
    p[2] += lo.z;
    p[4] += lo.phi;
    p[5] += lo.th;
#pragma unroll
    for (int i = 0; i < 6; ++i) A.out_par[(int64_t)i * A.n + t] = ok ? p[i] : nanv;
#pragma unroll
    for (int k = 0; k < 21; ++k) A.out_cov[(int64_t)k * A.n + t] = ok ? C[k] : nanv;
    A.chi2[t] = chi2;
    A.ndf[t] = 2 * used - (G.kb != 0.f ? 5 : 4);
    A.status[t] = st;
}

// ---------------------------------------------------------------------------
// Smoother: the state at every hit from all of the track's hits (two filters).

// Weighted mean of two independent estimates (pf, Cf), (pb, Cb) of the state on
// a surface, in its five free parameters P p: (u, z, q/pT, phi, theta) on a
// cylinder (u along the surface, perpendicular to the radius at pf), (x, y,
// q/pT, phi, theta) on a disk.  The mean is symmetric in the two; the one with
// the smaller q/pT variance is taken as base (a): with d = P (po - pa) (phi
// wrapped), S = P (Ca + Co) P^T, X = S^-1 P Ca (Cholesky of S scaled to unit
// diagonal) and K = X^T: ps = pa + K d, and Cs in the Joseph form
// (I - K P) Ca (I - K P)^T + K (P Co P^T) K^T, a sum of two positive terms
// instead of the FP32 difference Ca - K P Ca, which cancels where one estimate
// is much sharper than the other.  The mean lies on the surface (radius or
// z = rz): a move along the tangent at pa is put back on it, and the position
// block of Cs is projected onto the tangent plane there.  False if S is not
// positive definite.
__device__ __forceinline__ bool combine5(int kind, float rz, const float pf_[6], const float Cf_[21],
                                         const float pb_[6], const float Cb_[21], float ps[6], float Cs[21]) {
    const bool swap = Cb_[9] < Cf_[9];
    const float *pf = swap ? pb_ : pf_, *Cf = swap ? Cb_ : Cf_;  // base
    const float *pb = swap ? pf_ : pb_, *Cb = swap ? Cf_ : Cb_;  // other
    float c = 1.f, sn = 0.f;
    if (kind == 0) {
        const float ir = 1.f / sqrtf(fmaf(pf[0], pf[0], pf[1] * pf[1]));
        c = pf[0] * ir;
        sn = pf[1] * ir;
    }
    // P v for a 6-vector v
    auto proj = [&](const float v[6], float o[5]) {
        if (kind == 0) {
            o[0] = fmaf(c, v[1], -sn * v[0]);
            o[1] = v[2];
        } else {
            o[0] = v[0];
            o[1] = v[1];
        }
        o[2] = v[3];
        o[3] = v[4];
        o[4] = v[5];
    };
    float dp[6], d[5];
#pragma unroll
    for (int i = 0; i < 6; ++i) dp[i] = pb[i] - pf[i];
    dp[4] = wrap_pi(dp[4]);
    proj(dp, d);
    // PC = P Cf (5 x 6), PS = P (Cf + Cb) (5 x 6)
    float PC[5][6], PS[5][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float cf[6], cs[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            cf[i] = Cf[sym(i, j)];
            cs[i] = cf[i] + Cb[sym(i, j)];
        }
        float o[5], q[5];
        proj(cf, o);
        proj(cs, q);
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            PC[a][j] = o[a];
            PS[a][j] = q[a];
        }
    }
    // S = PS P^T, scaled to unit diagonal
    float S[5][5], sc[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        float row[5];
        proj(PS[a], row);
#pragma unroll
        for (int b = 0; b < 5; ++b) S[a][b] = row[b];
    }
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        if (!(S[a][a] > 0.f)) return false;
        sc[a] = 1.f / sqrtf(S[a][a]);
    }
    // Cholesky of the scaled S (lower triangle in place)
    float L[5][5];
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float v = S[a][b] * sc[a] * sc[b];
#pragma unroll
            for (int m = 0; m < b; ++m) v = fmaf(-L[a][m], L[b][m], v);
            if (a == b) {
                if (!(v > 0.f)) return false;
                L[a][a] = sqrtf(v);
            } else {
                L[a][b] = v / L[b][b];
            }
        }
    // X = S^-1 PC column by column (and S^-1 d), through the scaling
    float X[5][6], y[5];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        float r[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) r[a] = (j < 6 ? PC[a][j] : d[a]) * sc[a];
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            float v = r[a];
#pragma unroll
            for (int m = 0; m < a; ++m) v = fmaf(-L[a][m], r[m], v);
            r[a] = v / L[a][a];
        }
#pragma unroll
        for (int a = 4; a >= 0; --a) {
            float v = r[a];
#pragma unroll
            for (int m = a + 1; m < 5; ++m) v = fmaf(-L[m][a], r[m], v);
            r[a] = v / L[a][a];
        }
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            if (j < 6)
                X[a][j] = r[a] * sc[a];
            else
                y[a] = r[a] * sc[a];
        }
    }
    // ps = pf + Cf P^T S^-1 d = pf + PC^T y
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float v = pf[i];
#pragma unroll
        for (int a = 0; a < 5; ++a) v = fmaf(PC[a][i], y[a], v);
        ps[i] = v;
    }
    ps[4] = wrap_pi(ps[4]);
    if (kind == 0) {
        const float f = rz / sqrtf(fmaf(ps[0], ps[0], ps[1] * ps[1]));
        ps[0] *= f;
        ps[1] *= f;
    } else {
        ps[2] = rz;
    }
    // Joseph form with K[i][a] = X[a][i]: A = I - K P
    float Am[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float e[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        e[i] = 1.f;
        float kp[6];
        if (kind == 0) {
            kp[0] = -sn * X[0][i];
            kp[1] = c * X[0][i];
            kp[2] = X[1][i];
        } else {
            kp[0] = X[0][i];
            kp[1] = X[1][i];
            kp[2] = 0.f;
        }
        kp[3] = X[2][i];
        kp[4] = X[3][i];
        kp[5] = X[4][i];
#pragma unroll
        for (int j = 0; j < 6; ++j) Am[i][j] = e[j] - kp[j];
    }
    // R = P Co P^T = P (Cf + Cb) P^T - P Cf P^T would cancel: from Co directly
    float R[5][5];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float cb[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) cb[i] = Cb[sym(i, j)];
        float o[5];
        proj(cb, o);
#pragma unroll
        for (int a = 0; a < 5; ++a) PS[a][j] = o[a];  // reuse: P Co
    }
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        float row[5];
        proj(PS[a], row);
#pragma unroll
        for (int b = 0; b < 5; ++b) R[a][b] = row[b];
    }
    // M = A Ca, KR = K R
    float M[6][6], KR[6][5];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            float v = 0.f;
#pragma unroll
            for (int m = 0; m < 6; ++m) v = fmaf(Am[i][m], Cf[sym(m, j)], v);
            M[i][j] = v;
        }
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            float v = 0.f;
#pragma unroll
            for (int a = 0; a < 5; ++a) v = fmaf(X[a][i], R[a][b], v);
            KR[i][b] = v;
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float v = 0.f;
#pragma unroll
            for (int m = 0; m < 6; ++m) v = fmaf(M[i][m], Am[j][m], v);
#pragma unroll
            for (int b = 0; b < 5; ++b) v = fmaf(KR[i][b], X[b][j], v);
            Cs[sym(i, j)] = v;
        }
    // no variance along the surface normal n at ps: Cs -> (I - n n^T) Cs (I - n n^T)
    float nv[3] = {0.f, 0.f, 1.f};
    if (kind == 0) {
        const float ir = 1.f / sqrtf(fmaf(ps[0], ps[0], ps[1] * ps[1]));
        nv[0] = ps[0] * ir, nv[1] = ps[1] * ir, nv[2] = 0.f;
    }
    float Q[6][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float col[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) col[i] = Cs[sym(i, j)];
        const float v = fmaf(nv[0], col[0], fmaf(nv[1], col[1], nv[2] * col[2]));
#pragma unroll
        for (int i = 0; i < 3; ++i) col[i] = fmaf(-nv[i], v, col[i]);
#pragma unroll
        for (int i = 0; i < 6; ++i) Q[i][j] = col[i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float v = fmaf(nv[0], Q[i][0], fmaf(nv[1], Q[i][1], nv[2] * Q[i][2]));
#pragma unroll
        for (int j = 0; j < 3; ++j) Q[i][j] = fmaf(-nv[j], v, Q[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) Cs[sym(i, j)] = Q[i][j];
    return true;
}

// One thread per track: the forward filter writes its state after each hit
// into that hit's output row; the backward filter then starts from the state at
// the last hit (turned around, covariance times inflate), predicts each earlier
// hit from the later ones, replaces the row by the weighted mean of the two
// (combine5) and is updated with the hit, its material applied in reverse.  The
// last hit's row keeps the forward state.
template <int kPhys>
__global__ void __launch_bounds__(128, 4) smooth_kernel(const __grid_constant__ FitArgs A) {
    constexpr bool kMaterial = kPhys >= 1, kParamField = kPhys == 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= A.n) return;
    const Geom &G = A.G;
    const float nanv = __int_as_float(0x7fc00000);
    const int64_t n = A.n;
    for (int k = 0; k < A.max_hits; ++k) {
#pragma unroll
        for (int i = 0; i < 6; ++i) A.sm_par[((int64_t)k * 6 + i) * n + t] = nanv;
#pragma unroll
        for (int i = 0; i < 21; ++i) A.sm_cov[((int64_t)k * 21 + i) * n + t] = nanv;
    }
    constexpr int kSq = kMaterial ? 9 : 5;  // square-root columns through the seed hits
    float p[6], C[21];
    SqrtCov<kSq> Q;
    Lo lo{0.f, 0.f, 0.f, 0.f, 0.f};
    uint32_t st = 0;
    float chi2 = 0.f;
    int used = 0;
    int first[3] = {-1, -1, -1}, nfirst = 0;
    for (int k = 0; k < A.max_hits; ++k) {
        const int h = A.hit_idx[(int64_t)k * n + t];
        if (h < 0) continue;
        if (h >= A.n_hits) {
            record_fault(A.fault, kFaultBadHitIndex, t);
            continue;
        }
        if (nfirst < 3) first[nfirst++] = h;
    }
    bool ok = nfirst >= 3;
    if (ok) {
        const int l0 = A.hit_layer[first[0]];
        if (l0 < 0 || l0 >= G.n_layers) {
            record_fault(A.fault, kFaultBadLayer, first[0]);
            ok = false;
        } else if (A.seed_par) {
#pragma unroll
            for (int i = 0; i < 6; ++i) p[i] = A.seed_par[(int64_t)i * n + t];
#pragma unroll
            for (int k = 0; k < 21; ++k) C[k] = A.seed_cov[(int64_t)k * n + t];
        } else {
            float h1[3], h2[3], h3[3], eta;
            h1[0] = A.X[first[0]]; h1[1] = A.Y[first[0]]; h1[2] = A.Z[first[0]];
            h2[0] = A.X[first[1]]; h2[1] = A.Y[first[1]]; h2[2] = A.Z[first[1]];
            h3[0] = A.X[first[2]]; h3[1] = A.Y[first[2]]; h3[2] = A.Z[first[2]];
            const float kbs = kParamField ? G.kb * bz_factor(G.alpha, h2[0], h2[1], h2[2]) : G.kb;
            ok = seed_state(G.L[l0], kbs, h1, h2, h3, p, Q, eta);
        }
    }
    if (!ok) st |= MKF_ST_BADSEED;

    // forward filter, its state after each hit kept in the hit's row
    int lastk = -1;
    if (ok) {
        bool firsthit = true;
        // one hit; Cx is the covariance (float[21]) or, through the seed hits,
        // its square root
        auto fwd = [&](auto Cx, int k, int h) {
            const int l = A.hit_layer[h];
            if (l < 0 || l >= G.n_layers) {
                record_fault(A.fault, kFaultBadLayer, h);
                return;
            }
            const LayerDesc &Ld = G.L[l];
            if (!firsthit) {
                if (!move_to<kPhys>(G, Ld, p, lo, Cx)) {
                    st |= MKF_ST_UNREACHABLE;
                    return;
                }
                if (kMaterial) {
                    float mx0, mk;
                    material_at(G, Ld, p, mx0, mk);
                    add_scattering(Ld.kind, mx0, p, Cx);
                    apply_eloss(Ld.kind, mx0, mk, p, Cx, 1.f);
                }
            }
            firsthit = false;
            float dchi2;
            if (update_with(Ld, A.X[h], A.Y[h], A.Z[h], p, lo, Cx, dchi2)) {
                chi2 += dchi2;
                ++used;
                const float pw[6] = {p[0] + lo.x, p[1] + lo.y, p[2] + lo.z, p[3], p[4] + lo.phi, p[5] + lo.th};
#pragma unroll
                for (int i = 0; i < 6; ++i) A.sm_par[((int64_t)k * 6 + i) * n + t] = pw[i];
                float Cw[21];
                if constexpr (std::is_same_v<decltype(Cx), float *>) {
#pragma unroll
                    for (int i = 0; i < 21; ++i) Cw[i] = Cx[i];
                } else {
                    sqrt_to_cov(*Cx, Cw);
                }
#pragma unroll
                for (int i = 0; i < 21; ++i) A.sm_cov[((int64_t)k * 21 + i) * n + t] = Cw[i];
                lastk = k;
            } else {
                st |= MKF_ST_BADS;
            }
        };
        int k = 0;
        if (!A.seed_par) {  // from the seed prior: the seed hits with the square root
            for (; k < A.max_hits && used < 3; ++k) {
                const int h = A.hit_idx[(int64_t)k * n + t];
                if (h >= 0 && h < A.n_hits) fwd(&Q, k, h);
            }
            sqrt_to_cov(Q, C);
        }
        for (; k < A.max_hits; ++k) {
            const int h = A.hit_idx[(int64_t)k * n + t];
            if (h >= 0 && h < A.n_hits) fwd(C, k, h);
        }
    }

    // backward filter and the weighted means
    if (lastk >= 0 && finite_state(p) && isfinite(chi2)) {
#pragma unroll
        for (int i = 0; i < 6; ++i) p[i] = A.sm_par[((int64_t)lastk * 6 + i) * n + t];
#pragma unroll
        for (int i = 0; i < 21; ++i) C[i] = A.sm_cov[((int64_t)lastk * 21 + i) * n + t] * A.inflate;
        lo = Lo{0.f, 0.f, 0.f, 0.f, 0.f};
        reverse_state(p, lo, C);
        for (int k = lastk; k >= 0; --k) {
            const int h = A.hit_idx[(int64_t)k * n + t];
            if (h < 0 || h >= A.n_hits) continue;
            const int l = A.hit_layer[h];
            if (l < 0 || l >= G.n_layers) continue;
            const LayerDesc &Ld = G.L[l];
            if (k < lastk) {
                if (!move_to<kPhys>(G, Ld, p, lo, C)) {
                    st |= MKF_ST_UNREACHABLE;
                    continue;
                }
                const float c0 = A.sm_cov[((int64_t)k * 21) * n + t];
                if (c0 == c0) {  // the forward filter has a state here
                    float pb[6] = {p[0] + lo.x, p[1] + lo.y, p[2] + lo.z, p[3], p[4], p[5]}, Cb[21];
                    Lo lb{0.f, 0.f, 0.f, lo.phi, lo.th};
#pragma unroll
                    for (int i = 0; i < 21; ++i) Cb[i] = C[i];
                    reverse_state(pb, lb, Cb);
                    pb[4] += lb.phi;
                    pb[5] += lb.th;
                    float pf[6], Cf[21], ps[6], Cs[21];
#pragma unroll
                    for (int i = 0; i < 6; ++i) pf[i] = A.sm_par[((int64_t)k * 6 + i) * n + t];
#pragma unroll
                    for (int i = 0; i < 21; ++i) Cf[i] = A.sm_cov[((int64_t)k * 21 + i) * n + t];
                    const bool good = combine5(Ld.kind, Ld.rz, pf, Cf, pb, Cb, ps, Cs);
                    if (!good) st |= MKF_ST_BADS;
#pragma unroll
                    for (int i = 0; i < 6; ++i) A.sm_par[((int64_t)k * 6 + i) * n + t] = good ? ps[i] : nanv;
#pragma unroll
                    for (int i = 0; i < 21; ++i) A.sm_cov[((int64_t)k * 21 + i) * n + t] = good ? Cs[i] : nanv;
                }
            }
            float dchi2;
            if (!update_with(Ld, A.X[h], A.Y[h], A.Z[h], p, lo, C, dchi2)) st |= MKF_ST_BADS;
            if (kMaterial) {
                float mx0, mk;
                material_at(G, Ld, p, mx0, mk);
                apply_eloss(Ld.kind, mx0, mk, p, C, -1.f);
                add_scattering(Ld.kind, mx0, p, C);
            }
        }
    }
    if (!isfinite(chi2)) st |= MKF_ST_NONFINITE;
    A.chi2[t] = chi2;
    A.ndf[t] = 2 * used - (G.kb != 0.f ? 5 : 4);
    A.status[t] = st;
}

}  // namespace

// mode: 0 forward fit, 1 backward fit, 2 smoother (out_par / out_cov are then
// the per-hit arrays [max_hits][6][n] / [max_hits][21][n]).
static mkf_status launch_fit(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits,
                             const int32_t *hit_idx, int32_t max_hits, int32_t n, const float *seed_par,
                             const float *seed_cov, float inflate, int mode, float *out_par, float *out_cov,
                             float *chi2, int32_t *ndf, uint32_t *status) {
    const bool backward = mode == 1;
    if (!ctx) return MKF_ERR_ARG;
    if (!ctx->has_geom) return MKF_ERR_GEOMETRY;
    if (n < 0 || n_hits < 0 || max_hits < 1) return MKF_ERR_ARG;
    if (max_hits > MKF_MAX_LAYERS) return MKF_ERR_CAPACITY;
    if (n_hits > MKF_MAX_HITS) return MKF_ERR_CAPACITY;
    if ((seed_par == nullptr) != (seed_cov == nullptr)) return MKF_ERR_ARG;
    if (mode != 0 && !(inflate >= 1.f && inflate < 3.0e38f)) return MKF_ERR_ARG;
    if (n == 0) return MKF_OK;
    if (!xyz || !hit_layer || !hit_idx || !out_par || !out_cov || !chi2 || !ndf || !status) return MKF_ERR_ARG;
    if (backward && !seed_par) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    FitArgs A;
    A.G = ctx->geom;
    A.X = xyz;
    A.Y = xyz + n_hits;
    A.Z = xyz + 2 * (int64_t)n_hits;
    A.hit_layer = hit_layer;
    A.n_hits = n_hits;
    A.hit_idx = hit_idx;
    A.max_hits = max_hits;
    A.n = n;
    A.seed_par = seed_par;
    A.seed_cov = seed_cov;
    A.inflate = inflate;
    A.out_par = mode == 2 ? nullptr : out_par;
    A.out_cov = mode == 2 ? nullptr : out_cov;
    A.sm_par = mode == 2 ? out_par : nullptr;
    A.sm_cov = mode == 2 ? out_cov : nullptr;
    A.chi2 = chi2;
    A.ndf = ndf;
    A.status = status;
    A.fault = ctx->fault;
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    if (mode == 2) {
        switch (mkf_phys_variant(ctx->geom)) {
            case 0: smooth_kernel<0><<<blocks, threads, 0, ctx->stream>>>(A); break;
            case 1: smooth_kernel<1><<<blocks, threads, 0, ctx->stream>>>(A); break;
            default: smooth_kernel<2><<<blocks, threads, 0, ctx->stream>>>(A); break;
        }
        MKF_CUDA_TRY(cudaGetLastError());
        return MKF_OK;
    }
    switch (mkf_phys_variant(ctx->geom) + (backward ? 3 : 0)) {
        case 0: fit_kernel<false, 0><<<blocks, threads, 0, ctx->stream>>>(A); break;
        case 1: fit_kernel<false, 1><<<blocks, threads, 0, ctx->stream>>>(A); break;
        case 2: fit_kernel<false, 2><<<blocks, threads, 0, ctx->stream>>>(A); break;
        case 3: fit_kernel<true, 0><<<blocks, threads, 0, ctx->stream>>>(A); break;
        case 4: fit_kernel<true, 1><<<blocks, threads, 0, ctx->stream>>>(A); break;
        default: fit_kernel<true, 2><<<blocks, threads, 0, ctx->stream>>>(A); break;
    }
    MKF_CUDA_TRY(cudaGetLastError());
    return MKF_OK;
}

extern "C" mkf_status mkf_fit(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits,
                              const int32_t *hit_idx, int32_t max_hits, int32_t n, const float *seed_par,
                              const float *seed_cov, float *out_par, float *out_cov, float *chi2, int32_t *ndf,
                              uint32_t *status) {
    return launch_fit(ctx, xyz, hit_layer, n_hits, hit_idx, max_hits, n, seed_par, seed_cov, 1.f, 0, out_par,
                      out_cov, chi2, ndf, status);
}

extern "C" mkf_status mkf_fit_backward(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits,
                                       const int32_t *hit_idx, int32_t max_hits, int32_t n, const float *last_par,
                                       const float *last_cov, float inflate, float *out_par, float *out_cov,
                                       float *chi2, int32_t *ndf, uint32_t *status) {
    return launch_fit(ctx, xyz, hit_layer, n_hits, hit_idx, max_hits, n, last_par, last_cov, inflate, 1, out_par,
                      out_cov, chi2, ndf, status);
}

extern "C" mkf_status mkf_fit_smooth(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits,
                                     const int32_t *hit_idx, int32_t max_hits, int32_t n, const float *seed_par,
                                     const float *seed_cov, float inflate, float *sm_par, float *sm_cov, float *chi2,
                                     int32_t *ndf, uint32_t *status) {
    return launch_fit(ctx, xyz, hit_layer, n_hits, hit_idx, max_hits, n, seed_par, seed_cov, inflate, 2, sm_par,
                      sm_cov, chi2, ndf, status);
}
