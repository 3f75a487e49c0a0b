// Device-side Kalman-filter math for one track candidate, FP32, register
// resident.  Shared by the fit and find kernels of libmkf.
//
// State p = (x, y, z, w = q/pT, phi, theta); covariance C packed lower triangle,
// C[i (i + 1) / 2 + j], i >= j.  Uniform field Bz: a track turns at the rate
// h = -w K Bz per unit transverse path s (Sec. 1 of the paper names helix
// propagation to barrel and endcap layers; the formulas are the textbook helix).
//
// Formulation chosen for FP32 on sm_103a:
//  * the helix step is written with the half turning angle a = h s / 2 and the
//    chord L = s sinc(a) in the direction phi + a, which stays exact as h -> 0;
//  * the crossing with a cylinder r = R is the root of a quadratic in
//    tau = tan(h s / 2) / h (half-angle substitution), solved in the
//    cancellation-free form, s = 2 tau atan(h tau) / (h tau);
//  * the Jacobian of the propagate-to-surface map is J = A + d g^T, with A the
//    fixed-path Jacobian (identity plus six entries), d = dF/ds and g = ds/dp
//    from the surface constraint; C' = J C J^T is evaluated from that structure
//    (about 150 FMAs instead of 432 for dense 6x6 products);
//  * the r-phi residual is R atan2(P x H, P . H) from the difference vector, so
//    no large angle is subtracted;
//  * position (x, y, z), phi and theta are carried as unevaluated float pairs
//    (hi + lo): an FP32 coordinate at r ~ 100 cm is only good to 7.6e-6 cm, a
//    few thousandths of a 20 um resolution, so moves, updates, R^2 - r^2 and
//    the residuals are formed with exact two-sum / two-product steps instead;
//    an FP32 theta near 2 rad is only good to 1.2e-7 rad, which moves z by
//    0.2 um over a metre of path (2e-3 of a 100 um resolution).
#pragma once

#include <cstdint>

namespace mkf {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kField = 0.0029979245800f;  // GeV / (T cm)
constexpr int kMaxLayers = 64;
constexpr int kMaxRegions = 16;

struct LayerDesc {
    int kind;         // 0 cylinder, 1 disk
    float rz;         // R or Z
    float lo, hi;     // extent: z (cylinder) or r (disk)
    float su2, sv2;   // measurement variances
    float seed_sig2;  // seed position variance for a first hit on this layer
    int nphi, nzr;    // bin grid
    int bin_base;     // first bin of this layer inside an event's bin block
    float phi_scale;  // nphi / (2 pi)
    float zr_scale;   // nzr / (hi - lo)
    float x0;         // material: radiation lengths at normal incidence (0 = none)
    float eloss;      // mean energy loss per radiation length at minimum ionisation, GeV (0 = none)
};

struct Geom {
    int n_layers;
    float cyl_hi_beyond[kMaxLayers];  // max z-extent end of the cylinders at and after each sorted position
    float cyl_lo_beyond[kMaxLayers];  // min z-extent start of the same
    float kb;  // K * Bz (at the centre for the parameterised field)
    int field_kind;  // 0 uniform, 1 parameterised (RK4 propagation)
    float alpha;     // parameterised field: fall-off coefficient, 1/cm^2
    // r-z material map (device memory of the context; null = the layers' own
    // material): map_nr x map_nz cells over [0, r_max) x [z_min, z_max), cell
    // (ir, iz) at ir * map_nz + iz holding (x0, eloss)
    const float2 *mat_map;
    int map_nr, map_nz;
    float map_rinv, map_zmin, map_zinv;  // map_nr / r_max, z_min, map_nz / (z_max - z_min)
    int n_cyl, n_dsk;
    int bins_per_event;
    int n_regions;
    LayerDesc L[kMaxLayers];
    int8_t cyl[kMaxLayers];      // cylinder ids sorted by radius
    int8_t dsk[kMaxLayers];      // disk ids sorted by z
    int8_t cyl_pos[kMaxLayers];  // layer id -> position in cyl[] (-1 if a disk)
    int8_t dsk_pos[kMaxLayers];  // layer id -> position in dsk[] (-1 if a cylinder)
    float edges[kMaxRegions];
    unsigned long long mask[kMaxRegions];
};

__host__ __device__ constexpr int sym(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

__device__ __forceinline__ float wrap_pi(float a) {
    if (a > kPi) a -= kTwoPi;
    else if (a < -kPi) a += kTwoPi;
    return a;
}

// Error-free transformations (Knuth two-sum, FMA two-product).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

// (hi, lo) += d, renormalised.
__device__ __forceinline__ void df_add(float &hi, float &lo, float d) {
    float s, e;
    two_sum(hi, d, s, e);
    e += lo;
    hi = s + e;
    lo = e - (hi - s);
}

// phi pair wrapped into [-pi, pi] with 2 pi as a float pair (a plain float 2 pi
// is off by 1.7e-7 rad).
__device__ __forceinline__ void df_wrap_pi(float &hi, float &lo) {
    constexpr float kTwoPiHi = 6.28318548202514648438f;
    constexpr float kTwoPiLo = -1.74845553146951e-7f;
    if (hi > kPi) {
        df_add(hi, lo, -kTwoPiHi);
        df_add(hi, lo, -kTwoPiLo);
    } else if (hi < -kPi) {
        df_add(hi, lo, kTwoPiHi);
        df_add(hi, lo, kTwoPiLo);
    }
}

// a^2 + b^2 - c^2 - d^2 for floats a, b, c, d (exact products, compensated sum).
__device__ __forceinline__ float diff_sq2(float a, float b, float c, float d) {
    float pa, ea, pb, eb, pc, ec, pd, ed;
    two_prod(a, a, pa, ea);
    two_prod(b, b, pb, eb);
    two_prod(c, c, pc, ec);
    two_prod(d, d, pd, ed);
    float s1, e1, s2, e2, s3, e3;
    two_sum(pa, pb, s1, e1);
    two_sum(pc, pd, s2, e2);
    two_sum(s1, -s2, s3, e3);
    return s3 + (e3 + ((e1 - e2) + ((ea + eb) - (ec + ed))));
}

// Low parts of the pairs: (x, y, z) = hi + lo per coordinate; phi and theta
// = hi + lo.
struct Lo {
    float x, y, z, phi, th;
};

// The covariance through the seed hits, as a square root C = S S^T with K
// columns (five for the prior, two more for each layer of material on the
// way; unused columns hold zeros).  From the seed prior (variances 1e-4 rad^2
// on the angles, (10 % of q/pT)^2 on q/pT) the three seed-hit updates shrink
// C by up to six orders of magnitude in the directions the hits measure; the
// FP32 entries of the transported prior (relative rounding 6e-8) no longer fix
// the small eigenvalues that remain, and a track in a thousand came out with
// its chi2 off by several 1e-3 of itself.  Rounding in the square root
// perturbs C by FP32 precision times the square root of its condition number
// instead (the classical property of square-root filters).  The seed hits'
// updates are scalar steps in Potter's form (sqrt_update); C = S S^T after the
// third hit continues in the plain FP32 filter.
template <int K>
struct SqrtCov {
    float S[6][K];
    int k;  // columns in use
};

// sin(a)/a and its derivative (a cos a - sin a)/a^2, series near 0.
__device__ __forceinline__ void sinc_and_deriv(float a, float sa, float ca, float& sn, float& dsn) {
    float a2 = a * a;
    if (fabsf(a) < 0.25f) {
        sn = 1.f - a2 * (1.f / 6.f) * (1.f - a2 * (1.f / 20.f) * (1.f - a2 * (1.f / 42.f) * (1.f - a2 * (1.f / 72.f))));
        dsn = a * (-1.f / 3.f + a2 * (1.f / 30.f + a2 * (-1.f / 840.f + a2 * (1.f / 45360.f - a2 * (1.f / 3991680.f)))));
    } else {
        sn = sa / a;
        dsn = (a * ca - sa) / a2;
    }
}

// atan(x)/x, series near 0.
__device__ __forceinline__ float atanc(float x) {
    float x2 = x * x;
    if (fabsf(x) < 0.125f) return 1.f - x2 * (1.f / 3.f - x2 * (1.f / 5.f - x2 * (1.f / 7.f - x2 * (1.f / 9.f))));
    return atanf(x) / x;
}

// asin(x)/x, series near 0.
__device__ __forceinline__ float asinc(float x) {
    x = fminf(1.f, fmaxf(-1.f, x));
    float x2 = x * x;
    if (fabsf(x) < 0.125f)
        return 1.f + x2 * (1.f / 6.f + x2 * (3.f / 40.f + x2 * (5.f / 112.f + x2 * (35.f / 1152.f))));
    return asinf(x) / x;
}

// sin and cos of a bounded angle, |x| <= 8 (state angles, half turning
// angles): Cody-Waite reduction x = k pi/2 + r with pi/2 split into two floats
// (the FMA forms k * hi exactly; |k| <= 5 keeps the split's own error below
// 1e-14), then the Taylor series of sin to r^9 and of cos to r^10 on
// |r| <= pi/4 (truncation below 2e-9 relative), and the quadrant swap.
__device__ __forceinline__ void sincos_small(float x, float &s, float &c) {
    constexpr float kPio2Hi = 1.57079637050628662109375f;   // float(pi/2)
    constexpr float kPio2Lo = -4.37113900018624283e-8f;     // pi/2 - float(pi/2)
    const float k = rintf(x * 0.636619772367581343f);       // x * 2/pi
    float r = fmaf(k, -kPio2Hi, x);
    r = fmaf(k, -kPio2Lo, r);
    const float r2 = r * r;
    float ps = fmaf(r2, 1.f / 362880.f, -1.f / 5040.f);
    ps = fmaf(r2, ps, 1.f / 120.f);
    ps = fmaf(r2, ps, -1.f / 6.f);
    ps = fmaf(r2 * r, ps, r);
    float pc = fmaf(r2, -1.f / 3628800.f, 1.f / 40320.f);
    pc = fmaf(r2, pc, -1.f / 720.f);
    pc = fmaf(r2, pc, 1.f / 24.f);
    pc = fmaf(r2, pc, -0.5f);
    pc = fmaf(r2, pc, 1.f);
    const int q = static_cast<int>(k) & 3;
    const float sa = (q & 1) ? pc : ps, ca = (q & 1) ? ps : pc;
    s = (q & 2) ? -sa : sa;
    c = ((q + 1) & 2) ? -ca : ca;
}

// sin and cos of an angle pair hi + lo (first-order correction for the low part).
__device__ __forceinline__ void sincos_pair(float hi, float lo, float& s, float& c) {
    float s0, c0;
    sincos_small(hi, s0, c0);
    s = fmaf(c0, lo, s0);
    c = fmaf(-s0, lo, c0);
}

// cot of the theta pair hi + lo.
__device__ __forceinline__ float cot_pair(float hi, float lo) {
    float st, ct;
    sincos_pair(hi, lo, st, ct);
    return ct / st;
}

// Smallest s in (0, pi/|h|) (or s > 0 when h = 0) with |P(s)| = R.
// D = R^2 - |P|^2 is formed from the position pair without cancellation.
__device__ __forceinline__ bool path_cyl(float x, float y, const Lo &lo, float sphi, float cphi, float h, float R,
                                         float &s_out) {
    const float b = fmaf(x, cphi, y * sphi);   // P0 . u
    const float nn = fmaf(y, cphi, -x * sphi); // P0 . n
    const float D = diff_sq2(R, 0.f, x, y) - 2.f * fmaf(x, lo.x, y * lo.y);
    const float a2 = 2.f + 2.f * h * nn - 0.5f * h * h * D;
    const float disc = fmaf(b, b, 0.5f * a2 * D);
    if (!(disc >= 0.f)) return false;
    const float sq = sqrtf(disc);
    const float qq = -(b + copysignf(sq, b));
    // s = 2 tau atan(h tau) / (h tau) has the sign of tau: only positive roots
    // are converted
    float best = __int_as_float(0x7f800000);
    if (qq != 0.f) {
        const float t = (-0.5f * D) / qq;
        if (t > 0.f) best = 2.f * t * atanc(h * t);
    }
    if (a2 != 0.f) {
        const float t = qq / a2;
        if (t > 0.f) {
            const float st = 2.f * t * atanc(h * t);
            if (st > 0.f && st < best) best = st;
        }
    }
    if (!(best < __int_as_float(0x7f800000))) return false;
    s_out = best;
    return true;
}

// Path to the disk plane z = Z (less than half a turn ahead), or false.
__device__ __forceinline__ bool path_disk(float z, const Lo &lo, float cot, float h, float Z, float &s) {
    if (cot == 0.f) return false;
    const float sd = ((Z - z) - lo.z) / cot;
    if (!(sd > 0.f)) return false;
    if (h != 0.f && fabsf(h) * sd >= kPi) return false;
    s = sd;
    return true;
}

// Path from state p to the surface of layer l (no extent check).
__device__ __forceinline__ bool path_to_layer(const LayerDesc& Ld, float kb, const float p[6], const Lo& lo, float sphi,
                                              float cphi, float cot, float& s) {
    float h = -p[3] * kb;
    if (Ld.kind == 0) return path_cyl(p[0], p[1], lo, sphi, cphi, h, Ld.rz, s);
    return path_disk(p[2], lo, cot, h, Ld.rz, s);
}

// Position after a move by s (chord form), without touching the state.
__device__ __forceinline__ void helix_point(const float p[6], float sphi, float cphi, float cot, float h, float s,
                                            float& x, float& y, float& z) {
    float a = 0.5f * h * s, sa, ca, sn, dsn;
    sincos_small(a, sa, ca);
    sinc_and_deriv(a, sa, ca, sn, dsn);
    float L = s * sn;
    float cm = cphi * ca - sphi * sa, sm = sphi * ca + cphi * sa;
    x = fmaf(L, cm, p[0]);
    y = fmaf(L, sm, p[1]);
    z = fmaf(s, cot, p[2]);
}

// Jacobian of the move onto a surface, J = A + d g^T: the entries of the
// fixed-path Jacobian A that differ from the identity, d = dF/ds and the
// nonzero entries of g = ds/dp (kind 0: cylinder, 1: disk).
struct HelixJac {
    float Axw, Ayw, Axf, Ayf, Azt, Afw;
    float d0, d1, d2, d4;
    float g0, g1, g2, g3, g4, g5;
    int kind;
};

// C' = J C J^T from that structure (about 150 FMAs instead of 432).
__device__ __forceinline__ void transport_cov(const HelixJac& J, float C[21]) {
    // full symmetric C in registers
    float Cf[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) Cf[i][j] = C[sym(i, j)];

    // M = A C
    float M[6][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        M[0][j] = fmaf(J.Axw, Cf[3][j], fmaf(J.Axf, Cf[4][j], Cf[0][j]));
        M[1][j] = fmaf(J.Ayw, Cf[3][j], fmaf(J.Ayf, Cf[4][j], Cf[1][j]));
        M[2][j] = fmaf(J.Azt, Cf[5][j], Cf[2][j]);
        M[3][j] = Cf[3][j];
        M[4][j] = fmaf(J.Afw, Cf[3][j], Cf[4][j]);
        M[5][j] = Cf[5][j];
    }
    // M += d (g^T C)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float v;
        if (J.kind == 0) v = fmaf(J.g0, Cf[0][j], fmaf(J.g1, Cf[1][j], fmaf(J.g3, Cf[3][j], J.g4 * Cf[4][j])));
        else v = fmaf(J.g2, Cf[2][j], J.g5 * Cf[5][j]);
        M[0][j] = fmaf(J.d0, v, M[0][j]);
        M[1][j] = fmaf(J.d1, v, M[1][j]);
        M[2][j] = fmaf(J.d2, v, M[2][j]);
        M[4][j] = fmaf(J.d4, v, M[4][j]);
    }
    // C' = M A^T + (M g) d^T, lower triangle
    float u[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        if (J.kind == 0) u[i] = fmaf(J.g0, M[i][0], fmaf(J.g1, M[i][1], fmaf(J.g3, M[i][3], J.g4 * M[i][4])));
        else u[i] = fmaf(J.g2, M[i][2], J.g5 * M[i][5]);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        C[sym(i, 0)] = fmaf(u[i], J.d0, fmaf(J.Axw, M[i][3], fmaf(J.Axf, M[i][4], M[i][0])));
        if (i >= 1) C[sym(i, 1)] = fmaf(u[i], J.d1, fmaf(J.Ayw, M[i][3], fmaf(J.Ayf, M[i][4], M[i][1])));
        if (i >= 2) C[sym(i, 2)] = fmaf(u[i], J.d2, fmaf(J.Azt, M[i][5], M[i][2]));
        if (i >= 3) C[sym(i, 3)] = M[i][3];
        if (i >= 4) C[sym(i, 4)] = fmaf(u[i], J.d4, fmaf(J.Afw, M[i][3], M[i][4]));
        if (i >= 5) C[sym(i, 5)] = M[i][5];
    }
}

// S' = J S, column by column.
template <int K>
__device__ __forceinline__ void transport_cov(const HelixJac& J, SqrtCov<K>* Q) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        float c[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) c[i] = Q->S[i][j];
        const float v = J.kind == 0 ? fmaf(J.g0, c[0], fmaf(J.g1, c[1], fmaf(J.g3, c[3], J.g4 * c[4])))
                                    : fmaf(J.g2, c[2], J.g5 * c[5]);
        Q->S[0][j] = fmaf(J.d0, v, fmaf(J.Axw, c[3], fmaf(J.Axf, c[4], c[0])));
        Q->S[1][j] = fmaf(J.d1, v, fmaf(J.Ayw, c[3], fmaf(J.Ayf, c[4], c[1])));
        Q->S[2][j] = fmaf(J.d2, v, fmaf(J.Azt, c[5], c[2]));
        Q->S[4][j] = fmaf(J.d4, v, fmaf(J.Afw, c[3], c[4]));
    }
}

// Move state p by path s onto the surface of layer Ld and transport its
// covariance (C as float[21], or a square root SqrtCov<K>*) with the
// surface-constrained Jacobian J = A + d g^T.
template <class Cov>
__device__ __forceinline__ void propagate_transport(const LayerDesc& Ld, float kb, float p[6], Lo& lo, Cov C,
                                                   float sphi, float cphi, float cot, float s) {
    const float h = -p[3] * kb;
    const float a = 0.5f * h * s;
    float sa, ca, sn, dsn;
    sincos_small(a, sa, ca);
    sinc_and_deriv(a, sa, ca, sn, dsn);
    const float L = s * sn;
    const float cm = cphi * ca - sphi * sa, sm = sphi * ca + cphi * sa;  // direction phi + a
    const float dx = L * cm, dy = L * sm;
    const float c2a = 1.f - 2.f * sa * sa, s2a = 2.f * sa * ca;
    const float cpe = cphi * c2a - sphi * s2a, spe = sphi * c2a + cphi * s2a;  // direction at the end
    float st, ct_unused;
    sincos_small(p[5], st, ct_unused);
    const float xe = p[0] + dx, ye = p[1] + dy;

    HelixJac J;
    J.kind = Ld.kind;
    // fixed-path Jacobian entries
    const float dxdh = 0.5f * s * fmaf(s * dsn, cm, -dy);
    const float dydh = 0.5f * s * fmaf(s * dsn, sm, dx);
    J.Axw = -kb * dxdh;
    J.Ayw = -kb * dydh;
    J.Axf = -dy;
    J.Ayf = dx;
    J.Azt = -s / (st * st);
    J.Afw = -kb * s;
    // d = dF/ds
    J.d0 = cpe;
    J.d1 = spe;
    J.d2 = cot;
    J.d4 = h;
    // g = ds/dp (only the nonzero entries)
    J.g0 = J.g1 = J.g2 = J.g3 = J.g4 = J.g5 = 0.f;
    if (Ld.kind == 0) {
        const float inv = -1.f / fmaf(xe, cpe, ye * spe);
        J.g0 = xe * inv;
        J.g1 = ye * inv;
        J.g3 = fmaf(xe, J.Axw, ye * J.Ayw) * inv;
        J.g4 = fmaf(xe, J.Axf, ye * J.Ayf) * inv;
    } else {
        const float inv = -1.f / cot;
        J.g2 = inv;
        J.g5 = J.Azt * inv;
    }
    transport_cov(J, C);

    df_add(p[0], lo.x, dx);
    df_add(p[1], lo.y, dy);
    if (Ld.kind == 1) {
        p[2] = Ld.rz;  // on the disk by construction
        lo.z = 0.f;
    } else {
        df_add(p[2], lo.z, s * cot);
    }
    df_add(p[4], lo.phi, 2.f * a);
    df_wrap_pi(p[4], lo.phi);
}

// ---------------------------------------------------------------------------
// Parameterised field (Sec. 2.1: a constant or a parameterised field, chosen
// per propagation).  The field of a solenoid near its centre to second order,
// from an axially symmetric scalar potential (divergence- and curl-free):
// K B = kb (alpha x z, alpha y z, 1 - alpha (z^2 - r^2 / 2)), kb = K Bz(0).
// Propagation integrates the equation of motion with the path length S as
// variable, dr/dS = T, dT/dS = lambda T x (K B), lambda = q/p, by classical
// Runge-Kutta steps.

constexpr float kRkTurn = 0.05f;  // largest turning angle per step, rad
constexpr float kRkLen = 10.f;    // largest step, cm of path
constexpr int kRkMaxN = 16;       // most steps per propagation
constexpr int kRkNewton = 2;      // correction steps onto the surface

// C' = J C J^T for a dense Jacobian.
__device__ __forceinline__ void transport_cov(const float (&J)[6][6], float C[21]) {
    float M[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float a = 0.f;
#pragma unroll
            for (int m = 0; m < 6; ++m) a = fmaf(J[i][m], C[sym(m, k)], a);
            M[i][k] = a;
        }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) a = fmaf(M[i][k], J[j][k], a);
            C[sym(i, j)] = a;
        }
}

// S' = J S for a dense Jacobian.
template <int K>
__device__ __forceinline__ void transport_cov(const float (&J)[6][6], SqrtCov<K>* Q) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        float c[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) c[i] = Q->S[i][j];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            float a = 0.f;
#pragma unroll
            for (int m = 0; m < 6; ++m) a = fmaf(J[i][m], c[m], a);
            Q->S[i][j] = a;
        }
    }
}

// Bz(x, y, z) / Bz(0).
__device__ __forceinline__ float bz_factor(float alpha, float x, float y, float z) {
    return fmaf(-alpha, fmaf(z, z, -0.5f * fmaf(x, x, y * y)), 1.f);
}

__device__ __forceinline__ void kfield(float kb, float alpha, float x, float y, float z, float b[3]) {
    const float kaz = kb * alpha * z;
    b[0] = kaz * x;
    b[1] = kaz * y;
    b[2] = kb * bz_factor(alpha, x, y, z);
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = fmaf(a[1], b[2], -a[2] * b[1]);
    c[1] = fmaf(a[2], b[0], -a[0] * b[2]);
    c[2] = fmaf(a[0], b[1], -a[1] * b[0]);
}

// Trajectory data of one Runge-Kutta stage: position, direction, field K B,
// T x (K B).
struct RkStage {
    float x[3], T[3], b[3], tb[3];
};

__device__ __forceinline__ void rk_stage(float kb, float alpha, const float r0[3], const float d[3], const float T[3],
                                         RkStage &S) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        S.x[i] = r0[i] + d[i];
        S.T[i] = T[i];
    }
    kfield(kb, alpha, S.x[0], S.x[1], S.x[2], S.b);
    cross3(T, S.b, S.tb);
}

// Variational equation of the direction at a stage: d(dT)/dS = dlambda (T x b)
// + lambda (dT x b) + lambda T x (grad b . dr), with the field's gradient
// grad b . dr = kb alpha (z dx + x dz, z dy + y dz, x dx + y dy - 2 z dz).
__device__ __forceinline__ void tangent_rhs(const RkStage &S, float kba, float lam, float dlam, const float dr[3],
                                            const float dt[3], float out[3]) {
    const float x = S.x[0], y = S.x[1], z = S.x[2];
    const float g[3] = {kba * fmaf(z, dr[0], x * dr[2]), kba * fmaf(z, dr[1], y * dr[2]),
                        kba * fmaf(x, dr[0], fmaf(y, dr[1], -2.f * z * dr[2]))};
    float u[3], v[3];
    cross3(dt, S.b, u);
    cross3(S.T, g, v);
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i] = fmaf(dlam, S.tb[i], lam * (u[i] + v[i]));
}

// One classical Runge-Kutta step of path hs for the trajectory (d, T) and then,
// over the same stages, for the six tangent columns (Dr, DT) of the parameters
// (x, y, z, q/pT, phi, theta), whose lambda derivatives are dl.
// d is the displacement from r0, dlo the rounding error of its updates (a
// float pair, as the state's positions).
__device__ __forceinline__ void rk_step(float kb, float alpha, const float r0[3], float lam, const float dl[6],
                                        float d[3], float dlo[3], float T[3], float Dr[6][3], float DT[6][3],
                                        float hs) {
    RkStage S[4];
    const float hh = 0.5f * hs, h6 = hs * (1.f / 6.f);
    float dd[3], tt[3], sd[3], st[3];
    rk_stage(kb, alpha, r0, d, T, S[0]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dd[i] = fmaf(hh, T[i], d[i]);
        tt[i] = fmaf(hh * lam, S[0].tb[i], T[i]);
        sd[i] = T[i];
        st[i] = S[0].tb[i];
    }
    rk_stage(kb, alpha, r0, dd, tt, S[1]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dd[i] = fmaf(hh, S[1].T[i], d[i]);
        tt[i] = fmaf(hh * lam, S[1].tb[i], T[i]);
        sd[i] = fmaf(2.f, S[1].T[i], sd[i]);
        st[i] = fmaf(2.f, S[1].tb[i], st[i]);
    }
    rk_stage(kb, alpha, r0, dd, tt, S[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dd[i] = fmaf(hs, S[2].T[i], d[i]);
        tt[i] = fmaf(hs * lam, S[2].tb[i], T[i]);
        sd[i] = fmaf(2.f, S[2].T[i], sd[i]);
        st[i] = fmaf(2.f, S[2].tb[i], st[i]);
    }
    rk_stage(kb, alpha, r0, dd, tt, S[3]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        df_add(d[i], dlo[i], h6 * (sd[i] + S[3].T[i]));
        T[i] = fmaf(h6 * lam, st[i] + S[3].tb[i], T[i]);
    }
    const float kba = kb * alpha;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        float ar[3], at[3], ir[3], it[3], k[3];
        // stage 1
        tangent_rhs(S[0], kba, lam, dl[c], Dr[c], DT[c], k);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            ar[i] = DT[c][i];
            at[i] = k[i];
            ir[i] = fmaf(hh, DT[c][i], Dr[c][i]);
            it[i] = fmaf(hh, k[i], DT[c][i]);
        }
        // stage 2
        tangent_rhs(S[1], kba, lam, dl[c], ir, it, k);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            ar[i] = fmaf(2.f, it[i], ar[i]);
            at[i] = fmaf(2.f, k[i], at[i]);
            ir[i] = fmaf(hh, it[i], Dr[c][i]);
            it[i] = fmaf(hh, k[i], DT[c][i]);
        }
        // stage 3
        tangent_rhs(S[2], kba, lam, dl[c], ir, it, k);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            ar[i] = fmaf(2.f, it[i], ar[i]);
            at[i] = fmaf(2.f, k[i], at[i]);
            ir[i] = fmaf(hs, it[i], Dr[c][i]);
            it[i] = fmaf(hs, k[i], DT[c][i]);
        }
        // stage 4
        tangent_rhs(S[3], kba, lam, dl[c], ir, it, k);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Dr[c][i] = fmaf(h6, ar[i] + it[i], Dr[c][i]);
            DT[c][i] = fmaf(h6, at[i] + k[i], DT[c][i]);
        }
    }
}

// Root nearest 0 of a d^2 + b d + c = 0; the parabola's vertex when it has no
// real root, the linear root when a = 0.
__device__ __forceinline__ float nearest_root(float a, float b, float c) {
    const float disc = fmaf(b, b, -4.f * a * c);
    if (a == 0.f) return b != 0.f ? -c / b : 0.f;
    if (disc < 0.f) return -b / (2.f * a);
    const float q = -0.5f * (b + copysignf(sqrtf(disc), b));
    if (q == 0.f) return 0.f;
    const float r1 = q / a, r2 = c / q;
    return fabsf(r1) < fabsf(r2) ? r1 : r2;
}

// Move p onto the surface of layer Ld through the parameterised field and
// transport C.  n equal steps over the path s estimated by the helix in the
// local axial field (turning rate h), n from the turning angle and the path
// length, then kRkNewton correction steps onto the surface (on a cylinder the
// nearest root of the second-order expansion of x(S)^2 + y(S)^2 - R^2, whose
// bending term keeps grazing crossings converging; on a disk (Z - z) / Tz).  The Jacobian: the six
// parameter columns (dr, dT) integrated with the trajectory (the variational
// equations, the field's gradient included), then the surface constraint
// dS = -(n . dr) / (n . T) moves every column along (T, dT/dS) at the end.
template <class Cov>
__device__ __forceinline__ void propagate_field(const LayerDesc &Ld, float kb, float alpha, float p[6], Lo &lo,
                                                Cov C, float sphi, float cphi, float h, float s) {
    float st, ct;
    sincos_pair(p[5], lo.th, st, ct);
    const float lam = p[3] * st;
    const float dl[6] = {0.f, 0.f, 0.f, st, 0.f, p[3] * ct};  // d lambda / d(x, y, z, q/pT, phi, theta)
    float T[3] = {st * cphi, st * sphi, ct};
    float d[3] = {0.f, 0.f, 0.f}, dlo[3] = {0.f, 0.f, 0.f};
    float Dr[6][3], DT[6][3];
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Dr[c][i] = c == i ? 1.f : 0.f;
            DT[c][i] = 0.f;
        }
    DT[4][0] = -st * sphi, DT[4][1] = st * cphi;
    DT[5][0] = ct * cphi, DT[5][1] = ct * sphi, DT[5][2] = -st;
    const float r0[3] = {p[0], p[1], p[2]};
    const float S = s / st;
    const float nf = ceilf(fmaxf(fabsf(h) * s * (1.f / kRkTurn), fabsf(S) * (1.f / kRkLen)));
    const int n = nf >= 1.f ? (nf < static_cast<float>(kRkMaxN) ? static_cast<int>(nf) : kRkMaxN) : 1;
    const float hs = S / static_cast<float>(n);
    for (int i = 0; i < n; ++i) rk_step(kb, alpha, r0, lam, dl, d, dlo, T, Dr, DT, hs);
    for (int it = 0; it < kRkNewton; ++it) {
        float dn;
        if (Ld.kind == 0) {
            // r^2 - R^2 from the position pair without cancellation
            const float xl = (lo.x + dlo[0]) + d[0], yl = (lo.y + dlo[1]) + d[1];
            const float x = p[0] + xl, y = p[1] + yl;
            const float c = 2.f * fmaf(p[0], xl, p[1] * yl) + fmaf(xl, xl, yl * yl) - diff_sq2(Ld.rz, 0.f, p[0], p[1]);
            float b[3];
            kfield(kb, alpha, r0[0] + d[0], r0[1] + d[1], r0[2] + d[2], b);
            const float Fx = lam * fmaf(T[1], b[2], -T[2] * b[1]), Fy = lam * fmaf(T[2], b[0], -T[0] * b[2]);
            const float aq = fmaf(T[0], T[0], fmaf(T[1], T[1], fmaf(x, Fx, y * Fy)));
            dn = nearest_root(aq, 2.f * fmaf(x, T[0], y * T[1]), c);
        } else {
            dn = ((Ld.rz - p[2]) - ((lo.z + dlo[2]) + d[2])) / T[2];
        }
        rk_step(kb, alpha, r0, lam, dl, d, dlo, T, Dr, DT, dn);
    }

    // end point: dT/dS, surface normal, output conversions
    float b[3], F[3];
    kfield(kb, alpha, r0[0] + d[0], r0[1] + d[1], r0[2] + d[2], b);
    cross3(T, b, F);
#pragma unroll
    for (int i = 0; i < 3; ++i) F[i] *= lam;
    float nv[3] = {0.f, 0.f, 1.f};
    if (Ld.kind == 0) {
        const float x = p[0] + (lo.x + d[0]), y = p[1] + (lo.y + d[1]);
        const float ir = 1.f / sqrtf(fmaf(x, x, y * y));
        nv[0] = x * ir, nv[1] = y * ir, nv[2] = 0.f;
    }
    const float inT = -1.f / fmaf(nv[0], T[0], fmaf(nv[1], T[1], nv[2] * T[2]));
    const float tt2 = fmaf(T[0], T[0], T[1] * T[1]), tn2 = fmaf(T[2], T[2], tt2);
    const float tt = sqrtf(tt2), itt = 1.f / tt, itt2 = itt * itt;
    const float sth = tt / sqrtf(tn2);  // sin(theta) at the end
    // J columns (outputs x, y, z, q/pT, phi, theta) of a tangent (dr, dT, dlambda)
    float J[6][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const float *dr = Dr[j], *dT = DT[j];
        const float dlam = dl[j];
        const float dS = fmaf(nv[0], dr[0], fmaf(nv[1], dr[1], nv[2] * dr[2])) * inT;
        float r[3], t[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            r[i] = fmaf(T[i], dS, dr[i]);
            t[i] = fmaf(F[i], dS, dT[i]);
        }
        const float dtt = fmaf(T[0], t[0], T[1] * t[1]) * itt;
        J[0][j] = r[0];
        J[1][j] = r[1];
        J[2][j] = r[2];
        J[3][j] = fmaf(dlam, itt, -lam * dtt * itt2);
        J[4][j] = fmaf(T[0], t[1], -T[1] * t[0]) * itt2;
        J[5][j] = fmaf(T[2], dtt, -tt * t[2]) / tn2;
    }

    transport_cov(J, C);

    // state at the end: position pairs, azimuth turned by the angle between
    // the start and end transverse directions, theta and q/pT = lambda / sin(theta)
    df_add(p[0], lo.x, d[0]);
    df_add(p[0], lo.x, dlo[0]);
    df_add(p[1], lo.y, d[1]);
    df_add(p[1], lo.y, dlo[1]);
    if (Ld.kind == 1) {
        p[2] = Ld.rz;
        lo.z = 0.f;
    } else {
        df_add(p[2], lo.z, d[2]);
        df_add(p[2], lo.z, dlo[2]);
    }
    df_add(p[4], lo.phi, atan2f(fmaf(cphi, T[1], -sphi * T[0]), fmaf(cphi, T[0], sphi * T[1])));
    df_wrap_pi(p[4], lo.phi);
    // theta turned by the angle between the start and end polar directions
    // (sin, cos) = (st, ct) and (tt, T[2]) / |T|
    df_add(p[5], lo.th, atan2f(fmaf(tt, ct, -T[2] * st), fmaf(T[2], ct, tt * st)));
    p[3] = lam / sth;
}

// Multiple scattering in the layer's material, added to the covariance of a
// state on its surface (Sec. 2.1 takes radiation lengths from an r-z table;
// here each layer has one thickness): theta0 = 0.0136 GeV / (beta p) sqrt(x) (1 + 0.038 ln(x / beta^2))
// (Highland, as tabulated by the Particle Data Group; unit charge, pion mass)
// for the path x = x0 / |cos a| through the layer, a = angle between the
// direction and the surface normal; Var(theta) += theta0^2, Var(phi) +=
// theta0^2 / sin^2(theta), and with |p| unchanged q/pT follows theta:
// Var(q/pT) += (q/pT cot(theta) theta0)^2, Cov(q/pT, theta) += -(q/pT) cot(theta) theta0^2.
// Material where the state p crosses layer Ld: the r-z map's cell holding
// (r, z) when a map is loaded (cells of equal size; points outside it take the
// nearest edge cell), else the layer's own thickness x0 and loss coefficient k.
__device__ __forceinline__ void material_at(const Geom &G, const LayerDesc &Ld, const float p[6], float &x0, float &k) {
    if (G.mat_map == nullptr) {
        x0 = Ld.x0;
        k = Ld.eloss;
        return;
    }
    const float r = sqrtf(fmaf(p[0], p[0], p[1] * p[1]));
    const int ir = min(max(static_cast<int>(floorf(r * G.map_rinv)), 0), G.map_nr - 1);
    const int iz = min(max(static_cast<int>(floorf((p[2] - G.map_zmin) * G.map_zinv)), 0), G.map_nz - 1);
    const float2 m = G.mat_map[ir * G.map_nz + iz];
    x0 = m.x;
    k = m.y;
}

// t: thickness in radiation lengths at normal incidence (material_at).
// theta0, (q/pT) cot(theta) and sin(theta) of the crossing; false if no noise.
__device__ __forceinline__ bool scatter_angle(int kind, float t, const float p[6], float &th0, float &wc, float &st) {
    // q/pT = 0: no field, momentum not measured; taken as infinite (no noise)
    if (!(t > 0.f) || !(fabsf(p[3]) > 0.f)) return false;
    constexpr float kPionMass2 = 0.13957f * 0.13957f;
    float ct;
    sincos_small(p[5], st, ct);
    float cosa;
    if (kind == 0) {
        float sp, cp;
        sincos_small(p[4], sp, cp);
        cosa = fabsf(st * fmaf(cp, p[0], sp * p[1]) / sqrtf(fmaf(p[0], p[0], p[1] * p[1])));
    } else {
        cosa = fabsf(ct);
    }
    cosa = fmaxf(cosa, 1e-6f);
    const float pm = 1.f / (fabsf(p[3]) * st);
    const float beta = pm / sqrtf(fmaf(pm, pm, kPionMass2));
    const float x = t / cosa;
    th0 = 0.0136f / (beta * pm) * sqrtf(x) * (1.f + 0.038f * logf(x / (beta * beta)));
    wc = p[3] * ct / st;
    return true;
}

__device__ __forceinline__ void add_scattering(int kind, float t, const float p[6], float C[21]) {
    float th0, wc, st;
    if (!scatter_angle(kind, t, p, th0, wc, st)) return;
    const float v = th0 * th0;
    C[sym(5, 5)] += v;
    C[sym(4, 4)] += v / (st * st);
    C[sym(3, 3)] += wc * wc * v;
    C[sym(5, 3)] -= wc * v;
}

// The same noise as two columns of the square root: theta0 (-wc e_q/pT + e_theta)
// and theta0 / sin(theta) e_phi.  (Room for them is kept: material is met on
// arrival at the second and third seed hits' layers only.)
template <int K>
__device__ __forceinline__ void add_scattering(int kind, float t, const float p[6], SqrtCov<K> *Q) {
    float th0, wc, st;
    if (!scatter_angle(kind, t, p, th0, wc, st)) return;
    const int k = Q->k;
    if (k + 2 > K) return;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (j == k) {
            Q->S[3][j] = -wc * th0;
            Q->S[5][j] = th0;
        }
        if (j == k + 1) Q->S[4][j] = th0 / st;
    }
    Q->k = k + 2;
}

// Mean energy loss in the material (no straggling): dE = k * x / beta^2 for the
// path x = t / |cos a| (pion mass), at fixed direction; sign +1 loses it
// (forward in time), -1 gains it back (the backward fit).  q/pT scales by
// r = p / p'; C is transported with the derivative of q/pT' = q/pT g(p),
// g = p / p'(p), p = 1 / (|q/pT| sin theta), in q/pT and theta (the path held
// fixed): dp'/dp = (E' / p') (p / E + 2 k x m^2 / p^3), g' = 1 / p' - p dp'/dp / p'^2,
// d(q/pT')/d(q/pT) = g - p g', d(q/pT')/d(theta) = -(q/pT) p cot(theta) g'.
// q/pT scaled in place; (a, c) = the derivatives of q/pT' in q/pT and theta;
// false if nothing changes.
__device__ __forceinline__ bool eloss_map(int kind, float t, float k, float p[6], float sign, float &a, float &c) {
    if (!(k > 0.f) || !(t > 0.f) || !(fabsf(p[3]) > 0.f)) return false;
    constexpr float kPionMass = 0.13957f;
    float st, ct;
    sincos_small(p[5], st, ct);
    float cosa;
    if (kind == 0) {
        float sp, cp;
        sincos_small(p[4], sp, cp);
        cosa = fabsf(st * fmaf(cp, p[0], sp * p[1]) / sqrtf(fmaf(p[0], p[0], p[1] * p[1])));
    } else {
        cosa = fabsf(ct);
    }
    cosa = fmaxf(cosa, 1e-6f);
    const float pm = 1.f / (fabsf(p[3]) * st);
    const float e = sqrtf(fmaf(pm, pm, kPionMass * kPionMass));
    const float beta = pm / e;
    const float kx = sign * k * (t / cosa);
    const float e2 = e - kx / (beta * beta);
    if (!(e2 > kPionMass)) return false;  // stopped: left as it is
    const float p2 = sqrtf(fmaf(e2, e2, -kPionMass * kPionMass));
    const float r = pm / p2;
    const float dp2 = e2 / p2 * (pm / e + 2.f * kx * (kPionMass * kPionMass) / (pm * pm * pm));
    const float gp = 1.f / p2 - pm * dp2 / (p2 * p2);
    a = r - pm * gp;
    c = -p[3] * pm * (ct / st) * gp;
    p[3] *= r;
    return true;
}

__device__ __forceinline__ void apply_eloss(int kind, float t, float k, float p[6], float C[21], float sign) {
    float a, c;
    if (!eloss_map(kind, t, k, p, sign, a, c)) return;
    float row[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) row[j] = fmaf(a, C[sym(3, j)], c * C[sym(5, j)]);
    const float c33 = fmaf(a, row[3], c * row[5]);
#pragma unroll
    for (int j = 0; j < 6; ++j) C[sym(3, j)] = j == 3 ? c33 : row[j];
}

// The same map on the square root's q/pT row.
template <int K>
__device__ __forceinline__ void apply_eloss(int kind, float t, float k, float p[6], SqrtCov<K> *Q, float sign) {
    float a, c;
    if (!eloss_map(kind, t, k, p, sign, a, c)) return;
#pragma unroll
    for (int j = 0; j < K; ++j) Q->S[3][j] = fmaf(a, Q->S[3][j], c * Q->S[5][j]);
}

// Measurement frame at the state's position: unit radial vector (cp, sp), radius.
struct Frame {
    float cp, sp, rt, r2;
};

__device__ __forceinline__ Frame frame_of(const float p[6]) {
    Frame f;
    f.r2 = fmaf(p[0], p[0], p[1] * p[1]);
    f.rt = sqrtf(f.r2);
    float inv = 1.f / f.rt;
    f.cp = p[0] * inv;
    f.sp = p[1] * inv;
    return f;
}

// S = H C H^T + V (2x2), its inverse and H C (two rows); false if S is not
// positive definite.  H_u = (-sin, cos, 0...) of the position azimuth;
// H_v = (0, 0, 1, ...) on cylinders, (cos, sin, 0, ...) on disks.
struct Innov {
    float HCu[6], HCv[6];
    float Suu, Suv, Svv;
    float Iuu, Iuv, Ivv;
};

__device__ __forceinline__ bool innovation(int kind, float su2, float sv2, const Frame& f, const float C[21], Innov& I) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        I.HCu[j] = fmaf(-f.sp, C[sym(0, j)], f.cp * C[sym(1, j)]);
        I.HCv[j] = kind == 0 ? C[sym(2, j)] : fmaf(f.cp, C[sym(0, j)], f.sp * C[sym(1, j)]);
    }
    I.Suu = fmaf(-f.sp, I.HCu[0], f.cp * I.HCu[1]) + su2;
    if (kind == 0) {
        I.Suv = I.HCu[2];
        I.Svv = I.HCv[2] + sv2;
    } else {
        I.Suv = fmaf(f.cp, I.HCu[0], f.sp * I.HCu[1]);
        I.Svv = fmaf(f.cp, I.HCv[0], f.sp * I.HCv[1]) + sv2;
    }
    float det = fmaf(I.Suu, I.Svv, -I.Suv * I.Suv);
    if (!(I.Suu > 0.f && det > 0.f)) return false;
    float id = 1.f / det;
    I.Iuu = I.Svv * id;
    I.Ivv = I.Suu * id;
    I.Iuv = -I.Suv * id;
    return true;
}

// Residual (u, v) of a hit against the state on the layer surface.
// zr_hit = z (cylinder) or r of the hit (disk; recomputed here from x, y).
__device__ __forceinline__ void residual(int kind, float R, const float p[6], const Lo& lo, const Frame& f, float xh,
                                         float yh, float zr_hit, float& u, float& v) {
    const float dx = (xh - p[0]) - lo.x, dy = (yh - p[1]) - lo.y;
    const float cross = fmaf(p[0], dy, -p[1] * dx);
    const float dot = fmaf(p[0], dx, fmaf(p[1], dy, f.r2));
    // the angle between the two position vectors: a search window's hits are
    // within a small angle of the state, where atan(t), t = cross / dot, takes
    // its Taylor series to t^9 (truncation below 2e-11 relative for |t| < 1/8;
    // the fit 3.5 % faster, the finder unchanged)
    float dphi;
    if (fabsf(cross) < 0.125f * dot) {
        const float t = cross / dot, t2 = t * t;
        dphi = t * fmaf(-t2, fmaf(-t2, fmaf(-t2, fmaf(-t2, 1.f / 9.f, 1.f / 7.f), 1.f / 5.f), 1.f / 3.f), 1.f);
    } else {
        dphi = atan2f(cross, dot);
    }
    if (kind == 0) {
        u = R * dphi;
        v = (zr_hit - p[2]) - lo.z;
    } else {
        u = f.rt * dphi;
        // r_hit - r = (|H|^2 - |P|^2) / (r_hit + r), numerator without cancellation
        const float num = diff_sq2(xh, yh, p[0], p[1]) - 2.f * fmaf(p[0], lo.x, p[1] * lo.y);
        v = num / (sqrtf(fmaf(xh, xh, yh * yh)) + f.rt);
    }
}

__device__ __forceinline__ float chi2_of(const Innov& I, float u, float v) {
    return fmaf(u, fmaf(I.Iuu, u, I.Iuv * v), v * fmaf(I.Iuv, u, I.Ivv * v));
}

// Kalman gain K = C H^T S^-1 and the state update p += K r.
__device__ __forceinline__ void kf_gain_state(const Innov& I, float u, float v, float p[6], Lo& lo, float K0[6],
                                              float K1[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        K0[i] = fmaf(I.HCu[i], I.Iuu, I.HCv[i] * I.Iuv);
        K1[i] = fmaf(I.HCu[i], I.Iuv, I.HCv[i] * I.Ivv);
    }
    df_add(p[0], lo.x, fmaf(K0[0], u, K1[0] * v));
    df_add(p[1], lo.y, fmaf(K0[1], u, K1[1] * v));
    df_add(p[2], lo.z, fmaf(K0[2], u, K1[2] * v));
    p[3] = fmaf(K0[3], u, fmaf(K1[3], v, p[3]));
    df_add(p[4], lo.phi, fmaf(K0[4], u, K1[4] * v));
    df_wrap_pi(p[4], lo.phi);
    df_add(p[5], lo.th, fmaf(K0[5], u, K1[5] * v));
}

// Kalman update: K = C H^T S^-1, p += K r, C -= K (H C).
__device__ __forceinline__ void kf_apply(const Innov& I, float u, float v, float p[6], Lo& lo, float C[21]) {
    float K0[6], K1[6];
    kf_gain_state(I, u, v, p, lo, K0, K1);
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) C[sym(i, j)] = C[sym(i, j)] - fmaf(K0[i], I.HCu[j], K1[i] * I.HCv[j]);
}

// The same update with C in the Joseph form (I - K H) C (I - K H)^T + K V K^T,
// written C - K G^T - G K^T with G = (H C)^T - K S / 2 (equal to C - K H C
// for the optimal gain; about 50 more FMAs).  It holds for any gain, so the
// rounding of K enters C only at second order and C stays positive where an
// update shrinks a variance by orders of magnitude (the position along a
// layer after a long or scattered step), where C - K H C can turn a variance
// negative.  The fit kernels take it; the finder keeps the short form.
__device__ __forceinline__ void kf_apply_joseph(const Innov& I, float u, float v, float p[6], Lo& lo,
                                                float C[21]) {
    float K0[6], K1[6];
    kf_gain_state(I, u, v, p, lo, K0, K1);
    float G0[6], G1[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        G0[i] = fmaf(-0.5f * K0[i], I.Suu, fmaf(-0.5f * K1[i], I.Suv, I.HCu[i]));
        G1[i] = fmaf(-0.5f * K0[i], I.Suv, fmaf(-0.5f * K1[i], I.Svv, I.HCv[i]));
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j)
            C[sym(i, j)] = fmaf(-K0[i], G0[j], fmaf(-K1[i], G1[j], fmaf(-K0[j], G0[i], fmaf(-K1[j], G1[i], C[sym(i, j)]))));
}

// One measurement row h (variance r) through the square root, Potter's form:
// phi = S^T h, s = |phi|^2 + r, gain K = S phi / s, and
// S' = S - (gamma / s) (S phi) phi^T with gamma = 1 / (1 + sqrt(r / s)), so that
// S' S'^T = C - C h h^T C / s.  Adds the gain times the residual to dp and
// returns the residual's chi2 contribution.
template <int K>
__device__ __forceinline__ float potter_step(float (&S)[6][K], const float ph[K], float r, float res, float dp[6]) {
    float s = r;
#pragma unroll
    for (int j = 0; j < K; ++j) s = fmaf(ph[j], ph[j], s);
    float Sp[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) a = fmaf(S[i][j], ph[j], a);
        Sp[i] = a;
    }
    const float is = 1.f / s;
    const float kr = res * is;
    const float g = is / (1.f + sqrtf(r * is));
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        dp[i] = fmaf(Sp[i], kr, dp[i]);
        const float gs = -g * Sp[i];
#pragma unroll
        for (int j = 0; j < K; ++j) S[i][j] = fmaf(gs, ph[j], S[i][j]);
    }
    return res * kr;
}

// Kalman update with the square root: the residual (u, v) of the hit at the
// predicted state taken as two scalar measurements (their variances su2, sv2
// are independent), v's residual moved to the state after the u step.  The
// state changes as in the joint update and the two chi2 terms add up to
// r^T S^-1 r (exact algebra); returns that chi2.
template <int K>
__device__ __forceinline__ float sqrt_update(int kind, float su2, float sv2, const Frame& f, float u, float v,
                                             float p[6], Lo& lo, SqrtCov<K>* Q) {
    float dp[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float ph[K];
#pragma unroll
    for (int j = 0; j < K; ++j) ph[j] = fmaf(-f.sp, Q->S[0][j], f.cp * Q->S[1][j]);
    float chi2 = potter_step(Q->S, ph, su2, u, dp);
    const float v2 = v - (kind == 0 ? dp[2] : fmaf(f.cp, dp[0], f.sp * dp[1]));
#pragma unroll
    for (int j = 0; j < K; ++j) ph[j] = kind == 0 ? Q->S[2][j] : fmaf(f.cp, Q->S[0][j], f.sp * Q->S[1][j]);
    chi2 += potter_step(Q->S, ph, sv2, v2, dp);
    df_add(p[0], lo.x, dp[0]);
    df_add(p[1], lo.y, dp[1]);
    df_add(p[2], lo.z, dp[2]);
    p[3] += dp[3];
    df_add(p[4], lo.phi, dp[4]);
    df_wrap_pi(p[4], lo.phi);
    df_add(p[5], lo.th, dp[5]);
    return chi2;
}

// C = S S^T.
template <int K>
__device__ __forceinline__ void sqrt_to_cov(const SqrtCov<K>& Q, float C[21]) {
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float a = 0.f;
#pragma unroll
            for (int m = 0; m < K; ++m) a = fmaf(Q.S[i][m], Q.S[j][m], a);
            C[sym(i, j)] = a;
        }
}

// Seed state at hit 1 from three hits (circle in x-y, line in arc length-z),
// with a prior covariance whose position part lies in the first layer's
// surface, as its square root (five columns: the position along the surface's
// two directions, q/pT, phi, theta).  Returns false for degenerate hits.  Also
// returns eta of the estimate.
template <int K>
__device__ __forceinline__ bool seed_state(const LayerDesc& L1, float kb, const float h1[3], const float h2[3],
                                           const float h3[3], float p[6], SqrtCov<K>& Q, float& eta) {
    static_assert(K >= 5, "the prior takes five columns");
    float ax = h2[0] - h1[0], ay = h2[1] - h1[1];
    float bx = h3[0] - h1[0], by = h3[1] - h1[1];
    float cx = h3[0] - h2[0], cy = h3[1] - h2[1];
    float la = sqrtf(fmaf(ax, ax, ay * ay)), lb = sqrtf(fmaf(bx, bx, by * by)), lc = sqrtf(fmaf(cx, cx, cy * cy));
    if (!(la > 0.f && lb > 0.f && lc > 0.f)) return false;
    float h = 2.f * fmaf(ax, by, -ay * bx) / (la * lb * lc);
    float w = 0.f;
    if (kb != 0.f) w = -h / kb;
    else h = 0.f;
    float xa = 0.5f * h * la, xb = 0.5f * h * lb;
    float phi0 = atan2f(ay, ax) - xa * asinc(xa);
    float s13 = lb * asinc(xb);
    float cot = (h3[2] - h1[2]) / s13;
    p[0] = h1[0];
    p[1] = h1[1];
    p[2] = h1[2];
    p[3] = w;
    p[4] = wrap_pi(phi0);
    p[5] = atan2f(1.f, cot);
    eta = asinhf(cot);
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < K; ++j) Q.S[i][j] = 0.f;
    const float sg = sqrtf(L1.seed_sig2);
    if (L1.kind == 0) {
        float r = sqrtf(fmaf(h1[0], h1[0], h1[1] * h1[1]));
        float sp = h1[1] / r, cp = h1[0] / r;
        Q.S[0][0] = -sg * sp;  // along the cylinder's azimuth
        Q.S[1][0] = sg * cp;
        Q.S[2][1] = sg;
    } else {
        Q.S[0][0] = sg;
        Q.S[1][1] = sg;
    }
    Q.S[3][2] = sqrtf(fmaf(0.1f * w, 0.1f * w, 1e-4f));
    Q.S[4][3] = 0.01f;
    Q.S[5][4] = 0.01f;
    Q.k = 5;
    return true;
}


__device__ __forceinline__ bool finite_state(const float p[6]) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) ok = ok && isfinite(p[i]);
    return ok;
}

}  // namespace mkf
