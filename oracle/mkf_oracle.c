/*
 * FP64 oracle for the per-layer Kalman-filter step of mkFit-style track fitting
 * and finding ("Parallelized and Vectorized Tracking Using Kalman Filters with
 * CMS Detector Geometry and Events", sec. 1 and 2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the bench may load it.  It shares no code, header or constant
 * table with the CUDA library.
 *
 * The paper prints no equations: it names the Kalman filter (Fruhwirth), the
 * propagation of tracks to barrel and endcap layers (sec. 1), the selection of
 * the best chi2 extensions before the final Kalman updates (sec. 1, the "clone
 * engine"), per-layer hit search windows and layer plans (sec. 2.1) and a
 * constant field (sec. 2.1, sec. 3).  What follows writes out the textbook
 * definitions behind those words:
 *
 *  - state p = (x, y, z, q/pT, phi, theta), phi = azimuth of the momentum;
 *  - uniform field Bz: turning rate h = -(q/pT) * K * Bz per unit transverse path s,
 *    x(s) = x + (sin(phi + h s) - sin(phi)) / h,  y(s) = y - (cos(phi + h s) - cos(phi)) / h,
 *    z(s) = z + s cot(theta),  phi(s) = phi + h s  (straight line for h = 0);
 *  - propagation to a layer = the smallest s > 0 (less than half a turn) that puts
 *    the helix on the layer surface (cylinder r = R, or disk z = Z);
 *  - Jacobian of that map, J = dF/dp + (dF/ds)(ds/dp), ds/dp from the surface
 *    constraint; covariance transport C' = J C J^T;
 *  - 2-D measurement on the surface (r-phi and z on cylinders, r-phi and r on
 *    disks), Kalman gain update and chi2 of the predicted residual;
 *  - seeds from the circle through three hits;
 *  - finding: layer by layer, every hit of the layer is tested (no binning);
 *    candidates are ranked by score = chi2_cut * n_hits - chi2_total, the best
 *    N children are kept and only they receive the Kalman update.
 *
 * Beyond the uniform-field core (each written out where it is defined below):
 * the backward fit and the two-filter smoother; material effects (Highland
 * multiple scattering and the mean energy loss, per layer or from an r-z map);
 * a parameterised solenoid field with fourth-order Runge-Kutta propagation and
 * the Jacobian of that map by central differences; and the learned pruning of
 * the finder's branching (12 features of a candidate-hit pair, a 12-64-1 MLP
 * score, pairs below a threshold dropped before the N-best selection), pinned
 * against the separate MLP oracle and against features rebuilt from the
 * exported single-step calls (tests/test_oracle_pruning.py).
 *
 * Covariances are full 6x6 row-major arrays here.  Interfaces that exchange the
 * 21-value packed lower triangle use index i(i+1)/2 + j for i >= j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_K 0.0029979245800 /* GeV / (T cm) */
#define OR_MAXL 64
#define OR_MAXR 16
#define OR_PI 3.14159265358979323846

/* per-track status bits */
#define OR_ST_UNREACHABLE 1u   /* a requested layer could not be reached (fit) */
#define OR_ST_BADSEED 2u       /* seed hits degenerate */
#define OR_ST_NONFINITE 4u     /* a non-finite number appeared */
#define OR_ST_BADS 8u          /* residual covariance not positive definite */
#define OR_ST_MISSSTOP 16u     /* finding stopped by consecutive misses */
#define OR_ST_TRUNC 32u        /* output hit list truncated */

#define OR_HIT_MISS (-2)
#define OR_HIT_PASS (-3)

typedef struct {
    int n;
    int kind[OR_MAXL];
    double rz[OR_MAXL], lo[OR_MAXL], hi[OR_MAXL], su[OR_MAXL], sv[OR_MAXL];
    double x0[OR_MAXL]; /* material: radiation lengths at normal incidence */
    double eloss[OR_MAXL]; /* mean energy loss per radiation length at minimum ionisation, GeV */
    double bz;
    int field_kind; /* 0: uniform Bz; 1: parameterised field (field_at), RK4 propagation */
    double alpha;   /* parameterised field: fall-off coefficient, 1/cm^2 */
    /* r-z material map (sec. 2.1): map_nr x map_nz cells of equal size over
     * [0, map_rmax) x [map_zmin, map_zmax), x0 and eloss per cell (index
     * ir * map_nz + iz); map_nr = 0: the layers' own values */
    int map_nr, map_nz;
    double map_rmax, map_zmin, map_zmax;
    const double *map_x0, *map_eloss;
    int n_regions;
    double edges[OR_MAXR];
    uint64_t mask[OR_MAXR];
} geom_t;

static int geom_init(geom_t *g, int n_layers, const int32_t *kind, const double *rz, const double *lo,
                     const double *hi, const double *su, const double *sv, const double *x0,
                     const double *eloss, double bz, int field_kind, double alpha, int map_nr, int map_nz,
                     double map_rmax, double map_zmin, double map_zmax, const double *map_x0,
                     const double *map_eloss, int n_regions, const double *edges, const uint64_t *masks) {
    if (n_layers < 1 || n_layers > OR_MAXL) return -1;
    if (n_regions < 1 || n_regions > OR_MAXR) return -1;
    g->n = n_layers;
    for (int i = 0; i < n_layers; ++i) {
        g->kind[i] = kind[i];
        g->rz[i] = rz[i];
        g->lo[i] = lo[i];
        g->hi[i] = hi[i];
        g->su[i] = su[i];
        g->sv[i] = sv[i];
        g->x0[i] = x0 ? x0[i] : 0.0;
        g->eloss[i] = eloss ? eloss[i] : 0.0;
    }
    g->bz = bz;
    if (field_kind != 0 && field_kind != 1) return -1;
    g->field_kind = field_kind;
    g->alpha = field_kind ? alpha : 0.0;
    if (map_nr < 0 || map_nz < 0 || (map_nr > 0) != (map_nz > 0)) return -1;
    if (map_nr > 0 && (!map_x0 || !(map_rmax > 0.0) || !(map_zmax > map_zmin))) return -1;
    g->map_nr = map_nr;
    g->map_nz = map_nz;
    g->map_rmax = map_rmax;
    g->map_zmin = map_zmin;
    g->map_zmax = map_zmax;
    g->map_x0 = map_x0;
    g->map_eloss = map_eloss;
    g->n_regions = n_regions;
    for (int r = 0; r + 1 < n_regions; ++r) g->edges[r] = edges[r];
    for (int r = 0; r < n_regions; ++r) {
        uint64_t all = (n_layers == 64) ? ~0ull : ((1ull << n_layers) - 1ull);
        g->mask[r] = masks ? (masks[r] & all) : all;
    }
    return 0;
}

static double wrap_pi(double a) {
    a = fmod(a + OR_PI, 2.0 * OR_PI);
    if (a < 0) a += 2.0 * OR_PI;
    return a - OR_PI;
}

static double cot_of(double theta) { return cos(theta) / sin(theta); }

/* ------------------------------------------------------------------------- */
/* Helix and propagation                                                     */
/* ------------------------------------------------------------------------- */

/* Magnetic field.  Uniform: B = (0, 0, bz).  Parameterised (sec. 2.1: the
 * field type is chosen per propagation): the field of a solenoid near its
 * centre to second order, from the scalar potential that solves Laplace's
 * equation with axial symmetry,
 *   Bz = bz (1 - alpha (z^2 - r^2 / 2)),  Br = bz alpha r z,
 * i.e. Bx = bz alpha x z, By = bz alpha y z: divergence- and curl-free, Bz
 * falling off along z and rising slightly with r for alpha > 0. */
static void field_at(const geom_t *g, double x, double y, double z, double B[3]) {
    const double a = g->alpha;
    B[0] = g->bz * a * x * z;
    B[1] = g->bz * a * y * z;
    B[2] = g->bz * (1.0 - a * (z * z - 0.5 * (x * x + y * y)));
}

/* Turning rate per unit transverse path from the axial field at the state's
 * position (the uniform field's h in constant mode). */
static double turn_rate(const geom_t *g, const double p[6]) {
    double B[3];
    field_at(g, p[0], p[1], p[2], B);
    return -p[3] * OR_K * B[2];
}

/* Move state p along the helix by transverse path s (closed form). */
static void helix_move(const double p[6], double h, double s, double q[6]) {
    double phi = p[4], dx, dy;
    if (h == 0.0) {
        dx = s * cos(phi);
        dy = s * sin(phi);
    } else {
        dx = (sin(phi + h * s) - sin(phi)) / h;
        dy = -(cos(phi + h * s) - cos(phi)) / h;
    }
    q[0] = p[0] + dx;
    q[1] = p[1] + dy;
    q[2] = p[2] + s * cot_of(p[5]);
    q[3] = p[3];
    q[4] = wrap_pi(phi + h * s);
    q[5] = p[5];
}

/* Smallest s > 0 (and below half a turn) with x(s)^2 + y(s)^2 = R^2.
 * Circle of the track (centre C, radius 1/|h|) intersected with the layer circle. */
static int cyl_path(double x, double y, double phi, double h, double R, double *s_out) {
    double best = INFINITY;
    if (h == 0.0) {
        double b = x * cos(phi) + y * sin(phi);
        double c = x * x + y * y - R * R;
        double disc = b * b - c;
        if (disc < 0) return 0;
        double sq = sqrt(disc);
        double r1 = -b - sq, r2 = -b + sq;
        if (r1 > 0) best = r1;
        if (r2 > 0 && r2 < best) best = r2;
    } else {
        double rho = 1.0 / fabs(h);
        double cx = x - sin(phi) / h, cy = y + cos(phi) / h;
        double d = hypot(cx, cy);
        if (d == 0.0 || d > R + rho || d < fabs(R - rho)) return 0;
        double a = (R * R - rho * rho + d * d) / (2.0 * d);
        double hc2 = R * R - a * a;
        double hc = hc2 > 0 ? sqrt(hc2) : 0.0;
        double ux = cx / d, uy = cy / d;
        for (int k = -1; k <= 1; k += 2) {
            double X = a * ux - k * hc * uy, Y = a * uy + k * hc * ux;
            double ax = x - cx, ay = y - cy, bx = X - cx, by = Y - cy;
            double ang = atan2(ax * by - ay * bx, ax * bx + ay * by);
            double s = ang / h;
            if (s > 0 && s < best) best = s;
        }
    }
    if (!(best < INFINITY)) return 0;
    *s_out = best;
    return 1;
}

/* Path to the surface of layer l, or 0 if the helix does not reach it going
 * forward within half a turn.  No extent check. */
static int path_to_layer(const geom_t *g, const double p[6], int l, double *s) {
    double h = turn_rate(g, p);
    if (g->kind[l] == 0) return cyl_path(p[0], p[1], p[4], h, g->rz[l], s);
    double ct = cot_of(p[5]);
    if (ct == 0.0) return 0;
    double sd = (g->rz[l] - p[2]) / ct;
    if (!(sd > 0)) return 0;
    if (h != 0.0 && fabs(h) * sd >= OR_PI) return 0;
    *s = sd;
    return 1;
}

/* J = dF/dp + (dF/ds) (ds/dp), 6x6 row-major, for the move by s onto layer l. */
static void prop_jacobian(const geom_t *g, const double p[6], int l, double s, const double q[6],
                          double J[36]) {
    double A[36];
    memset(A, 0, sizeof(A));
    double h = turn_rate(g, p);
    double dhdw = -OR_K * g->bz;
    double phi = p[4], phis = phi + h * s;
    double dx = q[0] - p[0], dy = q[1] - p[1];
    double dxdh, dydh;
    if (h == 0.0) {
        dxdh = -0.5 * s * s * sin(phi);
        dydh = 0.5 * s * s * cos(phi);
    } else {
        dxdh = (s * cos(phis) - dx) / h;
        dydh = (s * sin(phis) - dy) / h;
    }
    double st = sin(p[5]);
    for (int i = 0; i < 6; ++i) A[i * 6 + i] = 1.0;
    A[0 * 6 + 3] = dxdh * dhdw;
    A[0 * 6 + 4] = -dy;
    A[1 * 6 + 3] = dydh * dhdw;
    A[1 * 6 + 4] = dx;
    A[2 * 6 + 5] = -s / (st * st);
    A[4 * 6 + 3] = s * dhdw;
    double d[6] = {cos(phis), sin(phis), cot_of(p[5]), 0.0, h, 0.0};
    double dsdp[6];
    if (g->kind[l] == 0) {
        double den = q[0] * d[0] + q[1] * d[1];
        for (int j = 0; j < 6; ++j) dsdp[j] = -(q[0] * A[0 * 6 + j] + q[1] * A[1 * 6 + j]) / den;
    } else {
        for (int j = 0; j < 6; ++j) dsdp[j] = -A[2 * 6 + j] / d[2];
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) J[i * 6 + j] = A[i * 6 + j] + d[i] * dsdp[j];
}

/* ------------------------------------------------------------------------- */
/* Propagation in the parameterised field: fourth-order Runge-Kutta          */
/* ------------------------------------------------------------------------- */

/* Equation of motion of a unit charge with lambda = q/p in the field, with the
 * path length S as variable: dr/dS = T, dT/dS = K lambda T x B(r) (T the unit
 * direction); lambda is constant.  X = (x, y, z, Tx, Ty, Tz, lambda). */
static void eom(const geom_t *g, const double X[7], double dX[7]) {
    double B[3];
    field_at(g, X[0], X[1], X[2], B);
    const double k = OR_K * X[6];
    dX[0] = X[3];
    dX[1] = X[4];
    dX[2] = X[5];
    dX[3] = k * (X[4] * B[2] - X[5] * B[1]);
    dX[4] = k * (X[5] * B[0] - X[3] * B[2]);
    dX[5] = k * (X[3] * B[1] - X[4] * B[0]);
    dX[6] = 0.0;
}

/* One classical Runge-Kutta step of length d (may be negative). */
static void rk4_step(const geom_t *g, double X[7], double d) {
    double k1[7], k2[7], k3[7], k4[7], Y[7];
    eom(g, X, k1);
    for (int i = 0; i < 7; ++i) Y[i] = X[i] + 0.5 * d * k1[i];
    eom(g, Y, k2);
    for (int i = 0; i < 7; ++i) Y[i] = X[i] + 0.5 * d * k2[i];
    eom(g, Y, k3);
    for (int i = 0; i < 7; ++i) Y[i] = X[i] + d * k3[i];
    eom(g, Y, k4);
    for (int i = 0; i < 7; ++i) X[i] += d / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

#define OR_RK_TURN 0.05  /* largest turning angle per step, rad */
#define OR_RK_LEN 10.0   /* largest step, cm of path */
#define OR_RK_MAXN 16    /* most steps per propagation */
#define OR_RK_NEWTON 2   /* correction steps onto the surface */

/* Number of equal steps over the estimated transverse path s (turning |h| s). */
static int rk_steps(const double p[6], double h, double s) {
    const double S = s / sin(p[5]);
    double n = ceil(fmax(fabs(h) * s / OR_RK_TURN, fabs(S) / OR_RK_LEN));
    if (!(n >= 1.0)) n = 1.0;
    return n > OR_RK_MAXN ? OR_RK_MAXN : (int)n;
}

/* Root nearest 0 of a d^2 + b d + c = 0; the parabola's vertex when it has no
 * real root, the linear root when a = 0. */
static double nearest_root(double a, double b, double c) {
    const double disc = b * b - 4.0 * a * c;
    if (a == 0.0) return b != 0.0 ? -c / b : 0.0;
    if (disc < 0.0) return -b / (2.0 * a);
    const double q = -0.5 * (b + copysign(sqrt(disc), b));
    if (q == 0.0) return 0.0;
    const double r1 = q / a, r2 = c / q;
    return fabs(r1) < fabs(r2) ? r1 : r2;
}

/* Move p onto layer l: n equal steps over the path s estimated by the helix in
 * the local axial field, then OR_RK_NEWTON correction steps onto the surface:
 * on a cylinder the nearest root of the second-order expansion of
 * x(S)^2 + y(S)^2 - R^2 about the current point (the bending term keeps it
 * exact enough where the track meets the cylinder at a grazing angle), on a
 * disk the linear (Z - z) / Tz. */
static void rk_move(const geom_t *g, const double p[6], int l, double s, int n, double q[6]) {
    const double st = sin(p[5]);
    double X[7] = {p[0], p[1], p[2], st * cos(p[4]), st * sin(p[4]), cos(p[5]), p[3] * st};
    const double S = s / st;
    for (int i = 0; i < n; ++i) rk4_step(g, X, S / n);
    for (int it = 0; it < OR_RK_NEWTON; ++it) {
        double d;
        if (g->kind[l] == 0) {
            double dX[7];
            eom(g, X, dX);
            const double c = X[0] * X[0] + X[1] * X[1] - g->rz[l] * g->rz[l];
            const double bq = 2.0 * (X[0] * X[3] + X[1] * X[4]);
            const double aq = X[3] * X[3] + X[4] * X[4] + X[0] * dX[3] + X[1] * dX[4];
            d = nearest_root(aq, bq, c);
        } else {
            d = (g->rz[l] - X[2]) / X[5];
        }
        rk4_step(g, X, d);
    }
    const double tn = sqrt(X[3] * X[3] + X[4] * X[4] + X[5] * X[5]);
    const double tt = hypot(X[3], X[4]) / tn;
    q[0] = X[0];
    q[1] = X[1];
    q[2] = X[2];
    q[3] = X[6] / tt;
    q[4] = atan2(X[4], X[3]);
    q[5] = atan2(tt, X[5] / tn);
}

/* Jacobian of rk_move by central differences (the step count held fixed), the
 * azimuth difference wrapped. */
static void rk_jacobian(const geom_t *g, const double p[6], int l, int n, double J[36]) {
    const double eps[6] = {1e-4, 1e-4, 1e-4, 1e-6 * fmax(fabs(p[3]), 1e-2), 1e-6, 1e-6};
    for (int j = 0; j < 6; ++j) {
        double pp[6], pm[6], qp[6], qm[6], s;
        memcpy(pp, p, sizeof(pp));
        memcpy(pm, p, sizeof(pm));
        pp[j] += eps[j];
        pm[j] -= eps[j];
        if (!path_to_layer(g, pp, l, &s)) s = 0.0;
        rk_move(g, pp, l, s, n, qp);
        if (!path_to_layer(g, pm, l, &s)) s = 0.0;
        rk_move(g, pm, l, s, n, qm);
        for (int i = 0; i < 6; ++i) {
            double dq = qp[i] - qm[i];
            if (i == 4) dq = wrap_pi(dq);
            J[i * 6 + j] = dq / (2.0 * eps[j]);
        }
    }
}

/* Move p by the estimated transverse path s onto layer l: the closed-form helix
 * and its Jacobian in the uniform field, Runge-Kutta steps and the Jacobian of
 * that map in the parameterised one. */
static void move_to_layer(const geom_t *g, const double p[6], int l, double s, double q[6], double J[36]) {
    if (g->field_kind == 0) {
        helix_move(p, turn_rate(g, p), s, q);
        prop_jacobian(g, p, l, s, q, J);
        return;
    }
    const int n = rk_steps(p, turn_rate(g, p), s);
    rk_move(g, p, l, s, n, q);
    rk_jacobian(g, p, l, n, J);
}

/* C' = J C J^T (full matrices), symmetrised. */
static void transport(const double J[36], const double C[36], double Co[36]) {
    double M[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double a = 0;
            for (int k = 0; k < 6; ++k) a += J[i * 6 + k] * C[k * 6 + j];
            M[i * 6 + j] = a;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double a = 0;
            for (int k = 0; k < 6; ++k) a += M[i * 6 + k] * J[j * 6 + k];
            Co[i * 6 + j] = a;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < i; ++j) {
            double m = 0.5 * (Co[i * 6 + j] + Co[j * 6 + i]);
            Co[i * 6 + j] = Co[j * 6 + i] = m;
        }
}

/* ------------------------------------------------------------------------- */
/* Measurement and update                                                    */
/* ------------------------------------------------------------------------- */

/* Residual (u, v) of hit (xh, yh, zh) against a state on layer l's surface and
 * the 2x6 projection H. */
/* Multiple scattering in the material where p crosses layer l (x0 radiation
 * lengths at normal incidence, material_at), added to the covariance of the state p on the layer's
 * surface.  theta0 = 0.0136 GeV / (beta p) sqrt(x) (1 + 0.038 ln(x / beta^2))
 * (Highland, as tabulated by the Particle Data Group; unit charge, pion mass
 * 0.13957 GeV) for the path x = x0 / |cos a|, a = the angle between the
 * direction and the surface normal (radial on a cylinder, z on a disk).  The
 * projected angles receive independent noise: Var(theta) += theta0^2,
 * Var(phi) += theta0^2 / sin^2(theta); the momentum magnitude is unchanged, so
 * q/pT = q / (p sin theta) follows theta: d(q/pT) = -(q/pT) cot(theta) d(theta),
 * giving Var(q/pT) += (q/pT cot theta theta0)^2 and
 * Cov(q/pT, theta) += -(q/pT) cot(theta) theta0^2.  Kicks along the path do not
 * move the position on the layer, so nothing else changes.  Without a field
 * q/pT is not measured (0 in the state): the momentum is taken as infinite and
 * no noise is added. */
#define OR_PION_MASS 0.13957

/* Material where the state p crosses layer l: from the r-z map's cell that
 * holds (r, z) when a map is loaded (points outside it take the nearest edge
 * cell), else the layer's own x0 and eloss. */
static void material_at(const geom_t *g, int l, const double p[6], double *x0, double *k) {
    if (g->map_nr == 0) {
        *x0 = g->x0[l];
        *k = g->eloss[l];
        return;
    }
    const double r = hypot(p[0], p[1]);
    int ir = (int)floor(r / g->map_rmax * g->map_nr);
    int iz = (int)floor((p[2] - g->map_zmin) / (g->map_zmax - g->map_zmin) * g->map_nz);
    ir = ir < 0 ? 0 : (ir >= g->map_nr ? g->map_nr - 1 : ir);
    iz = iz < 0 ? 0 : (iz >= g->map_nz ? g->map_nz - 1 : iz);
    *x0 = g->map_x0[ir * g->map_nz + iz];
    *k = g->map_eloss ? g->map_eloss[ir * g->map_nz + iz] : 0.0;
}

static void add_scattering(const geom_t *g, int l, const double p[6], double C[36]) {
    double t, k_unused;
    material_at(g, l, p, &t, &k_unused);
    /* q/pT = 0: no field, momentum not measured; taken as infinite (no noise) */
    if (!(t > 0.0) || !(fabs(p[3]) > 0.0)) return;
    const double st = sin(p[5]), ct = cos(p[5]);
    double cosa = g->kind[l] == 0 ? fabs(st * cos(p[4] - atan2(p[1], p[0]))) : fabs(ct);
    if (cosa < 1e-6) cosa = 1e-6;
    const double pm = 1.0 / (fabs(p[3]) * fabs(st));
    const double beta = pm / sqrt(pm * pm + OR_PION_MASS * OR_PION_MASS);
    const double x = t / cosa;
    const double th0 = 0.0136 / (beta * pm) * sqrt(x) * (1.0 + 0.038 * log(x / (beta * beta)));
    const double v = th0 * th0, wc = p[3] * ct / st;
    C[5 * 6 + 5] += v;
    C[4 * 6 + 4] += v / (st * st);
    C[3 * 6 + 3] += wc * wc * v;
    C[3 * 6 + 5] -= wc * v;
    C[5 * 6 + 3] -= wc * v;
}

/* Mean energy loss in the material where p crosses layer l (no straggling):
 * the particle loses dE = eloss * x / beta^2 for the path x = x0 / |cos a| (eloss =
 * the loss per radiation length at minimum ionisation; pion mass), at fixed
 * direction; sign +1 loses it (forward in time), -1 gains it back (the backward
 * pass).  q/pT scales by r = p / p'; C is transported with the derivative of
 * that map in (q/pT, theta) through the momentum (the loss grows as beta falls). */
static void add_eloss(const geom_t *g, int l, double p[6], double C[36], double sign) {
    double t, k;
    material_at(g, l, p, &t, &k);
    if (!(k > 0.0) || !(t > 0.0) || !(fabs(p[3]) > 0.0)) return;
    const double st = sin(p[5]), ct = cos(p[5]);
    double cosa = g->kind[l] == 0 ? fabs(st * cos(p[4] - atan2(p[1], p[0]))) : fabs(ct);
    if (cosa < 1e-6) cosa = 1e-6;
    const double pm = 1.0 / (fabs(p[3]) * fabs(st));
    const double e = sqrt(pm * pm + OR_PION_MASS * OR_PION_MASS);
    const double beta = pm / e;
    const double kx = sign * k * (t / cosa);
    const double e2 = e - kx / (beta * beta);
    if (!(e2 > OR_PION_MASS)) return; /* stopped: left as it is */
    const double p2 = sqrt(e2 * e2 - OR_PION_MASS * OR_PION_MASS);
    const double r = pm / p2;
    /* Jacobian of q/pT' = q/pT * g(p), g = p / p'(p), p = 1 / (|q/pT| sin theta):
     * dp'/dp = (E' / p') (p / E + 2 kx m^2 / p^3), g' = 1 / p' - p dp'/dp / p'^2;
     * d(q/pT')/d(q/pT) = g - p g', d(q/pT')/d(theta) = -(q/pT) p cot(theta) g'
     * (the path through the layer held fixed) */
    const double dp2 = e2 / p2 * (pm / e + 2.0 * kx * OR_PION_MASS * OR_PION_MASS / (pm * pm * pm));
    const double gp = 1.0 / p2 - pm * dp2 / (p2 * p2);
    const double a = r - pm * gp, c = -p[3] * pm * (ct / st) * gp;
    p[3] *= r;
    double row[6];
    for (int j = 0; j < 6; ++j) row[j] = a * C[3 * 6 + j] + c * C[5 * 6 + j];
    const double c33 = a * row[3] + c * row[5];
    for (int j = 0; j < 6; ++j) {
        C[3 * 6 + j] = row[j];
        C[j * 6 + 3] = row[j];
    }
    C[3 * 6 + 3] = c33;
}

static void residual(const geom_t *g, int l, const double p[6], double xh, double yh, double zh,
                     double r[2], double H[12]) {
    double phip = atan2(p[1], p[0]);
    double phih = atan2(yh, xh);
    double sp = sin(phip), cp = cos(phip);
    memset(H, 0, 12 * sizeof(double));
    H[0] = -sp;
    H[1] = cp;
    if (g->kind[l] == 0) {
        r[0] = g->rz[l] * wrap_pi(phih - phip);
        r[1] = zh - p[2];
        H[6 + 2] = 1.0;
    } else {
        double rt = hypot(p[0], p[1]);
        r[0] = rt * wrap_pi(phih - phip);
        r[1] = hypot(xh, yh) - rt;
        H[6 + 0] = cp;
        H[6 + 1] = sp;
    }
}

/* S = H C H^T + V and its inverse; returns 0 if S is not positive definite. */
static int residual_cov(const geom_t *g, int l, const double C[36], const double H[12], double S[4],
                        double Si[4], double HC[12]) {
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 6; ++j) {
            double acc = 0;
            for (int k = 0; k < 6; ++k) acc += H[a * 6 + k] * C[k * 6 + j];
            HC[a * 6 + j] = acc;
        }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double acc = 0;
            for (int k = 0; k < 6; ++k) acc += HC[a * 6 + k] * H[b * 6 + k];
            S[a * 2 + b] = acc;
        }
    S[0] += g->su[l] * g->su[l];
    S[3] += g->sv[l] * g->sv[l];
    double sym = 0.5 * (S[1] + S[2]);
    S[1] = S[2] = sym;
    double det = S[0] * S[3] - S[1] * S[2];
    if (!(S[0] > 0 && det > 0)) return 0;
    Si[0] = S[3] / det;
    Si[3] = S[0] / det;
    Si[1] = Si[2] = -S[1] / det;
    return 1;
}

static double chi2_of(const double r[2], const double Si[4]) {
    return r[0] * (Si[0] * r[0] + Si[1] * r[1]) + r[1] * (Si[2] * r[0] + Si[3] * r[1]);
}

/* Kalman update of (p, C) with residual r: K = C H^T S^-1, p += K r,
 * C -= K H C (symmetrised).  Returns chi2 of the predicted residual. */
static double kf_update(const double HC[12], const double Si[4], const double r[2], double p[6],
                        double C[36]) {
    double K[12]; /* 6x2 */
    for (int i = 0; i < 6; ++i)
        for (int b = 0; b < 2; ++b) K[i * 2 + b] = HC[0 * 6 + i] * Si[0 * 2 + b] + HC[1 * 6 + i] * Si[1 * 2 + b];
    for (int i = 0; i < 6; ++i) p[i] += K[i * 2 + 0] * r[0] + K[i * 2 + 1] * r[1];
    p[4] = wrap_pi(p[4]);
    double Cn[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Cn[i * 6 + j] = C[i * 6 + j] - (K[i * 2 + 0] * HC[0 * 6 + j] + K[i * 2 + 1] * HC[1 * 6 + j]);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double m = 0.5 * (Cn[i * 6 + j] + Cn[j * 6 + i]);
            C[i * 6 + j] = C[j * 6 + i] = m;
        }
    return chi2_of(r, Si);
}

/* ------------------------------------------------------------------------- */
/* Seeds                                                                      */
/* ------------------------------------------------------------------------- */

/* State at hit 1 from the circle through three hits (x-y) and the straight line
 * through hits 1 and 3 in (arc length, z); diagonal prior covariance. */
static int seed_state(const geom_t *g, const double *h1, const double *h2, const double *h3, int layer1,
                      double p[6], double C[36]) {
    double ax = h2[0] - h1[0], ay = h2[1] - h1[1];
    double bx = h3[0] - h1[0], by = h3[1] - h1[1];
    double cx = h3[0] - h2[0], cy = h3[1] - h2[1];
    double la = hypot(ax, ay), lb = hypot(bx, by), lc = hypot(cx, cy);
    if (!(la > 0 && lb > 0 && lc > 0)) return 0;
    double kappa = 2.0 * (ax * by - ay * bx) / (la * lb * lc); /* signed curvature = h */
    double h = kappa;
    double B2[3];
    field_at(g, h2[0], h2[1], h2[2], B2); /* the field at the middle hit sets the scale */
    double w = (B2[2] != 0.0) ? -h / (OR_K * B2[2]) : 0.0;
    if (B2[2] == 0.0) h = 0.0;
    double a12 = (h == 0.0) ? 0.0 : asin(fmax(-1.0, fmin(1.0, 0.5 * h * la)));
    double phi0 = atan2(ay, ax) - a12;
    double s13 = (h == 0.0) ? lb : 2.0 * asin(fmax(-1.0, fmin(1.0, 0.5 * h * lb))) / h;
    double cot = (h3[2] - h1[2]) / s13;
    p[0] = h1[0];
    p[1] = h1[1];
    p[2] = h1[2];
    p[3] = w;
    p[4] = wrap_pi(phi0);
    p[5] = atan2(1.0, cot);
    /* position prior lies in the surface of hit 1's layer (no variance along its
     * normal), so the state has 5 free parameters and ndf = 2 n_hits - 5 */
    double sig = 10.0 * fmax(g->su[layer1], g->sv[layer1]);
    double s2 = sig * sig;
    memset(C, 0, 36 * sizeof(double));
    if (g->kind[layer1] == 0) {
        double ph = atan2(h1[1], h1[0]), sp = sin(ph), cp = cos(ph);
        C[0] = s2 * sp * sp;
        C[1] = C[6] = -s2 * sp * cp;
        C[7] = s2 * cp * cp;
        C[14] = s2;
    } else {
        C[0] = C[7] = s2;
    }
    C[21] = (0.1 * w) * (0.1 * w) + 0.01 * 0.01;
    C[28] = 0.01 * 0.01;
    C[35] = 0.01 * 0.01;
    return 1;
}

static int finite6(const double p[6]) {
    for (int i = 0; i < 6; ++i)
        if (!isfinite(p[i])) return 0;
    return 1;
}

static void pack21(const double C[36], double *out, int64_t stride) {
    int k = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) out[(int64_t)(k++) * stride] = C[i * 6 + j];
}

static void unpack21(const double *in, int64_t stride, double C[36]) {
    int k = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = in[(int64_t)(k++) * stride];
            C[i * 6 + j] = C[j * 6 + i] = v;
        }
}

/* ------------------------------------------------------------------------- */
/* Exported single-step entry points (used by the pin tests)                  */
/* ------------------------------------------------------------------------- */

#define GEOM_ARGS                                                                                     \
    int n_layers, const int32_t *kind, const double *rz, const double *lo, const double *hi,        \
        const double *su, const double *sv, const double *x0, const double *eloss, double bz,         \
        int field_kind, double alpha, int map_nr, int map_nz, double map_rmax, double map_zmin,           \
        double map_zmax, const double *map_x0, const double *map_eloss, int n_regions, const double *edges, \
        const uint64_t *masks
#define GEOM_PASS                                                                                       \
    n_layers, kind, rz, lo, hi, su, sv, x0, eloss, bz, field_kind, alpha, map_nr, map_nz, map_rmax, map_zmin, \
        map_zmax, map_x0, map_eloss, n_regions, edges, masks

/* Propagate p to layer l: writes q, J (6x6 row-major) and s.  Returns 1 on
 * success, 0 if unreachable, -1 on bad arguments. */
int or_propagate(GEOM_ARGS, const double *p, int l, double *q, double *J, double *s) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS) || l < 0 || l >= g.n) return -1;
    double ss;
    if (!path_to_layer(&g, p, l, &ss)) return 0;
    move_to_layer(&g, p, l, ss, q, J);
    *s = ss;
    return 1;
}

/* The field at (x, y, z). */
int or_field(GEOM_ARGS, const double *r, double *B) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS)) return -1;
    field_at(&g, r[0], r[1], r[2], B);
    return 1;
}

/* Move p by transverse path s (closed-form helix). */
int or_helix_move(GEOM_ARGS, const double *p, double s, double *q) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS)) return -1;
    helix_move(p, turn_rate(&g, p), s, q);
    return 1;
}

void or_transport(const double *J, const double *C, double *Co) { transport(J, C, Co); }

/* One Kalman update on layer l with hit (xh, yh, zh).  Writes updated p, C,
 * the residual r[2], S[4], and returns chi2 (NaN if S is not positive definite).
 * Also writes the Joseph-form covariance into Cj for comparison. */
double or_update(GEOM_ARGS, int l, const double *hit, double *p, double *C, double *r_out, double *S_out,
                 double *Cj) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS)) return NAN;
    double H[12], r[2], S[4], Si[4], HC[12];
    residual(&g, l, p, hit[0], hit[1], hit[2], r, H);
    if (!residual_cov(&g, l, C, H, S, Si, HC)) return NAN;
    double C0[36];
    memcpy(C0, C, sizeof(C0));
    double chi2 = kf_update(HC, Si, r, p, C);
    if (Cj) {
        /* Joseph form: (I - K H) C0 (I - K H)^T + K V K^T */
        double K[12], IKH[36], T[36];
        for (int i = 0; i < 6; ++i)
            for (int b = 0; b < 2; ++b) K[i * 2 + b] = HC[i] * Si[b] + HC[6 + i] * Si[2 + b];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) IKH[i * 6 + j] = (i == j) - (K[i * 2] * H[j] + K[i * 2 + 1] * H[6 + j]);
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double a = 0;
                for (int k = 0; k < 6; ++k) a += IKH[i * 6 + k] * C0[k * 6 + j];
                T[i * 6 + j] = a;
            }
        double V0 = g.su[l] * g.su[l], V1 = g.sv[l] * g.sv[l];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double a = 0;
                for (int k = 0; k < 6; ++k) a += T[i * 6 + k] * IKH[j * 6 + k];
                Cj[i * 6 + j] = a + K[i * 2] * V0 * K[j * 2] + K[i * 2 + 1] * V1 * K[j * 2 + 1];
            }
    }
    if (r_out) { r_out[0] = r[0]; r_out[1] = r[1]; }
    if (S_out) memcpy(S_out, S, sizeof(S));
    return chi2;
}

/* Scattering noise of layer l at the state p (on its surface), added to C (6x6). */
int or_scattering(GEOM_ARGS, int l, const double *p, double *C) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS) || l < 0 || l >= g.n) return -1;
    add_scattering(&g, l, p, C);
    return 1;
}

/* Mean energy loss (sign +1) or gain (-1) in the material where p crosses
 * layer l, applied to p and C in place. */
int or_eloss(GEOM_ARGS, int l, double *p, double *C, double sign) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS) || l < 0 || l >= g.n) return -1;
    add_eloss(&g, l, p, C, sign);
    return 1;
}

/* Seed state and prior covariance (6x6) from three hits; returns 1 or 0. */
int or_seed(GEOM_ARGS, const double *h1, const double *h2, const double *h3, int layer1, double *p, double *C) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS)) return -1;
    return seed_state(&g, h1, h2, h3, layer1, p, C);
}

/* ------------------------------------------------------------------------- */
/* Fit: Kalman filter along fixed hit lists                                   */
/* ------------------------------------------------------------------------- */

/* xyz: [3][n_hits] SoA; hit_layer[n_hits]; hit_idx: [max_hits][n] (-1 = none,
 * hits in path order); seed_par [6][n] and seed_cov [21][n] (packed) or NULL to
 * seed from the first three hits.  Outputs: par [6][n], cov [21][n] (packed),
 * chi2[n], ndf[n], status[n].  The state is reported on the surface of the last
 * hit used. */
int or_fit(GEOM_ARGS, const double *xyz, int64_t n_hits, const int32_t *hit_layer, const int32_t *hit_idx,
           int max_hits, int64_t n, const double *seed_par, const double *seed_cov, double *out_par,
           double *out_cov, double *out_chi2, int32_t *out_ndf, uint32_t *out_status) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS)) return -1;
    const double *X = xyz, *Y = xyz + n_hits, *Z = xyz + 2 * n_hits;
    for (int64_t t = 0; t < n; ++t) {
        double p[6], C[36];
        uint32_t st = 0;
        int idx[OR_MAXL + 8];
        int nh = 0;
        for (int k = 0; k < max_hits && k < OR_MAXL + 8; ++k) {
            int32_t hi_ = hit_idx[(int64_t)k * n + t];
            if (hi_ >= 0 && hi_ < n_hits) idx[nh++] = hi_;
        }
        double chi2 = 0;
        int used = 0;
        if (nh < 3) st |= OR_ST_BADSEED;
        if (!(st & OR_ST_BADSEED)) {
            if (seed_par) {
                for (int i = 0; i < 6; ++i) p[i] = seed_par[(int64_t)i * n + t];
                unpack21(seed_cov + t, n, C);
            } else {
                double a[3] = {X[idx[0]], Y[idx[0]], Z[idx[0]]};
                double b[3] = {X[idx[1]], Y[idx[1]], Z[idx[1]]};
                double c[3] = {X[idx[2]], Y[idx[2]], Z[idx[2]]};
                if (!seed_state(&g, a, b, c, hit_layer[idx[0]], p, C)) st |= OR_ST_BADSEED;
            }
        }
        if (!(st & OR_ST_BADSEED)) {
            for (int k = 0; k < nh; ++k) {
                int hid = idx[k], l = hit_layer[hid];
                if (k > 0) {
                    double s, q[6], J[36], Cn[36];
                    if (!path_to_layer(&g, p, l, &s)) { st |= OR_ST_UNREACHABLE; continue; }
                    move_to_layer(&g, p, l, s, q, J);
                    transport(J, C, Cn);
                    memcpy(p, q, sizeof(q));
                    memcpy(C, Cn, sizeof(Cn));
                    add_scattering(&g, l, p, C);
                    add_eloss(&g, l, p, C, 1.0);
                }
                double H[12], r[2], S[4], Si[4], HC[12];
                residual(&g, l, p, X[hid], Y[hid], Z[hid], r, H);
                if (!residual_cov(&g, l, C, H, S, Si, HC)) { st |= OR_ST_BADS; continue; }
                chi2 += kf_update(HC, Si, r, p, C);
                used++;
            }
        }
        if (!finite6(p) || !isfinite(chi2)) st |= OR_ST_NONFINITE;
        for (int i = 0; i < 6; ++i) out_par[(int64_t)i * n + t] = (st & OR_ST_BADSEED) ? NAN : p[i];
        if (st & OR_ST_BADSEED) {
            for (int k = 0; k < 21; ++k) out_cov[(int64_t)k * n + t] = NAN;
        } else {
            pack21(C, out_cov + t, n);
        }
        out_chi2[t] = chi2;
        /* five free parameters on a surface; without a field q/pT is not measured */
        out_ndf[t] = 2 * used - (g.bz != 0.0 ? 5 : 4);
        out_status[t] = st;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Backward fit: the same filter through the hits in reverse order           */
/* ------------------------------------------------------------------------- */

/* The helix traversed the other way: the same curve with the momentum turned
 * around, p -> (x, y, z, -q/pT, phi + pi, pi - theta).  Its derivative is
 * F = diag(1, 1, 1, -1, 1, -1), so C -> F C F flips the sign of the covariances
 * between {q/pT, theta} and the other parameters. */
static void reverse_state(double p[6], double C[36]) {
    static const double f[6] = {1, 1, 1, -1, 1, -1};
    p[3] = -p[3];
    p[4] = wrap_pi(p[4] + OR_PI);
    p[5] = OR_PI - p[5];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) C[i * 6 + j] *= f[i] * f[j];
}

/* Backward fit along fixed hit lists (the reverse pass over a fitted or found
 * track, whose result is the state at its first hit with every hit used).
 * xyz, hit_layer, hit_idx as in or_fit (hits in path order).  last_par [6][n],
 * last_cov [21][n] (packed): the state on the surface of each track's last hit,
 * e.g. or_fit's output.  The state is turned around, its covariance multiplied
 * by inflate (>= 1), updated with the last hit, then moved to each earlier hit
 * in turn and updated; at the first hit it is turned back.  Outputs as or_fit,
 * reported on the surface of the first hit used. */
int or_fit_backward(GEOM_ARGS, const double *xyz, int64_t n_hits, const int32_t *hit_layer, const int32_t *hit_idx,
                    int max_hits, int64_t n, const double *last_par, const double *last_cov, double inflate,
                    double *out_par, double *out_cov, double *out_chi2, int32_t *out_ndf, uint32_t *out_status) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS)) return -1;
    if (!last_par || !last_cov || !(inflate >= 1.0)) return -1;
    const double *X = xyz, *Y = xyz + n_hits, *Z = xyz + 2 * n_hits;
    for (int64_t t = 0; t < n; ++t) {
        double p[6], C[36];
        uint32_t st = 0;
        int idx[OR_MAXL + 8];
        int nh = 0;
        for (int k = 0; k < max_hits && k < OR_MAXL + 8; ++k) {
            int32_t hi_ = hit_idx[(int64_t)k * n + t];
            if (hi_ >= 0 && hi_ < n_hits) idx[nh++] = hi_;
        }
        double chi2 = 0;
        int used = 0;
        if (nh < 3) st |= OR_ST_BADSEED;
        if (!(st & OR_ST_BADSEED)) {
            for (int i = 0; i < 6; ++i) p[i] = last_par[(int64_t)i * n + t];
            unpack21(last_cov + t, n, C);
            reverse_state(p, C);
            for (int i = 0; i < 36; ++i) C[i] *= inflate;
            for (int k = nh - 1; k >= 0; --k) {
                int hid = idx[k], l = hit_layer[hid];
                if (k < nh - 1) {
                    double s, q[6], J[36], Cn[36];
                    if (!path_to_layer(&g, p, l, &s)) { st |= OR_ST_UNREACHABLE; continue; }
                    move_to_layer(&g, p, l, s, q, J);
                    transport(J, C, Cn);
                    memcpy(p, q, sizeof(q));
                    memcpy(C, Cn, sizeof(Cn));
                }
                double H[12], r[2], S[4], Si[4], HC[12];
                residual(&g, l, p, X[hid], Y[hid], Z[hid], r, H);
                if (residual_cov(&g, l, C, H, S, Si, HC)) {
                    chi2 += kf_update(HC, Si, r, p, C);
                    used++;
                } else {
                    st |= OR_ST_BADS;
                }
                /* reversed in time, the layer's material follows its hit (at
                 * every hit, the last one included): the energy lost there is
                 * gained back, then the scattering noise is added */
                add_eloss(&g, l, p, C, -1.0);
                add_scattering(&g, l, p, C);
            }
            reverse_state(p, C);
        }
        if (!finite6(p) || !isfinite(chi2)) st |= OR_ST_NONFINITE;
        for (int i = 0; i < 6; ++i) out_par[(int64_t)i * n + t] = (st & OR_ST_BADSEED) ? NAN : p[i];
        if (st & OR_ST_BADSEED) {
            for (int k = 0; k < 21; ++k) out_cov[(int64_t)k * n + t] = NAN;
        } else {
            pack21(C, out_cov + t, n);
        }
        out_chi2[t] = chi2;
        out_ndf[t] = 2 * used - (g.bz != 0.0 ? 5 : 4);
        out_status[t] = st;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Smoothing: the state at every hit from all of the track's hits             */
/* ------------------------------------------------------------------------- */

/* Inverse of a symmetric positive definite n x n matrix (Gauss-Jordan with
 * partial pivoting); 0 if singular. */
static int invert_n(int n, const double *A, double *Ai) {
    double M[5 * 10];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j) M[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[r * 2 * n + c]) > fabs(M[piv * 2 * n + c])) piv = r;
        if (!(fabs(M[piv * 2 * n + c]) > 0.0)) return 0;
        if (piv != c)
            for (int j = 0; j < 2 * n; ++j) {
                double tmp = M[c * 2 * n + j];
                M[c * 2 * n + j] = M[piv * 2 * n + j];
                M[piv * 2 * n + j] = tmp;
            }
        const double d = M[c * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = M[r * 2 * n + c];
            for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[c * 2 * n + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ai[i * n + j] = M[i * 2 * n + n + j];
    return 1;
}

/* Weighted mean of two independent estimates of the state on layer l's
 * surface: (pf, Cf) and (pb, Cb), both in the forward direction.  On a surface
 * the state has five free parameters (the position along the normal is fixed),
 * so the mean is taken in P p, P = the 5 x 6 projection onto (u, z, q/pT, phi,
 * theta) on a cylinder (u along the surface, perpendicular to the radius at
 * pf) and (x, y, q/pT, phi, theta) on a disk: with d = P (pb - pf) (phi
 * wrapped), K = Cf P^T (P (Cf + Cb) P^T)^-1, ps = pf + K d (its position put
 * back on the surface), Cs = Cf - K P Cf (its position block projected onto
 * the tangent plane at ps). */
static int combine(const geom_t *g, int l, const double pf[6], const double Cf[36], const double pb[6],
                   const double Cb[36], double ps[6], double Cs[36]) {
    double P[30];
    memset(P, 0, sizeof(P));
    if (g->kind[l] == 0) {
        const double ph = atan2(pf[1], pf[0]);
        P[0] = -sin(ph);
        P[1] = cos(ph);
        P[6 + 2] = 1.0;
    } else {
        P[0] = 1.0;
        P[6 + 1] = 1.0;
    }
    P[12 + 3] = P[18 + 4] = P[24 + 5] = 1.0;
    double dp[6];
    for (int i = 0; i < 6; ++i) dp[i] = pb[i] - pf[i];
    dp[4] = wrap_pi(dp[4]);
    double d[5], S[25], Si[25], PC[30], K[30];
    for (int a = 0; a < 5; ++a) {
        d[a] = 0.0;
        for (int i = 0; i < 6; ++i) d[a] += P[a * 6 + i] * dp[i];
    }
    for (int a = 0; a < 5; ++a)
        for (int j = 0; j < 6; ++j) {
            double v = 0.0;
            for (int i = 0; i < 6; ++i) v += P[a * 6 + i] * (Cf[i * 6 + j] + Cb[i * 6 + j]);
            PC[a * 6 + j] = v;
        }
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) {
            double v = 0.0;
            for (int j = 0; j < 6; ++j) v += PC[a * 6 + j] * P[b * 6 + j];
            S[a * 5 + b] = v;
        }
    if (!invert_n(5, S, Si)) return 0;
    for (int i = 0; i < 6; ++i)
        for (int b = 0; b < 5; ++b) {
            double v = 0.0;
            for (int a = 0; a < 5; ++a) {
                double cp = 0.0;
                for (int j = 0; j < 6; ++j) cp += Cf[i * 6 + j] * P[a * 6 + j];
                v += cp * Si[a * 5 + b];
            }
            K[i * 5 + b] = v;
        }
    for (int i = 0; i < 6; ++i) {
        double v = pf[i];
        for (int a = 0; a < 5; ++a) v += K[i * 5 + a] * d[a];
        ps[i] = v;
    }
    ps[4] = wrap_pi(ps[4]);
    /* the mean lies on the surface: the position is put back on it (a move
     * along the tangent leaves it by a second-order amount) */
    if (g->kind[l] == 0) {
        const double f = g->rz[l] / hypot(ps[0], ps[1]);
        ps[0] *= f;
        ps[1] *= f;
    } else {
        ps[2] = g->rz[l];
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double v = Cf[i * 6 + j];
            for (int a = 0; a < 5; ++a) {
                double pc = 0.0;
                for (int m = 0; m < 6; ++m) pc += P[a * 6 + m] * Cf[m * 6 + j];
                v -= K[i * 5 + a] * pc;
            }
            Cs[i * 6 + j] = v;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < i; ++j) Cs[i * 6 + j] = Cs[j * 6 + i] = 0.5 * (Cs[i * 6 + j] + Cs[j * 6 + i]);
    /* no variance along the surface normal n at ps: Cs -> (I - n n^T) Cs (I - n n^T) */
    double nv[3] = {0.0, 0.0, 1.0};
    if (g->kind[l] == 0) {
        const double r = hypot(ps[0], ps[1]);
        nv[0] = ps[0] / r;
        nv[1] = ps[1] / r;
        nv[2] = 0.0;
    }
    double Pi[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Pi[i * 6 + j] = (i == j ? 1.0 : 0.0) - (i < 3 && j < 3 ? nv[i] * nv[j] : 0.0);
    double Tm[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double v = 0.0;
            for (int m = 0; m < 6; ++m) v += Pi[i * 6 + m] * Cs[m * 6 + j];
            Tm[i * 6 + j] = v;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double v = 0.0;
            for (int m = 0; m < 6; ++m) v += Tm[i * 6 + m] * Pi[j * 6 + m];
            Cs[i * 6 + j] = v;
        }
    return 1;
}

/* Smoothed states along fixed hit lists (two filters): the forward filter as
 * or_fit, keeping its state after each hit; then the backward filter from the
 * forward state at the last hit (turned around, covariance times inflate),
 * which at each earlier hit predicts the state from the later hits alone and
 * is then updated with that hit, as or_fit_backward.  The smoothed state at a
 * hit is the weighted mean (combine) of the forward state after the hit and the
 * backward prediction there; at the last hit it is the forward state.  Outputs:
 * sm_par [max_hits][6][n], sm_cov [max_hits][21][n] (packed) per row of hit_idx
 * (NaN where the row holds no hit or a step failed), and the forward fit's
 * chi2, ndf and status (with the backward pass's status bits added). */
int or_fit_smooth(GEOM_ARGS, const double *xyz, int64_t n_hits, const int32_t *hit_layer, const int32_t *hit_idx,
                  int max_hits, int64_t n, const double *seed_par, const double *seed_cov, double inflate,
                  double *sm_par, double *sm_cov, double *out_chi2, int32_t *out_ndf, uint32_t *out_status,
                  double *out_shrink) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS)) return -1;
    if (!(inflate >= 1.0) || max_hits > OR_MAXL + 8) return -1;
    const double *X = xyz, *Y = xyz + n_hits, *Z = xyz + 2 * n_hits;
    static double PF[OR_MAXL + 8][6], CF[OR_MAXL + 8][36];
    for (int64_t t = 0; t < n; ++t) {
        for (int k = 0; k < max_hits; ++k) {
            for (int i = 0; i < 6; ++i) sm_par[((int64_t)k * 6 + i) * n + t] = NAN;
            for (int i = 0; i < 21; ++i) sm_cov[((int64_t)k * 21 + i) * n + t] = NAN;
        }
        double p[6], C[36];
        uint32_t st = 0;
        int idx[OR_MAXL + 8], row[OR_MAXL + 8], ok[OR_MAXL + 8];
        int nh = 0;
        for (int k = 0; k < max_hits; ++k) {
            int32_t hi_ = hit_idx[(int64_t)k * n + t];
            if (hi_ >= 0 && hi_ < n_hits) {
                row[nh] = k;
                idx[nh++] = hi_;
            }
        }
        double chi2 = 0;
        int used = 0;
        if (nh < 3) st |= OR_ST_BADSEED;
        if (!(st & OR_ST_BADSEED)) {
            if (seed_par) {
                for (int i = 0; i < 6; ++i) p[i] = seed_par[(int64_t)i * n + t];
                unpack21(seed_cov + t, n, C);
            } else {
                double a[3] = {X[idx[0]], Y[idx[0]], Z[idx[0]]};
                double b[3] = {X[idx[1]], Y[idx[1]], Z[idx[1]]};
                double c[3] = {X[idx[2]], Y[idx[2]], Z[idx[2]]};
                if (!seed_state(&g, a, b, c, hit_layer[idx[0]], p, C)) st |= OR_ST_BADSEED;
            }
        }
        int last = -1;
        /* conditioning log: the largest ratio of a predicted residual variance
         * (H C H^T) to the hit's own variance over the backward filter's
         * updates -- the factor by which an update shrinks the prior */
        double shrink = 0.0;
        if (!(st & OR_ST_BADSEED)) {
            for (int k = 0; k < nh; ++k) {
                int hid = idx[k], l = hit_layer[hid];
                ok[k] = 0;
                if (k > 0) {
                    double s, q[6], J[36], Cn[36];
                    if (!path_to_layer(&g, p, l, &s)) { st |= OR_ST_UNREACHABLE; continue; }
                    move_to_layer(&g, p, l, s, q, J);
                    transport(J, C, Cn);
                    memcpy(p, q, sizeof(q));
                    memcpy(C, Cn, sizeof(Cn));
                    add_scattering(&g, l, p, C);
                    add_eloss(&g, l, p, C, 1.0);
                }
                double H[12], r[2], S[4], Si[4], HC[12];
                residual(&g, l, p, X[hid], Y[hid], Z[hid], r, H);
                if (!residual_cov(&g, l, C, H, S, Si, HC)) { st |= OR_ST_BADS; continue; }
                chi2 += kf_update(HC, Si, r, p, C);
                used++;
                memcpy(PF[k], p, sizeof(p));
                memcpy(CF[k], C, sizeof(C));
                ok[k] = 1;
                last = k;
            }
        }
        if (last >= 0 && finite6(p) && isfinite(chi2)) {
            /* backward filter from the forward state at the last hit */
            memcpy(p, PF[last], sizeof(p));
            memcpy(C, CF[last], sizeof(C));
            reverse_state(p, C);
            for (int i = 0; i < 36; ++i) C[i] *= inflate;
            for (int k = last; k >= 0; --k) {
                int hid = idx[k], l = hit_layer[hid];
                if (k < last) {
                    double s, q[6], J[36], Cn[36];
                    if (!path_to_layer(&g, p, l, &s)) { st |= OR_ST_UNREACHABLE; continue; }
                    move_to_layer(&g, p, l, s, q, J);
                    transport(J, C, Cn);
                    memcpy(p, q, sizeof(q));
                    memcpy(C, Cn, sizeof(Cn));
                }
                double ps[6], Cs[36];
                int have = 0;
                if (ok[k] && k == last) {
                    memcpy(ps, PF[k], sizeof(ps));
                    memcpy(Cs, CF[k], sizeof(Cs));
                    have = 1;
                } else if (ok[k]) {
                    double pb[6], Cb[36];
                    memcpy(pb, p, sizeof(pb));
                    memcpy(Cb, C, sizeof(Cb));
                    reverse_state(pb, Cb);
                    have = combine(&g, l, PF[k], CF[k], pb, Cb, ps, Cs);
                    if (!have) st |= OR_ST_BADS;
                }
                if (have) {
                    for (int i = 0; i < 6; ++i) sm_par[((int64_t)row[k] * 6 + i) * n + t] = ps[i];
                    pack21(Cs, sm_cov + (int64_t)row[k] * 21 * n + t, n);
                }
                double H[12], r[2], S[4], Si[4], HC[12];
                residual(&g, l, p, X[hid], Y[hid], Z[hid], r, H);
                if (residual_cov(&g, l, C, H, S, Si, HC)) {
                    const double vu = g.su[l] * g.su[l], vv = g.sv[l] * g.sv[l];
                    shrink = fmax(shrink, fmax((S[0] - vu) / vu, (S[3] - vv) / vv));
                    kf_update(HC, Si, r, p, C);
                } else {
                    st |= OR_ST_BADS;
                }
                add_eloss(&g, l, p, C, -1.0);
                add_scattering(&g, l, p, C);
            }
        }
        if (!isfinite(chi2)) st |= OR_ST_NONFINITE;
        out_chi2[t] = chi2;
        out_ndf[t] = 2 * used - (g.bz != 0.0 ? 5 : 4);
        out_status[t] = st;
        if (out_shrink) out_shrink[t] = shrink;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Finding                                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    double p[6], C[36];
    double chi2, score;
    int n_hits, n_miss, consec;
    int next_cyl, next_dsk; /* positions in the sorted cylinder / disk lists, -1 = none */
    int dir;                /* +1 / -1 along z for disks */
    int done;
    int path;               /* index of this candidate's last record in the history */
} cand_t;

typedef struct {
    int parent;   /* rank of the parent candidate */
    int hit;      /* global hit index, OR_HIT_MISS or OR_HIT_PASS */
    double chi2;  /* chi2 of the hit */
    double score;
    int layer;
    double u, v;  /* residual of the hit */
} child_t;

typedef struct {
    int prev;     /* previous record, -1 at the seed */
    int hit;
} hrec_t;

typedef struct {
    const geom_t *g;
    const double *X, *Y, *Z, *PHI, *RH;
    const int32_t *HL;        /* layer of each hit */
    const int32_t *lay_start; /* [n_events * n_layers + 1] into lay_hits */
    const int32_t *lay_hits;
    int cyl_sorted[OR_MAXL], n_cyl;
    int dsk_sorted[OR_MAXL], n_dsk;
    double cut;
    int max_consec;
    int n_best;
    const double *mlp;   /* 897 weights (bfloat16 values) or NULL */
    double tau;
    double *feat;        /* [cap][12] or NULL */
    int32_t *feat_ref;   /* [cap][2] */
    int64_t *feat_n;
    int64_t feat_cap;
    int seed_index;
} find_ctx_t;

static int cmp_child(const child_t *a, const child_t *b) {
    if (a->score != b->score) return a->score > b->score ? -1 : 1;
    if (a->parent != b->parent) return a->parent < b->parent ? -1 : 1;
    unsigned ha = a->hit < 0 ? 0xFFFFFFFFu : (unsigned)a->hit;
    unsigned hb = b->hit < 0 ? 0xFFFFFFFFu : (unsigned)b->hit;
    if (ha != hb) return ha < hb ? -1 : 1;
    return 0;
}

/* order of one parent's hit children: chi2, then hit index */
static int cmp_hit_child(const child_t *a, const child_t *b) {
    if (a->chi2 != b->chi2) return a->chi2 < b->chi2 ? -1 : 1;
    return a->hit < b->hit ? -1 : (a->hit > b->hit ? 1 : 0);
}

static int cmp_child_q(const void *a, const void *b) { return cmp_child((const child_t *)a, (const child_t *)b); }

/* chi2 total of the candidate a child would become */
static double child_chi2_total(const cand_t *parents, const child_t *ch) {
    return parents[ch->parent].chi2 + (ch->hit >= 0 ? ch->chi2 : 0.0);
}

static void upd_min(double *m, double v) {
    if (v < *m) *m = v;
}

/* Next layer of a candidate: the nearer (in path length) of the next cylinder
 * and the next disk allowed by the region mask.  Layers crossed outside their
 * extent are passed over (pointer advanced, no measurement, state unchanged),
 * and so are layers already behind the candidate.  Returns the layer id (and
 * its path s) or -1 when no layer is left. */
static int next_layer(const find_ctx_t *f, cand_t *c, uint64_t mask, double *s_out, double *mgeo) {
    const geom_t *g = f->g;
    const double rcur = hypot(c->p[0], c->p[1]), zcur = c->p[2];
    for (int guard = 0; guard < 2 * OR_MAXL + 2; ++guard) {
        /* layers outside the region's plan, and layers already behind the
         * candidate (a cylinder not beyond its radius, a disk not ahead in z),
         * are passed over */
        while (c->next_cyl >= 0 && c->next_cyl < f->n_cyl &&
               (!((mask >> f->cyl_sorted[c->next_cyl]) & 1ull) || g->rz[f->cyl_sorted[c->next_cyl]] <= rcur))
            c->next_cyl++;
        if (c->next_cyl >= f->n_cyl) c->next_cyl = -1;
        while (c->next_dsk >= 0 && c->next_dsk < f->n_dsk &&
               (!((mask >> f->dsk_sorted[c->next_dsk]) & 1ull) ||
                c->dir * (g->rz[f->dsk_sorted[c->next_dsk]] - zcur) <= 0))
            c->next_dsk += c->dir;
        if (c->next_dsk >= f->n_dsk) c->next_dsk = -1;
        double sc = INFINITY, sd = INFINITY;
        int lc = -1, ld = -1;
        if (c->next_cyl >= 0) {
            lc = f->cyl_sorted[c->next_cyl];
            if (!path_to_layer(g, c->p, lc, &sc)) { c->next_cyl = -1; sc = INFINITY; lc = -1; }
        }
        if (c->next_dsk >= 0) {
            ld = f->dsk_sorted[c->next_dsk];
            if (!path_to_layer(g, c->p, ld, &sd)) { c->next_dsk = -1; sd = INFINITY; ld = -1; }
        }
        if (lc < 0 && ld < 0) return -1;
        int use_cyl = (sc <= sd);
        if (lc >= 0 && ld >= 0) upd_min(mgeo, fabs(sc - sd) / fmax(sc, sd));
        int l = use_cyl ? lc : ld;
        double s = use_cyl ? sc : sd;
        double q[6];
        helix_move(c->p, turn_rate(g, c->p), s, q);
        double coord = (g->kind[l] == 0) ? q[2] : hypot(q[0], q[1]);
        double span = g->hi[l] - g->lo[l];
        upd_min(mgeo, fmin(fabs(coord - g->lo[l]), fabs(coord - g->hi[l])) / span);
        int inside = coord >= g->lo[l] && coord <= g->hi[l];
        if (use_cyl) c->next_cyl++;
        else c->next_dsk += c->dir;
        if (c->next_dsk >= f->n_dsk) c->next_dsk = -1;
        if (inside) {
            *s_out = s;
            return l;
        }
    }
    return -1;
}

/* Position of the first entry > v in a sorted list of values (or count). */
static int first_cyl_beyond(const find_ctx_t *f, double r) {
    for (int i = 0; i < f->n_cyl; ++i)
        if (f->g->rz[f->cyl_sorted[i]] > r) return i;
    return -1;
}

static int first_dsk_beyond(const find_ctx_t *f, double z, int dir) {
    if (dir > 0) {
        for (int i = 0; i < f->n_dsk; ++i)
            if (f->g->rz[f->dsk_sorted[i]] > z) return i;
    } else {
        for (int i = f->n_dsk - 1; i >= 0; --i)
            if (f->g->rz[f->dsk_sorted[i]] < z) return i;
    }
    return -1;
}

typedef struct {
    child_t *v;
    int n, cap;
} childvec_t;

static int push_child(childvec_t *cv, child_t c) {
    if (cv->n == cv->cap) {
        int nc = cv->cap ? 2 * cv->cap : 64;
        child_t *nv = (child_t *)realloc(cv->v, sizeof(child_t) * nc);
        if (!nv) return 0;
        cv->v = nv;
        cv->cap = nc;
    }
    cv->v[cv->n++] = c;
    return 1;
}

typedef struct {
    hrec_t *v;
    int n, cap;
} histvec_t;

static int push_hist(histvec_t *hv, int prev, int hit) {
    if (hv->n == hv->cap) {
        int nc = hv->cap ? 2 * hv->cap : 256;
        hrec_t *nv = (hrec_t *)realloc(hv->v, sizeof(hrec_t) * nc);
        if (!nv) return -1;
        hv->v = nv;
        hv->cap = nc;
    }
    hv->v[hv->n].prev = prev;
    hv->v[hv->n].hit = hit;
    return hv->n++;
}

/* Features of a (candidate, compatible hit) pair: residual pulls, chi2 of the
 * hit over the cut, the candidate's chi2 per degree of freedom, hit and miss
 * counts, layer, layer kind, q/pT, eta, and the log widths of the residual
 * covariance.  The miss count saturates at 15. */
static void pair_features(const find_ctx_t *f, const cand_t *c, int l, const double r[2], const double S[4], double x2,
                          double fe[12]) {
    const geom_t *g = f->g;
    double su = sqrt(S[0]), sv = sqrt(S[3]);
    int nm = c->n_miss < 15 ? c->n_miss : 15;
    int ndf = 2 * c->n_hits - 5;
    fe[0] = r[0] / su;
    fe[1] = r[1] / sv;
    fe[2] = x2 / f->cut;
    fe[3] = c->chi2 / (ndf > 1 ? ndf : 1);
    fe[4] = c->n_hits * 0.1;
    fe[5] = nm * 0.2;
    fe[6] = (double)l / g->n;
    fe[7] = g->kind[l] == 1 ? 1.0 : 0.0;
    fe[8] = c->p[3];
    fe[9] = asinh(cot_of(c->p[5])) / 3.0;
    fe[10] = log10(su);
    fe[11] = log10(sv);
}

/* 12 -> 64 ReLU -> 1; weights W1[64][12], b1[64], w2[64], b2. */
static double mlp_logit(const double *w, const double fe[12]) {
    double z = w[896];
    for (int j = 0; j < 64; ++j) {
        double a = w[768 + j];
        for (int k = 0; k < 12; ++k) a += w[j * 12 + k] * fe[k];
        z += w[832 + j] * (a > 0 ? a : 0.0);
    }
    return z;
}

/* Logits of n feature rows fe [n][12] with weights w [897] (the finder's
 * scoring function, exported for its pins). */
void or_mlp_logit(const double *w, const double *fe, int64_t n, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = mlp_logit(w, fe + 12 * i);
}

/* Find one seed.  Returns 0, or -1 on allocation failure. */
static int find_one(const find_ctx_t *f, int ev, const int32_t sh[3], double *outp, double *outC,
                    double *out_chi2, int32_t *out_nhits, int32_t *out_hits, int max_out, uint32_t *out_status,
                    int64_t cnt[3], double marg[4]) {
    const geom_t *g = f->g;
    const int L = g->n;
    uint32_t st = 0;
    cnt[0] = cnt[1] = cnt[2] = 0;
    marg[0] = marg[1] = marg[2] = marg[3] = INFINITY;
    cand_t *cands = (cand_t *)calloc((size_t)f->n_best, sizeof(cand_t));
    cand_t *nextc = (cand_t *)calloc((size_t)f->n_best, sizeof(cand_t));
    childvec_t cv = {0, 0, 0};
    histvec_t hv = {0, 0, 0};
    if (!cands || !nextc) { free(cands); free(nextc); return -1; }

    /* seed state + seed fit over the three seed hits */
    cand_t c0;
    memset(&c0, 0, sizeof(c0));
    double a[3] = {f->X[sh[0]], f->Y[sh[0]], f->Z[sh[0]]};
    double b[3] = {f->X[sh[1]], f->Y[sh[1]], f->Z[sh[1]]};
    double cc[3] = {f->X[sh[2]], f->Y[sh[2]], f->Z[sh[2]]};
    int seed_layer[3] = {f->HL[sh[0]], f->HL[sh[1]], f->HL[sh[2]]};
    int ok = 1;
    for (int k = 0; k < 3; ++k)
        if (seed_layer[k] < 0 || seed_layer[k] >= L) ok = 0;
    ok = ok && seed_state(g, a, b, cc, seed_layer[0], c0.p, c0.C);
    double eta = 0;
    if (ok) eta = asinh(cot_of(c0.p[5]));
    if (ok) {
        for (int k = 0; k < 3; ++k) {
            int l = seed_layer[k];
            int hid = sh[k];
            if (k > 0) {
                double s, q[6], J[36], Cn[36];
                if (!path_to_layer(g, c0.p, l, &s)) { ok = 0; break; }
                move_to_layer(g, c0.p, l, s, q, J);
                transport(J, c0.C, Cn);
                memcpy(c0.p, q, sizeof(q));
                memcpy(c0.C, Cn, sizeof(Cn));
                add_scattering(g, l, c0.p, c0.C);
                add_eloss(g, l, c0.p, c0.C, 1.0);
            }
            double H[12], r[2], S[4], Si[4], HC[12];
            residual(g, l, c0.p, f->X[hid], f->Y[hid], f->Z[hid], r, H);
            if (!residual_cov(g, l, c0.C, H, S, Si, HC)) { ok = 0; break; }
            c0.chi2 += kf_update(HC, Si, r, c0.p, c0.C);
        }
    }
    if (!ok || !finite6(c0.p)) {
        st |= OR_ST_BADSEED;
        for (int i = 0; i < 6; ++i) outp[i] = NAN;
        for (int i = 0; i < 36; ++i) outC[i] = NAN;
        *out_chi2 = NAN;
        *out_nhits = 0;
        for (int k = 0; k < max_out; ++k) out_hits[k] = -1;
        *out_status = st;
        free(cands); free(nextc);
        return 0;
    }
    c0.n_hits = 3;
    c0.score = f->cut * 3 - c0.chi2;
    c0.dir = cot_of(c0.p[5]) >= 0 ? 1 : -1;
    {
        int l3 = seed_layer[2];
        double r3 = hypot(f->X[sh[2]], f->Y[sh[2]]), z3 = f->Z[sh[2]];
        if (g->kind[l3] == 0) {
            int pos = -1;
            for (int i = 0; i < f->n_cyl; ++i)
                if (f->cyl_sorted[i] == l3) pos = i;
            c0.next_cyl = (pos + 1 < f->n_cyl) ? pos + 1 : -1;
        } else {
            c0.next_cyl = first_cyl_beyond(f, r3);
        }
        if (g->kind[l3] == 1) {
            int pos = -1;
            for (int i = 0; i < f->n_dsk; ++i)
                if (f->dsk_sorted[i] == l3) pos = i;
            int nx = pos + c0.dir;
            c0.next_dsk = (nx >= 0 && nx < f->n_dsk) ? nx : -1;
        } else {
            c0.next_dsk = first_dsk_beyond(f, z3, c0.dir);
        }
    }
    /* tracking region from the seed's eta */
    int region = 0;
    while (region + 1 < g->n_regions && eta >= g->edges[region]) region++;
    uint64_t mask = g->mask[region];

    c0.path = -1;
    int nc = 1;
    double last_gap = INFINITY;
    cands[0] = c0;
    for (int step = 0; step < 4 * OR_MAXL; ++step) {
        int any = 0;
        for (int r = 0; r < nc; ++r)
            if (!cands[r].done) any = 1;
        if (!any) break;
        cv.n = 0;
        for (int r = 0; r < nc; ++r) {
            cand_t *c = &cands[r];
            child_t ch;
            ch.parent = r;
            ch.chi2 = 0;
            ch.layer = -1;
            ch.u = ch.v = 0;
            if (c->done) {
                ch.hit = OR_HIT_PASS;
                ch.score = c->score;
                if (!push_child(&cv, ch)) goto oom;
                continue;
            }
            double s;
            int l = next_layer(f, c, mask, &s, &marg[2]);
            if (l < 0) {
                c->done = 1;
                ch.hit = OR_HIT_PASS;
                ch.score = c->score;
                if (!push_child(&cv, ch)) goto oom;
                continue;
            }
            /* propagate the parent in place: its children start from here */
            double q[6], J[36], Cn[36];
            move_to_layer(g, c->p, l, s, q, J);
            transport(J, c->C, Cn);
            memcpy(c->p, q, sizeof(q));
            memcpy(c->C, Cn, sizeof(Cn));
            add_scattering(g, l, c->p, c->C);
            add_eloss(g, l, c->p, c->C, 1.0);
            cnt[0]++;
            /* window half-widths from S at the predicted state */
            double H[12], rr[2], S[4], Si[4], HC[12];
            residual(g, l, c->p, c->p[0], c->p[1], c->p[2], rr, H);
            int sok = residual_cov(g, l, c->C, H, S, Si, HC);
            if (sok) {
                double wu = sqrt(f->cut * S[0]), wv = sqrt(f->cut * S[3]);
                int n_pend = 0;
                int32_t b0 = f->lay_start[(int64_t)ev * L + l], b1 = f->lay_start[(int64_t)ev * L + l + 1];
                for (int32_t j = b0; j < b1; ++j) {
                    int hid = f->lay_hits[j];
                    double u, v;
                    if (g->kind[l] == 0) {
                        u = g->rz[l] * wrap_pi(f->PHI[hid] - atan2(c->p[1], c->p[0]));
                        v = f->Z[hid] - c->p[2];
                    } else {
                        double rt = hypot(c->p[0], c->p[1]);
                        u = rt * wrap_pi(f->PHI[hid] - atan2(c->p[1], c->p[0]));
                        v = f->RH[hid] - rt;
                    }
                    if (fabs(u) > wu || fabs(v) > wv) continue;
                    cnt[1]++;
                    double rv[2] = {u, v};
                    double x2 = chi2_of(rv, Si);
                    upd_min(&marg[1], fabs(x2 - f->cut) / f->cut);
                    if (x2 < f->cut) {
                        ch.hit = hid;
                        ch.chi2 = x2;
                        ch.score = c->score + f->cut - x2;
                        ch.layer = l;
                        ch.u = rv[0];
                        ch.v = rv[1];
                        if (!push_child(&cv, ch)) goto oom;
                        n_pend++;
                    }
                }
                /* the parent's children: its N best compatible hits (by chi2, then
                 * hit index); with the MLP on and two or more compatible hits, those
                 * whose logit is below tau are dropped */
                int first = cv.n - n_pend;
                for (int i = first + 1; i < cv.n; ++i)
                    for (int j = i; j > first && cmp_hit_child(&cv.v[j - 1], &cv.v[j]) > 0; --j) {
                        child_t t = cv.v[j]; cv.v[j] = cv.v[j - 1]; cv.v[j - 1] = t;
                    }
                int n_compat = n_pend;
                if (n_pend > f->n_best) cv.n = first + f->n_best;
                int kept = first;
                for (int i = first; i < cv.n; ++i) {
                    int drop = 0;
                    if (f->feat || (f->mlp && n_compat >= 2)) {
                        double fe[12], rr2[2] = {cv.v[i].u, cv.v[i].v};
                        pair_features(f, c, l, rr2, S, cv.v[i].chi2, fe);
                        if (f->feat) {
                            int64_t at = (*f->feat_n)++;
                            if (at < f->feat_cap) {
                                for (int q = 0; q < 12; ++q) f->feat[at * 12 + q] = fe[q];
                                f->feat_ref[at * 3] = f->seed_index;
                                f->feat_ref[at * 3 + 1] = cv.v[i].hit;
                                f->feat_ref[at * 3 + 2] = n_compat;
                            }
                        }
                        if (f->mlp && n_compat >= 2) {
                            double z = mlp_logit(f->mlp, fe);
                            upd_min(&marg[3], fabs(z - f->tau));
                            if (z < f->tau) drop = 1;
                        }
                    }
                    if (!drop) cv.v[kept++] = cv.v[i];
                }
                cv.n = kept;
            } else {
                st |= OR_ST_BADS;
            }
            ch.hit = OR_HIT_MISS;
            ch.chi2 = 0;
            ch.score = c->score;
            ch.layer = l;
            if (!push_child(&cv, ch)) goto oom;
        }
        qsort(cv.v, (size_t)cv.n, sizeof(child_t), cmp_child_q);
        int keep = cv.n < f->n_best ? cv.n : f->n_best;
        /* ranking margins on the chi2 scale: the keep/drop boundary of this step,
         * and (kept until the end) the order of the two best */
        if (cv.n > f->n_best) {
            const child_t *u = &cv.v[f->n_best - 1], *w = &cv.v[f->n_best];
            upd_min(&marg[0], fabs(u->score - w->score) / fmax(1.0, child_chi2_total(cands, u)));
        }
        last_gap = INFINITY;
        if (cv.n > 1) last_gap = fabs(cv.v[0].score - cv.v[1].score) / fmax(1.0, child_chi2_total(cands, &cv.v[0]));
        for (int i = 0; i < keep; ++i) {
            const child_t *ch = &cv.v[i];
            cand_t n = cands[ch->parent];
            if (ch->hit >= 0) {
                int l = ch->layer;
                double H[12], r[2], S[4], Si[4], HC[12];
                residual(g, l, n.p, f->X[ch->hit], f->Y[ch->hit], f->Z[ch->hit], r, H);
                residual_cov(g, l, n.C, H, S, Si, HC);
                double x2 = kf_update(HC, Si, r, n.p, n.C);
                n.chi2 += x2;
                n.n_hits++;
                n.consec = 0;
                n.score = f->cut * n.n_hits - n.chi2;
                cnt[2]++;
            } else if (ch->hit == OR_HIT_MISS) {
                n.n_miss++;
                n.consec++;
                if (n.consec >= f->max_consec) n.done = 2;
            }
            if (ch->hit != OR_HIT_PASS) {
                int id = push_hist(&hv, n.path, ch->hit);
                if (id < 0) goto oom;
                n.path = id;
            }
            nextc[i] = n;
        }
        cand_t *tmp = cands;
        cands = nextc;
        nextc = tmp;
        nc = keep;
    }
    upd_min(&marg[0], last_gap);
    {
        const cand_t *best = &cands[0];
        /* walk the history of the best candidate back to the seed */
        int tmp[4 * OR_MAXL + 8];
        int nt = 0;
        for (int id = best->path; id >= 0 && nt < 4 * OR_MAXL; id = hv.v[id].prev)
            if (hv.v[id].hit >= 0) tmp[nt++] = hv.v[id].hit;
        int nh = 0;
        for (int k = 0; k < 3; ++k)
            if (nh < max_out) out_hits[nh++] = sh[k];
        for (int k = nt - 1; k >= 0; --k) {
            if (nh < max_out) out_hits[nh++] = tmp[k];
            else st |= OR_ST_TRUNC;
        }
        for (int k = nh; k < max_out; ++k) out_hits[k] = -1;
        memcpy(outp, best->p, sizeof(best->p));
        memcpy(outC, best->C, sizeof(best->C));
        *out_chi2 = best->chi2;
        *out_nhits = best->n_hits;
        if (best->done == 2) st |= OR_ST_MISSSTOP;
        if (!finite6(best->p)) st |= OR_ST_NONFINITE;
        *out_status = st;
    }
    free(cands); free(nextc); free(cv.v); free(hv.v);
    return 0;
oom:
    free(cands); free(nextc); free(cv.v); free(hv.v);
    return -1;
}

/* Track finding over a batch of events.
 * xyz [3][n_hits] (global hit index), hit_layer[n_hits], event_offsets[n_events+1];
 * seed_hits [3][n_seeds] (global hit indices, in path order), seed_event[n_seeds].
 * n_best = 1 is best-hit finding, n_best > 1 keeps the N best candidates.
 * Outputs per seed: par [6][n], cov [21][n] (packed), chi2, n_hits,
 * hits [max_out][n] (-1 padded), status, counters [3][n] (candidate-layers,
 * hits inside the window rectangle, Kalman updates), margins [4][n]
 * (closest score gap at a ranking decision, closest |chi2 - cut| / cut, closest
 * geometric decision, closest |logit - tau| of the pruning MLP).  mlp_w (897
 * values, or NULL) turns on learned pruning: a compatible hit whose logit is
 * below mlp_tau gives no child.  feat_out (or NULL) receives the 12 features of
 * every compatible hit, with (seed, hit) in feat_ref and the running count in
 * *feat_count (rows beyond feat_cap are counted, not written).  seed_list (or NULL for all) selects which seeds to run;
 * outputs are indexed by position in seed_list. */
int or_find(GEOM_ARGS, const double *xyz, int64_t n_hits, const int32_t *hit_layer, const int32_t *event_offsets,
            int n_events, const int32_t *seed_hits, const int32_t *seed_event, int64_t n_seeds,
            const int64_t *seed_list, int64_t n_list, int n_best, double chi2_cut, int max_consec,
            double *out_par, double *out_cov, double *out_chi2, int32_t *out_nhits, int32_t *out_hits, int max_out,
            uint32_t *out_status, int64_t *out_counters, double *out_margins, const double *mlp_w, double mlp_tau,
            double *feat_out, int32_t *feat_ref, int64_t *feat_count, int64_t feat_cap) {
    geom_t g;
    if (geom_init(&g, GEOM_PASS)) return -1;
    if (n_best < 1 || max_out < 3 || max_consec < 1) return -1;
    const int L = g.n;
    find_ctx_t f;
    memset(&f, 0, sizeof(f));
    f.g = &g;
    f.X = xyz;
    f.Y = xyz + n_hits;
    f.Z = xyz + 2 * n_hits;
    f.cut = chi2_cut;
    f.max_consec = max_consec;
    f.n_best = n_best;
    f.mlp = mlp_w;
    f.tau = mlp_tau;
    f.feat = feat_out;
    f.feat_ref = feat_ref;
    f.feat_n = feat_count;
    f.feat_cap = feat_cap;
    if (feat_out && (!feat_ref || !feat_count)) return -1;
    /* sorted layer lists */
    for (int l = 0; l < L; ++l) {
        if (g.kind[l] == 0) f.cyl_sorted[f.n_cyl++] = l;
        else f.dsk_sorted[f.n_dsk++] = l;
    }
    for (int i = 1; i < f.n_cyl; ++i)
        for (int j = i; j > 0 && g.rz[f.cyl_sorted[j - 1]] > g.rz[f.cyl_sorted[j]]; --j) {
            int t = f.cyl_sorted[j]; f.cyl_sorted[j] = f.cyl_sorted[j - 1]; f.cyl_sorted[j - 1] = t;
        }
    for (int i = 1; i < f.n_dsk; ++i)
        for (int j = i; j > 0 && g.rz[f.dsk_sorted[j - 1]] > g.rz[f.dsk_sorted[j]]; --j) {
            int t = f.dsk_sorted[j]; f.dsk_sorted[j] = f.dsk_sorted[j - 1]; f.dsk_sorted[j - 1] = t;
        }
    /* per-hit azimuth and radius; per (event, layer) hit lists */
    double *PHI = (double *)malloc(sizeof(double) * (size_t)(n_hits > 0 ? n_hits : 1));
    double *RH = (double *)malloc(sizeof(double) * (size_t)(n_hits > 0 ? n_hits : 1));
    int32_t *start = (int32_t *)calloc((size_t)n_events * L + 1, sizeof(int32_t));
    int32_t *fill = (int32_t *)calloc((size_t)n_events * L + 1, sizeof(int32_t));
    int32_t *lh = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_hits > 0 ? n_hits : 1));
    if (!PHI || !RH || !start || !fill || !lh) { free(PHI); free(RH); free(start); free(fill); free(lh); return -2; }
    for (int64_t i = 0; i < n_hits; ++i) {
        PHI[i] = atan2(f.Y[i], f.X[i]);
        RH[i] = hypot(f.X[i], f.Y[i]);
    }
    for (int e = 0; e < n_events; ++e)
        for (int32_t i = event_offsets[e]; i < event_offsets[e + 1]; ++i) start[(int64_t)e * L + hit_layer[i] + 1]++;
    for (int64_t k = 0; k < (int64_t)n_events * L; ++k) start[k + 1] += start[k];
    for (int e = 0; e < n_events; ++e)
        for (int32_t i = event_offsets[e]; i < event_offsets[e + 1]; ++i) {
            int64_t key = (int64_t)e * L + hit_layer[i];
            lh[start[key] + fill[key]++] = i;
        }
    f.PHI = PHI;
    f.RH = RH;
    f.lay_start = start;
    f.lay_hits = lh;
    f.HL = hit_layer;
    int64_t nl = seed_list ? n_list : n_seeds;
    int rc = 0;
    for (int64_t k = 0; k < nl && rc == 0; ++k) {
        int64_t sidx = seed_list ? seed_list[k] : k;
        int32_t sh[3] = {seed_hits[sidx], seed_hits[n_seeds + sidx], seed_hits[2 * n_seeds + sidx]};
        double p[6], C[36], chi2, marg[4];
        int32_t nh, hits[4 * OR_MAXL + 8];
        uint32_t st;
        int64_t cnt[3];
        int mo = max_out < 4 * OR_MAXL ? max_out : 4 * OR_MAXL;
        int ev = seed_event[sidx];
        if (ev < 0 || ev >= n_events || sh[0] < 0 || sh[1] < 0 || sh[2] < 0 || sh[0] >= n_hits || sh[1] >= n_hits ||
            sh[2] >= n_hits) {
            rc = -3;
            break;
        }
        f.seed_index = (int)sidx;
        if (find_one(&f, ev, sh, p, C, &chi2, &nh, hits, mo, &st, cnt, marg)) { rc = -2; break; }
        for (int i = 0; i < 6; ++i) out_par[(int64_t)i * nl + k] = p[i];
        pack21(C, out_cov + k, nl);
        out_chi2[k] = chi2;
        out_nhits[k] = nh;
        for (int j = 0; j < max_out; ++j) out_hits[(int64_t)j * nl + k] = j < mo ? hits[j] : -1;
        out_status[k] = st;
        for (int j = 0; j < 3; ++j) out_counters[(int64_t)j * nl + k] = cnt[j];
        for (int j = 0; j < 4; ++j) out_margins[(int64_t)j * nl + k] = marg[j];
    }
    free(PHI); free(RH); free(start); free(fill); free(lh);
    return rc;
}
