// Track finding: per-layer propagation, hit search in phi x z / phi x r bins,
// chi2 of compatible hits, best-hit or N-best branching and the Kalman update
// of the kept children only (Sec. 1: selection of the best chi2 extensions
// before the final Kalman updates; Sec. 2.1: layer plans per tracking region).
//
// GPU mapping: one lane per candidate; the N candidates of a seed occupy N
// consecutive lanes of a warp (32 / N seeds per warp).  A step of the layer loop
// is warp-synchronous:
//   1. every live candidate lane goes to its next layer, propagates, transports
//      its covariance and scans the bins of its chi2 window, keeping its best N
//      compatible hits in a shared-memory list sorted by (chi2, hit index);
//   2. the seed's N lanes pick the N best children in N rounds of a segmented
//      max over 32-bit keys exchanged by shuffles: the order-preserving integer
//      of the FP32 score with its low 4 bits replaced by the parent's rank, so
//      keys within a seed are unique and the maximum names its parent;
//   3. each lane becomes one child: it pulls its parent's propagated state by
//      shuffles and applies the Kalman update with its hit;
//   4. each lane records (parent rank, hit) in a per-step history in shared
//      memory, walked back at the end to produce the best candidate's hit list.
// The seed fit runs before, in its own kernel with one thread per seed (in the
// layer loop it would keep 9 of every 10 lanes idle for three steps).  A child
// reuses its parent's S^-1, H C and hit residual instead of recomputing them.
// No candidate state goes through global memory between layers.
#include <cuda_runtime.h>

#include <algorithm>

#include "mkf_internal.h"

namespace {

using namespace mkf;

constexpr uint32_t kHitMask = 0x0FFFFFFFu;
constexpr uint32_t kCodeMiss = 0x0FFFFFFEu;
constexpr uint32_t kCodePass = 0x0FFFFFFFu;
constexpr unsigned kFull = 0xffffffffu;

struct FindArgs {
    Geom G;
    const float4 *rec;
    const int32_t *inv;
    const uint8_t *layer8;
    const float *zhit;
    const int32_t *offsets;
    int32_t n_hits, n_events;
    const int32_t *seed_hits;
    const int32_t *seed_event;
    int32_t n_seeds;
    int32_t n_best;
    float cut;
    int32_t max_consec;
    int32_t max_steps;
    float *out_par, *out_cov, *out_chi2;
    int32_t *out_nhits, *out_hits;
    int32_t max_out;
    uint32_t *out_status;
    int32_t *counters;
    mkf_fault *fault;
    float *seedbuf;  // [kSeedFields][n_seeds] fitted seeds (written by seed_kernel)
    const uint16_t *mlp;  // bfloat16 weights or nullptr
    float mlp_tau;
    float *feat_out;
    int32_t *feat_ref;
    int32_t *feat_count;
    int32_t feat_cap;
    int32_t *work_counter;                // persistent warps' shared seed-group counter
    unsigned long long *event_times;      // [n_events + 1] or nullptr
    float *beam;                          // [n_best][kListFields][n_seeds] first-step hit lists
    int32_t step1;                        // the seed kernel takes the first step (plain finder)
    const int32_t *seed_list;             // seeds to find (or nullptr: all), *seed_count of them
    const int32_t *seed_count;
    int32_t mlp_mode;                     // 0 prune, 1 gate (flag MKF_ST_AMBIG, drop nothing)
    // processing order grouped by event and |eta| of the seed (or nullptr):
    // the seed kernel writes each seed's key and place, order_scatter_kernel
    // the order the finder's warps take the seeds in
    int32_t *order_key, *order_pos, *order_counts;
};

// Seeds are taken by the finder grouped by event and by the |eta| of their
// three-hit estimate in bins of 0.25 (16 bins): a warp's seeds then have
// similar numbers of layers ahead, so fewer lanes idle while the longest one
// ends (5 % on the uneven dense events), and each event's hits stay together.
constexpr int kOrderBuckets = 16;

// Number of seeds this call finds: all of them, or the device-side count of
// the seed list (clamped to n_seeds).
__device__ __forceinline__ int seeds_in_call(const FindArgs &A) {
    return A.seed_list ? min(max(*A.seed_count, 0), A.n_seeds) : A.n_seeds;
}

// Fitted-seed record, structure of arrays over seeds.
enum {
    SF_P = 0, SF_LO = 6, SF_C = 10, SF_CHI2 = 31, SF_BOOK = 32, SF_MASK_LO = 33, SF_MASK_HI = 34, SF_DIR = 35,
    SF_STATUS = 36, SF_HITS = 37, SF_BEAM = 40, SF_CCL = 41, SF_CHT = 42, SF_NLIST = 43, SF_SEARCHED = 44,
    SF_I = 45, SF_LOTH = 60, kSeedFields = 61
};

// First-step hit list of a seed, [entry][field][seed].
enum { LF_CHI2 = 0, LF_ORIG = 1, LF_U = 2, LF_V = 3, kListFields = 4 };

__device__ __forceinline__ void record_fault(mkf_fault *f, int code, int where) {
    if (atomicCAS(&f->code, 0, code) == 0) f->where = where;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Order-preserving map of a float to uint32 (larger float -> larger integer).
__device__ __forceinline__ uint32_t ord_float(float f) {
    if (!isfinite(f)) f = -3.0e38f;
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Selection key of a child: its score as an order-preserving integer, the low
// 4 bits holding a per-parent tag (larger key = better child).
__device__ __forceinline__ uint32_t sel_key(float score, uint32_t tag) { return (ord_float(score) & ~15u) | tag; }

// Candidate bookkeeping packed into one word for the lane-to-lane transfer.
struct Book {
    int nh, consec, ncyl, ndsk;
    bool done, missstop;
    int nmiss;  // misses so far (saturates at 15)
};

__device__ __forceinline__ uint32_t pack_book(const Book &b) {
    return static_cast<uint32_t>(b.nh & 0xFF) | (static_cast<uint32_t>(b.consec & 0xF) << 8) |
           (static_cast<uint32_t>((b.ncyl + 1) & 0x7F) << 12) | (static_cast<uint32_t>((b.ndsk + 1) & 0x7F) << 19) |
           (b.done ? (1u << 26) : 0u) | (b.missstop ? (1u << 27) : 0u) |
           (static_cast<uint32_t>(min(b.nmiss, 15)) << 28);
}

__device__ __forceinline__ Book unpack_book(uint32_t w) {
    Book b;
    b.nh = w & 0xFF;
    b.consec = (w >> 8) & 0xF;
    b.ncyl = static_cast<int>((w >> 12) & 0x7F) - 1;
    b.ndsk = static_cast<int>((w >> 19) & 0x7F) - 1;
    b.done = (w >> 26) & 1u;
    b.missstop = (w >> 27) & 1u;
    b.nmiss = static_cast<int>(w >> 28);
    return b;
}

// Next layer of a candidate (the nearer of its next cylinder and next disk in
// path length, within the region's layer mask); layers crossed outside their
// extent, and layers already behind the candidate, are passed over.  Returns
// the layer id and the path, or -1.  kbl: K Bz at the candidate (the helix of
// the local axial field estimates the paths in the parameterised field).
__device__ __forceinline__ int next_layer(const Geom &G, float kbl, unsigned long long mask, const float p[6],
                                          const Lo &lo, float sphi, float cphi, float cot, int dir, int &ncyl,
                                          int &ndsk, float &s_out) {
    const float h = -p[3] * kbl;
    const float rcur = sqrtf(fmaf(p[0], p[0], p[1] * p[1])), zcur = p[2] + lo.z;
    for (int guard = 0; guard < 2 * kMaxLayers + 2; ++guard) {
        // layers outside the region's plan, and layers already behind the
        // candidate (a cylinder not beyond its radius, a disk not ahead in z)
        while (ncyl >= 0 && ncyl < G.n_cyl && (!((mask >> G.cyl[ncyl]) & 1ull) || G.L[G.cyl[ncyl]].rz <= rcur)) ++ncyl;
        if (ncyl >= G.n_cyl) ncyl = -1;
        while (ndsk >= 0 && ndsk < G.n_dsk &&
               (!((mask >> G.dsk[ndsk]) & 1ull) || dir * (G.L[G.dsk[ndsk]].rz - zcur) <= 0.f))
            ndsk += dir;
        if (ndsk >= G.n_dsk) ndsk = -1;
        const float inf = __int_as_float(0x7f800000);
        float sc = inf, sd = inf;
        int lc = -1, ld = -1;
        if (ndsk >= 0) {
            ld = G.dsk[ndsk];
            if (!path_disk(p[2], lo, cot, h, G.L[ld].rz, sd)) {
                ndsk = -1;
                ld = -1;
                sd = inf;
            }
        }
        if (ncyl >= 0) {
            lc = G.cyl[ncyl];
            // the transverse arc to radius R is at least R - r: a disk reached
            // well before that comes first, and the cylinder waits
            const float R = G.L[lc].rz;
            if (sd < (R - rcur) * 0.99999f) {
                lc = -2;
            } else if (!path_cyl(p[0], p[1], lo, sphi, cphi, h, R, sc)) {
                ncyl = -1;
                lc = -1;
                sc = inf;
            }
        }
        if (lc < 0 && ld < 0) return -1;
        const bool use_cyl = sc <= sd;
        const int l = use_cyl ? lc : ld;
        const float s = use_cyl ? sc : sd;
        const LayerDesc &Ld = G.L[l];
        float coord;
        if (use_cyl) {
            coord = fmaf(s, cot, zcur);  // z along the helix
        } else {
            float x, y, z;
            helix_point(p, sphi, cphi, cot, h, s, x, y, z);
            coord = sqrtf(fmaf(x, x, y * y));
        }
        const bool inside = coord >= Ld.lo && coord <= Ld.hi;
        if (use_cyl) {
            // z changes monotonically along the helix and larger cylinders are
            // reached later: past the z-extent of every remaining cylinder, none
            // of them can be crossed inside its extent
            if ((cot > 0.f && coord > G.cyl_hi_beyond[ncyl]) || (cot < 0.f && coord < G.cyl_lo_beyond[ncyl]))
                ncyl = -1;
            else
                ++ncyl;
        } else {
            ndsk += dir;
        }
        if (ndsk >= G.n_dsk) ndsk = -1;
        if (inside) {
            s_out = s;
            return l;
        }
    }
    return -1;
}

// Segmented reductions over the N lanes [base, base + N) of a seed, by
// shuffles.  (The redux unit with one member mask per segment measured ~20 %
// slower for the whole finder.)
__device__ __forceinline__ uint32_t seg_max32(uint32_t v, int rank, int N, int base) {
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
        const uint32_t o = __shfl_down_sync(kFull, v, off);
        if (rank + off < N && o > v) v = o;
    }
    return __shfl_sync(kFull, v, base & 31);
}

__device__ __forceinline__ int seg_sum(int v, int rank, int N) {
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
        int o = __shfl_down_sync(kFull, v, off);
        if (rank + off < N) v += o;
    }
    return v;
}

__device__ __forceinline__ uint32_t seg_or(uint32_t v, int rank, int N) {
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
        uint32_t o = __shfl_down_sync(kFull, v, off);
        if (rank + off < N) v |= o;
    }
    return v;
}

// Features of a (candidate, compatible hit) pair (see mkf_find_params).
__device__ __forceinline__ void pair_features(float u, float v, const Innov &I, float x2, float cut, float chi2_tot,
                                              const Book &bk, int layer, int n_layers, int kind, const float p[6],
                                              float cot, float f[12]) {
    const float su = sqrtf(I.Suu), sv = sqrtf(I.Svv);
    f[0] = u / su;
    f[1] = v / sv;
    f[2] = x2 / cut;
    f[3] = chi2_tot / fmaxf(1.f, static_cast<float>(2 * bk.nh - 5));
    f[4] = static_cast<float>(bk.nh) * 0.1f;
    f[5] = static_cast<float>(bk.nmiss) * 0.2f;
    f[6] = static_cast<float>(layer) / static_cast<float>(n_layers);
    f[7] = kind == 1 ? 1.f : 0.f;
    f[8] = p[3];
    f[9] = asinhf(cot) * (1.f / 3.f);
    f[10] = log10f(su);
    f[11] = log10f(sv);
}

// MLP logit with FP32 weights in shared memory (layout of mkf.h).
__device__ __forceinline__ float mlp_logit(const float *ws, const float f[12]) {
    float z = ws[MKF_MLP_PARAMS - 1];
    for (int j = 0; j < MKF_MLP_HIDDEN; ++j) {
        float a = ws[MKF_MLP_IN * MKF_MLP_HIDDEN + j];
#pragma unroll
        for (int k = 0; k < MKF_MLP_IN; ++k) a = fmaf(ws[j * MKF_MLP_IN + k], f[k], a);
        z = fmaf(ws[MKF_MLP_IN * MKF_MLP_HIDDEN + MKF_MLP_HIDDEN + j], fmaxf(a, 0.f), z);
    }
    return z;
}

// A child of its (propagated) parent: the Kalman update with its hit, or the
// bookkeeping of a miss; a pass (no layer left) leaves the parent as it is.
__device__ __forceinline__ void make_child(uint32_t code, const Innov &I, float u, float v, float x2, int max_consec,
                                           float p[6], Lo &lo, float C[21], float &chi2, Book &bk, int &c_up) {
    if (code < kCodeMiss) {
        chi2 += x2;
        kf_apply(I, u, v, p, lo, C);
        bk.nh += 1;
        bk.consec = 0;
        ++c_up;
    } else if (code == kCodeMiss) {
        bk.consec += 1;
        bk.nmiss = min(bk.nmiss + 1, 15);
        if (bk.consec >= max_consec) {
            bk.done = true;
            bk.missstop = true;
        }
    }
}

// Result of expanding a candidate to its next layer.
struct Expansion {
    int layer;      // layer reached, or -1 (none left) / -2 (non-finite state)
    bool searched;  // propagated onto the layer and searched
    int nlist;      // compatible hits kept (at most N), sorted by (chi2, hit index)
    int n_compat;   // all compatible hits
    float cot;      // cot(theta) before the move
};

// One candidate to its next layer: next-layer choice, propagation and
// covariance transport, S^-1 and H C, the bins of the chi2 window, and the
// list of its N best compatible hits (chi2, hit index, residual u, v) at list
// stride `ls` (lane-interleaved shared memory in the finder, contiguous local
// arrays in the seed kernel).  p, lo, C move onto the layer; a candidate with no
// layer left is marked done.  kPhys: 0 uniform field, 1 material effects,
// 2 parameterised field (Runge-Kutta propagation) and material effects.
template <int kPhys>
__device__ __forceinline__ void expand(const FindArgs &A, const Geom &G, int ev, unsigned long long mask, int dir,
                                       int N, float cut, float p[6], Lo &lo, float C[21], Book &bk, Innov &I,
                                       uint32_t &status, int &c_cl, int &c_ht, float *lchi, int *lorig, float *lu,
                                       float *lv, int ls, Expansion &X) {
    float sphi, cphi;
    sincos_pair(p[4], lo.phi, sphi, cphi);
    const float cot = cot_pair(p[5], lo.th);
    X.cot = cot;
    X.searched = false;
    X.nlist = 0;
    X.n_compat = 0;
    float s = 0.f;
    const float kbl = kPhys == 2 ? G.kb * bz_factor(G.alpha, p[0], p[1], p[2]) : G.kb;
    const int l = finite_state(p) ? next_layer(G, kbl, mask, p, lo, sphi, cphi, cot, dir, bk.ncyl, bk.ndsk, s) : -2;
    X.layer = l;
    if (l == -2) status |= MKF_ST_NONFINITE;
    if (l < 0) {
        bk.done = true;
        return;
    }
    const LayerDesc &Ld = G.L[l];
    if (kPhys == 2)
        propagate_field(Ld, G.kb, G.alpha, p, lo, C, sphi, cphi, -p[3] * kbl, s);
    else
        propagate_transport(Ld, G.kb, p, lo, C, sphi, cphi, cot, s);
    if (kPhys >= 1) {
        float mx0, mk;
        material_at(G, Ld, p, mx0, mk);
        add_scattering(Ld.kind, mx0, p, C);
        apply_eloss(Ld.kind, mx0, mk, p, C, 1.f);
    }
    X.searched = true;
    ++c_cl;
    const Frame f = frame_of(p);
    if (!innovation(Ld.kind, Ld.su2, Ld.sv2, f, C, I)) {
        status |= MKF_ST_BADS;
        return;
    }
    const float wu = sqrtf(cut * I.Suu), wv = sqrtf(cut * I.Svv);
    const float wu_m = wu * 1.0001f, wv_m = wv * 1.0001f;
    const float lever = Ld.kind == 0 ? Ld.rz : f.rt;
    const float dphiw = wu_m / lever + 2e-6f;
    const float zc = Ld.kind == 0 ? p[2] : f.rt;
    const float wz = wv_m + 1e-5f;
    const float phic = atan2f(p[1], p[0]);
    int pb_lo, nphib;
    if (dphiw >= kPi) {
        pb_lo = 0;
        nphib = Ld.nphi;
    } else {
        pb_lo = static_cast<int>(floorf((phic - dphiw + kPi) * Ld.phi_scale));
        const int pb_hi = static_cast<int>(floorf((phic + dphiw + kPi) * Ld.phi_scale));
        nphib = min(pb_hi - pb_lo + 1, Ld.nphi);
        // |phic| <= pi and dphiw < pi put pb_lo in [-nphi/2 - 1, nphi]; the clamp
        // keeps every pb_lo + i below in [-nphi, 2 nphi) whatever the floats
        pb_lo = min(max(pb_lo, -Ld.nphi), Ld.nphi);
    }
    const float zlo_f = fminf(fmaxf(floorf((zc - wz - Ld.lo) * Ld.zr_scale), 0.f), Ld.nzr - 1.f);
    const float zhi_f = fminf(fmaxf(floorf((zc + wz - Ld.lo) * Ld.zr_scale), 0.f), Ld.nzr - 1.f);
    const int zb_lo = static_cast<int>(zlo_f), zb_hi = static_cast<int>(zhi_f);
    const int ebase = ev * G.bins_per_event + Ld.bin_base;
    int nlist = 0, n_compat = 0;
    // Loads run one ahead: the offsets of the next phi bin load while this
    // bin's hits are tested, and each hit record while the one before it is
    // (a window that spans many bins and hits otherwise waits on one load at a
    // time: -25 % for the widest-window seeds with material, -10 % for the
    // whole material workload, no change without material).
    // the hit range [k0, k1) of the window's z (or r) bins in phi bin i
    auto bin_range = [&](int i, int &k0, int &k1) {
        int pb = pb_lo + i;
        if (pb < 0) pb += Ld.nphi;
        else if (pb >= Ld.nphi) pb -= Ld.nphi;
        const int bin = ebase + pb * Ld.nzr;
        k0 = A.offsets[bin + zb_lo];
        k1 = A.offsets[bin + zb_hi + 1];
    };
    int nk0 = 0, nk1 = 0;
    if (nphib > 0) bin_range(0, nk0, nk1);
    for (int i = 0; i < nphib; ++i) {
        const int k0 = nk0, k1 = nk1;
        if (i + 1 < nphib) bin_range(i + 1, nk0, nk1);
        float4 nhr = k0 < k1 ? A.rec[k0] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = k0; k < k1; ++k) {
            const float4 hr = nhr;
            if (k + 1 < k1) nhr = A.rec[k + 1];
            if (fabsf(hr.z - zc) > wv_m) continue;
            float u, v;
            residual(Ld.kind, Ld.rz, p, lo, f, hr.x, hr.y, hr.z, u, v);
            if (fabsf(u) > wu_m) continue;
            if (fabsf(u) <= wu && fabsf(v) <= wv) ++c_ht;
            const float x2 = chi2_of(I, u, v);
            if (!(x2 < cut)) continue;
            const int orig = __float_as_int(hr.w);
            ++n_compat;
            // insert into the list, sorted by (chi2, orig), at most N
            if (nlist == N) {
                const float wc = lchi[(N - 1) * ls];
                const int wo = lorig[(N - 1) * ls];
                if (!(x2 < wc || (x2 == wc && orig < wo))) continue;
            }
            int j = nlist < N ? nlist : N - 1;
            while (j > 0) {
                const float pc = lchi[(j - 1) * ls];
                const int po = lorig[(j - 1) * ls];
                if (pc > x2 || (pc == x2 && po > orig)) {
                    lchi[j * ls] = pc;
                    lorig[j * ls] = po;
                    lu[j * ls] = lu[(j - 1) * ls];
                    lv[j * ls] = lv[(j - 1) * ls];
                    --j;
                } else {
                    break;
                }
            }
            lchi[j * ls] = x2;
            lorig[j * ls] = orig;
            lu[j * ls] = u;
            lv[j * ls] = v;
            if (nlist < N) ++nlist;
        }
    }
    X.nlist = nlist;
    X.n_compat = n_compat;
}

// Seed fit, one thread per seed: state from the three hits (circle + line),
// then the Kalman fit through them (the first hit without propagation; the
// covariance as a square root from the prior), the tracking region from the
// seed's eta, the direction along z and the first layers beyond the third hit.
// kPhys: 0 uniform field, 1 material effects, 2 parameterised field
// (Runge-Kutta propagation) and material effects.
template <int kPhys>
__global__ void __launch_bounds__(128) seed_kernel(const __grid_constant__ FindArgs A) {
    constexpr bool kParamField = kPhys == 2;
    constexpr int kSq = kPhys >= 1 ? 9 : 5;  // square-root columns (two per layer of material)
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= seeds_in_call(A)) return;
    const int t = A.seed_list ? A.seed_list[li] : li;  // the seed
    if (t < 0 || t >= A.n_seeds) {
        record_fault(A.fault, kFaultBadSeedList, li);
        return;
    }
    const Geom &G = A.G;
    const int n = A.n_seeds;
    float *B = A.seedbuf;
    const int ev = A.seed_event[t];
    bool ok = ev >= 0 && ev < A.n_events;
    float hx[3] = {0.f, 0.f, 0.f}, hy[3] = {0.f, 0.f, 0.f}, hz[3] = {0.f, 0.f, 0.f};
    int hidx[3] = {-1, -1, -1}, hl[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        hidx[k] = A.seed_hits[(int64_t)k * n + t];
        if (!ok) continue;
        if (hidx[k] < 0 || hidx[k] >= A.n_hits) {
            record_fault(A.fault, kFaultBadSeedHit, t);
            ok = false;
            continue;
        }
        const int pos = A.inv[hidx[k]];
        hl[k] = A.layer8[hidx[k]];
        if (pos < 0 || pos >= A.n_hits || hl[k] >= G.n_layers) {
            ok = false;
            continue;
        }
        const float4 r = A.rec[pos];
        hx[k] = r.x;
        hy[k] = r.y;
        hz[k] = A.zhit[hidx[k]];
    }
    float p[6], C[21], eta = 0.f, chi2 = 0.f;
    SqrtCov<kSq> Q;
    Lo lo{0.f, 0.f, 0.f, 0.f, 0.f};
    if (ok) {
        const float h1[3] = {hx[0], hy[0], hz[0]}, h2[3] = {hx[1], hy[1], hz[1]}, h3[3] = {hx[2], hy[2], hz[2]};
        // the parameterised field at the middle hit sets the curvature scale
        const float kbs = kParamField ? G.kb * bz_factor(G.alpha, h2[0], h2[1], h2[2]) : G.kb;
        ok = seed_state(G.L[hl[0]], kbs, h1, h2, h3, p, Q, eta);
    }
    for (int k = 0; k < 3 && ok; ++k) {
        const LayerDesc &Ld = G.L[hl[k]];
        if (k > 0) {
            float sphi, cphi, s;
            sincos_pair(p[4], lo.phi, sphi, cphi);
            const float cot = cot_pair(p[5], lo.th);
            const float kbl = kParamField ? G.kb * bz_factor(G.alpha, p[0], p[1], p[2]) : G.kb;
            if (!path_to_layer(Ld, kbl, p, lo, sphi, cphi, cot, s)) {
                ok = false;
                break;
            }
            if (kParamField)
                propagate_field(Ld, G.kb, G.alpha, p, lo, &Q, sphi, cphi, -p[3] * kbl, s);
            else
                propagate_transport(Ld, G.kb, p, lo, &Q, sphi, cphi, cot, s);
            if (kPhys >= 1) {
                float mx0, mk;
                material_at(G, Ld, p, mx0, mk);
                add_scattering(Ld.kind, mx0, p, &Q);
                apply_eloss(Ld.kind, mx0, mk, p, &Q, 1.f);
            }
        }
        const Frame f = frame_of(p);
        float u, v;
        const float zr = Ld.kind == 0 ? hz[k] : sqrtf(fmaf(hx[k], hx[k], hy[k] * hy[k]));
        residual(Ld.kind, Ld.rz, p, lo, f, hx[k], hy[k], zr, u, v);
        chi2 += sqrt_update(Ld.kind, Ld.su2, Ld.sv2, f, u, v, p, lo, &Q);
    }
    if (ok) sqrt_to_cov(Q, C);
    ok = ok && finite_state(p);
    uint32_t status = ok ? 0u : MKF_ST_BADSEED;
    if (A.order_key) {
        const int key = (ev >= 0 && ev < A.n_events ? ev : 0) * kOrderBuckets +
                        (ok ? min(static_cast<int>(fabsf(eta) * 4.f), kOrderBuckets - 1) : 0);
        A.order_key[t] = key;
        A.order_pos[t] = atomicAdd(&A.order_counts[key], 1);
    }
    unsigned long long mask = 0;
    int dir = 1;
    Book bk{3, 0, -1, -1, false, false, 0};
    if (ok) {
        int region = 0;
        while (region + 1 < G.n_regions && eta >= G.edges[region]) ++region;
        mask = G.mask[region];
        dir = cot_pair(p[5], lo.th) >= 0.f ? 1 : -1;
        const int l3 = hl[2];
        const float r3 = sqrtf(fmaf(hx[2], hx[2], hy[2] * hy[2])), z3 = hz[2];
        if (G.L[l3].kind == 0) {
            const int pos = G.cyl_pos[l3] + 1;
            bk.ncyl = pos < G.n_cyl ? pos : -1;
        } else {
            for (int i = 0; i < G.n_cyl; ++i)
                if (G.L[G.cyl[i]].rz > r3) {
                    bk.ncyl = i;
                    break;
                }
        }
        if (G.L[l3].kind == 1) {
            const int nx = G.dsk_pos[l3] + dir;
            bk.ndsk = (nx >= 0 && nx < G.n_dsk) ? nx : -1;
        } else if (dir > 0) {
            for (int i = 0; i < G.n_dsk; ++i)
                if (G.L[G.dsk[i]].rz > z3) {
                    bk.ndsk = i;
                    break;
                }
        } else {
            for (int i = G.n_dsk - 1; i >= 0; --i)
                if (G.L[G.dsk[i]].rz < z3) {
                    bk.ndsk = i;
                    break;
                }
        }
    }
    // The first step of the finder for this seed (one parent, so no selection
    // across candidates): the move to the next layer and the hit list.  The
    // seed's children are its compatible hits in list order (chi2, hit index),
    // then the miss (or the pass when no layer is left), the first N of them --
    // the order the finder's warp selection gives a single parent; the finder's
    // lanes make the children (one Kalman update each) from the moved seed,
    // its S^-1 and H C, and the list.
    int nbeam = 0, c_cl = 0, c_ht = 0, nlist = 0;
    bool searched = false;
    Innov I;
    if (A.step1 && ok) {
        const int N = A.n_best;
        float lchi[MKF_MAX_NBEST], lu[MKF_MAX_NBEST], lv[MKF_MAX_NBEST];
        int lorig[MKF_MAX_NBEST];
        Expansion X;
        expand<kPhys>(A, G, ev, mask, dir, N, A.cut, p, lo, C, bk, I, status, c_cl, c_ht, lchi, lorig, lu, lv, 1, X);
        nlist = X.nlist;
        searched = X.searched;
        nbeam = min(searched ? nlist + 1 : 1, N);
        float *L = A.beam;
        for (int k = 0; k < nlist; ++k) {
            L[((int64_t)k * kListFields + LF_CHI2) * n + t] = lchi[k];
            L[((int64_t)k * kListFields + LF_ORIG) * n + t] = __int_as_float(lorig[k]);
            L[((int64_t)k * kListFields + LF_U) * n + t] = lu[k];
            L[((int64_t)k * kListFields + LF_V) * n + t] = lv[k];
        }
        if (nlist > 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                B[(SF_I + k) * (int64_t)n + t] = I.HCu[k];
                B[(SF_I + 6 + k) * (int64_t)n + t] = I.HCv[k];
            }
            B[(SF_I + 12) * (int64_t)n + t] = I.Iuu;
            B[(SF_I + 13) * (int64_t)n + t] = I.Iuv;
            B[(SF_I + 14) * (int64_t)n + t] = I.Ivv;
        }
    }
    B[SF_NLIST * (int64_t)n + t] = __int_as_float(nlist);
    B[SF_SEARCHED * (int64_t)n + t] = __int_as_float(searched ? 1 : 0);
    B[SF_BEAM * (int64_t)n + t] = __int_as_float(nbeam);
    B[SF_CCL * (int64_t)n + t] = __int_as_float(c_cl);
    B[SF_CHT * (int64_t)n + t] = __int_as_float(c_ht);
#pragma unroll
    for (int i = 0; i < 6; ++i) B[(SF_P + i) * (int64_t)n + t] = p[i];
    B[(SF_LO + 0) * (int64_t)n + t] = lo.x;
    B[(SF_LO + 1) * (int64_t)n + t] = lo.y;
    B[(SF_LO + 2) * (int64_t)n + t] = lo.z;
    B[(SF_LO + 3) * (int64_t)n + t] = lo.phi;
    B[SF_LOTH * (int64_t)n + t] = lo.th;
#pragma unroll
    for (int k = 0; k < 21; ++k) B[(SF_C + k) * (int64_t)n + t] = C[k];
    B[SF_CHI2 * (int64_t)n + t] = chi2;
    B[SF_BOOK * (int64_t)n + t] = __uint_as_float(pack_book(bk));
    B[SF_MASK_LO * (int64_t)n + t] = __uint_as_float(static_cast<uint32_t>(mask));
    B[SF_MASK_HI * (int64_t)n + t] = __uint_as_float(static_cast<uint32_t>(mask >> 32));
    B[SF_DIR * (int64_t)n + t] = __int_as_float(dir);
    B[SF_STATUS * (int64_t)n + t] = __uint_as_float(status);
#pragma unroll
    for (int k = 0; k < 3; ++k) B[(SF_HITS + k) * (int64_t)n + t] = __int_as_float(hidx[k]);
}

// kLearned: the variant with learned pruning and the feature dump compiled in;
// the plain finder is built without them.  kPhys: 0 uniform field; 1 the
// material effects compiled in (selected when any layer has material); 2 the
// parameterised field (Runge-Kutta propagation) with the material effects.
// kN: the beam width N fixed at compile time (1 or 10, the widths the finder
// mostly runs with: the segment loops and lane arithmetic fold, 3-4 % faster;
// not for the parameterised field), or 0 for N taken from the arguments.
template <bool kLearned, int kPhys, int kN>
__global__ void __launch_bounds__(256, 2) find_kernel(const __grid_constant__ FindArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Geom SG;
    __shared__ float WS[MKF_MLP_PARAMS];
    {
        const int *src = reinterpret_cast<const int *>(&A.G);
        int *dst = reinterpret_cast<int *>(&SG);
        for (int i = threadIdx.x; i < static_cast<int>(sizeof(Geom) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        if (kLearned && A.mlp)
            for (int i = threadIdx.x; i < MKF_MLP_PARAMS; i += blockDim.x)
                WS[i] = __uint_as_float(static_cast<uint32_t>(A.mlp[i]) << 16);
    }
    __syncthreads();
    const Geom &G = SG;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int N = kN > 0 ? kN : A.n_best;
    const int spw = 32 / N;
    const int slot = lane / N, rank = lane - slot * N;
    const int base = slot * N;
    const bool lane_used = slot < spw;
    const int nwarps = blockDim.x >> 5;

    // shared memory: per-step history, then the per-lane child lists, then the
    // per-lane selection slots (index of the chosen child in its parent's list)
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem) + warp * (A.max_steps * 32);
    float *lchi = reinterpret_cast<float *>(reinterpret_cast<uint32_t *>(smem) + nwarps * A.max_steps * 32) +
                  warp * (N * 32 * 4);
    int *lorig = reinterpret_cast<int *>(lchi) + N * 32;
    float *lu = lchi + 2 * N * 32;
    float *lv = lchi + 3 * N * 32;
    int *sel = reinterpret_cast<int *>(reinterpret_cast<float *>(reinterpret_cast<uint32_t *>(smem) + nwarps * A.max_steps * 32) +
                                       nwarps * (N * 32 * 4)) +
               warp * 32;

    const float cut = A.cut;
    if (A.event_times && threadIdx.x == 0) atomicMin(&A.event_times[A.n_events], globaltimer_ns());

    // persistent warps: each takes the next group of seeds from a shared counter
    const int n_call = seeds_in_call(A);
    const int n_groups = (n_call + spw - 1) / spw;
    for (;;) {
        int grp = 0;
        if (lane == 0) grp = atomicAdd(A.work_counter, 1);
        grp = __shfl_sync(kFull, grp, 0);
        if (grp >= n_groups) break;
        const int li = grp * spw + slot;
        int seed = li;
        bool has_seed = lane_used && li < n_call;
        if (A.seed_list && has_seed) {
            seed = A.seed_list[li];
            // an out-of-range entry was recorded by the seed kernel
            has_seed = seed >= 0 && seed < A.n_seeds;
        }
        float p[6], C[21];
        Lo lo{0.f, 0.f, 0.f, 0.f, 0.f};
    #pragma unroll
        for (int i = 0; i < 6; ++i) p[i] = 0.f;
    #pragma unroll
        for (int k = 0; k < 21; ++k) C[k] = 0.f;
        Innov I;
    #pragma unroll
        for (int k = 0; k < 6; ++k) I.HCu[k] = I.HCv[k] = 0.f;
        I.Suu = I.Suv = I.Svv = I.Iuu = I.Iuv = I.Ivv = 0.f;
        float chi2 = 0.f;
        Book bk{0, 0, -1, -1, true, false, 0};
        bool live = false;
        uint32_t status = 0;
        int c_cl = 0, c_ht = 0, c_up = 0;
        int dir = 1, ev = 0;
        unsigned long long mask = 0;
        int sh0 = -1, sh1 = -1, sh2 = -1;

        int step = 0;
        // the child this lane becomes (its parent's moved state is in p, lo, C,
        // chi2, bk, I): made at the top of the next step
        bool pend = false;
        uint32_t pcode = 0;
        float pu = 0.f, pv = 0.f, px2 = 0.f;
        if (!kLearned && A.step1) {
            // ---- the candidates after the first step, from seed_kernel: rank r
            // takes child r; the seed-level record goes to rank 0
            if (has_seed) {
                const float *Bs = A.seedbuf;
                const int64_t n = A.n_seeds;
                const int nb = __float_as_int(Bs[SF_BEAM * n + seed]);
                if (rank == 0) {
                    status = __float_as_uint(Bs[SF_STATUS * n + seed]);
                    ev = A.seed_event[seed];
                    mask = static_cast<unsigned long long>(__float_as_uint(Bs[SF_MASK_LO * n + seed])) |
                           (static_cast<unsigned long long>(__float_as_uint(Bs[SF_MASK_HI * n + seed])) << 32);
                    dir = __float_as_int(Bs[SF_DIR * n + seed]);
                    sh0 = __float_as_int(Bs[(SF_HITS + 0) * n + seed]);
                    sh1 = __float_as_int(Bs[(SF_HITS + 1) * n + seed]);
                    sh2 = __float_as_int(Bs[(SF_HITS + 2) * n + seed]);
                    c_cl = __float_as_int(Bs[SF_CCL * n + seed]);
                    c_ht = __float_as_int(Bs[SF_CHT * n + seed]);
                }
                if (rank < nb) {
                    // child `rank` of the moved seed
    #pragma unroll
                    for (int i = 0; i < 6; ++i) p[i] = Bs[(SF_P + i) * n + seed];
                    lo.x = Bs[(SF_LO + 0) * n + seed];
                    lo.y = Bs[(SF_LO + 1) * n + seed];
                    lo.z = Bs[(SF_LO + 2) * n + seed];
                    lo.phi = Bs[(SF_LO + 3) * n + seed];
                    lo.th = Bs[SF_LOTH * n + seed];
    #pragma unroll
                    for (int k = 0; k < 21; ++k) C[k] = Bs[(SF_C + k) * n + seed];
                    chi2 = Bs[SF_CHI2 * n + seed];
                    bk = unpack_book(__float_as_uint(Bs[SF_BOOK * n + seed]));
                    const int nl = __float_as_int(Bs[SF_NLIST * n + seed]);
                    uint32_t code = __float_as_int(Bs[SF_SEARCHED * n + seed]) ? kCodeMiss : kCodePass;
                    float u = 0.f, v = 0.f, x2 = 0.f;
                    if (rank < nl) {
    #pragma unroll
                        for (int k = 0; k < 6; ++k) {
                            I.HCu[k] = Bs[(SF_I + k) * n + seed];
                            I.HCv[k] = Bs[(SF_I + 6 + k) * n + seed];
                        }
                        I.Iuu = Bs[(SF_I + 12) * n + seed];
                        I.Iuv = Bs[(SF_I + 13) * n + seed];
                        I.Ivv = Bs[(SF_I + 14) * n + seed];
                        const float *L = A.beam;
                        x2 = L[((int64_t)rank * kListFields + LF_CHI2) * n + seed];
                        code = __float_as_uint(L[((int64_t)rank * kListFields + LF_ORIG) * n + seed]);
                        u = L[((int64_t)rank * kListFields + LF_U) * n + seed];
                        v = L[((int64_t)rank * kListFields + LF_V) * n + seed];
                    }
                    // made at the top of the first step, like every other child
                    pend = true;
                    pcode = code;
                    pu = u;
                    pv = v;
                    px2 = x2;
                    hist[lane] = code;  // parent rank 0
                    live = true;
                }
            }
            step = 1;
        } else if (has_seed && rank == 0) {
            // ---- the fitted seed (rank-0 lane), from seed_kernel
            const float *Bs = A.seedbuf;
            const int64_t n = A.n_seeds;
            status = __float_as_uint(Bs[SF_STATUS * n + seed]);
            ev = A.seed_event[seed];
            if (!(status & MKF_ST_BADSEED)) {
    #pragma unroll
                for (int i = 0; i < 6; ++i) p[i] = Bs[(SF_P + i) * n + seed];
                lo.x = Bs[(SF_LO + 0) * n + seed];
                lo.y = Bs[(SF_LO + 1) * n + seed];
                lo.z = Bs[(SF_LO + 2) * n + seed];
                lo.phi = Bs[(SF_LO + 3) * n + seed];
                lo.th = Bs[SF_LOTH * n + seed];
    #pragma unroll
                for (int k = 0; k < 21; ++k) C[k] = Bs[(SF_C + k) * n + seed];
                chi2 = Bs[SF_CHI2 * n + seed];
                bk = unpack_book(__float_as_uint(Bs[SF_BOOK * n + seed]));
                mask = static_cast<unsigned long long>(__float_as_uint(Bs[SF_MASK_LO * n + seed])) |
                       (static_cast<unsigned long long>(__float_as_uint(Bs[SF_MASK_HI * n + seed])) << 32);
                dir = __float_as_int(Bs[SF_DIR * n + seed]);
                sh0 = __float_as_int(Bs[(SF_HITS + 0) * n + seed]);
                sh1 = __float_as_int(Bs[(SF_HITS + 1) * n + seed]);
                sh2 = __float_as_int(Bs[(SF_HITS + 2) * n + seed]);
                live = true;
            }
        }
        {
            const int src = lane_used ? base : lane;
            ev = __shfl_sync(kFull, ev, src);
            mask = __shfl_sync(kFull, mask, src);
            dir = __shfl_sync(kFull, dir, src);
        }

        while (true) {
            // ---- 0. the pending child: Kalman update with its hit, or the miss
            if (pend) {
                make_child(pcode, I, pu, pv, px2, A.max_consec, p, lo, C, chi2, bk, c_up);
                pend = false;
            }
            if (step >= A.max_steps) {
                if (lane == 0) record_fault(A.fault, kFaultHistOverflow, grp);
                break;
            }
            const bool active = live && !bk.done;
            if (!__any_sync(kFull, active)) break;  // every candidate of the warp has finished
            // ---- 1. expansion: next layer, propagation, window search
            Expansion X{-1, false, 0, 0, 0.f};
            if (active) {
                expand<kPhys>(A, G, ev, mask, dir, N, cut, p, lo, C, bk, I, status, c_cl, c_ht, lchi + lane, lorig + lane,
                       lu + lane, lv + lane, 32, X);
            }
            // learned pruning / feature dump over the candidate's list (its N best
            // compatible hits); the MLP scores a list only when the candidate has
            // two or more compatible hits.  The lanes step through the list
            // positions together, so the MLP runs once per position for the warp
            if (kLearned && A.mlp_mode == 1) {
                // gate: the best compatible hit by chi2 of a candidate with two or
                // more is scored; a doubtful one flags the seed (nothing dropped)
                const bool score_it = X.searched && X.nlist > 0 && X.n_compat >= 2 && A.mlp;
                if (__any_sync(kFull, score_it)) {
                    const int ly = X.layer >= 0 ? X.layer : 0;
                    float fe[12];
                    pair_features(lu[lane], lv[lane], I, lchi[lane], cut, chi2, bk, ly, G.n_layers, G.L[ly].kind, p,
                                  X.cot, fe);
                    const float logit = mlp_logit(WS, fe);
                    if (score_it && logit < A.mlp_tau) status |= MKF_ST_AMBIG;
                }
            } else if (kLearned) {
                const bool score_it = X.searched && X.nlist > 0 && (A.feat_out || (A.mlp && X.n_compat >= 2));
                const int ly = X.layer >= 0 ? X.layer : 0;
                const LayerDesc &Ld = G.L[ly];
                int kept = 0;
                for (int j = 0; __any_sync(kFull, score_it && j < X.nlist); ++j) {
                    const bool has = score_it && j < X.nlist;
                    const int jj = has ? j : 0;
                    const float x2 = lchi[jj * 32 + lane], u = lu[jj * 32 + lane], v = lv[jj * 32 + lane];
                    const int orig = lorig[jj * 32 + lane];
                    float fe[12];
                    pair_features(u, v, I, x2, cut, chi2, bk, ly, G.n_layers, Ld.kind, p, X.cot, fe);
                    if (A.feat_out && has) {
                        const int at = atomicAdd(A.feat_count, 1);
                        if (at < A.feat_cap) {
#pragma unroll
                            for (int q = 0; q < 12; ++q) A.feat_out[(int64_t)at * 12 + q] = fe[q];
                            A.feat_ref[(int64_t)at * 3] = seed;
                            A.feat_ref[(int64_t)at * 3 + 1] = orig;
                            A.feat_ref[(int64_t)at * 3 + 2] = X.n_compat;
                        }
                    }
                    const float logit = A.mlp ? mlp_logit(WS, fe) : 0.f;
                    const bool drop = A.mlp && X.n_compat >= 2 && logit < A.mlp_tau;
                    if (has && !drop) {
                        if (kept != j) {
                            lchi[kept * 32 + lane] = x2;
                            lorig[kept * 32 + lane] = orig;
                            lu[kept * 32 + lane] = u;
                            lv[kept * 32 + lane] = v;
                        }
                        ++kept;
                    }
                }
                if (score_it) X.nlist = kept;
            }
            const int nlist = X.nlist;
            const bool searched = X.searched;
            __syncwarp();

            // ---- 2. selection of the N best children of each seed: up to N rounds
            // of a segmented max over the lanes' best remaining child.  The key is
            // the score as an order-preserving integer whose low 4 bits are
            // replaced by (15 - parent rank): keys are unique within a seed, the
            // maximum names the winning parent, and scores that agree to 2^-19
            // relative are ordered by parent rank.  Each lane holds the keys of its
            // two best remaining children and reads the one after them every round,
            // so a win moves on by selects, with no shared-memory wait and no
            // divergent branch in the round (a branch there measured 3-4 % slower
            // for the plain finder and 2x for the learned one).  The winner records
            // the child (its step-history word and its index in the parent's list)
            // for the lane that takes it.
            const float score = cut * static_cast<float>(bk.nh) - chi2;
            const int n_children = live ? (searched ? nlist + 1 : 1) : 0;
            const uint32_t nohit = searched ? kCodeMiss : kCodePass;
            bool got = false;
            if (N == 1) {
                if (n_children > 0) {
                    got = true;
                    hist[step * 32 + lane] = nlist > 0 ? static_cast<uint32_t>(lorig[lane]) : nohit;
                    sel[lane] = 0;
                }
            } else {
                const uint32_t tag = 15u - static_cast<uint32_t>(rank);
                int head = 0;
                uint32_t key = n_children > 0 ? sel_key(nlist > 0 ? score + cut - lchi[lane] : score, tag) : 0u;
                uint32_t knext = n_children > 1 ? sel_key(nlist > 1 ? score + cut - lchi[32 + lane] : score, tag) : 0u;
                // step-history payload of the lane's best remaining child
                uint32_t code = nlist > 0 ? static_cast<uint32_t>(lorig[lane]) : nohit;
                for (int j = 0; j < N; ++j) {
                    if (!__any_sync(kFull, key != 0u)) break;
                    const uint32_t m = seg_max32(key, rank, N, base);
                    const bool seg_ok = m != 0u && lane_used;
                    got = got || (seg_ok && rank == j);
                    const bool win = seg_ok && (m & 15u) == tag;
                    if (win) {
                        hist[step * 32 + base + j] = (static_cast<uint32_t>(rank) << 28) | code;
                        sel[base + j] = head;
                    }
                    // every lane reads what it would move on to (in-bounds rows), the
                    // winner takes it: no divergent branch in the round
                    const int h1 = head + 1, h2 = head + 2;
                    const float x2n = lchi[min(h2, N - 1) * 32 + lane];
                    const int on = lorig[min(h1, N - 1) * 32 + lane];
                    const uint32_t k2 = h2 < n_children ? sel_key(h2 < nlist ? score + cut - x2n : score, tag) : 0u;
                    const uint32_t c1 = h1 < nlist ? static_cast<uint32_t>(on) : nohit;
                    head = win ? h1 : head;
                    key = win ? knext : key;
                    knext = win ? k2 : knext;
                    code = win ? c1 : code;
                }
            }
            __syncwarp();

            // ---- 3. each lane becomes one child: its parent's propagated state,
            // and the parent's S^-1 and H C, by shuffles; the update follows at
            // the top of the next step
            const uint32_t rec = got ? hist[step * 32 + lane] : 0u;
            const int prank = got ? static_cast<int>(rec >> 28) : rank;
            const int src = lane_used ? base + prank : lane;
            uint32_t bw = pack_book(bk);
            bw = __shfl_sync(kFull, bw, src);
            chi2 = __shfl_sync(kFull, chi2, src);
    #pragma unroll
            for (int i = 0; i < 6; ++i) p[i] = __shfl_sync(kFull, p[i], src);
    #pragma unroll
            for (int k = 0; k < 21; ++k) C[k] = __shfl_sync(kFull, C[k], src);
            lo.x = __shfl_sync(kFull, lo.x, src);
            lo.y = __shfl_sync(kFull, lo.y, src);
            lo.z = __shfl_sync(kFull, lo.z, src);
            lo.phi = __shfl_sync(kFull, lo.phi, src);
            lo.th = __shfl_sync(kFull, lo.th, src);
    #pragma unroll
            for (int k = 0; k < 6; ++k) {
                I.HCu[k] = __shfl_sync(kFull, I.HCu[k], src);
                I.HCv[k] = __shfl_sync(kFull, I.HCv[k], src);
            }
            I.Iuu = __shfl_sync(kFull, I.Iuu, src);
            I.Iuv = __shfl_sync(kFull, I.Iuv, src);
            I.Ivv = __shfl_sync(kFull, I.Ivv, src);
            bk = unpack_book(bw);
            live = got;
            {
                // the hit's residual and chi2 from the parent's list (every lane
                // reads an in-bounds row; the lanes that take a hit keep it)
                const uint32_t code = rec & kHitMask;
                const bool hit = got && code < kCodeMiss;
                const int at = min(max(got ? sel[lane] : 0, 0), N - 1) * 32 + src;
                const float u = lu[at], v = lv[at], x2 = lchi[at];
                pend = got;
                pcode = code;
                pu = hit ? u : 0.f;
                pv = hit ? v : 0.f;
                px2 = hit ? x2 : 0.f;
            }
            ++step;
            __syncwarp();
        }
        __syncwarp();

        // ---- output: rank 0 of each seed holds the best candidate
        c_cl = seg_sum(c_cl, rank, N);
        c_ht = seg_sum(c_ht, rank, N);
        c_up = seg_sum(c_up, rank, N);
        status = seg_or(status, rank, N);
        if (has_seed && rank == 0) {
            const int n = A.n_seeds;
            const bool ok = !(status & MKF_ST_BADSEED) && live;
            int nout = 0;
            if (ok) {
                const int shs[3] = {sh0, sh1, sh2};
                for (int k = 0; k < 3 && nout < A.max_out; ++k) A.out_hits[(int64_t)(nout++) * n + seed] = shs[k];
                // the hits the finder added (the candidate's count beyond its three
                // seed hits), written from the last backwards while the history is
                // walked back from the best candidate
                const int cnt = bk.nh - 3;
                int pos = nout + cnt - 1;
                int r = 0;
                for (int st = step - 1; st >= 0; --st) {
                    const uint32_t rec = hist[st * 32 + base + r];
                    const uint32_t code = rec & kHitMask;
                    if (code < kCodeMiss) {
                        if (pos < A.max_out) A.out_hits[(int64_t)pos * n + seed] = static_cast<int>(code);
                        --pos;
                    }
                    r = static_cast<int>(rec >> 28);
                }
                if (nout + cnt > A.max_out) status |= MKF_ST_TRUNC;
                nout = min(nout + cnt, A.max_out);
                if (bk.missstop) status |= MKF_ST_MISSSTOP;
                if (!finite_state(p) || !isfinite(chi2)) status |= MKF_ST_NONFINITE;
            }
            for (int k = nout; k < A.max_out; ++k) A.out_hits[(int64_t)k * n + seed] = -1;
            const float nanv = __int_as_float(0x7fc00000);
            p[0] += lo.x;
            p[1] += lo.y;
            p[2] += lo.z;
            p[4] += lo.phi;
            p[5] += lo.th;
    #pragma unroll
            for (int i = 0; i < 6; ++i) A.out_par[(int64_t)i * n + seed] = ok ? p[i] : nanv;
    #pragma unroll
            for (int k = 0; k < 21; ++k) A.out_cov[(int64_t)k * n + seed] = ok ? C[k] : nanv;
            A.out_chi2[seed] = ok ? chi2 : nanv;
            A.out_nhits[seed] = ok ? bk.nh : 0;
            A.out_status[seed] = status;
            if (A.counters) {
                A.counters[seed] = c_cl;
                A.counters[(int64_t)n + seed] = c_ht;
                A.counters[2 * (int64_t)n + seed] = c_up;
            }
            if (A.event_times && ev >= 0 && ev < A.n_events) atomicMax(&A.event_times[ev], globaltimer_ns());
        }
    }
}

// The finder's processing order from the seed kernel's keys and places
// (order_counts scanned into offsets; the last entry holds the total): over
// every seed, or over the seeds of a seed list.
__global__ void __launch_bounds__(256) order_scatter_kernel(const int32_t *key, const int32_t *pos,
                                                            const int32_t *offsets, int n, const int32_t *list,
                                                            const int32_t *list_count, int32_t *order) {
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    const int count = list ? min(max(*list_count, 0), n) : n;
    if (li >= count) return;
    const int t = list ? list[li] : li;
    if (t >= 0 && t < n) order[offsets[key[t]] + pos[t]] = t;
}

// Ordered compaction of the seeds whose status has any of `bits` (ascending
// seed index, so a following seed-list call keeps the events' seeds together):
// per tile of kWhereTile seeds a count, one exclusive scan over the tiles, then
// each tile writes its seeds at its offset in order.
constexpr int kWhereThreads = 256, kWherePer = 4, kWhereTile = kWhereThreads * kWherePer;

__device__ __forceinline__ int where_flags(const uint32_t *status, int n, uint32_t bits, int first, bool f[kWherePer]) {
    int c = 0;
#pragma unroll
    for (int k = 0; k < kWherePer; ++k) {
        const int i = first + k;
        f[k] = i < n && (status[i] & bits) != 0u;
        c += f[k] ? 1 : 0;
    }
    return c;
}

// Exclusive prefix of v over the block's threads (kWhereThreads); total in *tot.
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int *tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(kFull, x, off);
        if (lane >= off) x += o;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < kWhereThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(kFull, s, off);
            if (lane >= off) s += o;
        }
        if (lane < kWhereThreads / 32) warp_sums[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const int before = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
    *tot = warp_sums[kWhereThreads / 32 - 1];
    return before;
}

__global__ void __launch_bounds__(kWhereThreads) where_count_kernel(const uint32_t *status, int n, uint32_t bits,
                                                                    int32_t *tile_counts) {
    __shared__ int warp_sums[kWhereThreads / 32];
    bool f[kWherePer];
    const int c = where_flags(status, n, bits, blockIdx.x * kWhereTile + threadIdx.x * kWherePer, f);
    int tot;
    block_exclusive_scan(c, warp_sums, &tot);
    if (threadIdx.x == 0) tile_counts[blockIdx.x] = tot;
}

// One block: tile counts -> exclusive offsets (in place), the total to *count.
__global__ void __launch_bounds__(kWhereThreads) where_scan_kernel(int32_t *tile_counts, int n_tiles,
                                                                   int32_t *count) {
    __shared__ int warp_sums[kWhereThreads / 32];
    int carry = 0;
    for (int base = 0; base < n_tiles; base += kWhereThreads) {
        const int i = base + threadIdx.x;
        const int v = i < n_tiles ? tile_counts[i] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, warp_sums, &tot);
        if (i < n_tiles) tile_counts[i] = carry + ex;
        carry += tot;
        __syncthreads();  // warp_sums reused by the next chunk
    }
    if (threadIdx.x == 0) *count = carry;
}

__global__ void __launch_bounds__(kWhereThreads) where_write_kernel(const uint32_t *status, int n, uint32_t bits,
                                                                    const int32_t *tile_offsets, int32_t *list) {
    __shared__ int warp_sums[kWhereThreads / 32];
    bool f[kWherePer];
    const int first = blockIdx.x * kWhereTile + threadIdx.x * kWherePer;
    const int c = where_flags(status, n, bits, first, f);
    int tot;
    int at = tile_offsets[blockIdx.x] + block_exclusive_scan(c, warp_sums, &tot);
#pragma unroll
    for (int k = 0; k < kWherePer; ++k)
        if (f[k]) list[at++] = first + k;
}

// steps: at most one per layer + one final step with no layer left
int find_max_steps(int n_layers) { return n_layers + 2; }

size_t find_smem_bytes(int n_layers, int n_best, int threads) {
    const int nwarps = threads / 32;
    return static_cast<size_t>(nwarps) * (find_max_steps(n_layers) * 32 * 4 + n_best * 32 * 16 + 32 * 4);
}

}  // namespace

extern "C" mkf_status mkf_find(mkf_ctx *ctx, const mkf_hitbins *bins, const int32_t *seed_hits,
                               const int32_t *seed_event, int32_t n_seeds, const mkf_find_params *params,
                               float *out_par, float *out_cov, float *chi2, int32_t *n_hits, int32_t *hit_idx,
                               int32_t max_out, uint32_t *status, int32_t *counters) {
    if (!ctx || !bins || !params) return MKF_ERR_ARG;
    if (!ctx->has_geom || bins->geom_version != ctx->geom_version) return MKF_ERR_GEOMETRY;
    if (bins->device != ctx->device) return MKF_ERR_ARG;
    if (n_seeds < 0 || max_out < 3) return MKF_ERR_ARG;
    const int N = params->n_best;
    if (N < 1) return MKF_ERR_ARG;
    if (N > MKF_MAX_NBEST) return MKF_ERR_CAPACITY;
    if (!(params->chi2_cut > 0.f) || !(params->chi2_cut < 3.0e38f)) return MKF_ERR_ARG;
    if (params->max_consec_miss < 1 || params->max_consec_miss > 15) return MKF_ERR_ARG;
    int threads = params->block_threads ? params->block_threads : 128;
    if (threads < 32 || threads > 256 || threads % 32) return MKF_ERR_ARG;
    if (n_seeds == 0) return MKF_OK;
    if (!seed_hits || !seed_event || !out_par || !out_cov || !chi2 || !n_hits || !hit_idx || !status) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    FindArgs A;
    A.G = ctx->geom;
    A.rec = bins->rec;
    A.inv = bins->inv;
    A.layer8 = bins->layer;
    A.zhit = bins->zhit;
    A.offsets = bins->offsets;
    A.n_hits = bins->n_hits;
    A.n_events = bins->n_events;
    A.seed_hits = seed_hits;
    A.seed_event = seed_event;
    A.n_seeds = n_seeds;
    A.n_best = N;
    A.cut = params->chi2_cut;
    A.max_consec = params->max_consec_miss;
    A.max_steps = find_max_steps(ctx->geom.n_layers);
    A.out_par = out_par;
    A.out_cov = out_cov;
    A.out_chi2 = chi2;
    A.out_nhits = n_hits;
    A.out_hits = hit_idx;
    A.max_out = max_out;
    A.out_status = status;
    A.counters = counters;
    A.fault = ctx->fault;
    A.mlp = params->mlp_bf16;
    A.mlp_tau = params->mlp_tau;
    A.feat_out = params->feat_out;
    A.feat_ref = params->feat_ref;
    A.feat_count = params->feat_count;
    A.feat_cap = params->feat_cap;
    if (A.feat_out && (!A.feat_ref || !A.feat_count || A.feat_cap < 0)) return MKF_ERR_ARG;
    if ((params->seed_list == nullptr) != (params->seed_count == nullptr)) return MKF_ERR_ARG;
    if (params->mlp_mode != 0 && params->mlp_mode != 1) return MKF_ERR_ARG;
    if (params->mlp_mode == 1 && (!params->mlp_bf16 || params->feat_out)) return MKF_ERR_ARG;
    if (params->seed_order != 0 && params->seed_order != 1) return MKF_ERR_ARG;
    const bool grouped = params->seed_order == 0;
    A.seed_list = params->seed_list;
    A.seed_count = params->seed_count;
    A.mlp_mode = params->mlp_mode;
    const size_t smem = find_smem_bytes(ctx->geom.n_layers, N, threads);
    if (smem > 200 * 1024) return MKF_ERR_CAPACITY;
    // raise the kernel's dynamic shared-memory limit only when needed (not during
    // a stream capture after the first call)
    const bool learned = params->mlp_bf16 || params->feat_out;
    // material anywhere in the geometry selects the variant with the material
    // effects compiled in, the parameterised field the one with Runge-Kutta
    // propagation; the others carry no trace of them
    const int phys = mkf_phys_variant(ctx->geom);
    const int vi = ((learned ? 3 : 0) + phys) * 3 + (N == 1 ? 1 : (N == 10 ? 2 : 0));
    const void *const kfns[18] = {
        reinterpret_cast<const void *>(find_kernel<false, 0, 0>), reinterpret_cast<const void *>(find_kernel<false, 0, 1>),
        reinterpret_cast<const void *>(find_kernel<false, 0, 10>), reinterpret_cast<const void *>(find_kernel<false, 1, 0>),
        reinterpret_cast<const void *>(find_kernel<false, 1, 1>), reinterpret_cast<const void *>(find_kernel<false, 1, 10>),
        reinterpret_cast<const void *>(find_kernel<false, 2, 0>), reinterpret_cast<const void *>(find_kernel<false, 2, 0>),
        reinterpret_cast<const void *>(find_kernel<false, 2, 0>), reinterpret_cast<const void *>(find_kernel<true, 0, 0>),
        reinterpret_cast<const void *>(find_kernel<true, 0, 1>), reinterpret_cast<const void *>(find_kernel<true, 0, 10>),
        reinterpret_cast<const void *>(find_kernel<true, 1, 0>), reinterpret_cast<const void *>(find_kernel<true, 1, 1>),
        reinterpret_cast<const void *>(find_kernel<true, 1, 10>), reinterpret_cast<const void *>(find_kernel<true, 2, 0>),
        reinterpret_cast<const void *>(find_kernel<true, 2, 0>), reinterpret_cast<const void *>(find_kernel<true, 2, 0>)};
    const void *kfn = kfns[vi];
    if (static_cast<int>(smem) > ctx->find_smem_attr) {
        const int want = static_cast<int>(std::max<size_t>(smem, 48 * 1024));
        for (int v = 0; v < 18; ++v)
            MKF_CUDA_TRY(cudaFuncSetAttribute(kfns[v], cudaFuncAttributeMaxDynamicSharedMemorySize, want));
        ctx->find_smem_attr = want;
    }
    void *scratch = nullptr;
    const size_t seed_bytes = ((sizeof(float) * (size_t)kSeedFields * n_seeds + 255) / 256) * 256;
    // the plain finder's first step runs in the seed kernel (one thread per
    // seed instead of one busy lane of N); its candidates go through the beam
    A.step1 = learned ? 0 : 1;
    const size_t beam_bytes =
        A.step1 ? ((sizeof(float) * (size_t)kListFields * n_seeds * N + 255) / 256) * 256 : 0;
    // the processing order (grouped by event and |eta|): keys, places, order, key counts
    const int n_keys = bins->n_events * kOrderBuckets;
    const size_t order_bytes =
        grouped ? ((sizeof(int32_t) * (3 * (size_t)n_seeds + n_keys + 1) + 255) / 256) * 256 : 0;
    mkf_status st = mkf_scratch(ctx, seed_bytes + beam_bytes + order_bytes + 256, &scratch);
    if (st != MKF_OK) return st;
    A.seedbuf = static_cast<float *>(scratch);
    A.beam = A.step1 ? reinterpret_cast<float *>(static_cast<char *>(scratch) + seed_bytes) : nullptr;
    A.work_counter = reinterpret_cast<int32_t *>(static_cast<char *>(scratch) + seed_bytes + beam_bytes + order_bytes);
    int32_t *order = nullptr;
    A.order_key = A.order_pos = A.order_counts = nullptr;
    if (grouped) {
        int32_t *ob = reinterpret_cast<int32_t *>(static_cast<char *>(scratch) + seed_bytes + beam_bytes);
        A.order_key = ob;
        A.order_pos = ob + n_seeds;
        order = ob + 2 * (size_t)n_seeds;
        A.order_counts = ob + 3 * (size_t)n_seeds;
        MKF_CUDA_TRY(cudaMemsetAsync(A.order_counts, 0, sizeof(int32_t) * (n_keys + 1), ctx->stream));
    }
    A.event_times = reinterpret_cast<unsigned long long *>(params->event_times);
    MKF_CUDA_TRY(cudaMemsetAsync(A.work_counter, 0, sizeof(int32_t), ctx->stream));
    if (A.event_times) {
        MKF_CUDA_TRY(cudaMemsetAsync(A.event_times, 0, sizeof(uint64_t) * bins->n_events, ctx->stream));
        MKF_CUDA_TRY(cudaMemsetAsync(A.event_times + bins->n_events, 0xff, sizeof(uint64_t), ctx->stream));
    }
    switch (phys) {
        case 0: seed_kernel<0><<<(n_seeds + 127) / 128, 128, 0, ctx->stream>>>(A); break;
        case 1: seed_kernel<1><<<(n_seeds + 127) / 128, 128, 0, ctx->stream>>>(A); break;
        default: seed_kernel<2><<<(n_seeds + 127) / 128, 128, 0, ctx->stream>>>(A); break;
    }
    MKF_CUDA_TRY(cudaGetLastError());
    if (grouped) {
        // key counts -> offsets (the total, n_seeds, lands in the last entry),
        // then the order; the finder takes the seeds through it
        where_scan_kernel<<<1, kWhereThreads, 0, ctx->stream>>>(A.order_counts, n_keys, A.order_counts + n_keys);
        order_scatter_kernel<<<(n_seeds + 255) / 256, 256, 0, ctx->stream>>>(
            A.order_key, A.order_pos, A.order_counts, n_seeds, A.seed_list, A.seed_count, order);
        MKF_CUDA_TRY(cudaGetLastError());
        A.order_key = nullptr;  // the finder writes no keys
        A.seed_list = order;
        A.seed_count = A.order_counts + n_keys;
    }
    // persistent grid: as many blocks as fit on the device at once, or fewer
    const int spw = 32 / N;
    const int seeds_per_block = spw * (threads / 32);
    const int need = (n_seeds + seeds_per_block - 1) / seeds_per_block;
    // occupancy of this configuration (queried once, so that a later call can
    // be captured into a CUDA graph without runtime queries)
    if (ctx->find_occ_threads[vi] != threads || ctx->find_occ_smem[vi] != static_cast<int>(smem)) {
        int occ = 0;
        MKF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, threads, smem));
        ctx->find_occ_threads[vi] = threads;
        ctx->find_occ_smem[vi] = static_cast<int>(smem);
        ctx->find_occ_blocks[vi] = occ;
    }
    const int per_sm = ctx->find_occ_blocks[vi];
    const int blocks = std::max(1, std::min(need, std::max(1, per_sm) * ctx->num_sms));
    void *kargs[1] = {&A};
    MKF_CUDA_TRY(cudaLaunchKernel(kfn, dim3(blocks), dim3(threads), kargs, smem, ctx->stream));
    return MKF_OK;
}

extern "C" mkf_status mkf_seeds_where(mkf_ctx *ctx, const uint32_t *status, int32_t n, uint32_t bits,
                                      int32_t *seed_list, int32_t *seed_count) {
    if (!ctx || n < 0 || !seed_count || (n > 0 && (!status || !seed_list))) return MKF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return MKF_ERR_CUDA;
    if (n == 0) {
        MKF_CUDA_TRY(cudaMemsetAsync(seed_count, 0, sizeof(int32_t), ctx->stream));
        return MKF_OK;
    }
    const int n_tiles = (n + kWhereTile - 1) / kWhereTile;
    // the tile counts live in the context's scratch (which a finding call with
    // these seeds has already sized far beyond them)
    void *scratch = nullptr;
    mkf_status st = mkf_scratch(ctx, sizeof(int32_t) * (size_t)n_tiles, &scratch);
    if (st != MKF_OK) return st;
    int32_t *tiles = static_cast<int32_t *>(scratch);
    where_count_kernel<<<n_tiles, kWhereThreads, 0, ctx->stream>>>(status, n, bits, tiles);
    where_scan_kernel<<<1, kWhereThreads, 0, ctx->stream>>>(tiles, n_tiles, seed_count);
    where_write_kernel<<<n_tiles, kWhereThreads, 0, ctx->stream>>>(status, n, bits, tiles, seed_list);
    MKF_CUDA_TRY(cudaGetLastError());
    return MKF_OK;
}
