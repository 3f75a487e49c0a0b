/*
 * mkf.h -- C ABI of the GB300 (sm_103a) Kalman-filter track fitting and finding
 * library (libmkf.so).
 *
 * Method: "Parallelized and Vectorized Tracking Using Kalman Filters with CMS
 * Detector Geometry and Events" (mkFit).  The library runs the data-parallel
 * per-layer step of that method on every track candidate at once: helix
 * propagation in a uniform solenoid field to a barrel cylinder or an endcap
 * disk (Sec. 1, extension of the Kalman-filter and propagation equations to
 * the endcap case), transport of the 6x6 symmetric covariance, a hit search in
 * per-layer windows (Sec. 2.1, hit search windows in the layer description),
 * chi2 of each compatible hit, best-hit or N-best branching where only the
 * selected extensions receive the final Kalman update (Sec. 1, the selection of
 * the best chi2 extensions before the Kalman update), and the Kalman update.
 * The same update along fixed hit lists is the track fit (Sec. 1, vectorised
 * fitting).  Hits and seeds are provided by the caller and found tracks are
 * copied back to the caller (Sec. 2.2).
 *
 * Conventions (all entry points):
 *  - Every pointer documented as "device" is caller-owned CUDA device memory on
 *    the context's device; the library only borrows it for the duration of the
 *    work it enqueues.  "Host" pointers are read before the call returns.
 *  - Work is enqueued asynchronously on the context's stream; outputs are valid
 *    once that stream has been synchronised (mkf_sync does that and also reports
 *    faults that kernels recorded on the device).
 *  - Track state p = (x, y, z, q/pT, phi, theta) in cm, cm, cm, c/GeV, rad, rad:
 *    global position on the current layer surface, azimuth phi of the momentum,
 *    polar angle theta.  Arrays of states are structure-of-arrays with the track
 *    index fastest: par[i * n + t] for i in 0..5; covariances are the 21-value
 *    packed lower triangle, cov[k * n + t] with k = i (i + 1) / 2 + j, i >= j.
 *  - Errors: a negative mkf_status; nothing aborts, traps or prints.  Per-track
 *    problems are MKF_ST_* status bits, not call errors.
 */
#ifndef MKF_H
#define MKF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mkf_status;

#define MKF_OK 0
#define MKF_ERR_ARG (-1)          /* invalid argument (NULL, negative size, bad parameter) */
#define MKF_ERR_GEOMETRY (-2)     /* invalid geometry, or no geometry loaded, or bins built for another geometry */
#define MKF_ERR_CAPACITY (-3)     /* a size exceeds a documented maximum */
#define MKF_ERR_CUDA (-4)         /* a CUDA runtime call failed (allocation, launch, copy) */
#define MKF_ERR_DEVICE_CHECK (-5) /* a kernel found an invalid value in device input (see mkf_sync) */

/* Per-track status bits (outputs of mkf_fit / mkf_find). */
#define MKF_ST_UNREACHABLE 1u /* fit: a hit's layer could not be reached; the hit was skipped */
#define MKF_ST_BADSEED 2u     /* the three seed hits do not define a track; outputs are NaN */
#define MKF_ST_NONFINITE 4u   /* a non-finite value appeared in the state */
#define MKF_ST_BADS 8u        /* a residual covariance was not positive definite; that update was skipped */
#define MKF_ST_MISSSTOP 16u   /* find: the best candidate stopped after max_consec_miss misses in a row */
#define MKF_ST_TRUNC 32u      /* find: the hit list did not fit into max_out entries */
#define MKF_ST_AMBIG 64u      /* find, MLP gate mode: the MLP doubted a best-chi2 extension of this seed */

#define MKF_MAX_LAYERS 64
#define MKF_MAX_REGIONS 16
#define MKF_MAX_NBEST 16
#define MKF_MAX_HITS ((1 << 28) - 2) /* hit indices are carried in 28 bits */

typedef struct mkf_ctx mkf_ctx;         /* opaque, library-owned */
typedef struct mkf_hitbins mkf_hitbins; /* opaque, library-owned device storage */

/* Create a context on CUDA device `cuda_device`, enqueueing work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * *out receives the context.  Errors: MKF_ERR_ARG, MKF_ERR_CUDA. */
mkf_status mkf_create(mkf_ctx **out, int32_t cuda_device, void *cuda_stream);

/* Release the context and its scratch memory (after synchronising its stream). */
void mkf_destroy(mkf_ctx *ctx);

/* Change the stream later calls enqueue on. */
mkf_status mkf_set_stream(mkf_ctx *ctx, void *cuda_stream);

/* Synchronise the context's stream and report any fault a kernel recorded in
 * device memory since the last mkf_sync (MKF_ERR_DEVICE_CHECK; the record is
 * then cleared) or a CUDA error (MKF_ERR_CUDA). */
mkf_status mkf_sync(mkf_ctx *ctx);

/* Human-readable name of a status code (static string). */
const char *mkf_status_string(mkf_status s);

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 2.1: a vector of per-layer descriptions with dimensions,   */
/* hit-search parameters and type; per-region layer plans)                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t kind;      /* 0 = barrel cylinder, 1 = endcap disk */
    float r_or_z;      /* cylinder radius R > 0, or disk position Z (signed), cm */
    float lo, hi;      /* extent: z range (cylinder) or r range (disk), cm, lo < hi */
    float sigma_u;     /* hit resolution along r-phi, cm (> 0) */
    float sigma_v;     /* hit resolution along z (cylinder) or r (disk), cm (> 0) */
    int32_t n_phi_bins; /* hit bins in phi, 1..4096 */
    int32_t n_zr_bins;  /* hit bins in z (cylinder) or r (disk), 1..4096 */
} mkf_layer;

typedef struct {
    int32_t n_layers;         /* number of entries in layer_ids */
    const int32_t *layer_ids; /* host; the layers this region's candidates may visit */
} mkf_plan;

/* Load the detector description (host arrays, copied).
 *  layers[n_layers], 1 <= n_layers <= MKF_MAX_LAYERS.
 *  plans[n_plans]: tracking regions (Sec. 2.1: steering parameters per region;
 *  the paper uses five eta regions).  A seed belongs to region r when
 *  region_eta_edges[r-1] <= eta < region_eta_edges[r] (eta of the three-hit seed
 *  estimate); region_eta_edges has n_plans - 1 ascending entries.  Within its
 *  region a candidate visits only the plan's layers, in the order its helix
 *  reaches them.  n_plans = 0 (plans and edges may be NULL) is one region with
 *  every layer.
 *  bz_tesla: uniform solenoid field (0 allowed: straight tracks).
 * Errors: MKF_ERR_ARG, MKF_ERR_GEOMETRY, MKF_ERR_CAPACITY. */
mkf_status mkf_geometry_load(mkf_ctx *ctx, const mkf_layer *layers, int32_t n_layers, const mkf_plan *plans,
                             int32_t n_plans, const float *region_eta_edges, float bz_tesla);

/* Material (Sec. 2.1: multiple scattering and energy loss from the radiation
 * lengths of the detector; here one thickness per layer): x0 [n_layers] (host,
 * copied), each layer's thickness in radiation lengths at normal incidence,
 * 0 = none; eloss [n_layers] (host, copied, or NULL = none), the mean energy
 * loss per radiation length at minimum ionisation (GeV), for the geometry
 * loaded last (n_layers must match it; mkf_geometry_load resets every layer to
 * none; an r-z map from mkf_geometry_material_map takes precedence).  Fit and finding then apply, on arriving at a layer by propagation,
 * multiple scattering -- the Highland angle theta0 (unit charge, pion mass) for
 * the path through the layer: Var(theta) += theta0^2, Var(phi) += theta0^2 /
 * sin^2(theta), q/pT following theta at fixed |p| -- and then the mean energy
 * loss eloss * path / beta^2 (q/pT and its covariance row scaled by p / p');
 * the backward fit applies them after each hit in reverse (energy gained back,
 * then the noise).  Without a field q/pT is not measured (0) and nothing is
 * applied.  Hit bins stay valid.  Errors: MKF_ERR_ARG (n_layers differs, x0
 * NULL), MKF_ERR_GEOMETRY (no geometry, a value negative, not finite or
 * >= 1000). */
mkf_status mkf_geometry_material(mkf_ctx *ctx, const float *x0, const float *eloss, int32_t n_layers);

/* Field type (Sec. 2.1: a constant or a parameterised magnetic field, chosen
 * per propagation) for the geometry loaded last (mkf_geometry_load resets it to
 * the uniform field).  kind 0: uniform Bz = bz_tesla, propagation along the
 * closed-form helix.  kind 1: the field of a solenoid near its centre to
 * second order, Bz = bz (1 - alpha (z^2 - r^2 / 2)), Bx = bz alpha x z,
 * By = bz alpha y z (cm, tesla; divergence- and curl-free), alpha in 1/cm^2
 * (0 = the uniform field integrated numerically).  In it fit and finding
 * propagate by classical fourth-order Runge-Kutta steps in path length (at most
 * 0.05 rad of turning and 10 cm per step, at most 16 steps, over the path that
 * the helix in the local axial field estimates, then two Newton steps onto the
 * surface) and transport the covariance with the Jacobian integrated along the
 * trajectory (the variational equations, the field's gradient included);
 * layer order and extent checks
 * use the local helix, and seeds take their curvature scale from the field at
 * the middle hit.  The material effects apply as set.  Hit bins stay valid.
 * Errors: MKF_ERR_ARG (kind not 0 or 1, alpha not finite or |alpha| >= 1e-2),
 * MKF_ERR_GEOMETRY (no geometry). */
mkf_status mkf_geometry_field(mkf_ctx *ctx, int32_t kind, float alpha);

/* r-z material map (Sec. 2.1: radiation and interaction lengths from
 * two-dimensional arrays indexed in r and z) for the geometry loaded last
 * (mkf_geometry_load removes it): nr x nz cells of equal size over
 * [0, r_max) x [z_min, z_max) (cm), x0 [nr * nz] (host, copied; cell (ir, iz)
 * at ir * nz + iz) the thickness in radiation lengths at normal incidence that
 * a particle crossing a layer there traverses, eloss [nr * nz] (host, copied,
 * or NULL = none) the mean energy loss per radiation length at minimum
 * ionisation (GeV).  While a map is loaded it replaces the layers' own
 * material (mkf_geometry_material): each arrival at a layer takes x0 and eloss
 * from the cell holding the state's (r, z), points outside the map from the
 * nearest edge cell; the effects are those of mkf_geometry_material.  The
 * cell is chosen in FP32 on the device, so a crossing within rounding of a
 * cell edge may take either cell: keep edges away from layer surfaces.
 * nr = nz = 0 removes the map.  The copy waits for the context's stream.
 * Errors: MKF_ERR_ARG (sizes out of range or over 2^20 cells, x0 NULL,
 * r_max <= 0, z_max <= z_min), MKF_ERR_GEOMETRY (no geometry, a value negative,
 * not finite or >= 1000), MKF_ERR_CUDA. */
mkf_status mkf_geometry_material_map(mkf_ctx *ctx, int32_t nr, int32_t nz, float r_max, float z_min, float z_max,
                                     const float *x0, const float *eloss);

/* ------------------------------------------------------------------------ */
/* Hit binning (per event and layer, phi x z or phi x r bins)               */
/* ------------------------------------------------------------------------ */

/* Sort hits into per-(event, layer) bins of the loaded geometry: phi x z on
 * cylinders, phi x r on disks (the acceleration structure behind Sec. 2.1's hit
 * search windows).
 *  xyz:           device float [3][n_hits], SoA global coordinates.
 *  layer:         device int32 [n_hits], layer id of each hit.
 *  event_offsets: device int32 [n_events + 1], first hit of each event,
 *                 ascending, event_offsets[0] = 0, event_offsets[n_events] = n_hits.
 * *inout: NULL to allocate a new bin store, or a store from an earlier call to
 * refill (its device memory is reused, grown only when too small).  Hits with
 * an invalid layer id are dropped and recorded as a device fault (mkf_sync).
 * The store keeps the hits of a bin in the order the scatter placed them
 * (nothing the library computes depends on that order); mkf_hitbins_export
 * first puts every bin into ascending original index.
 * Errors: MKF_ERR_ARG, MKF_ERR_GEOMETRY (no geometry), MKF_ERR_CAPACITY
 * (n_hits > MKF_MAX_HITS), MKF_ERR_CUDA. */
mkf_status mkf_hits_bin(mkf_ctx *ctx, const float *xyz, const int32_t *layer, const int32_t *event_offsets,
                        int32_t n_events, int32_t n_hits, mkf_hitbins **inout);

/* Free a bin store (after the work that uses it has completed). */
void mkf_hitbins_free(mkf_hitbins *bins);

/* Sizes of a bin store: hits, events, bins (n_events * bins_per_event).
 * Errors: MKF_ERR_ARG. */
mkf_status mkf_hitbins_info(const mkf_hitbins *bins, int32_t *n_hits, int32_t *n_events, int64_t *n_bins);

/* Copy a bin store into caller-owned device buffers (asynchronous, on the
 * context's stream; any pointer may be NULL to skip that array).  When rec or
 * inv is requested, the store's bins are first put into ascending original
 * index in place (stream-ordered; a call on another stream that uses the store
 * at the same time must be ordered with this one):
 *  rec [n_hits][4] float: binned hits (x, y, z on cylinders or r on disks, the
 *      original index as int32 bits), grouped by bin, ascending original index
 *      within a bin;
 *  inv [n_hits] int32: binned position of each original hit (-1 if dropped);
 *  offsets [n_bins + 1] int32: CSR offsets; bin id = event * bins_per_event +
 *      layer_base + phi_bin * n_zr_bins + zr_bin, with layer_base the sum of
 *      n_phi_bins * n_zr_bins over lower layer ids, phi_bin =
 *      floor((phi + pi) * n_phi_bins / 2pi), zr_bin = floor((zr - lo) *
 *      n_zr_bins / (hi - lo)), both clamped into range.
 * Errors: MKF_ERR_ARG, MKF_ERR_CUDA. */
mkf_status mkf_hitbins_export(mkf_ctx *ctx, const mkf_hitbins *bins, float *rec, int32_t *inv, int32_t *offsets);

/* Largest input mkf_hits_bin_static accepts. */
#define MKF_STATIC_MAX_HITS (1 << 22)
#define MKF_STATIC_MAX_BINS (1 << 22) /* n_events * bins per event */

/* Hit binning for callers that cannot allocate GPU memory: the paper has no
 * counterpart; this is a deployment variant of mkf_hits_bin.
 *
 * Some callers cannot call cudaMalloc at all -- code that runs inside another
 * framework's memory pool or a real-time trigger process whose memory is fixed
 * at start-up, or a process that must not grow its footprint.  This entry point
 * allocates nothing: it writes the same arrays mkf_hitbins_export copies out of
 * a bin store straight into caller-owned buffers, and keeps its working memory
 * (histogram, scan partial sums, per-hit bin keys) in one statically sized
 * device array inside libmkf.  That array (about 52 MB) is reserved on a GPU
 * when the library's binning code is loaded onto it and stays reserved until
 * the process exits.  Under CUDA's lazy module loading (the default) that
 * happens at the first call of mkf_hits_bin or mkf_hits_bin_static on that GPU;
 * a caller with a fixed footprint should make one such call during start-up
 * (with CUDA_MODULE_LOADING=EAGER the runtime reserves it when it first sets
 * up the library's code on the GPU instead).
 *
 *  xyz, layer, event_offsets, n_events, n_hits: as for mkf_hits_bin.
 *  rec [n_hits][4] float, inv [n_hits] int32, offsets [n_bins + 1] int32:
 *      device, caller-owned outputs, same layout and contents as
 *      mkf_hitbins_export (n_bins = n_events * bins per event of the geometry).
 *      rec must start on a 16-byte boundary (it is written as 16-byte records;
 *      cudaMalloc'd and PyTorch buffers are); offsets must hold exactly
 *      n_bins + 1 entries, all of which are written.
 * Limits: n_hits <= MKF_STATIC_MAX_HITS and n_bins <= MKF_STATIC_MAX_BINS, else
 * MKF_ERR_CAPACITY and nothing is enqueued; a misaligned rec gives MKF_ERR_ARG
 * and nothing is enqueued.
 * The first call on a device looks up the device address of the working array
 * (a runtime call, no allocation); make that first call before capturing the
 * stream into a CUDA graph.  All calls on a device share the one working array:
 * two calls whose work overlaps on the GPU (different streams or contexts
 * without ordering between them) race and corrupt each other's results.
 * Errors: MKF_ERR_ARG, MKF_ERR_GEOMETRY, MKF_ERR_CAPACITY, MKF_ERR_CUDA. */
mkf_status mkf_hits_bin_static(mkf_ctx *ctx, const float *xyz, const int32_t *layer, const int32_t *event_offsets,
                               int32_t n_events, int32_t n_hits, float *rec, int32_t *inv, int32_t *offsets);

/* ------------------------------------------------------------------------ */
/* Fit (Sec. 1: Kalman-filter fitting along known hits)                      */
/* ------------------------------------------------------------------------ */

/* Kalman fit of n tracks along fixed hit lists.
 *  xyz [3][n_hits], hit_layer [n_hits]: device, as for mkf_hits_bin.
 *  hit_idx: device int32 [max_hits][n] (track fastest), the track's hits in
 *           path order; -1 entries are skipped.  1 <= max_hits <= 64.
 *  seed_par [6][n], seed_cov [21][n]: device, the starting state on the surface
 *           of the first hit; both NULL = seed each track from its first three
 *           hits (circle through three points, straight line in arc length-z).
 *  The first hit is applied without propagation; every later hit is reached by
 *  propagating to its layer's surface.
 *  Outputs (device, caller-owned): out_par [6][n], out_cov [21][n] -- state on
 *  the surface of the last hit used; chi2 [n] -- sum of the predicted-residual
 *  chi2 of all updates; ndf [n] = 2 * hits used - 5 (- 4 at zero field);
 *  status [n] -- MKF_ST_* bits.
 * Errors: MKF_ERR_ARG, MKF_ERR_GEOMETRY, MKF_ERR_CAPACITY, MKF_ERR_CUDA. */
mkf_status mkf_fit(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits, const int32_t *hit_idx,
                   int32_t max_hits, int32_t n, const float *seed_par, const float *seed_cov, float *out_par,
                   float *out_cov, float *chi2, int32_t *ndf, uint32_t *status);

/* Backward fit along fixed hit lists: the Kalman filter of mkf_fit run through
 * each track's hits in reverse order, the pass that delivers a fitted or found
 * track's parameters at its first (innermost) hit with every hit used (the
 * paper's layer plans carry layers used only during backward fitting, Sec. 2.1).
 * xyz, hit_layer, n_hits, hit_idx, max_hits, n and the outputs are as for
 * mkf_fit (hits listed in path order, -1 = none).  last_par [6][n], last_cov
 * [21][n] (device, packed as above): the state on the surface of each track's
 * last valid hit, e.g. mkf_fit's output.  That state is turned around (the same
 * helix with the momentum reversed: q/pT -> -q/pT, phi -> phi + pi, theta ->
 * pi - theta, and the matching sign changes of the covariance), its covariance
 * is multiplied by `inflate` (>= 1; large values make the pass independent of
 * the incoming covariance), it is updated with the last hit without moving,
 * then propagated to each earlier hit and updated; at the first hit it is turned
 * back.  Outputs: the state and covariance on the surface of the first hit used,
 * chi2 and ndf over the hits used, status bits as for mkf_fit (fewer than 3
 * valid hits: MKF_ST_BADSEED, NaN outputs).  Errors: MKF_ERR_ARG (inflate < 1
 * or not finite, last_par or last_cov NULL with n > 0, other arguments as for
 * mkf_fit), MKF_ERR_GEOMETRY, MKF_ERR_CAPACITY, MKF_ERR_CUDA. */
mkf_status mkf_fit_backward(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits,
                            const int32_t *hit_idx, int32_t max_hits, int32_t n, const float *last_par,
                            const float *last_cov, float inflate, float *out_par, float *out_cov, float *chi2,
                            int32_t *ndf, uint32_t *status);

/* Smoothed state at every hit of fixed hit lists (Sec. 2.1 mentions
 * back-fit layers): two filters.  The forward filter of mkf_fit (seeded as
 * there) keeps its state after each hit; the backward filter starts from the
 * forward state at the last hit, turned around with its covariance multiplied
 * by inflate (>= 1; large values make the two filters nearly independent, e.g.
 * 1e4), predicts each earlier hit from the later ones and is updated with it,
 * its material applied in reverse as in mkf_fit_backward.  The smoothed state
 * at a hit is the weighted mean of the forward state there and the backward
 * prediction, taken in the five free parameters on the surface ((u, z) on a
 * cylinder with u along it, (x, y) on a disk, then q/pT, phi, theta); at the
 * last hit it is the forward state.  sm_par [max_hits][6][n] and sm_cov
 * [max_hits][21][n] (device, caller-owned; packed lower triangles) are indexed
 * by the row of hit_idx; rows without a hit, or where a step failed, are NaN.
 * chi2, ndf, status: the forward fit's (status also gets the backward pass's
 * bits).  Errors: as mkf_fit, plus MKF_ERR_ARG for inflate < 1. */
mkf_status mkf_fit_smooth(mkf_ctx *ctx, const float *xyz, const int32_t *hit_layer, int32_t n_hits,
                          const int32_t *hit_idx, int32_t max_hits, int32_t n, const float *seed_par,
                          const float *seed_cov, float inflate, float *sm_par, float *sm_cov, float *chi2,
                          int32_t *ndf, uint32_t *status);

/* ------------------------------------------------------------------------ */
/* Seed cleaning and duplicate-track removal (Sec. 2.2: repeated seeds of one */
/* particle are removed using the identity of their hits and their fitted     */
/* pT, eta and phi; Sec. 3: duplicate tracks are to be removed after finding) */
/* ------------------------------------------------------------------------ */

/* Seed cleaning.  seed_hits [3][n_seeds] (device, hit indices; entries outside
 * [0, n_hits) are ignored), seed_par [6][n_seeds] (device, the seeds' fitted
 * states, e.g. mkf_fit over their three hits; rows 3, 4, 5 = q/pT, phi, theta
 * are used).  Two seeds are duplicates when they share at least one hit and
 * |d(q/pT)| <= max_dqpt, |d eta| <= max_deta, |d phi| (wrapped) <= max_dphi,
 * eta = -ln tan(theta/2), differences taken in double.  keep [n_seeds]
 * (device, written): 0 when a duplicate with a lower index exists, else 1 (a
 * rule that needs no processing order).  Errors: MKF_ERR_ARG (negative sizes
 * or tolerances, NULL pointers with n_seeds > 0), MKF_ERR_CAPACITY, MKF_ERR_CUDA. */
mkf_status mkf_seeds_clean(mkf_ctx *ctx, const int32_t *seed_hits, int32_t n_seeds, int32_t n_hits,
                           const float *seed_par, float max_dqpt, float max_deta, float max_dphi, int32_t *keep);

/* Duplicate-track removal.  hit_idx [max_hits][n] (device, each track's hits,
 * -1 = none; e.g. mkf_find's hit_idx), track_nhits [n] and chi2 [n] (device,
 * e.g. mkf_find's n_hits and chi2).  Two tracks are duplicates when the hits
 * they share number at least max(1, min_frac x the smaller of their hit
 * counts) (0 <= min_frac <= 1; a hit listed twice by one track counts once).
 * keep [n] (device, written): 0 when a duplicate ranks above the track -- more
 * hits, then lower chi2, then lower index -- else 1.  Errors: MKF_ERR_ARG,
 * MKF_ERR_CAPACITY (max_hits > MKF_MAX_LAYERS + 8, n_hits > MKF_MAX_HITS),
 * MKF_ERR_CUDA. */
mkf_status mkf_tracks_dedup(mkf_ctx *ctx, const int32_t *hit_idx, int32_t max_hits, int32_t n, int32_t n_hits,
                            const int32_t *track_nhits, const float *chi2, float min_frac, int32_t *keep);

/* ------------------------------------------------------------------------ */
/* Finding (Sec. 1: layer-by-layer finding with selection of the best chi2   */
/* extensions before the final Kalman updates)                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n_best;          /* candidates kept per seed: 1 = best hit, 2..MKF_MAX_NBEST = N best */
    float chi2_cut;          /* a hit is compatible when its chi2 < chi2_cut (> 0) */
    int32_t max_consec_miss; /* a candidate stops after this many misses in a row (1..15) */
    int32_t block_threads;   /* CUDA block size, multiple of 32 in 32..256; 0 = default (128) */
    /* Learned pruning (not in the paper): when mlp_bf16 is not NULL and a
     * candidate has two or more compatible hits on a layer, each of its N best
     * compatible hits (by chi2) is scored by the MLP (device, MKF_MLP_PARAMS
     * bfloat16 weights) and dropped when its logit < mlp_tau; the child without
     * a hit is never dropped.  Features of a (candidate, hit) pair, in order:
     * u/sqrt(S_uu), v/sqrt(S_vv), chi2/chi2_cut, chi2_total/max(1, 2 n_hits - 5),
     * n_hits/10, n_miss/5, layer/n_layers, is_disk, q/pT, eta/3,
     * log10 sqrt(S_uu), log10 sqrt(S_vv) -- candidate quantities before the hit. */
    const uint16_t *mlp_bf16;
    float mlp_tau;
    /* Feature dump (training data): when feat_out is not NULL, the features of
     * each candidate's N best compatible hits (before any pruning) go to
     * feat_out [feat_cap][12] (device) with (seed index, hit index, number of
     * compatible hits of the candidate on that layer) in feat_ref [feat_cap][3];
     * the device counter *feat_count (caller zeroes it) ends at the number of
     * pairs seen, of which min(count, feat_cap) were written, in no particular
     * order. */
    float *feat_out;
    int32_t *feat_ref;
    int32_t *feat_count;
    int32_t feat_cap;
    /* Per-event completion times (device [n_events + 1] or NULL): entry e is the
     * GPU global timer (ns) when the last seed of event e was written, entry
     * n_events the earliest start of a finding block; set by the call. */
    uint64_t *event_times;
    /* Seed subset (device, or both NULL for every seed): only the seeds
     * seed_list[0 .. *seed_count) (indices into seed_hits, each < n_seeds) are
     * found; their outputs are written at their own indices and every other
     * seed's outputs are left as they are.  The count is read on the device,
     * so a subset chosen by an earlier call (mkf_seeds_where) needs no host
     * round trip; *seed_count above n_seeds is taken as n_seeds, an index out
     * of range is a device fault (MKF_ERR_DEVICE_CHECK at mkf_sync). */
    const int32_t *seed_list;
    const int32_t *seed_count;
    /* With mlp_bf16: 0 prunes as described above; 1 (gate) drops nothing and
     * instead scores, on each layer where a candidate has two or more
     * compatible hits, its best one by chi2, setting MKF_ST_AMBIG on the seed
     * when that logit < mlp_tau (the learned cascade: best-hit finding with the
     * gate, then N-best finding of the flagged seeds only). */
    int32_t mlp_mode;
    /* Order in which the seeds are worked on (results do not depend on it):
     * 0 (default) grouped by event and by |eta| of the seed's three-hit
     * estimate (bins of 0.25), so that the seeds sharing a warp have similar
     * numbers of layers ahead; 1 the input order (with seed_list: its order). */
    int32_t seed_order;
} mkf_find_params;

/* Find tracks from seeds.
 *  bins: from mkf_hits_bin with the current geometry.
 *  seed_hits: device int32 [3][n_seeds], three hit indices per seed (path order).
 *  seed_event: device int32 [n_seeds], event of each seed.
 * Each seed is fitted through its three hits and then extended layer by layer:
 * a candidate goes to the next layer its helix reaches (the nearer of the next
 * cylinder and the next disk), every hit of that layer with chi2 < chi2_cut is
 * a child, plus one child without a hit; children are ranked by
 * score = chi2_cut * n_hits - chi2 (ties: lower parent rank, then lower hit
 * index, the child without a hit last) and the best n_best are kept; only kept
 * children receive the Kalman update.
 * Outputs (device, caller-owned): out_par [6][n_seeds], out_cov [21][n_seeds]
 * (best candidate's state at its last visited layer), chi2 [n_seeds],
 * n_hits [n_seeds], hit_idx [max_out][n_seeds] (hit indices in path order,
 * seed hits first, -1 padded; max_out >= 3), status [n_seeds],
 * counters [3][n_seeds] or NULL: candidate-layer steps, hits inside the chi2
 * window rectangle, Kalman updates.
 * Errors: MKF_ERR_ARG, MKF_ERR_GEOMETRY, MKF_ERR_CAPACITY, MKF_ERR_CUDA. */
mkf_status mkf_find(mkf_ctx *ctx, const mkf_hitbins *bins, const int32_t *seed_hits, const int32_t *seed_event,
                    int32_t n_seeds, const mkf_find_params *params, float *out_par, float *out_cov, float *chi2,
                    int32_t *n_hits, int32_t *hit_idx, int32_t max_out, uint32_t *status, int32_t *counters);

/* Seeds whose status has any of `bits` set (e.g. MKF_ST_AMBIG after a gated
 * best-hit pass, Sec. 1's selection of extensions done again with N
 * candidates for them): status [n] (device), seed_list [n] (device, written:
 * the indices in ascending order, so that the seeds of one event stay
 * together), *seed_count (device, written).  For the seed_list / seed_count
 * inputs of mkf_find; no host synchronisation.  Uses the context's scratch
 * memory (4 bytes per 1024 seeds; a preceding mkf_find call on these seeds has
 * sized it, so the call then allocates nothing and can be captured).
 * Errors: MKF_ERR_ARG, MKF_ERR_CUDA. */
mkf_status mkf_seeds_where(mkf_ctx *ctx, const uint32_t *status, int32_t n, uint32_t bits, int32_t *seed_list,
                           int32_t *seed_count);

/* ------------------------------------------------------------------------ */
/* Learned hit ranking (not in the paper: a small MLP that scores a          */
/* (candidate, compatible hit) pair so that branching can be pruned before   */
/* the Kalman update; trained here by these kernels)                         */
/* ------------------------------------------------------------------------ */

#define MKF_MLP_IN 12
#define MKF_MLP_HIDDEN 64
#define MKF_MLP_PARAMS (MKF_MLP_IN * MKF_MLP_HIDDEN + 2 * MKF_MLP_HIDDEN + 1) /* 897 */
/* Parameter layout: W1[64][12] (row = hidden unit), b1[64], w2[64], b2.
 * logit = w2 . relu(W1 x + b1) + b2, computed in FP32 with the weights rounded
 * to bfloat16 (round to nearest, ties to even). */

typedef struct {
    float lr, beta1, beta2, eps; /* Adam hyper-parameters (e.g. 1e-3, 0.9, 0.999, 1e-8) */
} mkf_adam;

/* FP32 -> bfloat16 (uint16 bit patterns), n values, device arrays.
 * Errors: MKF_ERR_ARG, MKF_ERR_CUDA. */
mkf_status mkf_mlp_to_bf16(mkf_ctx *ctx, const float *w, uint16_t *w_bf16, int32_t n);

/* Logits of n feature rows.  w_bf16 [MKF_MLP_PARAMS], feat [n][12], logit [n]:
 * device.  Errors: MKF_ERR_ARG, MKF_ERR_CUDA. */
mkf_status mkf_mlp_forward(mkf_ctx *ctx, const uint16_t *w_bf16, const float *feat, int32_t n, float *logit);

/* Mean binary cross-entropy of the logits against labels (0 or 1) and its
 * gradient with respect to the (bfloat16-rounded) weights.  feat [n][12],
 * label [n], grad [MKF_MLP_PARAMS], loss [1]: device.  The batch sum runs in a
 * fixed order: the result does not depend on scheduling.
 * Errors: MKF_ERR_ARG, MKF_ERR_CUDA. */
mkf_status mkf_mlp_grad(mkf_ctx *ctx, const uint16_t *w_bf16, const float *feat, const float *label, int32_t n,
                        float *grad, float *loss);

/* One Adam training step: gradient as mkf_mlp_grad with the weights w rounded
 * to bfloat16, then m, v and the FP32 master weights w updated in place (t is
 * the 1-based step number) and w_bf16 refreshed.  loss may be NULL.
 * Errors: MKF_ERR_ARG, MKF_ERR_CUDA. */
mkf_status mkf_mlp_train_step(mkf_ctx *ctx, const float *feat, const float *label, int32_t n, float *w, float *m,
                              float *v, int32_t t, const mkf_adam *hp, uint16_t *w_bf16, float *loss);

/* ------------------------------------------------------------------------ */
/* Measurement aid (not in the paper, which reports no roofline)             */
/* ------------------------------------------------------------------------ */

/* FP32 throughput probe: enqueues on the context stream one kernel in which
 * every thread runs 8 independent dependent-FMA chains for 16 * iters rounds
 * (8 blocks of 256 threads per SM), and returns in *flops (host) the number of
 * FP32 operations it performs (2 per FMA).  Timing the launch (e.g. with CUDA
 * events on the stream) gives the FP32 rate the fit and finder kernels are
 * measured against.  out: device buffer of at least 8 * (SM count) floats that
 * keeps the chains' result live (it is not written for these inputs).
 * Errors: MKF_ERR_ARG (iters < 1, NULL pointers), MKF_ERR_CUDA. */
mkf_status mkf_fp32_probe(mkf_ctx *ctx, int32_t iters, float *out, double *flops);

#ifdef __cplusplus
}
#endif

#endif /* MKF_H */
