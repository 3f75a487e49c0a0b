// Host build of the library's geometry-table construction (tests only).
#include "host_prelude.h"
#include "mkf_geom.h"

// out: [0] n_cyl, [1] n_dsk, [2] bins_per_event, [3..3+n) bin_base per layer,
//      [67..67+n_cyl) cylinder ids by radius, [131..131+n_dsk) disk ids by z,
//      [195..195+n_regions) region masks (low 32 bits), [211] n_regions
extern "C" int host_build_geom(const mkf_layer *layers, int n, const mkf_plan *plans, int np, const float *edges,
                               float bz, int *out, float *out_f) {
    static mkf::Geom G;
    const int st = mkf_build_geom(layers, n, plans, np, edges, bz, G);
    if (st != MKF_OK) return st;
    out[0] = G.n_cyl;
    out[1] = G.n_dsk;
    out[2] = G.bins_per_event;
    for (int l = 0; l < n; ++l) out[3 + l] = G.L[l].bin_base;
    for (int i = 0; i < G.n_cyl; ++i) out[67 + i] = G.cyl[i];
    for (int i = 0; i < G.n_dsk; ++i) out[131 + i] = G.dsk[i];
    for (int r = 0; r < G.n_regions; ++r) out[195 + r] = static_cast<int>(G.mask[r] & 0xffffffffu);
    out[211] = G.n_regions;
    out_f[0] = G.kb;
    for (int i = 0; i < G.n_cyl; ++i) {
        out_f[1 + i] = G.cyl_hi_beyond[i];
        out_f[65 + i] = G.cyl_lo_beyond[i];
    }
    return MKF_OK;
}
