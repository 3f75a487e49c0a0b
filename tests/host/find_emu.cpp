// Host driver of the finder's device code under warp emulation (tests only):
// the geometry table from the library's host header, the hit bins built on
// the host (ascending original index inside a bin, as the library's binning
// leaves them), the seed kernel run thread by thread, and the finder run as one
// persistent warp of 32 lane threads over all seeds.
#include "find_dev.inc"
#include "mkf_geom.h"

#include <thread>
#include <vector>

thread_local dim3 threadIdx, blockIdx;
dim3 blockDim;
WarpEmu *g_warp;
unsigned char *g_smem;

template <bool kLearned, int kPhys>
static void run_width(int kn, const FindArgs &A) {
    if (kn == 1) find_kernel<kLearned, kPhys, 1>(A);
    else if (kn == 10) find_kernel<kLearned, kPhys, 10>(A);
    else find_kernel<kLearned, kPhys, 0>(A);
}

static void run_variant(bool learned, int phys, int kn, const FindArgs &A) {
    if (learned) {
        if (phys == 0) run_width<true, 0>(kn, A);
        else if (phys == 1) run_width<true, 1>(kn, A);
        else find_kernel<true, 2, 0>(A);
    } else {
        if (phys == 0) run_width<false, 0>(kn, A);
        else if (phys == 1) run_width<false, 1>(kn, A);
        else find_kernel<false, 2, 0>(A);
    }
}

extern "C" int emu_find(const mkf_layer *layers, int nl, float bz, const float *X, const float *Y, const float *Z,
                        const int *layer, int n_hits, const int *event_offsets, int n_events, const int *seed_hits,
                        const int *seed_event, int n_seeds, int N, float cut, int max_consec, int max_out, int step1,
                        const uint16_t *mlp_bf16, float mlp_tau, float material, float eloss, int field_kind,
                        float alpha, int map_nr, int map_nz, float map_rmax, float map_zmin,
                        float map_zmax, const float *map_x0, const float *map_eloss, 
                        float *out_par, float *out_cov, float *out_chi2, int *out_nh, int *out_hits,
                        unsigned *out_status, int *counters, int *fault_out) {
    static Geom G;
    if (mkf_build_geom(layers, nl, nullptr, 0, nullptr, bz, G) != MKF_OK) return -1;
    for (int l = 0; l < nl; ++l) {  // as mkf_geometry_material sets them
        G.L[l].x0 = material;
        G.L[l].eloss = eloss;
    }
    G.field_kind = field_kind;  // as mkf_geometry_field sets it
    G.alpha = field_kind ? alpha : 0.f;
    static std::vector<float2> mapv;
    mapv.clear();
    if (map_nr > 0) {  // as mkf_geometry_material_map sets it
        mapv.resize(static_cast<size_t>(map_nr) * map_nz);
        for (size_t i = 0; i < mapv.size(); ++i) mapv[i] = make_float2(map_x0[i], map_eloss ? map_eloss[i] : 0.f);
        G.mat_map = mapv.data();
        G.map_nr = map_nr;
        G.map_nz = map_nz;
        G.map_rinv = static_cast<float>(map_nr) / map_rmax;
        G.map_zmin = map_zmin;
        G.map_zinv = static_cast<float>(map_nz) / (map_zmax - map_zmin);
    }
    const int phys = mkf_phys_variant(G);
    const int64_t n_bins = static_cast<int64_t>(n_events) * G.bins_per_event;
    std::vector<int> key(n_hits);
    for (int i = 0; i < n_hits; ++i) {
        int ev = 0;
        while (ev < n_events && event_offsets[ev + 1] <= i) ++ev;
        const LayerDesc &Ld = G.L[layer[i]];
        const float phi = atan2f(Y[i], X[i]);
        const float zr = Ld.kind == 0 ? Z[i] : sqrtf(fmaf(X[i], X[i], Y[i] * Y[i]));
        const int pb = std::min(std::max(static_cast<int>(floorf((phi + kPi) * Ld.phi_scale)), 0), Ld.nphi - 1);
        const int zb = std::min(std::max(static_cast<int>(floorf((zr - Ld.lo) * Ld.zr_scale)), 0), Ld.nzr - 1);
        key[i] = ev * G.bins_per_event + Ld.bin_base + pb * Ld.nzr + zb;
    }
    std::vector<int> offsets(n_bins + 1, 0), fill(n_bins, 0);
    for (int i = 0; i < n_hits; ++i) offsets[key[i] + 1]++;
    for (int64_t b = 0; b < n_bins; ++b) offsets[b + 1] += offsets[b];
    std::vector<float4> rec(n_hits);
    std::vector<int> inv(n_hits);
    std::vector<uint8_t> layer8(n_hits);
    std::vector<float> zhit(n_hits);
    for (int i = 0; i < n_hits; ++i) {
        const int k = offsets[key[i]] + fill[key[i]]++;
        const LayerDesc &Ld = G.L[layer[i]];
        rec[k] = float4{X[i], Y[i], Ld.kind == 0 ? Z[i] : sqrtf(fmaf(X[i], X[i], Y[i] * Y[i])), __int_as_float(i)};
        inv[i] = k;
        layer8[i] = static_cast<uint8_t>(layer[i]);
        zhit[i] = Z[i];
    }
    std::vector<float> seedbuf(static_cast<size_t>(kSeedFields) * n_seeds);
    std::vector<float> lists(static_cast<size_t>(kListFields) * n_seeds * N);
    mkf_fault fault{0, 0};
    int work = 0;
    FindArgs A;
    std::memset(&A, 0, sizeof(A));
    A.G = G;
    A.rec = rec.data();
    A.inv = inv.data();
    A.layer8 = layer8.data();
    A.zhit = zhit.data();
    A.offsets = offsets.data();
    A.n_hits = n_hits;
    A.n_events = n_events;
    A.seed_hits = seed_hits;
    A.seed_event = seed_event;
    A.n_seeds = n_seeds;
    A.n_best = N;
    A.cut = cut;
    A.max_consec = max_consec;
    A.max_steps = find_max_steps(nl);
    A.out_par = out_par;
    A.out_cov = out_cov;
    A.out_chi2 = out_chi2;
    A.out_nhits = out_nh;
    A.out_hits = out_hits;
    A.max_out = max_out;
    A.out_status = out_status;
    A.counters = counters;
    A.fault = &fault;
    A.seedbuf = seedbuf.data();
    A.beam = lists.data();
    A.step1 = mlp_bf16 ? 0 : step1;  // the learned variant takes its first step in the warp
    A.mlp = mlp_bf16;
    A.mlp_tau = mlp_tau;
    A.work_counter = &work;
    blockDim.x = 128;
    for (int t = 0; t < n_seeds; ++t) {
        blockIdx.x = t / 128;
        threadIdx.x = t % 128;
        if (phys == 2) seed_kernel<2>(A);
        else if (phys == 1) seed_kernel<1>(A);
        else seed_kernel<0>(A);
    }
    blockDim.x = 32;
    std::vector<unsigned char> smem(find_smem_bytes(nl, N, 32));
    g_smem = smem.data();
    WarpEmu w;
    g_warp = &w;
    std::vector<std::thread> lanes;
    for (int l = 0; l < 32; ++l)
        lanes.emplace_back([&, l] {
            threadIdx.x = l;
            blockIdx.x = 0;
            // the variant the library launches: fixed beam width 1 or 10 except in
            // the parameterised field
            const int kn = phys == 2 ? 0 : (N == 1 ? 1 : (N == 10 ? 10 : 0));
            run_variant(mlp_bf16 != nullptr, phys, kn, A);
        });
    for (auto &t : lanes) t.join();
    fault_out[0] = fault.code;
    fault_out[1] = fault.where;
    return 0;
}
