"""Run the finder's device code under host warp emulation on one synthetic
batch and save the outputs (a separate process: a warp divergence ends it)."""
import ctypes as C
import sys

import numpy as np


def main(so, cfg, event, n_tracks, n_noise, n_best, step1, out_path, mlp_path=None, tau=0.0, material=0.0, eloss=0.0,
         alpha=None, gen_field=False, map_path=None):
    sys.path.insert(0, sys.argv[-1])  # repository root
    from paper_1811_04141_gb300 import _native as NN
    from synth import make_batch
    mm = None
    if map_path is not None:
        z = np.load(map_path)
        mm = dict(r_max=float(z["r_max"]), z_min=float(z["z_min"]), z_max=float(z["z_max"]), x0=z["x0"],
                  eloss=z["eloss"] if "eloss" in z.files else None)
    if gen_field:
        b = make_batch(cfg, [event], n_tracks=n_tracks, n_noise=n_noise, field_alpha=alpha)
    elif mm is not None:
        b = make_batch(cfg, [event], n_tracks=n_tracks, n_noise=n_noise, material_map=mm)
    else:
        b = make_batch(cfg, [event], n_tracks=n_tracks, n_noise=n_noise)
    lib = C.CDLL(so)
    lay = b.layers
    arr = (NN.MkfLayer * len(lay))()
    for i, d in enumerate(lay):
        arr[i] = NN.MkfLayer(int(d["kind"]), float(d["r_or_z"]), float(d["lo"]), float(d["hi"]), float(d["sigma_u"]),
                             float(d["sigma_v"]), int(d["n_phi"]), int(d["n_zr"]))
    n, mo = b.n_seeds, len(lay) + 3
    out = dict(par=np.zeros((6, n), np.float32), cov=np.zeros((21, n), np.float32), chi2=np.zeros(n, np.float32),
               n_hits=np.zeros(n, np.int32), hits=np.full((mo, n), -7, np.int32), status=np.zeros(n, np.uint32),
               counters=np.zeros((3, n), np.int32), fault=np.zeros(2, np.int32))
    X, Y, Z = [np.ascontiguousarray(b.xyz[i], dtype=np.float32) for i in range(3)]
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    keep = [i32(b.layer), i32(b.event_offsets), i32(b.seed_hits), i32(b.seed_event)]
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    if mm is None:
        map_args = [0, 0, C.c_float(1.0), C.c_float(0.0), C.c_float(1.0), None, None]
    else:
        mx = np.ascontiguousarray(mm["x0"], dtype=np.float32)
        me = None if mm["eloss"] is None else np.ascontiguousarray(mm["eloss"], dtype=np.float32)
        map_args = [mx.shape[0], mx.shape[1], C.c_float(mm["r_max"]), C.c_float(mm["z_min"]), C.c_float(mm["z_max"]),
                    p(mx), None if me is None else p(me)]
    w = None if mlp_path is None else np.ascontiguousarray(np.load(mlp_path), dtype=np.uint16)
    rc = lib.emu_find(arr, len(lay), C.c_float(b.bz), p(X), p(Y), p(Z), p(keep[0]), b.n_hits, p(keep[1]),
                      len(b.event_offsets) - 1, p(keep[2]), p(keep[3]), n, n_best, C.c_float(30.0), 3, mo, step1,
                      None if w is None else p(w), C.c_float(tau), C.c_float(material), C.c_float(eloss),
                      0 if alpha is None else 1, C.c_float(0.0 if alpha is None else alpha), *map_args,
                      p(out["par"]), p(out["cov"]), p(out["chi2"]), p(out["n_hits"]), p(out["hits"]), p(out["status"]),
                      p(out["counters"]), p(out["fault"]))
    if rc != 0:
        raise SystemExit(f"emu_find failed: {rc}")
    np.savez(out_path, **out)


if __name__ == "__main__":
    a = sys.argv[1:]
    main(a[0], a[1], int(a[2]), int(a[3]), None if a[4] == "none" else int(a[4]), int(a[5]), int(a[6]), a[7],
         None if a[8] == "none" else a[8], float(a[9]), float(a[10]), float(a[11]),
         None if a[12] == "none" else float(a[12]), a[13] == "1", None if a[14] == "none" else a[14])
