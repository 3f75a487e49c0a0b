"""Binning without GPU allocation (mkf_hits_bin_static).

Some callers cannot allocate GPU memory: a process embedded in a host framework
that owns all device memory through its own pool, or a trigger process whose
footprint is fixed when it starts.  For them the library bins hits into buffers
the caller already owns and keeps its own working memory in a fixed device array
inside the library.  This test calls that entry point through the C ABI twice
in a row (a larger input, then a smaller one, so leftovers of the first call
would show) and checks that its output equals what the allocating path
(mkf_hits_bin followed by mkf_hitbins_export) produces for the same input, that
a call leaves the GPU's free memory unchanged, and that it refuses buffers it
could not write safely.
It lives in its own file, collected last, and works in a fresh process as well
as after the other tests.
"""
import numpy as np
import pytest
import torch

from synth import make_batch
from tests.gpu_helpers import make_ctx, upload

pytestmark = pytest.mark.gpu


def _allocating_path(ctx, d):
    bins = ctx.hits_bin(d["xyz"], d["layer"], d["event_offsets"])
    ex = bins.export(ctx)
    ctx.sync()
    return ex


def _static_path(ctx, d, n_bins):
    from paper_1811_04141_gb300.api import mkf_hits_bin_static
    n = d["xyz"].shape[1]
    rec = torch.full((n, 4), float("nan"), device="cuda")
    inv = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    off = torch.full((n_bins + 1,), -7, dtype=torch.int32, device="cuda")
    mkf_hits_bin_static(ctx.handle, d["xyz"], d["layer"], d["event_offsets"], rec, inv, off)
    ctx.sync()
    return rec, inv, off


def test_static_binning_matches_allocating_path_twice():
    big = make_batch("find20", [41, 42, 43], n_tracks=600)
    small = make_batch("find20", [44], n_tracks=120)
    ctx = make_ctx(big)
    for b in (big, small):
        d = upload(b)
        ref = _allocating_path(ctx, d)
        rec, inv, off = _static_path(ctx, d, ref["n_bins"])
        assert torch.equal(off, ref["offsets"])
        assert torch.equal(inv, ref["inv"])
        # bit-exact records (the original index travels as int32 bits in column 3)
        assert torch.equal(rec.view(torch.int32), ref["rec"].view(torch.int32))
        assert int(off[-1].item()) == b.n_hits
    ctx.close()


def test_static_binning_takes_no_device_memory():
    """After a first call (which may load the library's binning code onto the
    GPU), a call with preallocated outputs leaves the device's free memory
    unchanged: it allocates nothing."""
    from paper_1811_04141_gb300.api import mkf_hits_bin_static
    b = make_batch("find20", [46, 47], n_tracks=400)
    ctx = make_ctx(b)
    d = upload(b)
    n_bins = len(b.event_offsets[1:]) * sum(l["n_phi"] * l["n_zr"] for l in b.layers)
    n = d["xyz"].shape[1]
    rec = torch.empty((n, 4), device="cuda")
    inv = torch.empty((n,), dtype=torch.int32, device="cuda")
    off = torch.empty((n_bins + 1,), dtype=torch.int32, device="cuda")
    mkf_hits_bin_static(ctx.handle, d["xyz"], d["layer"], d["event_offsets"], rec, inv, off)
    ctx.sync()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    mkf_hits_bin_static(ctx.handle, d["xyz"], d["layer"], d["event_offsets"], rec, inv, off)
    ctx.sync()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(off[-1].item()) == b.n_hits
    ctx.close()


def test_static_binning_rejects_misaligned_or_short_buffers():
    """rec is written as 16-byte records: a buffer that does not start on a
    16-byte boundary is refused with MKF_ERR_ARG before anything runs; the
    binding refuses an offsets buffer of the wrong length."""
    from paper_1811_04141_gb300 import _native as N
    from paper_1811_04141_gb300.api import mkf_hits_bin_static
    b = make_batch("find20", [48], n_tracks=50)
    ctx = make_ctx(b)
    d = upload(b)
    n = d["xyz"].shape[1]
    n_bins = len(b.event_offsets[1:]) * sum(l["n_phi"] * l["n_zr"] for l in b.layers)
    flat = torch.zeros(n * 4 + 1, device="cuda")
    rec = flat[1:].view(n, 4)  # 4 bytes past a 16-byte boundary
    assert rec.data_ptr() % 16 == 4
    inv = torch.empty((n,), dtype=torch.int32, device="cuda")
    off = torch.empty((n_bins + 1,), dtype=torch.int32, device="cuda")
    with pytest.raises(N.MkfError) as e:
        mkf_hits_bin_static(ctx.handle, d["xyz"], d["layer"], d["event_offsets"], rec, inv, off)
    assert e.value.status == N.MKF_ERR_ARG
    assert torch.count_nonzero(flat) == 0
    with pytest.raises(ValueError):
        mkf_hits_bin_static(ctx, d["xyz"], d["layer"], d["event_offsets"], torch.empty((n, 4), device="cuda"), inv,
                            off[:-1])
    ctx.close()


def test_static_binning_rejects_oversized_input():
    from paper_1811_04141_gb300 import _native as N
    from paper_1811_04141_gb300.api import mkf_hits_bin_static
    b = make_batch("find20", [45], n_tracks=10)
    ctx = make_ctx(b)
    d = upload(b)
    # more events than the fixed working array has bins for
    n_ev = N.STATIC_MAX_BINS // sum(l["n_phi"] * l["n_zr"] for l in b.layers) + 1
    evo = torch.zeros(n_ev + 1, dtype=torch.int32, device="cuda")
    evo[1:] = d["xyz"].shape[1]
    n = d["xyz"].shape[1]
    with pytest.raises(N.MkfError) as e:
        mkf_hits_bin_static(ctx.handle, d["xyz"], d["layer"], evo, torch.empty(n, 4, device="cuda"),
                            torch.empty(n, dtype=torch.int32, device="cuda"),
                            torch.empty(8, dtype=torch.int32, device="cuda"))
    assert e.value.status == N.MKF_ERR_CAPACITY
    ctx.close()
