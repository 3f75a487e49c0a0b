"""Training and use of the hit-ranking MLP with the library's kernels.

The paper has no learned component; this is the configuration's learned-pruning
pattern: features of (candidate, compatible hit) pairs come from the finder
itself (mkf_find's feature dump), labels from the generator's truth (the hit
belongs to the seed's particle), the network is trained by mkf_mlp_train_step
(forward, backward and Adam run in libmkf's CUDA kernels; torch only holds the
buffers and draws the batch permutation), and the pruning threshold is the
largest one that keeps the finding efficiency within a tolerance of the plain
finder.  The plain chi2 selection stays the reference: efficiency and fake rate
are computed from the found hit lists and the truth.

Two uses of the trained network: pruning inside the N-best finder (pairs
below the threshold dropped before the selection), and the cascade
(`cascade`): best-hit finding of every seed with the network as a gate on its
best-chi2 extensions, then N-best finding, with the plain chi2 selection, of
the seeds whose extensions it doubted.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _native as N
from .api import feature_buffer, mkf_mlp_to_bf16, mkf_mlp_train_step


def collect_features(ctx, bins, seed_hits, seed_event, cap: int, **find_kw):
    """Run the plain finder with the feature dump on; returns (feat [m, 12], ref [m, 2])."""
    fb = feature_buffer(cap, seed_hits.device)
    ctx.find(bins, seed_hits, seed_event, feat=fb, **find_kw)
    ctx.sync()
    m = min(int(fb["count"].item()), cap)
    return fb["feat"][:m], fb["ref"][:m]


def label_pairs(ref, hit_particle, seed_particle):
    """1 when the hit belongs to the seed's particle (truth), else 0 (float32)."""
    return (hit_particle[ref[:, 1].long()] == seed_particle[ref[:, 0].long()]).float()


def init_weights(seed: int = 0) -> np.ndarray:
    """He-normal first layer, small second layer, zero biases (float32)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((N.MLP_HIDDEN, N.MLP_IN)) * np.sqrt(2.0 / N.MLP_IN)
    w2 = rng.standard_normal(N.MLP_HIDDEN) * np.sqrt(1.0 / N.MLP_HIDDEN)
    return np.concatenate([W1.ravel(), np.zeros(N.MLP_HIDDEN), w2, [0.0]]).astype(np.float32)


def train(ctx, feat, label, steps: int = 2000, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          state: dict | None = None):
    """Adam on shuffled mini-batches.  Returns a state dict (w, m, v, w_bf16,
    step, losses) that can be passed back in to resume."""
    dev = feat.device
    if state is None:
        w = torch.as_tensor(init_weights(seed), device=dev)
        state = dict(w=w, m=torch.zeros_like(w), v=torch.zeros_like(w), w_bf16=mkf_mlp_to_bf16(ctx, w), step=0,
                     losses=[])
    g = torch.Generator(device="cpu").manual_seed(seed + state["step"])
    n = feat.shape[0]
    loss = torch.zeros(1, device=dev)
    perm = torch.randperm(n, generator=g).to(dev)
    pos = 0
    for _ in range(steps):
        if pos + batch > n:
            perm = torch.randperm(n, generator=g).to(dev)
            pos = 0
        idx = perm[pos:pos + min(batch, n)]
        pos += batch
        fb = feat.index_select(0, idx).contiguous()
        lb = label.index_select(0, idx).contiguous()
        state["step"] += 1
        mkf_mlp_train_step(ctx, fb, lb, state["w"], state["m"], state["v"], state["step"], state["w_bf16"], lr=lr,
                           loss=loss)
        if state["step"] % 100 == 0:
            state["losses"].append(float(loss.item()))
    return state


def efficiency(hits, hit_particle, seed_particle, share: float = 0.75):
    """(efficiency, fake rate): a track is matched when at least `share` of its
    hits belong to its seed's particle; a fake has less than half."""
    h = hits.long()
    valid = h >= 0
    owner = torch.where(valid, hit_particle[h.clamp(min=0)], torch.full_like(h, -2))
    same = (owner == seed_particle.long()[None, :]) & valid
    n = valid.sum(0).clamp(min=1)
    frac = same.sum(0).float() / n.float()
    return float((frac >= share).float().mean().item()), float((frac < 0.5).float().mean().item())


def choose_tau(run_find, eff_plain: float, taus, tolerance: float = 0.005):
    """Largest tau whose efficiency stays within `tolerance` of the plain finder.
    run_find(tau) -> (efficiency, fake rate)."""
    best = None
    for tau in sorted(taus):
        eff, fake = run_find(tau)
        if eff >= eff_plain - tolerance:
            best = (tau, eff, fake)
    return best


def cascade(ctx, bins, seed_hits, seed_event, w_bf16, tau, n_best=10, out=None, subset=None, **find_kw):
    """The learned cascade, all on the device: best-hit finding of every seed
    with the MLP gate (a seed is flagged when, on a layer where its candidate
    has two or more compatible hits, the best one by chi2 scores below tau),
    then N-best finding of the flagged seeds only, written over their best-hit
    results.  Returns (out, (seed_list, seed_count)); pass both back in (`out`,
    `subset`) to reuse the buffers (e.g. inside a CUDA graph capture)."""
    out = ctx.find(bins, seed_hits, seed_event, n_best=1, mlp_bf16=w_bf16, mlp_tau=tau, mlp_mode=1, out=out,
                   **find_kw)
    lst, cnt = ctx.seeds_where(out["status"], N.ST_AMBIG, *(subset or (None, None)))
    ctx.find(bins, seed_hits, seed_event, n_best=n_best, out=out, seed_list=lst, seed_count=cnt, **find_kw)
    return out, (lst, cnt)


def choose_gate_tau(run_cascade, eff_plain: float, fake_plain: float, taus, tolerance: float = 0.005):
    """Smallest gate threshold (fewest seeds sent to N-best finding) whose
    efficiency and fake rate stay within `tolerance` of the plain finder's.
    run_cascade(tau) -> (efficiency, fake rate)."""
    for tau in sorted(taus):
        eff, fake = run_cascade(tau)
        if eff >= eff_plain - tolerance and fake <= fake_plain + tolerance:
            return tau, eff, fake
    return None
