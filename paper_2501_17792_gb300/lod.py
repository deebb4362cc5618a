"""Ranked level of detail: choose each distance band's Gaussians by a
learned score instead of keeping a fixed prefix.

CrowdSplat (Sec. 2, Fig. 3) renders each distance band with its own,
separately fitted template of fewer Gaussians.  Without the videos to fit
those templates, this module ranks the Gaussians of the full template per
band and keeps the top ones:

1. render views of each band at full detail and record, per template
   Gaussian, the sum of its compositing weights alpha * T
   (``Renderer.render_contrib``);
2. train the 48-64-64-1 MLP (``binding.Mlp``) to predict the log of that
   contribution relative to its template's mean (``Renderer.lod_targets``)
   from 32 per-Gaussian features (``Renderer.lod_features``) and the band;
3. score every Gaussian for every band, rank per template
   (``Renderer.lod_rank``) and give each level its top round(f_l N)
   Gaussians (``Renderer.set_lod_subset``).

All arithmetic of these steps runs in the library's kernels; this module
moves tensors and slices index lists.  The ranking depends on neither pose
nor view, so it runs once; frames pay nothing extra.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import scene as S


@dataclasses.dataclass
class Bands:
    """Distance ranges (m) of the LoD levels used to collect training views."""
    lo: tuple = (2.5, 10.0, 30.0)
    hi: tuple = (10.0, 30.0, 110.0)


def collect_contributions(renderer, n_templates: int, camera, *, bands: Bands = Bands(),
                          views_per_band: int = 34, instances_per_view: int = 100, seed: int = 0):
    """Per band, the summed contribution of every template Gaussian over
    `views_per_band` full-detail renders of `instances_per_view` random
    instances placed in that band's distance range.  Returns a CUDA float32
    tensor [n_bands, n_total].  Leaves the renderer at single-level LoD."""
    import torch
    renderer.set_lod(S.single_lod())
    for t in range(n_templates):
        renderer.set_lod_subset(t, 0, np.zeros(0, np.uint32))
    n_total = renderer.n_gauss_total
    out = torch.zeros((len(bands.lo), n_total), dtype=torch.float32, device=f"cuda:{renderer.device}")
    img = None
    for b, (lo, hi) in enumerate(zip(bands.lo, bands.hi)):
        for v in range(views_per_band):
            inst = S.band_instances(n_templates, instances_per_view, lo, hi, seed + 7919 * b + 104729 * v)
            renderer.set_instances(inst.template_id, inst.root, inst.pose)
            img = renderer.render_contrib(camera, out[b], out=img)
    torch.cuda.synchronize(renderer.device)
    return out


def train_ranker(mlp, feat, targets, *, steps: int = 1500, lr: float = 2e-3, log_every: int = 0):
    """Full-batch Adam on every (band, Gaussian) row; the learning rate
    halves at 50% and 75% of the steps.  feat [n_total, 32] and targets
    [n_bands, n_total] CUDA tensors.  Returns the loss history (every
    `log_every` steps, plus first and last)."""
    import torch
    nb, n = targets.shape
    f = feat.repeat(nb, 1).contiguous()
    band = torch.arange(nb, dtype=torch.int32, device=feat.device).repeat_interleave(n).contiguous()
    tg = targets.reshape(-1).contiguous()
    hist = []
    for s in range(steps):
        rate = lr * (0.5 if s >= steps // 2 else 1.0) * (0.5 if s >= 3 * steps // 4 else 1.0)
        want = s == 0 or s == steps - 1 or (log_every and s % log_every == 0)
        L = mlp.train_step(f, band, tg, rate, want_loss=bool(want))
        if want:
            hist.append((s, L))
    return hist


def band_scores(mlp, feat, n_bands: int):
    """[n_bands, n_total] MLP scores of every Gaussian for every band."""
    import torch
    n = feat.shape[0]
    out = torch.empty((n_bands, n), dtype=torch.float32, device=feat.device)
    for b in range(n_bands):
        band = torch.full((n,), b, dtype=torch.int32, device=feat.device)
        mlp.forward(feat, band, out=out[b])
    return out


def ranked_subsets(renderer, scores, fractions, template_sizes, levels=None):
    """{(template, level): top round(f_l N) Gaussians by that level's score}
    (round half up, at least one Gaussian).  scores: [n_levels, n_total]."""
    subs = {}
    levels = range(len(fractions)) if levels is None else levels
    for l in levels:
        order = renderer.lod_rank(scores[l]).cpu().numpy().view(np.uint32)
        off = 0
        for t, n in enumerate(template_sizes):
            k = min(n, max(1, int(math.floor(float(np.float32(fractions[l])) * n + 0.5))))
            subs[(t, l)] = order[off:off + k].copy()
            off += n
    return subs


def apply_subsets(renderer, subsets):
    for (t, l), idx in subsets.items():
        renderer.set_lod_subset(t, l, idx)


def clear_subsets(renderer, n_templates: int, n_levels: int = 4):
    for t in range(n_templates):
        for l in range(n_levels):
            renderer.set_lod_subset(t, l, np.zeros(0, np.uint32))


def psnr(a, b) -> float:
    """PSNR (dB, peak 1) between two RGB(A) images (CUDA tensors or arrays);
    RGB channels only."""
    import torch
    if isinstance(a, torch.Tensor):
        d = (a[..., :3].double() - b[..., :3].double()).pow(2).mean().item()
    else:
        d = float(np.mean((np.asarray(a, np.float64)[..., :3] - np.asarray(b, np.float64)[..., :3]) ** 2))
    return float(10 * math.log10(1.0 / max(d, 1e-30)))


def prefix_orders(scores, fractions, template_sizes):
    """Per template, a storage order whose prefixes are ranked levels: the
    top round(f_L N) Gaussians of the coarsest band's score first, then the
    next best of each finer band's score among those not yet placed, up to
    that level's size, then the rest by the finest band's score.  Levels are
    nested by construction (each coarser level is a prefix of the finer
    ones), so a template re-uploaded in this order renders its levels as
    plain prefixes, with no per-level index list to gather through.
    scores: [n_levels, n_total] (CUDA tensor or array); fractions: one per
    level, finest first.  Returns a list of int64 permutations (storage
    position -> original index)."""
    sc = scores.cpu().numpy() if hasattr(scores, "cpu") else np.asarray(scores)
    out, off = [], 0
    L = len(fractions)
    for n in template_sizes:
        s = sc[:, off:off + n].astype(np.float64)
        placed = np.zeros(n, bool)
        order = []
        for l in range(L - 1, -1, -1):
            k = n if l == 0 else min(n, max(1, int(math.floor(float(np.float32(fractions[l])) * n + 0.5))))
            need = k - len(order)
            if need <= 0:
                continue
            cand = np.nonzero(~placed)[0]
            # highest score first; ties by index (stable)
            pick = cand[np.argsort(-s[min(l, s.shape[0] - 1), cand], kind="stable")[:need]]
            order.extend(pick.tolist())
            placed[pick] = True
        out.append(np.asarray(order, np.int64))
        off += n
    return out


def permute_template(tpl, perm):
    """The template with its Gaussians stored in the order `perm`."""
    return dataclasses.replace(tpl, means=tpl.means[perm], scales=tpl.scales[perm], quats=tpl.quats[perm],
                               opacity=tpl.opacity[perm], sh=tpl.sh[perm], skin_idx=tpl.skin_idx[perm],
                               skin_w=tpl.skin_w[perm])
