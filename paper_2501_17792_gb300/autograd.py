"""torch.autograd wrapper of the differentiable render (cs_render_train +
cs_backward): image = render(template attributes, joint poses).

The template attributes go to the library through ``upload_templates`` (a
host copy, as every upload), the poses through ``set_instances`` on the
device; all arithmetic of the forward and the backward runs in the
library's kernels.  One template set and one camera per call; the instances'
template ids and roots are fixed inputs (no gradient).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import scene as S


class CrowdRender(torch.autograd.Function):
    """forward(renderer, camera, template_id, root, template, means, scales,
    quats, opacity, sh, pose) -> RGBA image [H, W, 4].

    ``template`` supplies the non-differentiable attributes (skinning,
    rest joints, parents, SH degree); means [N,3], scales [N,3], quats
    [N,4], opacity [N], sh [N,K,3] and pose [I,24,3] are tensors (any device)
    whose gradients are returned."""

    @staticmethod
    def forward(ctx, renderer, camera, template_id, root, template, means, scales, quats, opacity, sh, pose):
        t = dataclasses.replace(
            template,
            means=means.detach().float().cpu().numpy(), scales=scales.detach().float().cpu().numpy(),
            quats=quats.detach().float().cpu().numpy(), opacity=opacity.detach().float().cpu().numpy(),
            sh=sh.detach().float().cpu().numpy())
        renderer.upload_templates([t])
        dev = f"cuda:{renderer.device}"
        p = pose.detach().to(device=dev, dtype=torch.float32).contiguous()
        renderer.set_instances(torch.as_tensor(template_id, dtype=torch.int32, device=dev),
                               torch.as_tensor(np.asarray(root, np.float32).reshape(-1, 12), device=dev), p)
        img = renderer.render_train(camera)
        ctx.renderer = renderer
        ctx.n_inst = int(p.shape[0])
        ctx.K = int(sh.shape[1])
        ctx.devices = [x.device for x in (means, scales, quats, opacity, sh, pose)]
        return img

    @staticmethod
    def backward(ctx, grad_img):
        g = ctx.renderer.backward(grad_img.contiguous(), ctx.n_inst)
        outs = (g["means"], g["scales"], g["quats"], g["opacity"], g["sh"][:, :ctx.K, :], g["pose"])
        outs = tuple(o.to(d) for o, d in zip(outs, ctx.devices))
        return (None, None, None, None, None) + outs


def render(renderer, camera, instances: S.Instances, template: S.Template, means, scales, quats, opacity, sh,
           pose):
    """Differentiable render of one template's instances; see CrowdRender."""
    return CrowdRender.apply(renderer, camera, instances.template_id, instances.root, template, means, scales,
                             quats, opacity, sh, pose)
