"""torch.autograd binding of d4dgs_render / d4dgs_render_backward.

``render(params, cam, t, renderer)`` returns the H x W x 3 image and, on
``backward()``, fills ``.grad`` of the raw parameter tensors through the
library's backward kernels (per-tile back-to-front replay + preprocess
adjoint).  The forward keeps its workspace (records, sorted lists, final
transmittance, last contributors) for the backward, so the Renderer passed in
must not render another frame in between.
"""
from __future__ import annotations

import torch

from . import SCENE_FIELDS, DeviceScene, Renderer, d4dgs_render_backward


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cam, t, renderer: Renderer, sh_degree: int, *tensors):
        scene = DeviceScene(dict(zip(SCENE_FIELDS, [x.detach() for x in tensors])), sh_degree)
        img = renderer.render(scene, cam, t)
        ctx.cam, ctx.t, ctx.renderer, ctx.scene = cam, t, renderer, scene
        ctx.ws_id = renderer.ws.data_ptr()
        return img.clone()

    @staticmethod
    def backward(ctx, grad_img):
        r = ctx.renderer
        if r.ws.data_ptr() != ctx.ws_id:
            raise RuntimeError("the renderer's workspace changed between forward and backward")
        grads = ctx.scene.zeros_like_grad()
        d4dgs_render_backward(ctx.scene, ctx.cam, ctx.t, r.cfg, r.ws, grad_img.contiguous(), grads)
        return (None, None, None, None) + tuple(grads[k] for k in SCENE_FIELDS)


def render(params: dict, cam, t: float, renderer: Renderer, sh_degree: int) -> torch.Tensor:
    """Differentiable render of one view; ``params`` maps SCENE_FIELDS to
    contiguous float32 CUDA tensors (leaf tensors with requires_grad)."""
    return _RenderFn.apply(cam, float(t), renderer, int(sh_degree), *[params[k] for k in SCENE_FIELDS])


def l1_training_step(params: dict, views, targets, renderers, sh_degree: int, optimizer=None) -> float:
    """One differentiable step over a batch of views: mean L1 between each
    render and its target image, backward through every view, optional
    optimizer step.  ``views`` is a list of (camera, t); one Renderer per view
    (each view's workspace must survive until its backward)."""
    loss = 0.0
    for (cam, t), target, r in zip(views, targets, renderers):
        img = render(params, cam, t, r, sh_degree)
        loss = loss + (img - target).abs().mean()
    loss = loss / len(views)
    if optimizer is not None:
        optimizer.zero_grad(set_to_none=True)
    loss.backward()
    if optimizer is not None:
        optimizer.step()
    return float(loss.detach())
