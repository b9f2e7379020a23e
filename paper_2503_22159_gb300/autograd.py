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

from . import (SCENE_FIELDS, DeviceScene, Renderer, d4dgs_l1_loss, d4dgs_render_backward,
               d4dgs_render_backward_accumulate)


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


def l1_step(scene: DeviceScene, views, targets, renderers, grads: dict, stream=None) -> float:
    """One step of the differentiable training workload through the C ABI, without autograd:
    for each view (camera, t) render, the L1 loss against its target and dL/dI (the loss kernel,
    scale 1 / (values per image x views): the mean over the step), then the backward, added into
    `grads` (zeroed here first).  Returns the loss (read back once, after the last view)."""
    for k in grads:
        grads[k].zero_()
    loss = torch.zeros(1, dtype=torch.float32, device=next(iter(grads.values())).device)
    scale = 1.0 / sum(int(t.numel()) for t in targets)
    for (cam, t), target, r in zip(views, targets, renderers):
        img = r.render(scene, cam, t, stream=stream)
        dl = torch.empty_like(img)
        d4dgs_l1_loss(img, target, scale, dl, loss, stream)
        d4dgs_render_backward_accumulate(scene, cam, t, r.cfg, r.ws, dl, grads, stream)
    return float(loss.item())


class _L1Fn(torch.autograd.Function):
    """Mean L1 of an image against a target through the loss kernel (dL/dI computed in the
    forward, scaled by the incoming gradient in the backward)."""

    @staticmethod
    def forward(ctx, img, target, scale):
        loss = torch.zeros(1, dtype=torch.float32, device=img.device)
        dl = torch.empty_like(img)
        d4dgs_l1_loss(img.contiguous(), target.contiguous(), float(scale), dl, loss)
        ctx.save_for_backward(dl)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (dl,) = ctx.saved_tensors
        return dl * g, None, None


def l1_training_step(params: dict, views, targets, renderers, sh_degree: int, optimizer=None) -> float:
    """One differentiable step over a batch of views: mean L1 between each
    render and its target image (the loss kernel), backward through every view,
    optional optimizer step.  ``views`` is a list of (camera, t); one Renderer
    per view (each view's workspace must survive until its backward)."""
    scale = 1.0 / sum(int(t.numel()) for t in targets)
    loss = 0.0
    for (cam, t), target, r in zip(views, targets, renderers):
        img = render(params, cam, t, r, sh_degree)
        loss = loss + _L1Fn.apply(img, target, scale)
    if optimizer is not None:
        optimizer.zero_grad(set_to_none=True)
    loss.backward()
    if optimizer is not None:
        optimizer.step()
    return float(loss.detach())
