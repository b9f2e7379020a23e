"""Optical-flow channel and flow-gradient consistency loss on the GPU (needs a
GPU): the flow image against the oracle's, the loss and dL/dF against the
oracle's loss and its central differences, and the backward through the flow
channel against central differences of the oracle's loss with respect to the
raw parameters (the image-edge guide held fixed, as in the loss)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu
from tests.test_oracle_adjoint import FIELDS, fd_scene

pytestmark = pytest.mark.gpu


def gpu_flow(scene, cam, t, tile=16):
    m = gu.d4()
    ds = m.DeviceScene.from_host(scene)
    r = m.Renderer(scene.n, cam, tile=tile)
    r.render(ds, cam, t)   # sizes the workspace
    img = torch.empty((cam.height, cam.width, 3), device="cuda")
    fl = torch.empty((cam.height, cam.width, 2), device="cuda")
    m.d4dgs_render_flow(ds, cam, t, r.cfg, r.ws, img, fl)
    torch.cuda.synchronize()
    assert r.stats(cam)["status"] == 0
    return r, ds, img, fl


@pytest.mark.parametrize("tile", [16, 32])
def test_flow_image_matches_oracle(tile):
    sc = synth.make_scene(1500, 61, "tiny", sh_degree=0)
    cam, t = synth.pinhole(128, 128), 0.4
    r, ds, img, fl = gpu_flow(sc, cam, t, tile)
    ref = oracle.render_flow(sc, cam, t)
    f = fl.cpu().numpy().astype(np.float64)
    scale = float(np.abs(ref["flow"]).max())
    assert scale > 0.1
    err = np.abs(f - ref["flow"])
    assert (err <= 2e-3 * scale + ref["slack"][..., None]).all(), float(err.max())
    assert err.mean() <= 1e-4 * scale
    # the image of the flow render is the plain render's, bit for bit
    assert torch.equal(img, r.render(ds, cam, t))


def test_flow_loss_and_its_gradient_match_oracle():
    rng = np.random.default_rng(62)
    H, W = 40, 48
    rgb = rng.uniform(0.0, 0.5, (H, W, 3))
    rgb[:, 20:, :] += 0.5                       # a vertical edge
    flow = rng.normal(0.0, 2.0, (H, W, 2)) + np.linspace(0.0, 6.0, W)[None, :, None]
    m = gu.d4()
    trgb = torch.tensor(rgb, dtype=torch.float32, device="cuda")
    tflow = torch.tensor(flow, dtype=torch.float32, device="cuda")
    dl = torch.empty_like(tflow)
    L = float(m.d4dgs_flow_loss(trgb, tflow, lam=0.7, eps=1e-6, dl_dflow=dl).cpu())
    r64, f64 = trgb.cpu().numpy().astype(np.float64), tflow.cpu().numpy().astype(np.float64)
    wgt = oracle.image_edge_weight(r64)
    assert L == pytest.approx(oracle.flow_gradient_loss(f64, wgt, 0.7, 1e-6), rel=1e-5)
    g = dl.cpu().numpy().astype(np.float64).reshape(-1)
    flat = f64.reshape(-1).copy()
    gmax = np.abs(g).max()
    for j in rng.choice(flat.size, 400, replace=False):
        x0 = flat[j]
        h = 1e-5 * max(1.0, abs(x0))
        flat[j] = x0 + h
        lp = oracle.flow_gradient_loss(flat.reshape(H, W, 2), wgt, 0.7, 1e-6)
        flat[j] = x0 - h
        lm = oracle.flow_gradient_loss(flat.reshape(H, W, 2), wgt, 0.7, 1e-6)
        flat[j] = x0
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[j]) <= 2e-3 * abs(fd) + 1e-4 * gmax, (int(j), fd, g[j])


def test_flow_backward_matches_oracle_central_differences():
    sc, cam = fd_scene(deg=0)
    t, lam, eps = 0.5, 1.0, 1e-6
    sc32 = synth.Scene(**{k: np.asarray(v, np.float32).astype(np.float64) for k, v in sc.arrays().items()},
                       sh_degree=0)
    m = gu.d4()
    r, ds, img, fl = gpu_flow(sc32, cam, t)
    dlf = torch.empty_like(fl)
    m.d4dgs_flow_loss(img, fl, lam=lam, eps=eps, dl_dflow=dlf)
    grads = ds.zeros_like_grad()
    m.d4dgs_render_backward_flow(ds, cam, t, r.cfg, r.ws, torch.zeros_like(img), dlf, grads)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    wgt = oracle.image_edge_weight(img.cpu().numpy().astype(np.float64))
    loss = lambda s: oracle.flow_gradient_loss(oracle.render_flow(s, cam, t)["flow"], wgt, lam, eps)
    base_fp = oracle.fingerprint(sc32, cam, t)
    rng = np.random.default_rng(63)
    checked = 0
    for field in ("means", "velocity", "t_mean", "log_scales", "opacity_logit", "quats"):
        arr = getattr(sc32, field)
        flat = arr.reshape(-1)
        ref_scale = 0.0
        pairs = []
        for j in rng.choice(flat.size, min(flat.size, 60), replace=False):
            x0 = flat[j]
            h = 1e-6 * max(1.0, abs(x0))
            flat[j] = x0 + h
            ok = np.array_equal(oracle.fingerprint(sc32, cam, t), base_fp)
            lp = loss(sc32)
            flat[j] = x0 - h
            ok = ok and np.array_equal(oracle.fingerprint(sc32, cam, t), base_fp)
            lm = loss(sc32)
            flat[j] = x0
            if ok:
                fd = (lp - lm) / (2 * h)
                pairs.append((fd, got[field].reshape(-1)[j]))
                ref_scale = max(ref_scale, abs(fd))
        assert ref_scale > 0, field
        for fd, g in pairs:
            assert abs(fd - g) <= 2e-2 * abs(fd) + 2e-3 * ref_scale, (field, fd, g)
            checked += 1
    assert checked > 250
