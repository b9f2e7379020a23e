"""A training step's pieces on the GPU (needs a GPU): the L1 loss kernel
against its plain definition, the accumulating backward against the sum of
single-view backwards, the launch timer, and the 4-view L1 step through the
C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("count,offset", [(1352 * 1014 * 3, 0), (1001, 0), (4099, 1)])
def test_l1_loss_matches_its_definition(count, offset):
    """Gradient bit for bit (scale times the sign of an exact float difference); loss within the
    FP32 accumulation of `count` terms.  Odd counts and an offset start (no 16-byte alignment)
    take the scalar path."""
    m = gu.d4()
    rng = np.random.default_rng(count)
    a = rng.uniform(0, 1, count + offset).astype(np.float32)
    b = rng.uniform(0, 1, count + offset).astype(np.float32)
    b[::97] = a[::97]   # exact ties: sign 0
    img = torch.from_numpy(a).cuda()[offset:]
    tgt = torch.from_numpy(b).cuda()[offset:]
    grad = torch.full((count,), 7.0, device="cuda")
    loss = torch.full((1,), 0.25, device="cuda")
    scale = 1.0 / count
    m.d4dgs_l1_loss(img, tgt, scale, grad, loss)
    torch.cuda.synchronize()
    ref_loss, ref_grad = oracle.l1_loss(a[offset:], b[offset:], np.float32(scale))
    assert np.array_equal(grad.cpu().numpy(), ref_grad.astype(np.float32))
    assert abs(float(loss.item()) - (0.25 + ref_loss)) <= 2e-6 * (0.25 + ref_loss)


def test_backward_accumulate_adds_views():
    """d4dgs_render_backward_accumulate of a second view adds exactly that view's gradients."""
    m = gu.d4()
    sc = synth.make_scene(6000, 61, "box20", sh_degree=3)
    ds = m.DeviceScene.from_host(sc)
    views = [synth.orbit(3, 200, 150, 300)[k] for k in (30, 200)]
    G = [torch.randn((150, 200, 3), generator=torch.Generator().manual_seed(k)).cuda() for k in range(2)]
    single = []
    for (cam, t), g in zip(views, G):
        r = m.Renderer(sc.n, cam, tile=32, batch=256)
        r.render(ds, cam, t)
        out = ds.zeros_like_grad()
        m.d4dgs_render_backward(ds, cam, t, r.cfg, r.ws, g, out)
        single.append({k: v.double() for k, v in out.items()})
    acc = ds.zeros_like_grad()
    for k in acc:
        acc[k].fill_(123.0)   # overwritten by the first call
    for j, ((cam, t), g) in enumerate(zip(views, G)):
        r = m.Renderer(sc.n, cam, tile=32, batch=256)
        r.render(ds, cam, t)
        fn = m.d4dgs_render_backward if j == 0 else m.d4dgs_render_backward_accumulate
        fn(ds, cam, t, r.cfg, r.ws, g, acc)
    torch.cuda.synchronize()
    for k in acc:
        want = single[0][k] + single[1][k]
        scale = float(want.abs().max())
        assert scale > 0
        # float atomics: the accumulation order differs between runs
        assert torch.allclose(acc[k].double(), want, rtol=1e-4, atol=1e-6 * scale), k


def test_launch_timer_times_every_launch_of_a_frame():
    m = gu.d4()
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    ds = m.DeviceScene.from_host(w.scene)
    r = m.Renderer(w.scene.n, cam)
    out = torch.empty((cam.height, cam.width, 3), device="cuda")
    r.render(ds, cam, t, out)
    with m.LaunchTimer() as lt:
        m.d4dgs_render(ds, cam, t, r.cfg, r.ws, out)
    torch.cuda.synchronize()
    ms = lt.times_ms()
    assert len(ms) == m.d4dgs_launches_per_frame(w.scene.n, cam, r.cfg)
    assert all(x >= 0 for x in ms) and sum(ms) > 0
    # nothing is recorded once the timer is stopped
    with m.LaunchTimer() as lt2:
        pass
    assert lt2.count == 0


def test_l1_training_step_over_four_views():
    """The step of the differentiable training workload on a small scene: 4 views, L1 against a
    seeded target scene's renders, backward accumulated over the views; the gradient equals the
    oracle adjoint of the mean L1 loss (dL/dI from the loss kernel), per element within 1e-3
    relative / 1e-5 absolute plus the oracle's gradient slack."""
    from paper_2503_22159_gb300.autograd import l1_step
    m = gu.d4()
    sc = synth.make_scene(3000, 71, "box20", sh_degree=1)
    target_sc = synth.make_scene(3000, 72, "box20", sh_degree=1)
    views = [(synth.orbit(4, 96, 72, 300)[k][0], float(np.float32(t))) for k, t in
             ((10, 0.2), (90, 0.45), (170, 0.6), (250, 0.9))]
    ds, tds = m.DeviceScene.from_host(sc), m.DeviceScene.from_host(target_sc)
    targets = [m.Renderer(target_sc.n, c).render(tds, c, t).clone() for c, t in views]
    renderers = [m.Renderer(sc.n, c) for c, _ in views]
    grads = ds.zeros_like_grad()
    loss = l1_step(ds, views, targets, renderers, grads)
    torch.cuda.synchronize()
    imgs = [oracle.render(sc, c, t)["rgb"] for c, t in views]
    scale = 1.0 / (len(views) * 96 * 72 * 3)
    ref_loss = sum(oracle.l1_loss(img, tg.cpu().numpy(), scale)[0] for img, tg in zip(imgs, targets))
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    want = {k: 0.0 for k in grads}
    slack = {k: 0.0 for k in grads}
    for (c, t), tg, r in zip(views, targets, renderers):
        # dL/dI from the GPU image (the step's decisions), the adjoint from the oracle
        img = r.render(ds, c, t).cpu().numpy()
        _, G = oracle.l1_loss(img, tg.cpu().numpy(), scale)
        g, s = oracle.backward(sc, c, t, G, with_slack=True)
        for k in grads:
            want[k] = want[k] + g[k]
            slack[k] = slack[k] + s[k]
    for k, v in grads.items():
        got, o = v.cpu().numpy().astype(np.float64), want[k]
        err = np.abs(got - o)
        assert np.all(err <= 1e-3 * np.abs(o) + 1e-5 + slack[k]), (k, float(err.max()))
