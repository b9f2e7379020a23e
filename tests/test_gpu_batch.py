"""Batched multi-view rendering and serving (needs a GPU): every view of a
mixed batch -- different scenes, cameras, timestamps and resolutions in one
launch per kernel -- equals the same view rendered alone, with and without
CUDA-graph replay, and the serving loops return every request intact."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def host_scenes_small():
    return {"A": synth.make_scene(6000, 51, "box20", sh_degree=3), "B": synth.make_scene(9000, 52, "box20", sh_degree=1)}


def scenes_small():
    m = gu.d4()
    return {k: m.DeviceScene.from_host(v) for k, v in host_scenes_small().items()}


def solo(scene, cam, t, cfg):
    m = gu.d4()
    r = m.Renderer(scene.n, cam, tile=cfg.tile, batch=cfg.batch)
    return r.render(scene, cam, t).clone()


def mixed_views(scenes, seed=0, k=6):
    rng = np.random.default_rng(seed)
    res = [(160, 120), (333, 257), (256, 256), (96, 200)]
    out = []
    for i in range(k):
        name = "AB"[i % 2]
        cam, _ = synth.orbit(int(rng.integers(0, 1000)), *res[i % len(res)], 300)[int(rng.integers(0, 300))]
        out.append((name, cam, float(np.float32(rng.uniform(0, 1)))))
    return out


@pytest.mark.parametrize("graph,tile,trim", [(False, 16, False), (True, 16, False), (True, 32, True)])
def test_mixed_batch_equals_each_view_alone(graph, tile, trim):
    m = gu.d4()
    scenes = scenes_small()
    cfg = m.config_struct(tile, 256, trim=trim)
    br = m.BatchRenderer(cfg)
    for seed in (0, 1):   # two different batches through the same (graph) path
        vs = mixed_views(scenes, seed)
        views, outs = [], []
        for name, cam, t in vs:
            sc = scenes[name]
            ws = torch.empty(m.d4dgs_workspace_bytes(sc.n, cam, cfg, 40 * sc.n), dtype=torch.uint8, device="cuda")
            out = torch.full((cam.height, cam.width, 3), -1.0, device="cuda")
            views.append((sc, cam, t, ws, out))
            outs.append(out)
        br.render(views, graph=graph)
        torch.cuda.synchronize()
        for (name, cam, t), (sc, _, _, ws, out) in zip(vs, views):
            assert m.d4dgs_read_stats(sc.n, cam, cfg, ws)["status"] == 0
            assert torch.equal(out, solo(sc, cam, t, cfg)), (name, cam.width, cam.height)


@pytest.mark.parametrize("graph", [False, True])
def test_time_groups_equal_each_time_alone(graph):
    """Consecutive views of one scene and camera at different times form time groups (up to 4 views,
    preprocessed together, each Gaussian read once; Algorithm 1's camera-change caching and the
    parallel multi-frame rendering of Sec. IV-C); a view of another camera splits them.  Every
    view's image and tile lists equal, bit for bit, those of the view rendered alone, and every
    view's image matches the oracle's render of that time."""
    m = gu.d4()
    hosts = host_scenes_small()
    scenes = {k: m.DeviceScene.from_host(v) for k, v in hosts.items()}
    cfg = m.config_struct(16, 256)
    cam_a, _ = synth.orbit(7, 320, 240, 300)[40]
    cam_b, _ = synth.orbit(8, 200, 160, 300)[200]
    spec = [("A", cam_a, 0.05), ("A", cam_a, 0.3), ("A", cam_a, 0.55), ("A", cam_a, 0.8), ("A", cam_a, 0.95),
            ("B", cam_b, 0.5), ("A", cam_a, 0.42), ("A", cam_a, 0.43)]
    views = []
    for name, cam, t in spec:
        sc = scenes[name]
        ws = torch.empty(m.d4dgs_workspace_bytes(sc.n, cam, cfg, 40 * sc.n), dtype=torch.uint8, device="cuda")
        views.append((sc, cam, float(np.float32(t)), ws, torch.full((cam.height, cam.width, 3), -1.0, device="cuda")))
    m.BatchRenderer(cfg).render(views, graph=graph)
    torch.cuda.synchronize()
    for (name, cam, t), (sc, _, tt, ws, out) in zip(spec, views):
        assert m.d4dgs_read_stats(sc.n, cam, cfg, ws)["status"] == 0
        r = m.Renderer(sc.n, cam, tile=cfg.tile, batch=cfg.batch, key_capacity=40 * sc.n)
        alone = r.render(sc, cam, tt).clone()
        assert torch.equal(out, alone), (name, t)
        L = m.d4dgs_workspace_layout(sc.n, cam, cfg, ws.numel())
        k = m.d4dgs_read_stats(sc.n, cam, cfg, ws)["n_keys"]
        La = r.layout(cam)
        got = ws[L["tile_keys"]: L["tile_keys"] + 4 * k]
        ref = r.ws[La["tile_keys"]: La["tile_keys"] + 4 * k]
        assert k == r.stats(cam)["n_keys"] and torch.equal(got, ref), (name, t)
        if not graph:
            gu.compare_image(out.cpu().numpy(), oracle.render(hosts[name], cam, tt), f"group view {name} t={tt}")


def test_batch_rejects_mixed_layout_classes():
    m = gu.d4()
    cfg = m.config_struct(16, 256)
    big = m.DeviceScene.from_host(synth.make_scene(70_000, 3, "tiny"))
    small = m.DeviceScene.from_host(synth.make_scene(100, 3, "tiny"))
    cam_big = synth.pinhole(256, 8192)   # 512 tile rows: two row passes, against one for the small view
    cam_small = synth.pinhole(64, 64)
    views = []
    for sc, cam in ((big, cam_big), (small, cam_small)):
        ws = torch.empty(m.d4dgs_workspace_bytes(sc.n, cam, cfg, 1000), dtype=torch.uint8, device="cuda")
        views.append((sc, cam, 0.5, ws, torch.empty((cam.height, cam.width, 3), device="cuda")))
    with pytest.raises(m.D4DGSError):
        m.BatchRenderer(cfg).render(views)


@pytest.mark.parametrize("mode,trim", [("batched", False), ("loop", False), ("batched", True)])
def test_serving_returns_every_request_as_rendered_alone(mode, trim):
    from paper_2503_22159_gb300 import serving
    m = gu.d4()
    scenes = scenes_small()
    cfg = m.config_struct(32 if trim else 16, 256, trim=trim)
    reqs = serving.make_trace(scenes, n_requests=48, rate_hz=2000.0, seed=9,
                              resolutions=((160, 120), (320, 240), (256, 192)))
    caps = serving.calibrate_capacity(scenes, reqs, cfg, "cuda")
    got = {}

    def keep(r, out):
        # the slot is reused as soon as this returns: finish reading first
        got[r.rid] = out.clone()
        torch.cuda.current_stream().synchronize()

    if mode == "batched":
        st = serving.serve_batched(scenes, reqs, cfg, caps, max_views=8, budget_bytes=2 << 30, on_done=keep)
        assert st.batches < len(reqs) and st.mean_batch > 1.0
    else:
        st = serving.serve_loop(scenes, reqs, cfg, caps, on_done=keep)
    torch.cuda.synchronize()
    assert st.n == len(reqs) and np.isfinite(st.p99_ms)
    assert all(r.status == 0 for r in reqs)
    for r in reqs[:16]:
        assert torch.equal(got[r.rid], solo(scenes[r.scene], r.cam, r.t, cfg)), r.rid


def test_serving_isolates_a_poisoned_and_a_cancelled_request():
    """Faults injected on the host stay with their request.  In a trace replayed by continuous
    batching, one request carries a camera with a NaN principal point and another is cancelled
    while its batch is on the GPU: the first is refused on arrival (D4DGS_ERR_INVALID_ARG, no
    image), the second's image is discarded (cancelled), and every other request -- the views
    batched around them included -- returns its image bit for bit as rendered alone.  The
    per-frame loop refuses the same poisoned request and serves the rest likewise."""
    from paper_2503_22159_gb300 import serving
    m = gu.d4()
    scenes = scenes_small()
    cfg = m.config_struct(16, 256)
    for mode in ("batched", "loop"):
        reqs = serving.make_trace(scenes, n_requests=32, rate_hz=4000.0, seed=11,
                                  resolutions=((160, 120), (256, 192)))
        caps = serving.calibrate_capacity(scenes, reqs, cfg, "cuda")
        bad = reqs[5]
        bad.cam = synth.Camera(R=bad.cam.R, T=bad.cam.T, fx=bad.cam.fx, fy=bad.cam.fy, cx=float("nan"),
                               cy=bad.cam.cy, width=bad.cam.width, height=bad.cam.height)
        got, none = {}, set()
        victim = []

        def keep(r, out):
            if out is None:
                none.add(r.rid)
                return
            got[r.rid] = out.clone()
            torch.cuda.current_stream().synchronize()

        def cancel_one(batch):
            # the first multi-view batch: cancel its second request while the batch runs
            if not victim and len(batch) > 1:
                victim.append(batch[1])
                batch[1].cancelled = True

        if mode == "batched":
            st = serving.serve_batched(scenes, reqs, cfg, caps, max_views=8, budget_bytes=2 << 30, on_done=keep,
                                       on_launch=cancel_one, realtime=False)
            assert victim and victim[0].status == serving.STATUS_CANCELLED and victim[0].rid in none
            assert st.extra["cancelled"] == 1 and st.mean_batch > 1.0
        else:
            st = serving.serve_loop(scenes, reqs, cfg, caps, on_done=keep, realtime=False)
        torch.cuda.synchronize()
        assert bad.status == m.D4DGS_ERR_INVALID_ARG and bad.rid in none and st.extra["refused"] == 1
        served = [r for r in reqs if r is not bad and r not in victim]
        assert all(r.status == 0 for r in served) and set(got) == {r.rid for r in served}
        for r in served:
            assert torch.equal(got[r.rid], solo(scenes[r.scene], r.cam, r.t, cfg)), (mode, r.rid)


def test_colour_cache_time_group():
    """config colour_cache (Algorithm 1's per-camera caching carried to the colour): SH evaluated
    towards the static mean, once per time group.  Each grouped view matches the oracle's render with
    the same colour rule within the image tolerance and equals the same view rendered alone bit for
    bit; against the definition (colour towards the time-shifted mean) it stays within the stated
    approximation bound, max-abs 0.05 and mean-abs 0.005 (on the 300k benchmark frames the oracle
    measures at most 0.023 and 0.0019)."""
    m = gu.d4()
    hosts = host_scenes_small()
    sc = hosts["A"]
    ds = m.DeviceScene.from_host(sc)
    cfg = m.config_struct(16, 256, colour_cache=True)
    cam, _ = synth.orbit(7, 320, 240, 300)[40]
    times = [float(np.float32(t)) for t in (0.05, 0.3, 0.55, 0.8)]
    views = []
    for t in times:
        ws = torch.empty(m.d4dgs_workspace_bytes(sc.n, cam, cfg, 40 * sc.n), dtype=torch.uint8, device="cuda")
        views.append((ds, cam, t, ws, torch.full((cam.height, cam.width, 3), -1.0, device="cuda")))
    m.BatchRenderer(cfg).render(views)
    torch.cuda.synchronize()
    for (_, _, t, ws, out) in views:
        assert m.d4dgs_read_stats(sc.n, cam, cfg, ws)["status"] == 0
        img = out.cpu().numpy()
        gu.compare_image(img, oracle.render(sc, cam, t, colour_static=True), f"colour cache t={t}")
        exact = oracle.render(sc, cam, t)["rgb"]
        assert np.abs(img - exact).max() <= 0.05 and np.abs(img - exact).mean() <= 0.005
        r = m.Renderer(sc.n, cam, tile=16, batch=256, key_capacity=40 * sc.n)
        r.cfg = cfg
        assert torch.equal(r.render(ds, cam, t), out)
