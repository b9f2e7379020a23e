"""Parity of the CUDA forward path with the CPU oracle (needs a GPU).

Stage by stage: the preprocess records against the FP64 oracle, the tile/key
lists bit for bit against the FP32 binning mirror, and the image against the
FP64 per-pixel brute force; then edge cases and invariants."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def medium(n=20_000, w=333, h=257, seed=5, deg=1, frame=40):
    """A ragged medium case: image sizes that are not tile multiples, several
    sort partitions, SH degree 1 on the 20-unit box seen from the orbit."""
    scene = synth.make_scene(n, seed, "box20", sh_degree=deg)
    cam, t = synth.orbit(1, w, h, 300)[frame]
    return scene, cam, t


# ---------------------------------------------------------------------------
# stage parity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("trim", [False, True])
def test_preprocess_matches_oracle(trim):
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    m = gu.d4()
    ds = m.DeviceScene.from_host(w.scene)
    r = m.Renderer(w.scene.n, cam, trim=trim)
    m.d4dgs_preprocess(ds, cam, t, r.cfg, r.ws)
    torch.cuda.synchronize()
    rec = gu.gpu_records(r, w.scene.n, cam)
    L = r.layout(cam)
    keys = r.view("depth_keys", torch.int32, w.scene.n, cam).cpu().numpy().view(np.uint32)
    tt = r.view("tiles_touched", torch.int32, w.scene.n, cam).cpu().numpy()
    rect = r.view("rect", torch.int16, 4 * w.scene.n, cam).cpu().numpy().view(np.uint16).reshape(-1, 4)
    trims = r.view("trims", torch.int64, w.scene.n, cam).cpu().numpy().view(np.uint64)
    b = oracle.bin_f32(w.scene, cam, t, 16, trim=trim)
    g = oracle.preprocess(w.scene, cam, t)
    # integer / bit outputs: exact against the FP32 mirror, every Gaussian
    assert np.array_equal(keys, b["depth_key"])
    assert np.array_equal(tt, b["tiles_touched"].astype(np.int32))
    vis = b["tiles_touched"] > 0
    assert np.array_equal(rect[vis].astype(np.int32), b["rect"][vis])
    assert np.array_equal(trims[vis], b["trims"][vis])
    assert np.any(trims[vis] != 0) == trim
    assert np.array_equal(rec[vis, 7].astype(np.int32), b["radius"][vis])
    # the binary32 footprint itself: mean, opacity at t and depth bit for bit; the conic
    # within 4 ulp of the exact inverse of the mirror's Sigma'
    assert np.array_equal(rec[vis, 0:2], b["uv"][vis])
    assert np.array_equal(rec[vis, 5], b["foot"][vis, 0])
    s00, s01, s11 = (b["foot"][vis, k].astype(np.float64) for k in (1, 2, 3))
    det = s00 * s11 - s01 * s01
    inv = np.stack([s11 / det, -s01 / det, s00 / det], 1)
    np.testing.assert_allclose(rec[vis][:, [2, 3, 4]], inv, rtol=2.4e-7, atol=0)
    # float outputs: against FP64
    np.testing.assert_allclose(rec[vis, 0], g["u"][vis], atol=2e-4)
    np.testing.assert_allclose(rec[vis, 1], g["v"][vis], atol=2e-4)
    np.testing.assert_allclose(rec[vis, 2:4], g["conic"][vis, :2], rtol=2e-4, atol=1e-6)
    np.testing.assert_allclose(rec[vis, 4], g["conic"][vis, 2], rtol=2e-4, atol=1e-6)
    np.testing.assert_allclose(rec[vis, 5], g["opacity_t"][vis], rtol=2e-6)
    np.testing.assert_allclose(rec[vis, 6], g["depth"][vis], rtol=1e-6)
    np.testing.assert_allclose(rec[vis, 8:11], g["rgb"][vis], atol=2e-6)
    assert L["key_capacity"] > 0


@pytest.mark.parametrize("binning", [1, 2, 3])
@pytest.mark.parametrize("trim", [False, True])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_lists_bit_exact_tiny(tile, trim, binning):
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    r, _, _ = gu.render(w.scene, cam, t, tile=tile, batch=64, trim=trim, binning=binning)
    assert (r.layout(cam)["tile_passes"] == 1) == (binning == 2)
    assert (r.layout(cam)["tile_passes"] == 0) == (binning == 3)
    got = gu.gpu_lists(r, cam)
    b, exp = gu.expected_lists(w.scene, cam, t, tile, trim=trim)
    assert got["stats"]["status"] == 0
    assert got["stats"]["n_keys"] == len(exp["tile"])
    gu.compare_lists(got, b, exp)


@pytest.mark.parametrize("binning", [1, 2, 3])
@pytest.mark.parametrize("trim", [False, True])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_lists_bit_exact_medium_ragged(tile, trim, binning):
    scene, cam, t = medium()
    r, _, _ = gu.render(scene, cam, t, tile=tile, batch=128, trim=trim, binning=binning)
    assert (r.layout(cam)["tile_passes"] == 1) == (binning == 2)
    assert (r.layout(cam)["tile_passes"] == 0) == (binning == 3)
    got = gu.gpu_lists(r, cam)
    b, exp = gu.expected_lists(scene, cam, t, tile, trim=trim)
    assert len(exp["tile"]) > 10 * 5120, "the case should span many sort partitions"
    gu.compare_lists(got, b, exp)


def test_lists_bit_exact_wide_grid():
    """40,000 Gaussians on 2560x2048 at 8-px tiles (320 x 256 tiles): the pairs pack as
    (tile row << 16 | id); the column order comes from the emission's buckets."""
    scene = synth.make_scene(40_000, 8, "box20", sh_degree=0)
    scene.log_scales -= 1.5   # smaller splats keep the pair count moderate
    cam, t = synth.orbit(2, 2560, 2048, 300)[100]
    r, _, _ = gu.render(scene, cam, t, tile=8, batch=64)
    got = gu.gpu_lists(r, cam)
    assert got["packed"] and r.layout(cam)["tile_passes"] == 2
    b, exp = gu.expected_lists(scene, cam, t, 8)
    gu.compare_lists(got, b, exp)


def test_lists_bit_exact_unpacked_pairs():
    """2^21 + 1 Gaussians (22 id bits) on a 64 x 16384 image at 8-px tiles (2048 tile rows, 11 bits):
    a pair does not fit 32 bits, so the sort carries row keys and id values separately, with two
    row passes."""
    scene = synth.make_scene(2 ** 21 + 1, 12, "tiny", sh_degree=0)
    cam, t = synth.pinhole(64, 16384), 0.5
    r, _, _ = gu.render(scene, cam, t, tile=8, batch=64)
    L = r.layout(cam)
    assert L["id_bits"] == 22 and not L["packed"] and L["tile_passes"] == 3
    got = gu.gpu_lists(r, cam)
    assert got["stats"]["status"] == 0 and got["stats"]["n_keys"] > 1_000_000
    b, exp = gu.expected_lists(scene, cam, t, 8)
    gu.compare_lists(got, b, exp)


def test_image_parity_tiny():
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    r, _, img = gu.render(w.scene, cam, t)
    ref = oracle.render(w.scene, cam, t)
    s = gu.compare_image(img.cpu().numpy(), ref, "tiny")
    assert s["flagged"] < 0.02 * cam.width * cam.height
    gu.compare_T(gu.gpu_final_T(r, cam), ref, "tiny")


def test_image_parity_medium_sampled():
    scene, cam, t = medium()
    r, _, img = gu.render(scene, cam, t)
    rng = np.random.default_rng(0)
    pix = np.column_stack([rng.integers(0, cam.width, 2500), rng.integers(0, cam.height, 2500)])
    pix = np.concatenate([pix, np.column_stack([np.arange(cam.width), np.full(cam.width, cam.height - 1)])])
    ref = oracle.render(scene, cam, t, pixels=pix)
    got = img.cpu().numpy()[pix[:, 1], pix[:, 0]]
    gu.compare_image(got, ref, "medium")
    gu.compare_T(gu.gpu_final_T(r, cam)[pix[:, 1], pix[:, 0]], ref, "medium")


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_image_identical_with_and_without_column_cuts(tile):
    """The cuts drop only tiles where no pixel passes the alpha test: the image, the final
    transmittance and the blend's visits are the same bits, with fewer pairs."""
    scene, cam, t = medium(n=5000, w=200, h=150)
    r0, _, base = gu.render(scene, cam, t, tile=tile)
    r1, _, img = gu.render(scene, cam, t, tile=tile, trim=True)
    assert torch.equal(base, img)
    assert np.array_equal(gu.gpu_final_T(r0, cam), gu.gpu_final_T(r1, cam))
    assert r1.stats(cam)["n_keys"] < r0.stats(cam)["n_keys"]


@pytest.mark.parametrize("tile,batch", [(8, 64), (8, 256), (16, 64), (16, 128), (32, 128), (32, 256)])
def test_image_identical_across_tile_and_batch(tile, batch):
    """Every pixel walks the same (depth, id)-ordered Gaussians with the same
    FP32 operations whatever the tile size and staging depth: bit-identical."""
    scene, cam, t = medium(n=5000, w=200, h=150)
    _, _, base = gu.render(scene, cam, t, tile=16, batch=256)
    _, _, img = gu.render(scene, cam, t, tile=tile, batch=batch)
    assert torch.equal(base, img)


# ---------------------------------------------------------------------------
# edge cases and invariants
# ---------------------------------------------------------------------------

def test_empty_scene_is_background():
    scene = synth.make_scene(0, 0, "tiny")
    cam = synth.pinhole(40, 30)
    r, _, img = gu.render(scene, cam, 0.5, bg=(0.25, 0.5, 0.75))
    assert torch.equal(img, torch.tensor([0.25, 0.5, 0.75], device=img.device).expand_as(img))
    assert r.stats(cam)["n_keys"] == 0


def test_all_behind_camera_is_background():
    w = synth.tiny_workload(300)
    cam = synth.pinhole(64, 64)
    cam.T = np.array([0.0, 0.0, -10.0], np.float32)   # every Gaussian ends at z < 0.2
    r, _, img = gu.render(w.scene, cam, 0.5)
    assert float(img.abs().max()) == 0.0
    assert r.stats(cam)["n_visible"] == 0


def test_background_colour_parity():
    w = synth.tiny_workload(500)
    cam, t = w.frames[0]
    bg = (0.2, 0.5, 0.8)
    _, _, img = gu.render(w.scene, cam, t, bg=bg)
    ref = oracle.render(w.scene, cam, t, bg=bg)
    gu.compare_image(img.cpu().numpy(), ref, "bg")


def test_huge_and_near_plane_gaussians():
    """Gaussians that cover every tile, sit just beyond the near plane, or
    straddle it."""
    sc = synth.make_scene(64, 9, "tiny")
    sc.means[:8] = [[0.0, 0.0, 0.3]] * 8
    sc.log_scales[:8] = math.log(0.5)
    sc.means[8:16, 2] = np.linspace(0.15, 0.25, 8)
    sc.velocity[:16] = 0
    cam = synth.pinhole(96, 80)
    r, _, img = gu.render(sc, cam, 0.5)
    ref = oracle.render(sc, cam, 0.5)
    gu.compare_image(img.cpu().numpy(), ref, "huge")
    b, exp = gu.expected_lists(sc, cam, 0.5, 16)
    gu.compare_lists(gu.gpu_lists(r, cam), b, exp)


def test_single_gaussian():
    sc = synth.make_scene(1, 3, "tiny")
    sc.means[0] = [0.05, -0.02, 3.0]
    cam = synth.pinhole(64, 48)
    _, _, img = gu.render(sc, cam, float(sc.t_mean[0]))
    ref = oracle.render(sc, cam, float(sc.t_mean[0]))
    gu.compare_image(img.cpu().numpy(), ref, "single")
    assert float(img.max()) > 0.01


def test_capacity_overflow_reported_without_writing_out_of_bounds():
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    m = gu.d4()
    ds = m.DeviceScene.from_host(w.scene)
    r = m.Renderer(w.scene.n, cam, key_capacity=1000)
    guard = torch.full((1 << 20,), 7, dtype=torch.uint8, device="cuda")
    out = torch.empty((cam.height, cam.width, 3), device="cuda")
    m.d4dgs_render(ds, cam, t, r.cfg, r.ws, out)
    st = m.d4dgs_read_stats(w.scene.n, cam, r.cfg, r.ws)
    assert st["status"] == m.D4DGS_ERR_CAPACITY
    assert st["n_keys"] > 1000
    assert int((guard != 7).sum()) == 0
    img = r.render(ds, cam, t)   # grows the workspace and re-renders
    ref = oracle.render(w.scene, cam, t)
    gu.compare_image(img.cpu().numpy(), ref, "after-grow")


def test_near_plane_setting_matches_oracle():
    """config near = 1.0 (the oracle's camera plane likewise): Gaussians whose time-shifted mean
    is not beyond z = 1 are not drawn; the lists bit for bit against the mirror with that plane,
    the image against the oracle; the frame differs from the one with the default plane."""
    sc = synth.make_scene(3000, 27, "tiny")
    sc.means[:, 2] = np.random.default_rng(27).uniform(0.4, 3.0, sc.n).astype(np.float32)
    cam, t = synth.pinhole(160, 120), 0.5
    cam.near = 1.0
    r, _, img = gu.render(sc, cam, t)
    b, exp = gu.expected_lists(sc, cam, t, 16)
    gu.compare_lists(gu.gpu_lists(r, cam), b, exp)
    gu.compare_image(img.cpu().numpy(), oracle.render(sc, cam, t), "near 1.0")
    _, _, img02 = gu.render(sc, synth.pinhole(160, 120), t)
    assert float((img - img02).abs().max()) > 0.05


def test_bounded_spin_wait_gives_up_and_reports_timeout():
    """config spin_limit = 1 on the 300k benchmark frame (hundreds of sort partitions per pass, so
    decoupled look-backs wait): every wait gives up after one poll, the call returns, the frame
    reports D4DGS_ERR_TIMEOUT, and no byte past the workspace is written; the next frame on the
    same workspace with the default limit is correct."""
    m = gu.d4()
    w = synth.scene_workload()
    cam, t = w.frames[150]
    n = w.scene.n
    ds = m.DeviceScene.from_host(w.scene)
    impatient = m.config_struct(32, 256, spin_limit=1)
    nbytes = m.d4dgs_workspace_bytes(n, cam, impatient, 40 * n)
    buf = torch.full((nbytes + (1 << 20),), 0xA5, dtype=torch.uint8, device="cuda")
    ws = buf[:nbytes]
    out = torch.empty((cam.height, cam.width, 3), device="cuda")
    m.d4dgs_render(ds, cam, t, impatient, ws, out)
    torch.cuda.synchronize()
    assert m.d4dgs_read_stats(n, cam, impatient, ws)["status"] == m.D4DGS_ERR_TIMEOUT
    assert int((buf[nbytes:] != 0xA5).sum()) == 0
    cfg = m.config_struct(32, 256)
    m.d4dgs_render(ds, cam, t, cfg, ws, out)
    torch.cuda.synchronize()
    assert m.d4dgs_read_stats(n, cam, cfg, ws)["status"] == m.D4DGS_OK
    assert int((buf[nbytes:] != 0xA5).sum()) == 0
    pix = np.column_stack([np.random.default_rng(2).integers(0, cam.width, 400),
                           np.random.default_rng(3).integers(0, cam.height, 400)])
    ref = oracle.render(w.scene, cam, t, pixels=pix)
    gu.compare_image(out.cpu().numpy()[pix[:, 1], pix[:, 0]], ref, "after a timed-out frame")


def test_deterministic():
    scene, cam, t = medium(n=8000, w=160, h=120)
    _, _, a = gu.render(scene, cam, t)
    _, _, b = gu.render(scene, cam, t)
    assert torch.equal(a, b)


def test_static_reduction_bit_identical_over_time():
    """V = 0 and s_t -> infinity: the GPU image must not depend on t at all."""
    sc = synth.make_scene(2000, 21, "tiny")
    sc.velocity[:] = 0
    sc.log_t_scale[:] = 30.0
    cam = synth.pinhole(128, 96)
    imgs = [gu.render(sc, cam, t)[2] for t in (0.0, 0.31, 1.0)]
    assert float(imgs[0].max()) > 0.05
    assert torch.equal(imgs[0], imgs[1]) and torch.equal(imgs[0], imgs[2])


def test_nan_camera_rejected():
    w = synth.tiny_workload(10)
    cam = synth.pinhole(32, 32)
    m = gu.d4()
    ds = m.DeviceScene.from_host(w.scene)
    r = m.Renderer(10, cam)
    bad = synth.pinhole(32, 32)
    bad.cx = float("nan")
    out = torch.empty((32, 32, 3), device="cuda")
    with pytest.raises(m.D4DGSError) as e:
        m.d4dgs_render(ds, bad, 0.5, r.cfg, r.ws, out)
    assert e.value.code == m.D4DGS_ERR_INVALID_ARG


def test_render_host_matches_device_path():
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    r, ds, img = gu.render(w.scene, cam, t)
    m = gu.d4()
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(w.scene, k))).pin_memory() for k in m.SCENE_FIELDS}
    host["sh_degree"] = w.scene.sh_degree
    buf = torch.empty(m.d4dgs_scene_bytes(w.scene.n, w.scene.sh_degree), dtype=torch.uint8, device="cuda")
    dev_rgb = torch.empty_like(img)
    out = torch.empty(img.shape, dtype=torch.float32).pin_memory()
    m.d4dgs_render_host(host, cam, t, r.cfg, buf, r.ws, dev_rgb, out)
    assert torch.equal(out, img.cpu())


def test_render_host_async_two_slots_match_device_path():
    """Frames queued alternately on two slots (staging buffer, workspace, device image, stream)
    overlap on the device; after each slot's wait its host image equals the device-path render."""
    w = synth.tiny_workload()
    m = gu.d4()
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(w.scene, k))).pin_memory() for k in m.SCENE_FIELDS}
    host["sh_degree"] = w.scene.sh_degree
    frames = [(w.frames[0][0], t) for t in (0.5, 0.1, 0.9, 0.3)]
    refs = [gu.render(w.scene, cam, t)[2].cpu() for cam, t in frames]
    cam0 = frames[0][0]
    slots = []
    for _ in range(2):
        r = m.Renderer(w.scene.n, cam0)
        slots.append(dict(r=r, buf=torch.empty(m.d4dgs_scene_bytes(w.scene.n, w.scene.sh_degree), dtype=torch.uint8,
                                               device="cuda"),
                          rgb=torch.empty((cam0.height, cam0.width, 3), device="cuda"),
                          out=torch.empty((cam0.height, cam0.width, 3)).pin_memory(), st=torch.cuda.Stream()))
    got = [None] * len(frames)
    pending = [None, None]
    for k, (cam, t) in enumerate(frames):
        s = slots[k % 2]
        if pending[k % 2] is not None:
            s["st"].synchronize()
            got[pending[k % 2]] = s["out"].clone()
        m.d4dgs_render_host_async(host, cam, t, s["r"].cfg, s["buf"], s["r"].ws, s["rgb"], s["out"], s["st"])
        pending[k % 2] = k
    for j in range(2):
        slots[j]["st"].synchronize()
        got[pending[j]] = slots[j]["out"].clone()
    for a, b in zip(got, refs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("trim", [False, True])
def test_staging_depth_512_renders_as_256(trim):
    """32-px tiles also stage 512 Gaussians a batch: the walk, its stops and the image are the
    ones a 256-deep staging gives, bit for bit."""
    scene, cam, t = medium()
    r256, _, a = gu.render(scene, cam, t, tile=32, batch=256, trim=trim)
    r512, _, b = gu.render(scene, cam, t, tile=32, batch=512, trim=trim)
    assert torch.equal(a, b)
    px = cam.width * cam.height
    for name in ("final_T", "n_contrib"):
        assert torch.equal(r256.view(name, torch.int32, px, cam), r512.view(name, torch.int32, px, cam)), name
