"""Parity at the benchmark's full size and launch configuration (needs a GPU):
300,000 SH-3 Gaussians, 1352x1014, tile 16, batch 256, frames of the orbit.

The whole preprocess and the whole (tile, Gaussian) list are compared (bit for
bit where the arithmetic is fixed); the image on sampled pixels that the
oracle computes one by one."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene_w():
    return synth.scene_workload()


@pytest.fixture(scope="module")
def gpu_renderer(scene_w):
    m = gu.d4()
    ds = m.DeviceScene.from_host(scene_w.scene)
    cam0 = scene_w.frames[0][0]
    r = m.Renderer(scene_w.scene.n, cam0, tile=16, batch=256, key_capacity=40 * scene_w.scene.n)
    return m, ds, r


@pytest.mark.parametrize("k,trim,tile,binning", [(150, False, 16, 0), (150, True, 16, 0), (150, False, 32, 0),
                                                  (150, False, 32, 2), (150, True, 32, 2), (150, False, 32, 3),
                                                  (150, True, 16, 3)])
def test_scene_preprocess_and_lists(scene_w, gpu_renderer, k, trim, tile, binning):
    """Tile 16 and 32 (the benchmark's launch configuration) with the column binning; tile 32
    (1376 tiles) with the direct binning and the rank lists too."""
    m, ds, r = gpu_renderer
    if trim or tile != 16 or binning:
        r = m.Renderer(scene_w.scene.n, scene_w.frames[0][0], tile=tile, batch=256, key_capacity=40 * scene_w.scene.n,
                       trim=trim, binning=binning)
    cam, t = scene_w.frames[k]
    r.render(ds, cam, t)
    torch.cuda.synchronize()
    assert (r.layout(cam)["tile_passes"] == 1) == (binning == 2)
    assert (r.layout(cam)["tile_passes"] == 0) == (binning == 3)
    n = scene_w.scene.n
    rec = gu.gpu_records(r, n, cam)
    b = oracle.bin_f32(scene_w.scene, cam, t, tile, trim=trim)
    g = oracle.preprocess(scene_w.scene, cam, t)
    vis = b["tiles_touched"] > 0
    assert vis.sum() > 100_000
    assert np.array_equal(rec[vis, 7].astype(np.int32), b["radius"][vis])
    assert np.array_equal(rec[vis, 6].view(np.uint32), b["depth_key"][vis])
    assert np.array_equal(rec[vis, 0:2], b["uv"][vis])
    assert np.array_equal(rec[vis, 5], b["foot"][vis, 0])
    trims = r.view("trims", torch.int64, n, cam).cpu().numpy().view(np.uint64)
    assert np.array_equal(trims[vis], b["trims"][vis])
    np.testing.assert_allclose(rec[vis, 0], g["u"][vis], atol=2e-3)
    np.testing.assert_allclose(rec[vis, 1], g["v"][vis], atol=2e-3)
    np.testing.assert_allclose(rec[vis, 5], g["opacity_t"][vis], rtol=5e-6)
    np.testing.assert_allclose(rec[vis, 8:11], g["rgb"][vis], atol=1e-5)
    np.testing.assert_allclose(rec[vis, 2], g["conic"][vis, 0], rtol=1e-3, atol=1e-7)
    np.testing.assert_allclose(rec[vis, 4], g["conic"][vis, 2], rtol=1e-3, atol=1e-7)
    got = gu.gpu_lists(r, cam)
    exp = oracle.tile_list(b)
    assert got["stats"]["status"] == 0
    # every Gaussian, every tile: the whole list and every range bit for bit
    gu.compare_lists(got, b, exp)


@pytest.mark.parametrize("k", [0, 150, 299])
def test_scene_image_sampled(scene_w, gpu_renderer, k):
    m, ds, r = gpu_renderer
    cam, t = scene_w.frames[k]
    img = r.render(ds, cam, t)
    torch.cuda.synchronize()
    rng = np.random.default_rng(k)
    pix = np.column_stack([rng.integers(0, cam.width, 1500), rng.integers(0, cam.height, 1500)])
    pix = np.concatenate([pix, np.column_stack([np.arange(cam.width), np.full(cam.width, 7 * k % cam.height)])])
    # the last column and row (ragged bottom tile row: 1014 = 63 * 16 + 6)
    pix = np.concatenate([pix, np.column_stack([np.full(cam.height, cam.width - 1), np.arange(cam.height)])])
    ref = oracle.render(scene_w.scene, cam, t, pixels=pix)
    got = img.cpu().numpy()[pix[:, 1], pix[:, 0]]
    s = gu.compare_image(got, ref, f"scene frame {k}")
    gu.compare_T(gu.gpu_final_T(r, cam)[pix[:, 1], pix[:, 0]], ref, f"scene frame {k}")
    assert float(np.abs(ref["rgb"]).max()) > 0.1
    # pixels with a decision within FP32 reach of its threshold (slack > 0) get the slack on top
    # of 2e-3; at most 5% of the sampled pixels may be such (measured: 0.2-2.8% on frames 0, 150
    # and 299 at 3000 random pixels)
    share = s["flagged"] / len(pix)
    print(f"scene frame {k}: flagged share {share:.4f}, max err {s['max']:.3g}, mean err {s['mean']:.3g}")
    assert share <= 0.05, f"frame {k}: {share:.3f} of the sampled pixels flagged"
