"""Slicing-first baseline on the GPU (needs a GPU): the kernel that slices every
4D Gaussian at each frame (Eq. 5-7) renders the oracle's slicing-first image,
and the disentangled kernel on the converted scene renders the same image."""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import convert
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def render_slicing(sc4, cam, t, tile=16):
    m = gu.d4()
    ds = m.DeviceScene4D.from_host(sc4)
    cfg = m.config_struct(tile, 256)
    ws = torch.empty(m.d4dgs_workspace_bytes(sc4.n, cam, cfg, 64 * sc4.n + 4096), dtype=torch.uint8, device="cuda")
    out = torch.empty((cam.height, cam.width, 3), device="cuda")
    m.d4dgs_render_slicing(ds, cam, t, cfg, ws, out)
    assert m.d4dgs_read_stats(sc4.n, cam, cfg, ws)["status"] == 0
    return out.cpu().numpy()


@pytest.mark.parametrize("tile", [16, 32])
def test_slicing_first_matches_oracle_tiny(tile):
    sc4 = synth.make_scene4d(800, 41, "tiny", mix=0.3)
    cam = synth.pinhole(128, 128)
    for t in (0.25, 0.6):
        ref = oracle.render_slicing(sc4, cam, t)
        gu.compare_image(render_slicing(sc4, cam, t, tile), ref, f"slicing tiny t={t}")
        assert np.abs(ref["rgb"]).max() > 0.05


def test_slicing_first_and_converted_disentangled_match_oracle_sampled():
    sc4 = synth.make_scene4d(20000, 42, "box20")
    cam, t = synth.orbit(3, 400, 300, 300)[120]
    rng = np.random.default_rng(1)
    pix = np.column_stack([rng.integers(0, cam.width, 1200), rng.integers(0, cam.height, 1200)])
    ref = oracle.render_slicing(sc4, cam, t, pixels=pix)
    img4 = render_slicing(sc4, cam, t)
    gu.compare_image(img4[pix[:, 1], pix[:, 0]], ref, "slicing-first")
    dis = convert.disentangle(sc4)
    _, _, img = gu.render(dis, cam, t)
    gu.compare_image(img.cpu().numpy()[pix[:, 1], pix[:, 0]], ref, "converted disentangled")
