"""d4dgs_render_static: the render entry point for callers that cannot
allocate device memory when they render (its scratch is a fixed array inside
the library), checked against d4dgs_render with a caller-owned workspace.

It runs last (file name) so that a failure here cannot hide the others, and
must pass both alone in a fresh process and after every other test."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _render_static(m, ds, cam, t, cfg, out):
    st = m._abi.d4dgs_stats()
    rc = m._abi.load().d4dgs_render_static(ctypes.byref(ds.struct()), ctypes.byref(m.camera_struct(cam)),
                                           float(t), ctypes.byref(cfg), ctypes.c_void_p(out.data_ptr()),
                                           ctypes.byref(st), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, st


def test_render_static_matches_workspace_path_twice():
    m = gu.d4()
    sc = synth.make_scene(3000, 31, "tiny", sh_degree=1)
    cam = synth.pinhole(160, 120)
    ds = m.DeviceScene.from_host(sc)
    for t in (0.25, 0.75):   # two calls in a row; the second must not see the first's leftovers
        _, _, ref = gu.render(sc, cam, t)
        out = torch.full_like(ref, -1.0)
        rc, st = _render_static(m, ds, cam, t, m.config_struct(16, 256), out)
        torch.cuda.synchronize()
        assert rc == 0, m._abi.strerror(rc)
        assert st.status == 0 and st.n_keys > 0
        # the same kernels on the same inputs: bit for bit
        assert torch.equal(out, ref), (out - ref).abs().max().item()


def test_render_static_refuses_sizes_beyond_its_scratch():
    m = gu.d4()
    sc = synth.make_scene(8, 1, "tiny")
    ds = m.DeviceScene.from_host(sc)
    cam = synth.pinhole(8192, 8192)            # 8 B/pixel of per-pixel state alone exceeds 64 MiB
    out = torch.empty((1, 1, 3), device="cuda")
    rc, _ = _render_static(m, ds, cam, 0.5, m.config_struct(16, 256), out)
    assert rc == m.D4DGS_ERR_WORKSPACE_TOO_SMALL


def test_render_static_reports_an_overflowing_frame_through_stats():
    """The 300k benchmark scene at 16-px tiles makes ~30 M (tile, Gaussian) pairs, more than the
    fixed array's key capacity: with stats the call reports D4DGS_ERR_CAPACITY (it cannot grow
    the array; the image is incomplete)."""
    m = gu.d4()
    w = synth.scene_workload()
    cam, t = w.frames[150]
    ds = m.DeviceScene.from_host(w.scene)
    out = torch.empty((cam.height, cam.width, 3), device="cuda")
    rc, st = _render_static(m, ds, cam, t, m.config_struct(16, 256), out)
    assert rc == m.D4DGS_ERR_CAPACITY and st.status == m.D4DGS_ERR_CAPACITY
    assert st.n_keys > st.key_capacity > 0
