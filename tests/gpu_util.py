"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and read its workspace buffers back; compare against the oracle."""
from __future__ import annotations

import numpy as np
import torch

import oracle

# Image tolerances (max-abs and mean-abs in [0,1] RGB) plus the oracle's
# per-pixel slack for decisions within FP32 reach of a threshold.
MAX_ABS = 2e-3
MEAN_ABS = 1e-4


def d4():
    import paper_2503_22159_gb300 as m
    return m


def render(scene, cam, t, tile=16, batch=256, bg=(0.0, 0.0, 0.0), cap=None, trim=False, binning=0):
    m = d4()
    ds = m.DeviceScene.from_host(scene)
    r = m.Renderer(scene.n, cam, tile=tile, batch=batch, bg=bg, key_capacity=cap, trim=trim,
                   near=getattr(cam, "near", 0.2), binning=binning)
    img = r.render(ds, cam, t)
    torch.cuda.synchronize()
    return r, ds, img


def _u32(r, name, count, cam):
    if count == 0:
        return np.zeros(0, np.uint32)
    return r.view(name, torch.int32, count, cam).cpu().numpy().view(np.uint32)


def gpu_records(r, n, cam):
    return r.view("records", torch.float32, 12 * n, cam).cpu().numpy().reshape(n, 12)


def gpu_lists(r, cam):
    st = r.stats(cam)
    k = int(st["n_keys"])
    L = r.layout(cam)
    ntiles = L["tiles_x"] * L["tiles_y"]
    keys = _u32(r, "tile_keys", k, cam)
    if L["packed"]:
        rows = keys >> np.uint32(L["id_bits"])
        ids = keys & np.uint32((1 << L["id_bits"]) - 1)
    else:
        rows = keys
        ids = _u32(r, "tile_vals", k, cam)
    ranges = _u32(r, "ranges", 2 * ntiles, cam).reshape(ntiles, 2)
    # the tile of each position from the ranges; the key carries the tile row
    starts = ranges[:, 0].astype(np.int64)
    counts = (ranges[:, 1].astype(np.int64) - starts)
    assert np.all(counts >= 0) and counts.sum() == k
    assert np.array_equal(starts[counts > 0], np.concatenate([[0], np.cumsum(counts)[:-1]])[counts > 0])
    tiles = np.repeat(np.arange(ntiles, dtype=np.uint32), counts)
    assert np.array_equal(rows, tiles // np.uint32(L["tiles_x"])), "pair keys disagree with the tile ranges"
    return dict(tile=tiles, id=ids, ranges=ranges, stats=st, packed=bool(L["packed"]))


def expected_lists(scene, cam, t, tile, trim=False):
    b = oracle.bin_f32(scene, cam, t, tile, trim=trim)
    return b, oracle.tile_list(b)


def compare_lists(got, b, exp):
    """The (tile, id) sequence and every non-empty tile's [start, end) bit for bit
    (empty tiles: any empty range).  The mirror's arithmetic, exp and log included,
    is the kernel's, so no Gaussian is left out."""
    assert len(got["tile"]) == len(exp["tile"]), (len(got["tile"]), len(exp["tile"]))
    assert np.array_equal(got["tile"], exp["tile"])
    assert np.array_equal(got["id"], exp["id"])
    gr, er = got["ranges"].astype(np.int64), exp["ranges"].astype(np.int64)
    full = er[:, 1] > er[:, 0]
    assert np.array_equal(gr[full], er[full])
    assert np.all(gr[~full, 1] == gr[~full, 0])
    return 0


def compare_image(got, ref, where=""):
    """|gpu - oracle| <= MAX_ABS + slack per pixel channel; mean-abs <= MEAN_ABS."""
    got = np.asarray(got, np.float64)
    err = np.abs(got - ref["rgb"])
    slack = ref["slack"][..., None]
    bad = err > MAX_ABS + slack
    assert not bad.any(), f"{where}: {int(bad.sum())} channels beyond tolerance, max err {err.max():.3g}"
    flagged = ref["slack"] > 0
    strict = err[~flagged]
    if strict.size:
        assert strict.max() <= MAX_ABS, f"{where}: unflagged max err {strict.max():.3g}"
    assert err.mean() <= MEAN_ABS, f"{where}: mean abs err {err.mean():.3g}"
    return dict(max=float(err.max()), mean=float(err.mean()), flagged=int(flagged.sum()))


def gpu_final_T(r, cam):
    """Per-pixel transmittance the blend stored for the backward (H x W)."""
    return r.view("final_T", torch.float32, cam.width * cam.height, cam).cpu().numpy().reshape(cam.height, cam.width)


def compare_T(got_T, ref, where=""):
    """Final transmittance within the oracle's accumulated FP32 budget Tw
    (twice it, plus 1e-6 relative) on pixels without a near-threshold
    decision.  A dropped or extra alpha >= 1/255 term moves T by at least
    0.39% relative, so every pixel whose bound is tighter than that also
    checks that no such term was lost; require most pixels to be of that kind."""
    got_T = np.asarray(got_T, np.float64)
    T = ref["T"]
    tol = (2.0 * ref["Tw"] + 1e-6) * T + 1e-9
    strict = ref["slack"] == 0
    err = np.abs(got_T - T)
    bad = strict & (err > tol)
    assert not bad.any(), f"{where}: {int(bad.sum())} pixels with T beyond budget, worst rel {float((err / np.maximum(T, 1e-30))[bad].max()):.3g}"
    sharp = strict & (tol < (1.0 / 255.0) * T)
    assert sharp.sum() >= 0.2 * T.size, f"{where}: only {int(sharp.sum())} of {T.size} pixels can see a dropped term"
    return dict(strict=int(strict.sum()), sharp=int(sharp.sum()))
