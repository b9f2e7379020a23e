"""The C ABI without a GPU: the library loads, exports every symbol that
include/d4dgs.h declares, and its host-side logic (workspace sizing, layout,
argument checks) behaves as documented.  No kernel is launched here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def d4():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_22159_gb300 as d4
    return d4


def declared_functions():
    src = open(os.path.join(ROOT, "include", "d4dgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(d4dgs_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("d4dgs_preprocess", "d4dgs_render", "d4dgs_render_backward", "d4dgs_sort", "d4dgs_blend",
              "d4dgs_workspace_bytes", "d4dgs_read_stats", "d4dgs_strerror"):
        assert f in names


def test_library_exports_every_declared_symbol(d4):
    lib = d4._abi.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(d4._abi.PROTOTYPES), "binding misses a declared function"


def test_strerror(d4):
    assert d4._abi.strerror(0) == "ok"
    assert "capacity" in d4._abi.strerror(d4.D4DGS_ERR_CAPACITY)


def test_workspace_bytes_monotone_and_layout(d4):
    cam = synth.pinhole(1352, 1014)
    cfg = d4.config_struct(16, 256)
    b0 = d4.d4dgs_workspace_bytes(300_000, cam, cfg, 0)
    b1 = d4.d4dgs_workspace_bytes(300_000, cam, cfg, 1_000_000)
    assert b1 > b0 + 8 * 1_000_000   # two packed uint32 pair buffers
    L = d4.d4dgs_workspace_layout(300_000, cam, cfg, b1)
    assert L["key_capacity"] == 1_000_000
    assert (L["tiles_x"], L["tiles_y"]) == (85, 64)
    assert L["tile_passes"] == 2 and L["depth_passes"] == 4
    assert L["id_bits"] == 19 and L["packed"] == 1 and L["tile_vals"] == -1
    offs = [L[k] for k in ("records", "depth_keys", "tiles_touched", "rect", "trims", "depth_order", "tile_keys",
                           "ranges", "final_T", "n_contrib", "control")]
    assert all(o % 256 == 0 for o in offs)
    assert max(offs) < b1
    with pytest.raises(d4.D4DGSError):
        d4.d4dgs_workspace_layout(300_000, cam, cfg, b0 - 1)


@pytest.mark.parametrize("w,h,tile,passes", [(128, 128, 16, 2), (1352, 1014, 16, 2), (2704, 2028, 8, 2),
                                             (16, 16, 16, 2), (7, 5, 32, 2), (4096, 4096, 8, 3),
                                             (16384, 2048, 8, 2)])
def test_tile_pass_count(d4, w, h, tile, passes):
    """Column binning: pass 0 buckets the pairs by tile column; 8-bit passes over the row bits
    follow (at least one)."""
    cam = synth.pinhole(w, h)
    cfg = d4.config_struct(tile, 64, binning=1)
    L = d4.d4dgs_workspace_layout(10, cam, cfg, d4.d4dgs_workspace_bytes(10, cam, cfg, 100))
    cols, rows = math.ceil(w / tile), math.ceil(h / tile)
    assert L["tile_passes"] == passes
    assert 2 ** (8 * (passes - 1)) >= rows
    assert 2 ** L["col_bits"] >= cols > 2 ** (L["col_bits"] - 1) or cols == 1


@pytest.mark.parametrize("w,h,tile,fits", [(128, 128, 16, True), (1352, 1014, 32, True),
                                                  (1920, 1080, 32, True), (1352, 1014, 16, False),
                                                  (2704, 2028, 32, False), (7, 5, 32, True), (1440, 1440, 32, True),
                                                  (1472, 1440, 32, False)])
def test_binning_choice(d4, w, h, tile, fits):
    """Direct binning (pairs straight into the tiles' lists, tile_passes 1) on request for grids of
    at most 2048 tiles, where it is an invalid config beyond; binning 0 takes the column path."""
    cam = synth.pinhole(w, h)
    ntiles = math.ceil(w / tile) * math.ceil(h / tile)
    assert fits == (ntiles <= 2048)
    for binning, direct in ((0, False), (1, False), (2, True), (3, False)):
        cfg = d4.config_struct(tile, 64, binning=binning)
        if binning == 2 and not fits:
            assert d4._abi.load().d4dgs_workspace_bytes(10, ctypes.byref(d4.camera_struct(cam)), ctypes.byref(cfg),
                                                        100) == 0
            continue
        L = d4.d4dgs_workspace_layout(10, cam, cfg, d4.d4dgs_workspace_bytes(10, cam, cfg, 100))
        assert (L["tile_passes"] == 1) == direct
        # rank lists (binning 3, any grid): no pass sorts the pairs; the lists end in the first buffer
        assert (L["tile_passes"] == 0) == (binning == 3)
    assert d4._abi.load().d4dgs_workspace_bytes(10, ctypes.byref(d4.camera_struct(cam)),
                                                ctypes.byref(d4.config_struct(tile, 64, binning=4)), 100) == 0


def test_invalid_arguments_rejected_on_host(d4):
    cfg = d4.config_struct(16, 256)
    cam = synth.pinhole(64, 64)
    assert d4._abi.load().d4dgs_workspace_bytes(10, ctypes.byref(d4.camera_struct(cam)),
                                                ctypes.byref(d4.config_struct(12, 256)), 10) == 0
    assert d4._abi.load().d4dgs_workspace_bytes(10, ctypes.byref(d4.camera_struct(cam)),
                                                ctypes.byref(d4.config_struct(16, 100)), 10) == 0
    bad = synth.pinhole(64, 64)
    bad.fx = float("nan")
    assert d4._abi.load().d4dgs_workspace_bytes(10, ctypes.byref(d4.camera_struct(bad)), ctypes.byref(cfg), 10) == 0
    # a render call with a NaN camera or NaN time is refused before anything is launched
    s = d4._abi.d4dgs_scene(*([0] * 8), 0, 0)
    lib = d4._abi.load()
    rc = lib.d4dgs_render(ctypes.byref(s), ctypes.byref(d4.camera_struct(bad)), 0.0, ctypes.byref(cfg),
                          ctypes.c_void_p(256), 1 << 20, ctypes.c_void_p(256), None)
    assert rc == d4.D4DGS_ERR_INVALID_ARG
    rc = lib.d4dgs_render(ctypes.byref(s), ctypes.byref(d4.camera_struct(cam)), float("nan"), ctypes.byref(cfg),
                          ctypes.c_void_p(256), 1 << 20, ctypes.c_void_p(256), None)
    assert rc == d4.D4DGS_ERR_INVALID_ARG
    # misaligned quaternion pointer
    s = d4._abi.d4dgs_scene(256, 256, 256, 256, 256, 260, 256, 256, 5, 0)
    rc = lib.d4dgs_preprocess(ctypes.byref(s), ctypes.byref(d4.camera_struct(cam)), 0.0, ctypes.byref(cfg),
                              ctypes.c_void_p(256), 1 << 20, None)
    assert rc == d4.D4DGS_ERR_INVALID_ARG
    # too-small workspace
    s = d4._abi.d4dgs_scene(256, 256, 256, 256, 256, 256, 256, 256, 5, 0)
    rc = lib.d4dgs_preprocess(ctypes.byref(s), ctypes.byref(d4.camera_struct(cam)), 0.0, ctypes.byref(cfg),
                              ctypes.c_void_p(256), 1024, None)
    assert rc == d4.D4DGS_ERR_WORKSPACE_TOO_SMALL


def test_launch_count(d4):
    cfg = d4.config_struct(16, 256)
    # clear + preprocess + 4 depth passes (the first also does the tile counts: 86 x 65 grid cells)
    # + column emit + 1 row pass + blend
    assert d4.d4dgs_launches_per_frame(300_000, synth.pinhole(1352, 1014), cfg) == 9
    # 2704 x 2028 at 16 px: 171 x 128 grid cells are too many to ride along, tile counts launch alone
    assert d4.d4dgs_launches_per_frame(300_000, synth.pinhole(2704, 2028), cfg) == 10
    # 1352 x 1014 at 32 px (1376 tiles), direct binning: counts + scan + emission instead of the
    # column emission and the row pass
    assert d4.d4dgs_launches_per_frame(300_000, synth.pinhole(1352, 1014), d4.config_struct(32, 256, binning=2)) == 10
    assert d4.d4dgs_launches_per_frame(300_000, synth.pinhole(1352, 1014), d4.config_struct(32, 256)) == 9
    # rank lists: the rank emission and the list building instead of the column emission and the row pass
    assert d4.d4dgs_launches_per_frame(300_000, synth.pinhole(1352, 1014), d4.config_struct(32, 256, binning=3)) == 9
    # an empty scene: clear and blend around one launch of the tile counts
    assert d4.d4dgs_launches_per_frame(0, synth.pinhole(1352, 1014), d4.config_struct(32, 512)) == 3


def test_packing_decision(d4):
    """A pair's key holds its tile row only (the emission has bucketed the columns): packed into one
    uint32 with the id whenever row bits + id bits <= 32."""
    cfg8 = d4.config_struct(8, 64)
    cam = synth.pinhole(2560, 2048)   # 320 tile columns, 256 rows (8 bits)
    L = d4.d4dgs_workspace_layout(40_000, cam, cfg8, d4.d4dgs_workspace_bytes(40_000, cam, cfg8, 1000))
    assert L["id_bits"] == 16 and L["packed"] == 1 and L["tile_vals"] == -1 and L["tile_passes"] == 2
    assert L["col_bits"] == 9
    tall = synth.pinhole(64, 16384)   # 2048 tile rows (11 bits)
    for n, ids, packed in ((2 ** 21, 21, 1), (2 ** 21 + 1, 22, 0)):
        L = d4.d4dgs_workspace_layout(n, tall, cfg8, d4.d4dgs_workspace_bytes(n, tall, cfg8, 1000))
        assert L["id_bits"] == ids and L["packed"] == packed and (L["tile_vals"] > 0) == (not packed)
        assert L["tile_passes"] == 3   # 11 row bits: two row passes


def test_product_does_not_import_oracle():
    """The product package never reaches the CPU oracle (no fallback path)."""
    pkg = os.path.join(ROOT, "paper_2503_22159_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "orc_" not in src, f


def test_staging_depth_512_only_at_32px_tiles(d4):
    """The blend stages 64, 128 or 256 Gaussians a batch at any tile size and 512 at 32-px tiles."""
    cam = synth.pinhole(640, 480)
    lib = d4._abi.load()
    for tile in (8, 16, 32):
        for batch in (64, 128, 256, 512, 1024):
            ok = batch in (64, 128, 256) or (batch == 512 and tile == 32)
            n = lib.d4dgs_workspace_bytes(10, ctypes.byref(d4.camera_struct(cam)),
                                          ctypes.byref(d4.config_struct(tile, batch)), 100)
            assert (n > 0) == ok, (tile, batch)

