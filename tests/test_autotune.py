"""Autotuner: cache keys and persistence and the sweep on the CPU (with a
fake timer); on the GPU, a real sweep picks a valid configuration whose image
equals every other configuration's."""
import numpy as np
import pytest
import torch

import synth


@pytest.fixture()
def at(tmp_path, monkeypatch):
    monkeypatch.setenv("D4DGS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_22159_gb300 import autotune
    return autotune


def test_sweep_picks_fastest_and_cache_roundtrip(at, tmp_path):
    fake = {(8, 64, False): 3.0, (16, 128, True): 1.5, (32, 256, False): 2.0}
    best, table = at.sweep(lambda t, b, c: fake.get((t, b, c), 9.0))
    assert best == (16, 128, True) and len(table) == 20 and table["16/128/cut"] == 1.5
    assert "32/512" in table and "16/512" not in table
    key = at.cache_key("GB300", 1352, 1014, 300_000)
    assert key == "GB300|1352x1014|n<=524288"
    c = at.TuneCache()
    c.put(key, *best, table)
    assert at.TuneCache().get(key) == (16, 128, True)
    assert at.TuneCache().get(at.cache_key("GB300", 1352, 1014, 600_000)) is None   # other N bucket


def test_sweep_skips_configurations_that_cannot_render(at):
    """A tile size whose frames need more pairs than a workspace can hold is reported as None."""
    best, table = at.sweep(lambda t, b, c: None if t == 8 else float(t + b / 1000 + c))
    assert best == (16, 64, False)
    assert all(table[at.config_name(8, b, c)] is None for b in at.BATCHES if b != 512 for c in at.TRIMS)
    with pytest.raises(RuntimeError):
        at.sweep(lambda t, b, c: None)


@pytest.mark.gpu
def test_gpu_sweep_choice_renders_identically(at):
    import paper_2503_22159_gb300 as d4
    sc = synth.make_scene(20_000, 61, "box20", sh_degree=1)
    frames = synth.orbit(3, 320, 240, 300)[100:103]
    ds = d4.DeviceScene.from_host(sc)
    (tile, batch, trim), table = at.tune(ds, frames, force=True)
    assert tile in at.TILES and batch in at.BATCHES and len(table) == 20
    assert at.tune(ds, frames)[1] is None   # cached
    cam, t = frames[0]
    ref = d4.Renderer(sc.n, cam, tile=16, batch=256).render(ds, cam, t).clone()
    img = d4.Renderer(sc.n, cam, tile=tile, batch=batch, trim=trim).render(ds, cam, t)
    assert torch.equal(img, ref)
