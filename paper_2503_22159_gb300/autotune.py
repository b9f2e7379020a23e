"""Tile-size / blend-batch / column-cut autotuner.

For a resolution and scene size it times whole frames (preprocess + binning +
blend, CUDA events, after warm-up) for every tile size in {8, 16, 32}, blend
staging depth in {64, 128, 256} and binning with or without the per-column
cuts of the rectangles, on a few representative frames, keeps the fastest,
and caches the choice per (GPU name, width, height, N bucket) in a JSON file.
The image does not depend on the choice: every pixel walks the same
depth-ordered Gaussians with the same operations whatever the tiling.
"""
from __future__ import annotations

import json
import math
import os
from pathlib import Path

TILES = (8, 16, 32)
BATCHES = (64, 128, 256, 512)   # 512: 32-px tiles only
TRIMS = (False, True)


def default_cache_path() -> Path:
    base = os.environ.get("D4DGS_AUTOTUNE_CACHE")
    if base:
        return Path(base)
    return Path(os.environ.get("XDG_CACHE_HOME", str(Path.home() / ".cache"))) / "d4dgs" / "autotune.json"


def n_bucket(n: int) -> int:
    """Scene sizes are bucketed by powers of two."""
    return 1 << max(0, int(math.ceil(math.log2(max(n, 1)))))


def cache_key(gpu: str, width: int, height: int, n: int) -> str:
    return f"{gpu}|{width}x{height}|n<={n_bucket(n)}"


class TuneCache:
    def __init__(self, path: Path | None = None):
        self.path = Path(path) if path else default_cache_path()
        self.data = {}
        if self.path.exists():
            try:
                self.data = json.loads(self.path.read_text())
            except (OSError, ValueError):
                self.data = {}

    def get(self, key: str):
        e = self.data.get(key)
        return (int(e["tile"]), int(e["batch"]), bool(e.get("trim", False))) if e else None

    def put(self, key: str, tile: int, batch: int, trim: bool, table: dict):
        self.data[key] = {"tile": tile, "batch": batch, "trim": bool(trim), "ms": table}
        self.path.parent.mkdir(parents=True, exist_ok=True)
        tmp = self.path.with_suffix(f".{os.getpid()}.tmp")
        tmp.write_text(json.dumps(self.data, indent=1, sort_keys=True))
        os.replace(tmp, self.path)


def config_name(tile: int, batch: int, trim: bool) -> str:
    return f"{tile}/{batch}" + ("/cut" if trim else "")


def sweep(time_config, tiles=TILES, batches=BATCHES, trims=TRIMS):
    """time_config(tile, batch, trim) -> ms per frame, or None when the configuration cannot
    render these frames; returns (best (tile, batch, trim), {config_name: ms or None})."""
    table, cfgs = {}, {}
    for t in tiles:
        for b in batches:
            if b == 512 and t != 32:   # the library stages 512 at 32-px tiles only
                continue
            for c in trims:
                ms = time_config(t, b, c)
                name = config_name(t, b, c)
                table[name] = None if ms is None else float(ms)
                cfgs[name] = (int(t), int(b), bool(c))
    feasible = {k: v for k, v in table.items() if v is not None}
    if not feasible:
        raise RuntimeError("no tile / batch configuration can render these frames")
    return cfgs[min(feasible, key=feasible.get)], table


def time_frames(scene, frames, tile: int, batch: int, trim: bool = False, warmup: int = 2, reps: int = 2,
                device="cuda") -> float:
    """Mean ms per frame of d4dgs_render for one (tile, batch) over `frames` [(camera, t)];
    None when a frame has more (tile, Gaussian) pairs than a workspace can hold at this tile size.
    Each timed render follows an untimed render of the same frame, so the blend's tile order comes
    from that frame's own work, as it does from its predecessor's in an animation (the probe frames
    are far apart: timed one after another, each would take the order of an unrelated frame)."""
    import torch

    from . import D4DGS_ERR_CAPACITY, D4DGSError, Renderer, d4dgs_render
    cam0 = frames[0][0]
    r = Renderer(scene.n, cam0, tile=tile, batch=batch, device=device, trim=trim)
    try:
        for cam, t in frames:                  # size the workspace for these frames
            r.render(scene, cam, t)
    except D4DGSError as e:
        if e.code != D4DGS_ERR_CAPACITY:
            raise
        return None
    out = torch.empty((cam0.height, cam0.width, 3), dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device)
    for k in range(warmup):
        cam, t = frames[k % len(frames)]
        d4dgs_render(scene, cam, t, r.cfg, r.ws, out, stream)
    evs = []
    for _ in range(reps):
        for cam, t in frames:
            d4dgs_render(scene, cam, t, r.cfg, r.ws, out, stream)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            d4dgs_render(scene, cam, t, r.cfg, r.ws, out, stream)
            ev1.record(stream)
            evs.append((ev0, ev1))
    evs[-1][1].synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / len(evs)


def tune(scene, frames, cache: TuneCache | None = None, device="cuda", force: bool = False):
    """Best (tile, batch, trim) for this scene size and the frames' resolution (cached)."""
    import torch
    cam = frames[0][0]
    gpu = torch.cuda.get_device_name(device)
    key = cache_key(gpu, cam.width, cam.height, scene.n)
    cache = cache or TuneCache()
    hit = cache.get(key)
    if hit and not force:
        return hit, None
    best, table = sweep(lambda t, b, c: time_frames(scene, frames, t, b, c, device=device))
    cache.put(key, best[0], best[1], best[2], table)
    return best, table
