"""Tile-size / blend-batch autotuner.

For a resolution and scene size it times whole frames (preprocess + binning +
blend, CUDA events, after warm-up) for every tile size in {8, 16, 32} and
blend staging depth in {64, 128, 256} on a few representative frames, keeps
the fastest, and caches the choice per (GPU name, width, height, N bucket) in
a JSON file.  The image does not depend on the choice: every pixel walks the
same depth-ordered Gaussians with the same operations whatever the tiling.
"""
from __future__ import annotations

import json
import math
import os
from pathlib import Path

TILES = (8, 16, 32)
BATCHES = (64, 128, 256)


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
        return (int(e["tile"]), int(e["batch"])) if e else None

    def put(self, key: str, tile: int, batch: int, table: dict):
        self.data[key] = {"tile": tile, "batch": batch, "ms": table}
        self.path.parent.mkdir(parents=True, exist_ok=True)
        tmp = self.path.with_suffix(f".{os.getpid()}.tmp")
        tmp.write_text(json.dumps(self.data, indent=1, sort_keys=True))
        os.replace(tmp, self.path)


def sweep(time_config, tiles=TILES, batches=BATCHES):
    """time_config(tile, batch) -> ms per frame, or None when the configuration cannot render
    these frames; returns (best (tile, batch), {"tile/batch": ms or None})."""
    table = {}
    for t in tiles:
        for b in batches:
            ms = time_config(t, b)
            table[f"{t}/{b}"] = None if ms is None else float(ms)
    feasible = {k: v for k, v in table.items() if v is not None}
    if not feasible:
        raise RuntimeError("no tile / batch configuration can render these frames")
    best = min(feasible, key=feasible.get)
    t, b = best.split("/")
    return (int(t), int(b)), table


def time_frames(scene, frames, tile: int, batch: int, warmup: int = 2, reps: int = 1, device="cuda") -> float:
    """Mean ms per frame of d4dgs_render for one (tile, batch) over `frames` [(camera, t)];
    None when a frame has more (tile, Gaussian) pairs than a workspace can hold at this tile size."""
    import torch

    from . import D4DGS_ERR_CAPACITY, D4DGSError, Renderer, d4dgs_render
    cam0 = frames[0][0]
    r = Renderer(scene.n, cam0, tile=tile, batch=batch, device=device)
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
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        for cam, t in frames:
            d4dgs_render(scene, cam, t, r.cfg, r.ws, out, stream)
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / (reps * len(frames))


def tune(scene, frames, cache: TuneCache | None = None, device="cuda", force: bool = False):
    """Best (tile, batch) for this scene size and the frames' resolution (cached)."""
    import torch
    cam = frames[0][0]
    gpu = torch.cuda.get_device_name(device)
    key = cache_key(gpu, cam.width, cam.height, scene.n)
    cache = cache or TuneCache()
    hit = cache.get(key)
    if hit and not force:
        return hit, None
    best, table = sweep(lambda t, b: time_frames(scene, frames, t, b, device=device))
    cache.put(key, best[0], best[1], table)
    return best, table
