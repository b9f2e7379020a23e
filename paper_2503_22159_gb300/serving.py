"""Serving: render requests of mixed scene, camera, timestamp and resolution
against device-resident scenes, with continuous batching.

* Scenes stay resident on the device (DeviceScene).
* Admission by memory: each request needs a workspace of its class
  (scene, resolution); workspaces are pooled per class and allocated lazily
  under a byte budget, so a request waits until a slot of its class is free.
* Continuous batching: whenever one of the pipeline's streams is free, the
  queued requests that have a slot and share the head request's layout class
  (packed pairs, tile passes) form the next batch -- up to 32 views rendered
  by one launch of each kernel (d4dgs_render_batch, optionally replayed from a
  captured CUDA graph).  Requests that arrive while batches run on the GPU
  join the next batch; batches on the two streams overlap on the device.
* The per-frame loop renders the same trace one request at a time (FIFO),
  for comparison.

Latency = completion (observed by event query on the host) - arrival.
``on_done(request, image)`` is called when a request completes; the image's
buffer goes back to the pool when it returns, so it must finish reading it
(e.g. copy and synchronise) before returning.

Faults stay with the request that has them.  A request whose camera or time
is not finite (or whose size is out of range) is refused when it arrives
(status D4DGS_ERR_INVALID_ARG, ``on_done(request, None)``) and never joins a
batch, so the views around it render as they would alone.  A request whose
``cancelled`` flag is set is dropped while it waits, or, if it is already on
the GPU, its image is discarded when its batch retires (status
STATUS_CANCELLED, ``on_done(request, None)``); its workspace slot goes back
to the pool either way.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (D4DGS_ERR_CAPACITY, D4DGS_ERR_INVALID_ARG, D4DGS_OK, BatchRenderer, DeviceScene, config_struct, d4dgs_read_stats,
               d4dgs_render, d4dgs_workspace_bytes, d4dgs_workspace_layout)


# A request its caller cancelled (a serving status, not a library error code).
STATUS_CANCELLED = -100


@dataclass
class Request:
    rid: int
    scene: str
    cam: object
    t: float
    arrival: float                   # seconds from the start of the trace
    done: float = math.nan           # completion time (same clock)
    status: int = D4DGS_OK
    cancelled: bool = False          # set by the caller at any time

    @property
    def res(self):
        return (int(self.cam.width), int(self.cam.height))


@dataclass
class Slot:
    key: tuple
    ws: torch.Tensor
    out: torch.Tensor
    cap: int
    nbytes: int = 0


class WorkspacePool:
    """Workspaces per (scene, width, height), allocated lazily under a byte
    budget.  When a class needs room, idle slots of other classes are freed
    (oldest first); a request whose class can never fit is refused."""

    def __init__(self, cfg, scenes: dict, caps: dict, budget_bytes: int, device):
        self.cfg, self.scenes, self.caps, self.device = cfg, scenes, caps, device
        self.budget, self.used = int(budget_bytes), 0
        self.free = collections.defaultdict(list)
        self.count = collections.Counter()
        self.evicted = 0

    def _bytes(self, key, cam):
        n = self.scenes[key[0]].n
        return d4dgs_workspace_bytes(n, cam, self.cfg, self.caps[key]) + cam.width * cam.height * 12

    def _evict_one(self, keep_key) -> bool:
        for k, lst in self.free.items():
            if k != keep_key and lst:
                slot = lst.pop(0)
                self.used -= slot.nbytes
                self.evicted += 1
                del slot
                return True
        return False

    def acquire(self, key, cam):
        if self.free[key]:
            return self.free[key].pop()
        need = self._bytes(key, cam)
        if need > self.budget:
            raise MemoryError(f"a {key} workspace ({need / 2**30:.1f} GiB) exceeds the serving budget")
        while self.used + need > self.budget and self._evict_one(key):
            pass
        if self.used + need > self.budget:
            return None   # wait for an in-flight batch to release its slots
        n = self.scenes[key[0]].n
        nb = d4dgs_workspace_bytes(n, cam, self.cfg, self.caps[key])
        ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device=self.device)
        self.used += need
        self.count[key] += 1
        return Slot(key, ws, out, self.caps[key], need)

    def release(self, slot: "Slot"):
        self.free[slot.key].append(slot)

    def layout_class(self, key, cam):
        n = self.scenes[key[0]].n
        L = d4dgs_workspace_layout(n, cam, self.cfg, d4dgs_workspace_bytes(n, cam, self.cfg, 1024))
        return (L["packed"], L["tile_passes"])


def request_valid(r: Request) -> bool:
    """The checks the library's entry points make on a view (finite camera and time, image size
    1..16384, positive focal lengths), made on the host before the request joins a batch."""
    c = r.cam
    vals = list(np.asarray(c.R, np.float64).reshape(-1)) + list(np.asarray(c.T, np.float64).reshape(-1))
    vals += [c.fx, c.fy, c.cx, c.cy, r.t]
    return (all(math.isfinite(float(v)) for v in vals) and c.fx > 0 and c.fy > 0
            and 1 <= int(c.width) <= 16384 and 1 <= int(c.height) <= 16384)


def make_trace(scenes: dict, n_requests: int = 2000, rate_hz: float = 500.0, seed: int = 4,
               resolutions=((640, 480), (1352, 1014), (1920, 1080), (2704, 2028)), radius: float = 30.0):
    """Poisson arrivals; each request draws a scene, an orbit pose, t ~ U[0,1] and a resolution."""
    import synth
    rng = np.random.default_rng(seed)
    names = sorted(scenes)
    t_arr = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    reqs = []
    for i in range(n_requests):
        name = names[rng.integers(len(names))]
        w, h = resolutions[rng.integers(len(resolutions))]
        az, el = rng.uniform(0, 2 * math.pi), rng.uniform(-0.2, 0.2)
        pos = radius * np.array([math.cos(el) * math.sin(az), -math.sin(el), math.cos(el) * math.cos(az)])
        cam = synth.look_at(pos, np.zeros(3), w, h)
        reqs.append(Request(i, name, cam, float(np.float32(rng.uniform(0, 1))), float(t_arr[i])))
    return reqs


def calibrate_capacity(scenes: dict, requests, cfg, device, margin: float = 1.3, per_class: int = 6) -> dict:
    """Key capacity per (scene, resolution) class from renders of a few of its requests."""
    by_class = collections.defaultdict(list)
    for r in requests:
        by_class[(r.scene, *r.res)].append(r)
    caps = {}
    for key, rs in by_class.items():
        scene = scenes[key[0]]
        best = 1 << 16
        for r in rs[:per_class]:
            cap = 64 * scene.n
            while True:
                ws = torch.empty(d4dgs_workspace_bytes(scene.n, r.cam, cfg, cap), dtype=torch.uint8, device=device)
                out = torch.empty((r.cam.height, r.cam.width, 3), device=device)
                d4dgs_render(scene, r.cam, r.t, cfg, ws, out)
                st = d4dgs_read_stats(scene.n, r.cam, cfg, ws)
                del ws, out
                if st["status"] == D4DGS_ERR_CAPACITY:
                    cap = int(st["n_keys"] * 1.1) + 1024
                    continue
                best = max(best, int(st["n_keys"]))
                break
        caps[key] = min(int(best * margin) + 4096, (1 << 30) - 1)
    return caps


@dataclass
class ServeStats:
    mode: str
    n: int
    frames_per_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    batches: int = 0
    mean_batch: float = 0.0
    rerendered: int = 0
    extra: dict = field(default_factory=dict)

    def as_dict(self):
        return {k: v for k, v in self.__dict__.items()}


def _summary(mode, reqs, t_first, t_last, **kw):
    lat = np.array([(r.done - r.arrival) * 1e3 for r in reqs])
    return ServeStats(mode, len(reqs), len(reqs) / (t_last - t_first), float(np.percentile(lat, 50)),
                      float(np.percentile(lat, 99)), float(lat.mean()), **kw)


def _redo_overflow(r: Request, scene, cfg, device, slot: Slot):
    """A frame whose pairs overflowed its slot is rendered again alone with room for all of them."""
    st = d4dgs_read_stats(scene.n, r.cam, cfg, slot.ws)
    if st["status"] != D4DGS_ERR_CAPACITY:
        r.status = st["status"]
        return False
    ws = torch.empty(d4dgs_workspace_bytes(scene.n, r.cam, cfg, int(st["n_keys"] * 1.1) + 1024), dtype=torch.uint8,
                     device=device)
    d4dgs_render(scene, r.cam, r.t, cfg, ws, slot.out)
    torch.cuda.synchronize(device)
    r.status = d4dgs_read_stats(scene.n, r.cam, cfg, ws)["status"]
    return True


def serve_loop(scenes: dict, requests, cfg, caps: dict, device="cuda", realtime: bool = True,
               on_done=None) -> ServeStats:
    """Per-frame loop: requests in arrival order, one d4dgs_render each."""
    device = torch.device(device)
    pool = WorkspacePool(cfg, scenes, caps, 1 << 62, device)
    stream = torch.cuda.Stream(device)
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    redo = refused = cancelled = 0
    for r in reqs:
        if realtime:
            while time.perf_counter() - t0 < r.arrival:
                pass
        if r.cancelled or not request_valid(r):
            r.status = STATUS_CANCELLED if r.cancelled else D4DGS_ERR_INVALID_ARG
            cancelled += r.cancelled
            refused += not r.cancelled
            r.done = time.perf_counter() - t0
            if on_done:
                on_done(r, None)
            continue
        key = (r.scene, *r.res)
        slot = pool.acquire(key, r.cam)
        d4dgs_render(scenes[r.scene], r.cam, r.t, cfg, slot.ws, slot.out, stream)
        stream.synchronize()
        r.done = time.perf_counter() - t0
        st = d4dgs_read_stats(scenes[r.scene].n, r.cam, cfg, slot.ws, stream)
        if st["status"] != D4DGS_OK:
            redo += _redo_overflow(r, scenes[r.scene], cfg, device, slot)
            r.done = time.perf_counter() - t0
        if on_done:
            on_done(r, slot.out)
        pool.release(slot)
    t_first = min(r.arrival for r in reqs) if realtime else 0.0
    return _summary("per-frame loop", reqs, t_first, max(r.done for r in reqs), rerendered=redo,
                    extra={"refused": refused, "cancelled": cancelled})


def serve_batched(scenes: dict, requests, cfg, caps: dict, device="cuda", max_views: int = 16,
                  budget_bytes: int = 120 << 30, n_streams: int = 2, graph: bool = True,
                  realtime: bool = True, on_done=None, stall_s: float = 30.0, on_launch=None) -> ServeStats:
    """Continuous batching (see the module docstring).  ``on_launch(requests)`` is called with the
    requests of each batch right after it is launched."""
    device = torch.device(device)
    pool = WorkspacePool(cfg, scenes, caps, budget_bytes, device)
    br = BatchRenderer(cfg, device)
    streams = [torch.cuda.Stream(device) for _ in range(n_streams)]
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    queue: list[Request] = []
    inflight = []   # (stream index, event, [(request, slot)])
    busy = [False] * n_streams
    classes = {}
    nb, nviews_total, redo = 0, 0, 0
    refused = cancelled = 0
    total = len(pending)
    finished = 0
    t0 = time.perf_counter()
    last_progress = t0
    while finished < total:
        now = time.perf_counter() - t0
        if inflight or not queue:
            last_progress = time.perf_counter()
        elif time.perf_counter() - last_progress > stall_s:
            raise RuntimeError(f"serving made no progress for {stall_s} s with {len(queue)} queued requests")
        while pending and (not realtime or pending[0].arrival <= now):
            r = pending.popleft()
            if not request_valid(r):   # refused on arrival: it never joins a batch
                r.status = D4DGS_ERR_INVALID_ARG
                r.done = time.perf_counter() - t0
                refused += 1
                finished += 1
                if on_done:
                    on_done(r, None)
                continue
            queue.append(r)
        # requests cancelled while they wait leave the queue
        if any(r.cancelled for r in queue):
            for r in queue:
                if r.cancelled:
                    r.status = STATUS_CANCELLED
                    r.done = time.perf_counter() - t0
                    cancelled += 1
                    finished += 1
                    if on_done:
                        on_done(r, None)
            queue = [r for r in queue if not r.cancelled]
        # retire completed batches
        still = []
        for si, ev, items in inflight:
            if ev.query():
                tdone = time.perf_counter() - t0
                for r, slot in items:
                    r.done = tdone
                    if r.cancelled:   # cancelled while on the GPU: the image is discarded
                        r.status = STATUS_CANCELLED
                        cancelled += 1
                        if on_done:
                            on_done(r, None)
                        pool.release(slot)
                        finished += 1
                        continue
                    st = d4dgs_read_stats(scenes[r.scene].n, r.cam, cfg, slot.ws, streams[si])
                    if st["status"] != D4DGS_OK:
                        redo += _redo_overflow(r, scenes[r.scene], cfg, device, slot)
                        r.done = time.perf_counter() - t0
                    if on_done:
                        on_done(r, slot.out)
                    pool.release(slot)
                    finished += 1
                busy[si] = False
            else:
                still.append((si, ev, items))
        inflight = still
        # form and launch a batch on a free stream
        free = [i for i in range(n_streams) if not busy[i]]
        if free and queue:
            head_cls = None
            batch, rest = [], []
            for r in queue:
                key = (r.scene, *r.res)
                cls = classes.get(key)
                if cls is None:
                    cls = classes[key] = pool.layout_class(key, r.cam)
                if len(batch) < max_views and (head_cls is None or cls == head_cls):
                    slot = pool.acquire(key, r.cam)
                    if slot is not None:
                        head_cls = cls
                        batch.append((r, slot))
                        continue
                rest.append(r)
            queue = rest
            if batch:
                si = free[0]
                views = [(scenes[r.scene], r.cam, r.t, slot.ws, slot.out) for r, slot in batch]
                br.render(views, stream=streams[si], graph=graph)
                ev = torch.cuda.Event()
                ev.record(streams[si])
                inflight.append((si, ev, batch))
                busy[si] = True
                if on_launch:
                    on_launch([r for r, _ in batch])
                nb += 1
                nviews_total += len(batch)
                continue
        if not queue and not inflight and pending and realtime:
            # idle until the next arrival
            while time.perf_counter() - t0 < pending[0].arrival:
                pass
    reqs = sorted(requests, key=lambda r: r.rid)
    t_first = min(r.arrival for r in reqs) if realtime else 0.0
    return _summary("continuous batching" + (" + CUDA graphs" if graph else ""), reqs, t_first,
                    max(r.done for r in reqs), batches=nb, mean_batch=nviews_total / max(nb, 1), rerendered=redo,
                    extra={"workspace_gb": pool.used / 2**30, "evicted": pool.evicted, "refused": refused,
                           "cancelled": cancelled,
                           "slots": dict((f"{k[0]}@{k[1]}x{k[2]}", v) for k, v in pool.count.items())})
