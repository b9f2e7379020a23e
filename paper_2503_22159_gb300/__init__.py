"""GB300-native (sm_103a) renderer for disentangled 4D Gaussian splatting.

Thin Python binding over the C ABI of ``include/d4dgs.h`` (libd4dgs.so).
PyTorch provides device memory and the current CUDA stream; every step of the
frame runs in the library's own kernels.  The functions keep the C names:

    d4dgs_workspace_bytes, d4dgs_workspace_layout, d4dgs_preprocess,
    d4dgs_sort, d4dgs_blend, d4dgs_render, d4dgs_render_backward,
    d4dgs_read_stats, d4dgs_render_host, d4dgs_launches_per_frame

plus two conveniences: :class:`DeviceScene` (the scene's arrays as device
tensors) and :class:`Renderer` (workspace ownership and key-capacity sizing).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import (D4DGS_ERR_CAPACITY, D4DGS_ERR_CUDA, D4DGS_ERR_INVALID_ARG, D4DGS_ERR_TIMEOUT,
                   D4DGS_ERR_WORKSPACE_TOO_SMALL, D4DGS_OK, D4DGSError)

SCENE_FIELDS = ("means", "t_mean", "velocity", "log_scales", "log_t_scale", "quats", "opacity_logit", "sh")

__all__ = ["DeviceScene", "Renderer", "BatchRenderer", "camera_struct", "config_struct", "d4dgs_workspace_bytes",
           "d4dgs_workspace_layout", "d4dgs_preprocess", "d4dgs_sort", "d4dgs_blend", "d4dgs_blend_profile",
           "DeviceScene4D", "d4dgs_preprocess_slicing", "d4dgs_render_slicing",
           "d4dgs_render_flow", "d4dgs_render_backward_flow", "d4dgs_flow_loss", "d4dgs_split_accumulate",
           "d4dgs_split",
           "d4dgs_render",
           "d4dgs_render_backward", "d4dgs_read_stats", "d4dgs_render_host", "d4dgs_render_host_async",
           "d4dgs_launches_per_frame", "d4dgs_render_backward_accumulate", "d4dgs_l1_loss", "LaunchTimer",
           "D4DGSError", "D4DGS_OK", "D4DGS_ERR_CAPACITY", "D4DGS_ERR_TIMEOUT", "D4DGS_ERR_INVALID_ARG",
           "D4DGS_ERR_WORKSPACE_TOO_SMALL", "D4DGS_ERR_CUDA"]


def _stream_handle(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


class DeviceScene:
    """The raw parameters of one scene as contiguous float32 device tensors."""

    def __init__(self, tensors: dict, sh_degree: int):
        self.t = {k: tensors[k] for k in SCENE_FIELDS}
        self.sh_degree = int(sh_degree)
        self.n = int(self.t["means"].shape[0])
        for k, v in self.t.items():
            if v.dtype != torch.float32 or not v.is_contiguous() or not v.is_cuda:
                raise ValueError(f"scene field {k} must be a contiguous float32 CUDA tensor")

    @classmethod
    def from_host(cls, scene, device="cuda") -> "DeviceScene":
        """From any object with the SCENE_FIELDS arrays (e.g. synth.Scene)."""
        t = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), dtype=np.float32)).to(device)
             for k in SCENE_FIELDS}
        return cls(t, scene.sh_degree)

    def struct(self) -> _abi.d4dgs_scene:
        s = _abi.d4dgs_scene(*[self.t[k].data_ptr() for k in SCENE_FIELDS], self.n, self.sh_degree)
        return s

    def zeros_like_grad(self) -> dict:
        return {k: torch.zeros_like(v) for k, v in self.t.items()}


SCENE4D_FIELDS = ("means4", "log_scales4", "quat_l", "quat_r", "opacity_logit", "sh")


class DeviceScene4D:
    """A slicing-first scene (4D means, 4D log-scales, rotation quaternion pair) on the device."""

    def __init__(self, tensors: dict, sh_degree: int):
        self.t = {k: tensors[k] for k in SCENE4D_FIELDS}
        self.sh_degree = int(sh_degree)
        self.n = int(self.t["means4"].shape[0])
        for k, v in self.t.items():
            if v.dtype != torch.float32 or not v.is_contiguous() or not v.is_cuda:
                raise ValueError(f"scene field {k} must be a contiguous float32 CUDA tensor")

    @classmethod
    def from_host(cls, scene, device="cuda") -> "DeviceScene4D":
        t = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), dtype=np.float32)).to(device)
             for k in SCENE4D_FIELDS}
        return cls(t, scene.sh_degree)

    def struct(self) -> _abi.d4dgs_scene4d:
        return _abi.d4dgs_scene4d(*[self.t[k].data_ptr() for k in SCENE4D_FIELDS], self.n, self.sh_degree)


def d4dgs_preprocess_slicing(scene: DeviceScene4D, cam, t: float, cfg, ws: torch.Tensor, stream=None):
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_preprocess_slicing(ctypes.byref(scene.struct()), ctypes.byref(camera_struct(cam)),
                                                    float(t), ctypes.byref(cfg), p, nb, _stream_handle(stream)),
               "d4dgs_preprocess_slicing")


def d4dgs_render_slicing(scene: DeviceScene4D, cam, t: float, cfg, ws: torch.Tensor, out: torch.Tensor, stream=None):
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_render_slicing(ctypes.byref(scene.struct()), ctypes.byref(camera_struct(cam)),
                                                float(t), ctypes.byref(cfg), p, nb, ctypes.c_void_p(out.data_ptr()),
                                                _stream_handle(stream)), "d4dgs_render_slicing")


def camera_struct(cam) -> _abi.d4dgs_camera:
    c = _abi.d4dgs_camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).reshape(9)]
    c.T[:] = [float(x) for x in np.asarray(cam.T, np.float32).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def config_struct(tile: int = 16, batch: int = 256, bg=(0.0, 0.0, 0.0), trim: bool = False, near: float = 0.2,
                  spin_limit: int = 0, colour_cache: bool = False, binning: int = 0) -> _abi.d4dgs_config:
    """binning: 0 the library's choice (column), 1 column buckets + row passes, 2 straight into the
    tiles' lists (<= 2048 tiles), 3 depth ranks into the tiles' ranges, each list read back in depth
    order from a bitmap."""
    g = _abi.d4dgs_config()
    g.tile, g.batch = int(tile), int(batch)
    g.bg[:] = [float(x) for x in bg]
    g.trim = 1 if trim else 0
    g.near = float(near)
    g.spin_limit = int(spin_limit)
    g.colour_cache = 1 if colour_cache else 0
    g.binning = int(binning)
    return g


def d4dgs_workspace_bytes(n: int, cam, cfg, key_capacity: int) -> int:
    b = _abi.load().d4dgs_workspace_bytes(int(n), ctypes.byref(camera_struct(cam)), ctypes.byref(cfg),
                                          int(key_capacity))
    if b == 0:
        raise D4DGSError(D4DGS_ERR_INVALID_ARG, "d4dgs_workspace_bytes")
    return int(b)


def d4dgs_workspace_layout(n: int, cam, cfg, ws_bytes: int) -> dict:
    L = _abi.d4dgs_layout()
    _abi.check(_abi.load().d4dgs_workspace_layout(int(n), ctypes.byref(camera_struct(cam)), ctypes.byref(cfg),
                                                  int(ws_bytes), ctypes.byref(L)), "d4dgs_workspace_layout")
    return {k: getattr(L, k) for k, _ in L._fields_}


def _ws(ws: torch.Tensor):
    if ws.dtype != torch.uint8 or not ws.is_cuda or not ws.is_contiguous():
        raise ValueError("workspace must be a contiguous uint8 CUDA tensor")
    return ctypes.c_void_p(ws.data_ptr()), ws.numel()


def d4dgs_preprocess(scene: DeviceScene, cam, t: float, cfg, ws: torch.Tensor, stream=None):
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_preprocess(ctypes.byref(scene.struct()), ctypes.byref(camera_struct(cam)),
                                            float(t), ctypes.byref(cfg), p, nb, _stream_handle(stream)),
               "d4dgs_preprocess")


def d4dgs_sort(n: int, cam, cfg, ws: torch.Tensor, stream=None):
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_sort(int(n), ctypes.byref(camera_struct(cam)), ctypes.byref(cfg), p, nb,
                                      _stream_handle(stream)), "d4dgs_sort")


def d4dgs_blend(n: int, cam, cfg, ws: torch.Tensor, out: torch.Tensor, stream=None):
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_blend(int(n), ctypes.byref(camera_struct(cam)), ctypes.byref(cfg), p, nb,
                                       ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "d4dgs_blend")


def d4dgs_blend_profile(n: int, cam, cfg, ws: torch.Tensor, out: torch.Tensor, counts: torch.Tensor, stream=None):
    """Instrumented blend: also totals the evaluated and blended (pixel, Gaussian) pairs and the
    plain tile algorithm's pair count into ``counts`` (a 3-element int64 CUDA tensor)."""
    if counts.numel() < 3 or counts.dtype != torch.int64 or not counts.is_cuda:
        raise ValueError("counts must be a CUDA int64 tensor with at least 3 elements")
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_blend_profile(int(n), ctypes.byref(camera_struct(cam)), ctypes.byref(cfg), p, nb,
                                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(counts.data_ptr()),
                                               _stream_handle(stream)), "d4dgs_blend_profile")


def d4dgs_render(scene: DeviceScene, cam, t: float, cfg, ws: torch.Tensor, out: torch.Tensor, stream=None):
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_render(ctypes.byref(scene.struct()), ctypes.byref(camera_struct(cam)), float(t),
                                        ctypes.byref(cfg), p, nb, ctypes.c_void_p(out.data_ptr()),
                                        _stream_handle(stream)), "d4dgs_render")


def d4dgs_render_backward(scene: DeviceScene, cam, t: float, cfg, ws: torch.Tensor, dl_drgb: torch.Tensor,
                          grads: dict, stream=None):
    p, nb = _ws(ws)
    g = _abi.d4dgs_scene_grad(*[grads[k].data_ptr() for k in SCENE_FIELDS])
    _abi.check(_abi.load().d4dgs_render_backward(ctypes.byref(scene.struct()), ctypes.byref(camera_struct(cam)),
                                                 float(t), ctypes.byref(cfg), p, nb,
                                                 ctypes.c_void_p(dl_drgb.data_ptr()), ctypes.byref(g),
                                                 _stream_handle(stream)), "d4dgs_render_backward")


def d4dgs_render_backward_accumulate(scene: DeviceScene, cam, t: float, cfg, ws: torch.Tensor,
                                     dl_drgb: torch.Tensor, grads: dict, stream=None):
    """d4dgs_render_backward adding into `grads` (a step over several views)."""
    p, nb = _ws(ws)
    g = _abi.d4dgs_scene_grad(*[grads[k].data_ptr() for k in SCENE_FIELDS])
    _abi.check(_abi.load().d4dgs_render_backward_accumulate(
        ctypes.byref(scene.struct()), ctypes.byref(camera_struct(cam)), float(t), ctypes.byref(cfg), p, nb,
        ctypes.c_void_p(dl_drgb.data_ptr()), ctypes.byref(g), _stream_handle(stream)),
        "d4dgs_render_backward_accumulate")


def d4dgs_l1_loss(img: torch.Tensor, target: torch.Tensor, scale: float, dl_dimg: torch.Tensor,
                  loss: torch.Tensor, stream=None):
    """loss (one device float) += scale * sum |img - target|; dl_dimg = scale * sign(img - target)."""
    for x in (img, target, dl_dimg):
        if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
            raise ValueError("d4dgs_l1_loss takes contiguous float32 CUDA tensors")
    if img.numel() != target.numel() or img.numel() != dl_dimg.numel() or loss.numel() < 1:
        raise ValueError("d4dgs_l1_loss: sizes differ")
    _abi.check(_abi.load().d4dgs_l1_loss(ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                         int(img.numel()), float(scale), ctypes.c_void_p(dl_dimg.data_ptr()),
                                         ctypes.c_void_p(loss.data_ptr()), _stream_handle(stream)), "d4dgs_l1_loss")


class LaunchTimer:
    """Per-launch device times of the library calls made inside ``with`` on this host thread:
    ``times_ms()`` after the stream has been synchronised (d4dgs_launch_timer)."""

    def __init__(self, stream=None, max_launches: int = 64):
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self.events = [torch.cuda.Event(enable_timing=True) for _ in range(max_launches + 1)]
        for e in self.events:        # creates the underlying events
            e.record(self.stream)
        self.count = 0

    def __enter__(self):
        arr = (ctypes.c_void_p * (len(self.events) - 1))(*[e.cuda_event for e in self.events[1:]])
        self._arr = arr
        self.events[0].record(self.stream)
        _abi.check(_abi.load().d4dgs_launch_timer(arr, len(arr)), "d4dgs_launch_timer")
        return self

    def __exit__(self, *exc):
        self.count = int(_abi.load().d4dgs_launch_timer_stop())
        return False

    def times_ms(self):
        return [self.events[i].elapsed_time(self.events[i + 1]) for i in range(self.count)]


def d4dgs_render_flow(scene: DeviceScene, cam, t: float, cfg, ws: torch.Tensor, out: torch.Tensor,
                      out_flow: torch.Tensor, stream=None):
    """Render the image and the optical-flow channel (H x W x 2, pixels per unit time)."""
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_render_flow(ctypes.byref(scene.struct()), ctypes.byref(camera_struct(cam)), float(t),
                                             ctypes.byref(cfg), p, nb, ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(out_flow.data_ptr()), _stream_handle(stream)),
               "d4dgs_render_flow")


def d4dgs_render_backward_flow(scene: DeviceScene, cam, t: float, cfg, ws: torch.Tensor, dl_drgb: torch.Tensor,
                               dl_dflow: torch.Tensor, grads: dict, stream=None):
    p, nb = _ws(ws)
    g = _abi.d4dgs_scene_grad(*[grads[k].data_ptr() for k in SCENE_FIELDS])
    _abi.check(_abi.load().d4dgs_render_backward_flow(ctypes.byref(scene.struct()), ctypes.byref(camera_struct(cam)),
                                                      float(t), ctypes.byref(cfg), p, nb,
                                                      ctypes.c_void_p(dl_drgb.data_ptr()),
                                                      ctypes.c_void_p(dl_dflow.data_ptr()), ctypes.byref(g),
                                                      _stream_handle(stream)), "d4dgs_render_backward_flow")


def d4dgs_flow_loss(rgb: torch.Tensor, flow: torch.Tensor, lam: float = 1.0, eps: float = 1e-6,
                    dl_dflow: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Flow-gradient consistency loss (a 1-element device tensor); fills dl_dflow when given."""
    H, W = int(rgb.shape[0]), int(rgb.shape[1])
    lib = _abi.load()
    scratch = torch.empty(int(lib.d4dgs_flow_loss_scratch_bytes(W, H)), dtype=torch.uint8, device=rgb.device)
    loss = torch.empty(1, dtype=torch.float32, device=rgb.device)
    _abi.check(lib.d4dgs_flow_loss(ctypes.c_void_p(rgb.data_ptr()), ctypes.c_void_p(flow.data_ptr()), W, H,
                                   float(lam), float(eps), ctypes.c_void_p(scratch.data_ptr()), scratch.numel(),
                                   ctypes.c_void_p(loss.data_ptr()),
                                   ctypes.c_void_p(dl_dflow.data_ptr()) if dl_dflow is not None else None,
                                   _stream_handle(stream)), "d4dgs_flow_loss")
    return loss


def d4dgs_split_accumulate(grads: dict, stats: torch.Tensor, stream=None):
    """Add |dL/d mean|, |dL/d t_mean| and 1 to stats (N x 3) for Gaussians with a nonzero gradient."""
    n = int(grads["means"].shape[0])
    g = _abi.d4dgs_scene_grad(*[grads[k].data_ptr() for k in SCENE_FIELDS])
    _abi.check(_abi.load().d4dgs_split_accumulate(ctypes.byref(g), n, ctypes.c_void_p(stats.data_ptr()),
                                                  _stream_handle(stream)), "d4dgs_split_accumulate")


def d4dgs_split(scene: DeviceScene, stats: torch.Tensor, normals: torch.Tensor, tau_xyz: float, tau_t: float,
                log_min_xyz: float, log_min_t: float, factor: float = 1.6, stream=None):
    """Temporal / spatial splitting: returns (the new scene, its Gaussian count) -- the scene's tensors
    have room for 2N Gaussians, the first `count` are valid (the count is read back)."""
    n, dev = scene.n, scene.t["means"].device
    cap = max(2 * n, 1)
    K = (scene.sh_degree + 1) ** 2
    shapes = {"means": (cap, 3), "t_mean": (cap,), "velocity": (cap, 3), "log_scales": (cap, 3),
              "log_t_scale": (cap,), "quats": (cap, 4), "opacity_logit": (cap,), "sh": (cap, K, 3)}
    out = {k: torch.empty(v, dtype=torch.float32, device=dev) for k, v in shapes.items()}
    g = _abi.d4dgs_scene_grad(*[out[k].data_ptr() for k in SCENE_FIELDS])
    lib = _abi.load()
    scratch = torch.empty(max(int(lib.d4dgs_split_scratch_bytes(n)), 4), dtype=torch.uint8, device=dev)
    out_n = torch.zeros(1, dtype=torch.int32, device=dev)
    prm = _abi.d4dgs_split_params(float(tau_xyz), float(tau_t), float(log_min_xyz), float(log_min_t), float(factor))
    _abi.check(lib.d4dgs_split(ctypes.byref(scene.struct()), ctypes.c_void_p(stats.data_ptr()),
                               ctypes.c_void_p(normals.data_ptr()), ctypes.byref(prm), ctypes.byref(g), cap,
                               ctypes.c_void_p(out_n.data_ptr()), ctypes.c_void_p(scratch.data_ptr()), scratch.numel(),
                               _stream_handle(stream)), "d4dgs_split")
    m = int(out_n.item())
    return DeviceScene({k: v[:m] for k, v in out.items()}, scene.sh_degree), m


def d4dgs_read_stats(n: int, cam, cfg, ws: torch.Tensor, stream=None) -> dict:
    p, nb = _ws(ws)
    s = _abi.d4dgs_stats()
    _abi.load().d4dgs_read_stats(int(n), ctypes.byref(camera_struct(cam)), ctypes.byref(cfg), p, nb,
                                 ctypes.byref(s), _stream_handle(stream))
    return {k: getattr(s, k) for k, _ in s._fields_}


def d4dgs_scene_bytes(n: int, sh_degree: int) -> int:
    return int(_abi.load().d4dgs_scene_bytes(int(n), int(sh_degree)))


def d4dgs_render_host(host_scene, cam, t: float, cfg, dev_scene_buf: torch.Tensor, ws: torch.Tensor,
                      dev_rgb: torch.Tensor, out_host: torch.Tensor, stream=None):
    """Render from HOST scene arrays (torch CPU tensors, ideally pinned) into a host image; the
    host->device copies, the frame and the device->host copy all run inside the call."""
    s = _abi.d4dgs_scene(*[host_scene[k].data_ptr() for k in SCENE_FIELDS], int(host_scene["means"].shape[0]),
                         int(host_scene["sh_degree"]))
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_render_host(ctypes.byref(s), ctypes.byref(camera_struct(cam)), float(t),
                                             ctypes.byref(cfg), ctypes.c_void_p(dev_scene_buf.data_ptr()),
                                             dev_scene_buf.numel(), p, nb, ctypes.c_void_p(dev_rgb.data_ptr()),
                                             ctypes.c_void_p(out_host.data_ptr()), _stream_handle(stream)),
               "d4dgs_render_host")


def d4dgs_render_host_async(host_scene, cam, t: float, cfg, dev_scene_buf: torch.Tensor, ws: torch.Tensor,
                            dev_rgb: torch.Tensor, out_host: torch.Tensor, stream=None):
    """d4dgs_render_host queued on `stream` without waiting: out_host holds the image once the
    stream has passed this point; the host and device buffers belong to the call until then."""
    s = _abi.d4dgs_scene(*[host_scene[k].data_ptr() for k in SCENE_FIELDS], int(host_scene["means"].shape[0]),
                         int(host_scene["sh_degree"]))
    p, nb = _ws(ws)
    _abi.check(_abi.load().d4dgs_render_host_async(ctypes.byref(s), ctypes.byref(camera_struct(cam)), float(t),
                                                   ctypes.byref(cfg), ctypes.c_void_p(dev_scene_buf.data_ptr()),
                                                   dev_scene_buf.numel(), p, nb, ctypes.c_void_p(dev_rgb.data_ptr()),
                                                   ctypes.c_void_p(out_host.data_ptr()), _stream_handle(stream)),
               "d4dgs_render_host_async")


def d4dgs_launches_per_frame(n: int, cam, cfg) -> int:
    return int(_abi.load().d4dgs_launches_per_frame(int(n), ctypes.byref(camera_struct(cam)), ctypes.byref(cfg)))


class BatchRenderer:
    """Renders up to 32 views with one launch per kernel (d4dgs_render_batch).

    Views share the config and the layout class (packed pairs, tile passes).
    ``graph=True`` captures the launch sequence once per stream as a CUDA
    graph whose first node copies the freshly encoded descriptors (pinned host
    buffer -> device) before the kernels run, so one graph serves every batch
    of its class."""

    def __init__(self, cfg, device="cuda"):
        lib = _abi.load()
        self.cfg, self.device = cfg, torch.device(device)
        self.args_bytes = int(lib.d4dgs_batch_args_bytes())
        self.area_bytes = int(lib.d4dgs_batch_area_bytes())
        self._graphs = {}
        self._slots = {}

    def _slot(self, stream):
        key = int(stream.cuda_stream)
        if key not in self._slots:
            self._slots[key] = dict(
                area=torch.empty(self.area_bytes, dtype=torch.uint8, device=self.device),
                host=torch.empty(self.args_bytes, dtype=torch.uint8).pin_memory(),
                dev=torch.empty(self.args_bytes, dtype=torch.uint8, device=self.device))
        return self._slots[key]

    def encode(self, views, host: torch.Tensor):
        """views: list of (DeviceScene, camera, t, workspace tensor, output tensor)."""
        n = len(views)
        arr = (_abi.d4dgs_view * n)()
        keep = []
        for i, (scene, cam, t, ws, out) in enumerate(views):
            st = scene.struct()
            keep.append(st)
            arr[i].scene = ctypes.addressof(st)
            arr[i].cam = camera_struct(cam)
            arr[i].t = float(t)
            arr[i].ws = ws.data_ptr()
            arr[i].ws_bytes = ws.numel()
            arr[i].out_rgb = out.data_ptr()
        _abi.check(_abi.load().d4dgs_batch_encode(n, arr, ctypes.byref(self.cfg), ctypes.c_void_p(host.data_ptr()),
                                                  self.args_bytes), "d4dgs_batch_encode")

    def render_stages(self, views, stages: int, stream=None):
        """Launch some stages of an eager batch render (1 = preprocess, 2 = binning, 4 = blend; in that
        order, on one stream): a profiling hook."""
        stream = torch.cuda.current_stream(self.device) if stream is None else stream
        slot = self._slot(stream)
        host = slot.setdefault("stage_host", torch.empty(self.args_bytes, dtype=torch.uint8))
        if stages & 1:
            self.encode(views, host)
        _abi.check(_abi.load().d4dgs_render_batch_stages(ctypes.c_void_p(host.data_ptr()), None,
                                                         ctypes.c_void_p(slot["area"].data_ptr()), self.area_bytes,
                                                         int(stages), _stream_handle(stream)),
                   "d4dgs_render_batch_stages")

    def render(self, views, stream=None, graph: bool = False):
        stream = torch.cuda.current_stream(self.device) if stream is None else stream
        slot = self._slot(stream)
        if not graph:
            host = torch.empty(self.args_bytes, dtype=torch.uint8)
            self.encode(views, host)
            _abi.check(_abi.load().d4dgs_render_batch(ctypes.c_void_p(host.data_ptr()), None,
                                                      ctypes.c_void_p(slot["area"].data_ptr()), self.area_bytes,
                                                      _stream_handle(stream)), "d4dgs_render_batch")
            return
        # graph mode: the pinned host copy must not change while an earlier replay may still read it
        if "event" in slot:
            slot["event"].synchronize()
        self.encode(views, slot["host"])
        key = (int(stream.cuda_stream), self._class_key(slot["host"]))
        g = self._graphs.get(key)
        if g is None:
            # one eager launch first: the library's one-time queries must not run under capture
            _abi.check(_abi.load().d4dgs_render_batch(ctypes.c_void_p(slot["host"].data_ptr()), None,
                                                      ctypes.c_void_p(slot["area"].data_ptr()), self.area_bytes,
                                                      _stream_handle(stream)), "d4dgs_render_batch")
            stream.synchronize()
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream(self.device)
            side.wait_stream(stream)
            with torch.cuda.graph(g, stream=side):
                slot["dev"].copy_(slot["host"], non_blocking=True)
                _abi.check(_abi.load().d4dgs_render_batch(ctypes.c_void_p(slot["host"].data_ptr()),
                                                          ctypes.c_void_p(slot["dev"].data_ptr()),
                                                          ctypes.c_void_p(slot["area"].data_ptr()), self.area_bytes,
                                                          _stream_handle(side)), "d4dgs_render_batch")
            stream.wait_stream(side)
            self._graphs[key] = g
        with torch.cuda.stream(stream):
            g.replay()
        ev = torch.cuda.Event()
        ev.record(stream)
        slot["event"] = ev

    @staticmethod
    def _class_key(host: torch.Tensor):
        # nviews, tile, batch, packed, tile_passes, column capacity, trim, tile and grid-cell capacities
        # (leading int32 fields of the encoded batch)
        head = host[:36].view(torch.int32).tolist()
        return tuple(head[1:9])


class Renderer:
    """Owns a workspace for (N, camera size, tile, batch) and grows its key
    capacity when a frame reports D4DGS_ERR_CAPACITY."""

    def __init__(self, n: int, cam, tile: int = 16, batch: int = 256, bg=(0.0, 0.0, 0.0),
                 key_capacity: int | None = None, device="cuda", trim: bool = False, near: float = 0.2,
                 binning: int = 0):
        self.n, self.device = int(n), torch.device(device)
        self.cfg = config_struct(tile, batch, bg, trim, near, binning=binning)
        self.width, self.height = int(cam.width), int(cam.height)
        self.cam0 = cam
        cap = key_capacity if key_capacity is not None else max(1 << 16, 16 * self.n)
        self._alloc(cap)

    def _alloc(self, cap: int):
        self.key_capacity = int(min(cap, (1 << 30) - 1))
        nbytes = d4dgs_workspace_bytes(self.n, self.cam0, self.cfg, self.key_capacity)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def layout(self, cam=None) -> dict:
        return d4dgs_workspace_layout(self.n, cam or self.cam0, self.cfg, self.ws.numel())

    def render(self, scene: DeviceScene, cam, t: float, out: torch.Tensor | None = None, check: bool = True,
               stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device=self.device)
        for _ in range(8):
            d4dgs_render(scene, cam, t, self.cfg, self.ws, out, stream)
            if not check:
                return out
            st = d4dgs_read_stats(self.n, cam, self.cfg, self.ws, stream)
            if st["status"] == D4DGS_ERR_CAPACITY:
                if self.key_capacity >= (1 << 30) - 1:   # the largest capacity the workspace format allows
                    break
                self._alloc(int(st["n_keys"] * 1.25) + 1024)
                continue
            if st["status"] != D4DGS_OK:
                raise D4DGSError(st["status"], "render")
            return out
        raise D4DGSError(D4DGS_ERR_CAPACITY, "render")

    def stats(self, cam=None, stream=None) -> dict:
        return d4dgs_read_stats(self.n, cam or self.cam0, self.cfg, self.ws, stream)

    def view(self, name: str, dtype, count: int, cam=None) -> torch.Tensor:
        """A typed view of one workspace buffer (test and profiling hook)."""
        off = self.layout(cam)[name]
        itemsize = torch.empty((), dtype=dtype).element_size()
        return self.ws[off: off + count * itemsize].view(dtype)
