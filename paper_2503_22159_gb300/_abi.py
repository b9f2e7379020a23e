"""ctypes view of include/d4dgs.h and the loader of the in-tree libd4dgs.so.

The library is the only compute path: if it has not been built this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_HERE = Path(__file__).resolve().parent
LIB_PATH = _HERE / "_build" / "libd4dgs.so"

D4DGS_OK = 0
D4DGS_ERR_INVALID_ARG = -1
D4DGS_ERR_WORKSPACE_TOO_SMALL = -2
D4DGS_ERR_CAPACITY = -3
D4DGS_ERR_TIMEOUT = -4
D4DGS_ERR_CUDA = -5

_fp = ctypes.POINTER(ctypes.c_float)


class d4dgs_scene(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("means", "t_mean", "velocity", "log_scales", "log_t_scale",
                                                "quats", "opacity_logit", "sh")] + [
        ("n", ctypes.c_int32), ("sh_degree", ctypes.c_int32)]


class d4dgs_scene4d(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("means4", "log_scales4", "quat_l", "quat_r", "opacity_logit",
                                                "sh")] + [("n", ctypes.c_int32), ("sh_degree", ctypes.c_int32)]


class d4dgs_split_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("tau_xyz", "tau_t", "log_min_xyz", "log_min_t", "factor")]


class d4dgs_scene_grad(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("means", "t_mean", "velocity", "log_scales", "log_t_scale",
                                                "quats", "opacity_logit", "sh")]


class d4dgs_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("T", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class d4dgs_config(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("batch", ctypes.c_int32), ("bg", ctypes.c_float * 3),
                ("trim", ctypes.c_int32), ("near", ctypes.c_float), ("spin_limit", ctypes.c_uint32),
                ("colour_cache", ctypes.c_int32),
                ("binning", ctypes.c_int32)]


class d4dgs_view(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("cam", d4dgs_camera), ("t", ctypes.c_float), ("ws", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t), ("out_rgb", ctypes.c_void_p)]


class d4dgs_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_keys", ctypes.c_int64), ("key_capacity", ctypes.c_int64),
                ("n_visible", ctypes.c_int64)]


class d4dgs_layout(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("records", "depth_keys", "tiles_touched", "rect", "depth_order",
                                               "tile_keys", "tile_vals", "ranges", "final_T", "n_contrib",
                                               "control", "key_capacity")] + [
        ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32), ("depth_passes", ctypes.c_int32),
        ("tile_passes", ctypes.c_int32), ("id_bits", ctypes.c_int32), ("packed", ctypes.c_int32),
        ("col_bits", ctypes.c_int32), ("trims", ctypes.c_int64), ("tile_order", ctypes.c_int64)]


# name -> (restype, argtypes); the exported symbols of include/d4dgs.h
_P = ctypes.POINTER
_vp = ctypes.c_void_p
PROTOTYPES = {
    "d4dgs_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, _P(d4dgs_camera), _P(d4dgs_config), ctypes.c_int64]),
    "d4dgs_workspace_layout": (ctypes.c_int, [ctypes.c_int32, _P(d4dgs_camera), _P(d4dgs_config), ctypes.c_size_t,
                                              _P(d4dgs_layout)]),
    "d4dgs_preprocess": (ctypes.c_int, [_P(d4dgs_scene), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config), _vp,
                                        ctypes.c_size_t, _vp]),
    "d4dgs_sort": (ctypes.c_int, [ctypes.c_int32, _P(d4dgs_camera), _P(d4dgs_config), _vp, ctypes.c_size_t, _vp]),
    "d4dgs_blend": (ctypes.c_int, [ctypes.c_int32, _P(d4dgs_camera), _P(d4dgs_config), _vp, ctypes.c_size_t, _vp,
                                   _vp]),
    "d4dgs_blend_profile": (ctypes.c_int, [ctypes.c_int32, _P(d4dgs_camera), _P(d4dgs_config), _vp,
                                           ctypes.c_size_t, _vp, _vp, _vp]),
    "d4dgs_render": (ctypes.c_int, [_P(d4dgs_scene), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config), _vp,
                                    ctypes.c_size_t, _vp, _vp]),
    "d4dgs_render_backward": (ctypes.c_int, [_P(d4dgs_scene), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config),
                                             _vp, ctypes.c_size_t, _vp, _P(d4dgs_scene_grad), _vp]),
    "d4dgs_render_backward_accumulate": (ctypes.c_int, [_P(d4dgs_scene), _P(d4dgs_camera), ctypes.c_float,
                                                        _P(d4dgs_config), _vp, ctypes.c_size_t, _vp,
                                                        _P(d4dgs_scene_grad), _vp]),
    "d4dgs_l1_loss": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_float, _vp, _vp, _vp]),
    "d4dgs_launch_timer": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32]),
    "d4dgs_launch_timer_stop": (ctypes.c_int32, []),
    "d4dgs_read_stats": (ctypes.c_int, [ctypes.c_int32, _P(d4dgs_camera), _P(d4dgs_config), _vp, ctypes.c_size_t,
                                        _P(d4dgs_stats), _vp]),
    "d4dgs_scene_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "d4dgs_render_host": (ctypes.c_int, [_P(d4dgs_scene), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config), _vp,
                                         ctypes.c_size_t, _vp, ctypes.c_size_t, _vp, _vp, _vp]),
    "d4dgs_render_host_async": (ctypes.c_int, [_P(d4dgs_scene), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config), _vp,
                                         ctypes.c_size_t, _vp, ctypes.c_size_t, _vp, _vp, _vp]),
    "d4dgs_render_static": (ctypes.c_int, [_P(d4dgs_scene), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config),
                                           _vp, _P(d4dgs_stats), _vp]),
    "d4dgs_batch_args_bytes": (ctypes.c_size_t, []),
    "d4dgs_batch_area_bytes": (ctypes.c_size_t, []),
    "d4dgs_batch_encode": (ctypes.c_int, [ctypes.c_int32, _P(d4dgs_view), _P(d4dgs_config), _vp, ctypes.c_size_t]),
    "d4dgs_render_batch": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "d4dgs_split_accumulate": (ctypes.c_int, [_P(d4dgs_scene_grad), ctypes.c_int32, _vp, _vp]),
    "d4dgs_split_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int32]),
    "d4dgs_split": (ctypes.c_int, [_P(d4dgs_scene), _vp, _vp, _P(d4dgs_split_params), _P(d4dgs_scene_grad),
                                   ctypes.c_int32, _vp, _vp, ctypes.c_size_t, _vp]),
    "d4dgs_render_flow": (ctypes.c_int, [_P(d4dgs_scene), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config), _vp,
                                         ctypes.c_size_t, _vp, _vp, _vp]),
    "d4dgs_render_backward_flow": (ctypes.c_int, [_P(d4dgs_scene), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config),
                                                  _vp, ctypes.c_size_t, _vp, _vp, _P(d4dgs_scene_grad), _vp]),
    "d4dgs_flow_loss_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "d4dgs_flow_loss": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _vp,
                                       ctypes.c_size_t, _vp, _vp, _vp]),
    "d4dgs_preprocess_slicing": (ctypes.c_int, [_P(d4dgs_scene4d), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config),
                                                _vp, ctypes.c_size_t, _vp]),
    "d4dgs_render_slicing": (ctypes.c_int, [_P(d4dgs_scene4d), _P(d4dgs_camera), ctypes.c_float, _P(d4dgs_config),
                                            _vp, ctypes.c_size_t, _vp, _vp]),
    "d4dgs_render_batch_stages": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t, ctypes.c_int32, _vp]),
    "d4dgs_launches_per_frame": (ctypes.c_int, [ctypes.c_int32, _P(d4dgs_camera), _P(d4dgs_config)]),
    "d4dgs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def load(path: Path | None = None):
    """Load libd4dgs.so (built in-tree by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path is not None else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                           "(there is no fallback path)")
    lib = ctypes.CDLL(str(p))
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().d4dgs_strerror(code).decode()


class D4DGSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


def check(code: int, where: str):
    if code != D4DGS_OK:
        raise D4DGSError(code, where)
