"""CPU oracle for the disentangled 4D Gaussian frame renderer.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never imports, links or executes it, and it
imports nothing from the product package.

``oracle.c`` holds the arithmetic (FP64 renderer, FP32 binning mirror, FP64
adjoint); this module only marshals numpy arrays into it.  Scenes and cameras
are the containers from :mod:`synth` (float32 arrays); the FP64 functions
widen them exactly to double.

Parity status of each function (see the pin tests in ``tests/test_oracle_*``):
  preprocess        pinned (closed-form single Gaussian, SH vs scipy, quaternion
                    vs scipy Rotation, Jacobian vs finite differences, conic vs
                    numpy inverse, slicing-first equivalence)
  render            pinned (closed-form footprint, two-Gaussian Eq. 4, static
                    reduction, time-shift equivalence, monotone transmittance)
  bin_f32           pinned (agrees with the FP64 preprocess; rectangle covers
                    every pixel with alpha >= 1/255)
  backward          pinned (central finite differences of ``render``)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB_PATH = _HERE / "_build" / "liboracle.so"
_lib = None

c_double_p = ctypes.POINTER(ctypes.c_double)
c_float_p = ctypes.POINTER(ctypes.c_float)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_uint32_p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> Path:
    """Compile oracle.c into a shared library (gcc, OpenMP, no FP contraction)."""
    _LIB_PATH.parent.mkdir(parents=True, exist_ok=True)
    if not force and _LIB_PATH.exists() and _LIB_PATH.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB_PATH
    tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-std=c11", str(_SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("sh_degree", ctypes.c_int32)] + [
        (k, c_double_p) for k in ("means", "t_mean", "velocity", "log_scales", "log_t_scale",
                                  "quats", "opacity_logit", "sh", "cov3d", "in_err")] + [
        ("colour_static", ctypes.c_int32)]


class _SceneF32(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("sh_degree", ctypes.c_int32)] + [
        (k, c_float_p) for k in ("means", "t_mean", "velocity", "log_scales", "log_t_scale",
                                 "quats", "opacity_logit")]


class _SceneGrad(ctypes.Structure):
    _fields_ = [(k, c_double_p) for k in ("means", "t_mean", "velocity", "log_scales", "log_t_scale", "quats",
                                          "opacity_logit", "sh")]


class _Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("T", ctypes.c_double * 3), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("near", ctypes.c_double)]


class _CameraF32(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("T", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("near", ctypes.c_float)]


_G2D_FIELDS = ("u", "v", "depth", "conic", "cov2d", "opacity_t", "rgb", "lambda_max", "err")


class _G2D(ctypes.Structure):
    _fields_ = [("drawn", c_int32_p)] + [(k, c_double_p) for k in _G2D_FIELDS]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        _lib.orc_num_threads.restype = ctypes.c_int
        _lib.orc_preprocess.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Camera), ctypes.c_double,
                                        ctypes.c_int, ctypes.POINTER(_G2D)]
        _lib.orc_render_pixels.argtypes = [ctypes.POINTER(_G2D), ctypes.c_int, ctypes.POINTER(_Camera),
                                           c_double_p, ctypes.c_int64, c_int32_p, c_int32_p,
                                           c_double_p, c_double_p, c_int32_p, c_double_p, c_double_p]
        _lib.orc_pair_windows.argtypes = [ctypes.POINTER(_G2D), ctypes.c_int64, c_int32_p, c_int32_p, c_int32_p,
                                          c_double_p]
        c_uint64_p = ctypes.POINTER(ctypes.c_uint64)
        _lib.orc_bin_f32.argtypes = [ctypes.POINTER(_SceneF32), ctypes.POINTER(_CameraF32), ctypes.c_float,
                                     ctypes.c_int32, ctypes.c_int32, c_uint32_p, c_int32_p, c_int32_p, c_uint32_p, c_uint64_p,
                                     c_float_p, c_float_p]
        _lib.orc_expf.restype = ctypes.c_float
        _lib.orc_expf.argtypes = [ctypes.c_float]
        _lib.orc_logf.restype = ctypes.c_float
        _lib.orc_logf.argtypes = [ctypes.c_float]
        _lib.orc_emit_keys.restype = ctypes.c_int64
        _lib.orc_emit_keys.argtypes = [ctypes.c_int32, c_uint32_p, c_int32_p, c_uint64_p, c_uint32_p,
                                       ctypes.c_int32, ctypes.c_int64, c_uint32_p, c_uint32_p, c_uint32_p]
        _lib.orc_sh_basis.argtypes = [c_double_p, ctypes.c_int, c_double_p]
        _lib.orc_quat_to_rot.argtypes = [c_double_p, c_double_p]
        _lib.orc_backward.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Camera), ctypes.c_double,
                                      c_double_p, c_double_p, ctypes.POINTER(_SceneGrad), ctypes.POINTER(_SceneGrad)]
        _lib.orc_fingerprint.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Camera), ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_uint64)]
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def expf32(x) -> np.ndarray:
    """The binary32 exp of the binning contract (Cody-Waite reduction + Taylor series), elementwise."""
    x = np.asarray(x, np.float32)
    f = lib().orc_expf
    return np.array([f(float(v)) for v in x.ravel()], np.float32).reshape(x.shape)


def logf32(x) -> np.ndarray:
    """The binary32 log of the binning contract (atanh series), elementwise."""
    x = np.asarray(x, np.float32)
    f = lib().orc_logf
    return np.array([f(float(v)) for v in x.ravel()], np.float32).reshape(x.shape)


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Keep:
    """Holds the arrays a ctypes struct points into."""

    def __init__(self):
        self.refs = []

    def d(self, a):
        if a is None:
            return None
        a = _d(a)
        self.refs.append(a)
        return _p(a, ctypes.c_double)


def _scene64(scene, keep: _Keep, cov3d=None, in_err=None, colour_static=False):
    s = _Scene()
    s.colour_static = 1 if colour_static else 0
    s.n = scene.n
    s.sh_degree = scene.sh_degree
    for k in ("means", "t_mean", "velocity", "log_scales", "log_t_scale", "quats", "opacity_logit", "sh"):
        setattr(s, k, keep.d(getattr(scene, k)))
    s.cov3d = keep.d(cov3d)
    if in_err is not None:
        assert cov3d is not None and np.asarray(in_err).shape == (scene.n, 10)
    s.in_err = keep.d(in_err)
    return s


def _camera64(cam):
    c = _Camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float64).reshape(9)]
    c.T[:] = [float(x) for x in np.asarray(cam.T, np.float64).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near = float(getattr(cam, "near", 0.2))
    return c


def sh_basis(d, degree: int = 3) -> np.ndarray:
    d = _d(d)
    out = np.zeros(16)
    lib().orc_sh_basis(_p(d, ctypes.c_double), degree, _p(out, ctypes.c_double))
    return out[: (degree + 1) ** 2]


def quat_to_rot(q) -> np.ndarray:
    q = _d(q)
    R = np.zeros(9)
    lib().orc_quat_to_rot(_p(q, ctypes.c_double), _p(R, ctypes.c_double))
    return R.reshape(3, 3)


def preprocess(scene, cam, t: float, temporal_cull: bool = True, cov3d=None, in_err=None,
               colour_static: bool = False) -> dict:
    """FP64 dynamic 2D Gaussians at time t (dict of numpy arrays, length N), with ``err``
    (N x 16): what a binary32 evaluation makes of each Gaussian (oracle.c, orc_preprocess):
    u, v, Z, o_hat and the inverse of Sigma' of its binary32 footprint, the mode (0 both
    draw it, 1 only the definition, 2 only binary32), in cov3d mode a-priori bounds instead.
    ``cov3d`` (N x 6) replaces scales and quaternions; ``in_err`` (N x 10, with ``cov3d``)
    bounds the FP32 error of the mean at t (3), the relative error of the opacity at t (1)
    and of Sigma3D (6) that an FP32 evaluation starts from.  ``colour_static``: the SH colour in the
    direction of the static mean instead of the time-shifted one (the per-camera colour cache of the
    time-grouped renderer, an approximation of the definition)."""
    n = scene.n
    keep = _Keep()
    s = _scene64(scene, keep, cov3d, in_err, colour_static)
    c = _camera64(cam)
    out = dict(drawn=np.zeros(n, np.int32), u=np.zeros(n), v=np.zeros(n), depth=np.zeros(n),
               conic=np.zeros((n, 3)), cov2d=np.zeros((n, 3)), opacity_t=np.zeros(n),
               rgb=np.zeros((n, 3)), lambda_max=np.zeros(n), err=np.zeros((n, 16)))
    g = _G2D(_p(out["drawn"], ctypes.c_int32), *[_p(out[k], ctypes.c_double) for k in _G2D_FIELDS])
    lib().orc_preprocess(ctypes.byref(s), ctypes.byref(c), float(t), int(temporal_cull), ctypes.byref(g))
    out["drawn"] = out["drawn"].astype(bool)
    return out


def _g2d_struct(g: dict):
    fields = {k: _d(g[k]) for k in _G2D_FIELDS}
    drawn = np.ascontiguousarray(g["drawn"], dtype=np.int32)
    s = _G2D(_p(drawn, ctypes.c_int32), *[_p(fields[k], ctypes.c_double) for k in _G2D_FIELDS])
    return s, [drawn] + list(fields.values())


def pair_windows(g: dict, gid, pixels) -> dict:
    """For (Gaussian, pixel) pairs: the FP64 exponent p and unclamped alpha o_hat e^min(p,0),
    the same for the binary32 footprint (p_f, alpha_f), and the relative window of an FP32
    blend's alpha around alpha_f that the slack uses."""
    gid = np.ascontiguousarray(gid, np.int32)
    pixels = np.asarray(pixels, np.int32).reshape(-1, 2)
    assert len(gid) == len(pixels)
    px = np.ascontiguousarray(pixels[:, 0])
    py = np.ascontiguousarray(pixels[:, 1])
    s, keep = _g2d_struct(g)
    out = np.zeros((len(gid), 5))
    lib().orc_pair_windows(ctypes.byref(s), len(gid), _p(gid, ctypes.c_int32), _p(px, ctypes.c_int32),
                           _p(py, ctypes.c_int32), _p(out, ctypes.c_double))
    del keep
    return dict(p=out[:, 0], alpha=out[:, 1], p_f=out[:, 2], alpha_f=out[:, 3], w=out[:, 4])


def render_g2d(g: dict, cam, pixels=None, bg=(0.0, 0.0, 0.0)) -> dict:
    """Per-pixel brute-force compositing of precomputed FP64 2D Gaussians.

    ``pixels`` is None (whole image, row-major) or an (M, 2) int array of (x, y).
    Returns rgb (H,W,3) or (M,3), T, ncontrib, slack and Tw (see oracle.c)."""
    n = len(g["u"])
    s, keep = _g2d_struct(g)
    c = _camera64(cam)
    if pixels is None:
        m = cam.width * cam.height
        px = py = None
        shape = (cam.height, cam.width)
    else:
        pixels = np.asarray(pixels, np.int32).reshape(-1, 2)
        m = pixels.shape[0]
        px = np.ascontiguousarray(pixels[:, 0])
        py = np.ascontiguousarray(pixels[:, 1])
        shape = (m,)
    rgb = np.zeros(shape + (3,))
    T = np.zeros(shape)
    nc = np.zeros(shape, np.int32)
    slack = np.zeros(shape)
    Tw = np.zeros(shape)
    bgv = _d(np.asarray(bg, np.float64))
    lib().orc_render_pixels(ctypes.byref(s), n, ctypes.byref(c), _p(bgv, ctypes.c_double), m,
                            _p(px, ctypes.c_int32), _p(py, ctypes.c_int32),
                            _p(rgb, ctypes.c_double), _p(T, ctypes.c_double), _p(nc, ctypes.c_int32),
                            _p(slack, ctypes.c_double), _p(Tw, ctypes.c_double))
    del keep
    return dict(rgb=rgb, T=T, ncontrib=nc, slack=slack, Tw=Tw)


def render(scene, cam, t: float, pixels=None, bg=(0.0, 0.0, 0.0), temporal_cull: bool = True,
           cov3d=None, in_err=None, colour_static: bool = False) -> dict:
    """Render one frame (or the listed pixels) of ``scene`` at time ``t`` in FP64 (``colour_static``:
    the colour-cache approximation, SH evaluated towards the static mean)."""
    g = preprocess(scene, cam, t, temporal_cull=temporal_cull, cov3d=cov3d, in_err=in_err,
                   colour_static=colour_static)
    out = render_g2d(g, cam, pixels=pixels, bg=bg)
    out["g2d"] = g
    return out


def bin_f32(scene, cam, t: float, tile: int, trim: bool = False) -> dict:
    """FP32 binning mirror: depth key bits, radius, rect, column trims (``trim``: the renderer's
    config trim; all zero otherwise), tile count, uv and ``foot`` (o_hat, Sigma'_00, Sigma'_01,
    Sigma'_11 of the binary32 footprint) of every binned Gaussian."""
    n = scene.n
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    arrs = {k: f(getattr(scene, k)) for k in ("means", "t_mean", "velocity", "log_scales", "log_t_scale",
                                               "quats", "opacity_logit")}
    s = _SceneF32(n, scene.sh_degree, *[_p(arrs[k], ctypes.c_float) for k in (
        "means", "t_mean", "velocity", "log_scales", "log_t_scale", "quats", "opacity_logit")])
    c = _CameraF32()
    c.R[:] = [float(x) for x in f(cam.R).reshape(9)]
    c.T[:] = [float(x) for x in f(cam.T).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = int(cam.width), int(cam.height)
    c.near = float(getattr(cam, "near", 0.2))
    out = dict(depth_key=np.zeros(n, np.uint32), radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
               tiles_touched=np.zeros(n, np.uint32), trims=np.zeros(n, np.uint64), uv=np.zeros((n, 2), np.float32),
               foot=np.zeros((n, 4), np.float32))
    lib().orc_bin_f32(ctypes.byref(s), ctypes.byref(c), ctypes.c_float(t), int(tile), 1 if trim else 0,
                      _p(out["depth_key"], ctypes.c_uint32), _p(out["radius"], ctypes.c_int32),
                      _p(out["rect"], ctypes.c_int32), _p(out["tiles_touched"], ctypes.c_uint32),
                      _p(out["trims"], ctypes.c_uint64), _p(out["uv"], ctypes.c_float), _p(out["foot"], ctypes.c_float))
    out["tiles_x"] = (cam.width + tile - 1) // tile
    out["tiles_y"] = (cam.height + tile - 1) // tile
    return out


def tile_list(b: dict) -> dict:
    """Sorted (tile, depth_bits, id) list of an ``bin_f32`` result (sort by tile,
    then depth bits, then id), plus per-tile [start, end) ranges."""
    n = len(b["depth_key"])
    total = int(b["tiles_touched"].astype(np.int64).sum())
    tile = np.zeros(total, np.uint32)
    depth = np.zeros(total, np.uint32)
    ids = np.zeros(total, np.uint32)
    k = lib().orc_emit_keys(n, _p(b["depth_key"], ctypes.c_uint32), _p(np.ascontiguousarray(b["rect"]), ctypes.c_int32),
                            _p(np.ascontiguousarray(b["trims"]), ctypes.c_uint64),
                            _p(b["tiles_touched"], ctypes.c_uint32), int(b["tiles_x"]), total,
                            _p(tile, ctypes.c_uint32), _p(depth, ctypes.c_uint32), _p(ids, ctypes.c_uint32))
    assert k == total
    order = np.lexsort((ids, depth, tile))
    tile, depth, ids = tile[order], depth[order], ids[order]
    ntiles = int(b["tiles_x"] * b["tiles_y"])
    starts = np.searchsorted(tile, np.arange(ntiles), side="left")
    ends = np.searchsorted(tile, np.arange(ntiles), side="right")
    return dict(tile=tile, depth=depth, id=ids, ranges=np.stack([starts, ends], axis=1).astype(np.uint32))


def backward(scene, cam, t: float, dl_drgb, bg=(0.0, 0.0, 0.0), with_slack: bool = False):
    """FP64 adjoint: gradients of sum(dl_drgb * image) w.r.t. every raw parameter
    (dl_drgb: (H, W, 3); the render uses the temporal cull, as render() does).
    with_slack: also the per-element gradient slack (same keys and shapes): how far an FP32
    renderer's gradient may move because a decision near its threshold goes the other way
    (oracle.c, orc_backward); returns (grads, slack)."""
    keep = _Keep()
    s = _scene64(scene, keep)
    c = _camera64(cam)
    names = ("means", "t_mean", "velocity", "log_scales", "log_t_scale", "quats", "opacity_logit", "sh")
    grads = {k: np.zeros(np.asarray(getattr(scene, k)).shape) for k in names}
    gs = _SceneGrad(*[_p(grads[k], ctypes.c_double) for k in names])
    slack = {k: np.zeros(np.asarray(getattr(scene, k)).shape) for k in names} if with_slack else None
    ss = _SceneGrad(*[_p(slack[k], ctypes.c_double) for k in names]) if with_slack else None
    dl = _d(dl_drgb)
    assert dl.shape == (cam.height, cam.width, 3)
    bgv = _d(np.asarray(bg, np.float64))
    lib().orc_backward(ctypes.byref(s), ctypes.byref(c), float(t), _p(dl, ctypes.c_double),
                       _p(bgv, ctypes.c_double), ctypes.byref(gs), ctypes.byref(ss) if with_slack else None)
    return (grads, slack) if with_slack else grads


def l1_loss(img, target, scale: float):
    """The L1 photometric term of a training step and its gradient (the 3DGS image loss the
    paper's training keeps, Sec. III-C), FP64: (scale * sum |img - target|,
    scale * sign(img - target))."""
    d = _d(img) - _d(target)
    return float(scale * np.abs(d).sum()), scale * np.sign(d)


def fingerprint(scene, cam, t: float) -> np.ndarray:
    """Per-pixel hash of the blended contributor list (and of active alpha clamps)."""
    keep = _Keep()
    s = _scene64(scene, keep)
    c = _camera64(cam)
    out = np.zeros(cam.width * cam.height, np.uint64)
    lib().orc_fingerprint(ctypes.byref(s), ctypes.byref(c), float(t), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))


# ---------------------------------------------------------------------------
# Slicing-first 4D Gaussians (Eq. 5-7), FP64.  The 4D rotation is the
# isoclinic pair of unit quaternions acting as p -> q_l p q_r on
# p = t + x i + y j + z k (the paper does not fix the 4D rotation's
# parameterisation; q_r = conj(q_l) is the 3D rotation of q_l with time fixed).

def _hamilton(a, b):
    """Quaternion products a b for (..., 4) arrays in (w, x, y, z) order."""
    aw, ax, ay, az = np.moveaxis(a, -1, 0)
    bw, bx, by, bz = np.moveaxis(b, -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def rot4(quat_l, quat_r) -> np.ndarray:
    """(N, 4, 4) rotation matrices in (x, y, z, t) order of p -> q_l p q_r (both normalised)."""
    ql = _d(quat_l).reshape(-1, 4)
    qr = _d(quat_r).reshape(-1, 4)
    ql = ql / np.linalg.norm(ql, axis=1, keepdims=True)
    qr = qr / np.linalg.norm(qr, axis=1, keepdims=True)
    n = len(ql)
    R = np.zeros((n, 4, 4))
    # basis vectors x, y, z, t as quaternions i, j, k, 1
    basis = np.array([[0.0, 1, 0, 0], [0.0, 0, 1, 0], [0.0, 0, 0, 1], [1.0, 0, 0, 0]])
    for c in range(4):
        img = _hamilton(_hamilton(ql, np.broadcast_to(basis[c], (n, 4))), qr)
        R[:, :, c] = img[:, [1, 2, 3, 0]]
    return R


def slice4d(scene4d, t: float):
    """The slicing-first step at time t (Eq. 5-7): Sigma4D = R4 diag(s4^2) R4^T = [[U, V], [V^T, W]],
    Sigma3D = U - V V^T / W, mean mu_xyz + (t - mu_t) V / W and opacity times
    exp(-(t - mu_t)^2 / (2 W)).  Returns (a static FP64 scene at t, its 3D covariances as N x 6)."""
    import synth
    m4 = _d(scene4d.means4).reshape(-1, 4)
    s4 = np.exp(_d(scene4d.log_scales4).reshape(-1, 4))
    R = rot4(scene4d.quat_l, scene4d.quat_r)
    S4 = np.einsum("nik,nk,njk->nij", R, s4 * s4, R)
    U, V, W = S4[:, :3, :3], S4[:, :3, 3], S4[:, 3, 3]
    S3 = U - np.einsum("ni,nj->nij", V, V) / W[:, None, None]
    tau = t - m4[:, 3]
    mean_t = m4[:, :3] + tau[:, None] * V / W[:, None]
    op = 1.0 / (1.0 + np.exp(-_d(scene4d.opacity_logit))) * np.exp(-0.5 * tau * tau / W)
    with np.errstate(divide="ignore"):
        logit = np.where(op >= 1.0, 60.0, np.log(op / (1.0 - op)))
    n = len(m4)
    static = synth.Scene(means=mean_t, t_mean=np.full(n, float(t)), velocity=np.zeros((n, 3)),
                         log_scales=np.zeros((n, 3)), log_t_scale=np.zeros(n),
                         quats=np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), opacity_logit=logit,
                         sh=_d(scene4d.sh), sh_degree=scene4d.sh_degree)
    cov6 = S3[:, [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
    return static, cov6


_U32 = 2.0 ** -24        # unit roundoff of binary32
_FN_REL = 4.0 * _U32     # exp / log within 2 ulp


def slice4d_fp32_bounds(scene4d, t: float) -> np.ndarray:
    """(N, 10) bounds on the FP32 error of what an FP32 evaluation of the slice (Eq. 5-7)
    hands to the projection: the mean at t (3, absolute), the opacity at t (1, relative) and
    Sigma3D (6, absolute; xx, xy, xz, yy, yz, zz).  Same model as the oracle's projection
    bounds (correctly rounded operations, a sum of k terms within k u of their magnitudes,
    exp within 2 ulp).  Two FP32 routes are covered, so each bound is the sum of both:
      * slicing first: R4 from the normalised quaternion pair (4u per component, 12u per
        entry), M4 = R4 diag(e^s4), Sigma4D = M4 M4^T, V/W, Sigma3D = U - V (V/W)^T,
        mean mu + tau V/W, opacity sigmoid(lg) exp(-tau^2 / (2W));
      * the disentangled parameters rounded to binary32 (scales e^ls and quaternions of the
        eigen-decomposition of Sigma3D, V/W, log sqrt(W)) and then the disentangled
        projection, whose factor M3 = R(q) diag(s) the oracle's Sigma' bound takes as
        64u |M3| |M3|^T on Sigma3D."""
    u, E = _U32, _FN_REL
    m4 = _d(scene4d.means4).reshape(-1, 4)
    s4 = np.exp(_d(scene4d.log_scales4).reshape(-1, 4))
    R4 = rot4(scene4d.quat_l, scene4d.quat_r)
    M4 = R4 * s4[:, None, :]
    dM4 = (16 * u + E) * np.broadcast_to(s4[:, None, :], M4.shape)
    aM4 = np.abs(M4)
    S4 = np.einsum("nik,njk->nij", M4, M4)
    dS4 = (np.einsum("nik,njk->nij", aM4, dM4) + np.einsum("nik,njk->nij", dM4, aM4)
           + 4 * u * np.einsum("nik,njk->nij", aM4, aM4))
    V, W = S4[:, :3, 3], S4[:, 3, 3]
    dV, dW = dS4[:, :3, 3], dS4[:, 3, 3]
    v = V / W[:, None]
    dv = (dV + np.abs(v) * dW[:, None]) / W[:, None] + u * np.abs(v)
    S3 = S4[:, :3, :3] - V[:, :, None] * v[:, None, :]
    dS3 = (dS4[:, :3, :3] + dV[:, :, None] * np.abs(v)[:, None, :] + np.abs(V)[:, :, None] * dv[:, None, :]
           + u * np.abs(V[:, :, None] * v[:, None, :]) + u * np.abs(S3))
    # the converted route: Sigma3D's factor and the rounding of its scales to binary32
    evals, evecs = np.linalg.eigh(0.5 * (S3 + np.swapaxes(S3, 1, 2)))
    M3 = evecs * np.sqrt(np.maximum(evals, 0.0))[:, None, :]
    ls = 0.5 * np.log(np.maximum(evals, 1e-30))
    aM3 = np.abs(M3)
    dS3 = dS3 + (64 * u + 2 * u * np.abs(ls).max(axis=1))[:, None, None] * np.einsum("nik,njk->nij", aM3, aM3)
    tau = t - m4[:, 3]
    m = m4[:, :3] + tau[:, None] * v
    dm = (np.abs(tau)[:, None] * dv + 2 * u * np.abs(tau[:, None] * v) + u * np.abs(m)
          + 3 * u * np.abs(tau[:, None] * v) + u * np.abs(m))
    x = 0.5 * tau * tau / W
    lst = np.abs(0.5 * np.log(W))
    dop = (2 * E + 3 * u + x * (5 * u + dW / W)) + (2 * E + 3 * u + x * (5 * u + 2 * E + 2 * u * lst))
    out = np.zeros((len(m4), 10))
    out[:, :3] = dm
    out[:, 3] = dop
    out[:, 4:] = dS3[:, [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
    return out


def render_slicing(scene4d, cam, t: float, pixels=None, bg=(0.0, 0.0, 0.0)) -> dict:
    """Slice every 4D Gaussian at t (Eq. 5-7), then render the static 3D result in FP64
    (the slack covers an FP32 slice as well as FP32 disentangled parameters)."""
    static, cov6 = slice4d(scene4d, t)
    return render(static, cam, t, pixels=pixels, bg=bg, cov3d=cov6, in_err=slice4d_fp32_bounds(scene4d, t))


# ---------------------------------------------------------------------------
# Optical-flow channel and the flow-gradient consistency loss (Sec. III-C,
# Eq. 13, 17-18), FP64.  Readings: a Gaussian's flow is its ray-space velocity
# (Eq. 13) in pixels, (fx V_x / Z, fy V_y / Z) with V the camera-frame velocity
# and Z the depth of the time-shifted mean; it is blended with the colour
# weights (alpha_i T_i, background 0).  Gradients use the 3x3 Sobel operator
# with replicated borders; the flow-magnitude gradient is divided by the
# kernel weight 8; the image-gradient magnitude (over the three channels) is
# divided by its maximum over the image and held fixed as a guide.

def flow_g2d(scene, cam, t: float) -> np.ndarray:
    """(N, 2) screen velocity in pixels per unit time of every Gaussian at t."""
    m = _d(scene.means).reshape(-1, 3) + (t - _d(scene.t_mean))[:, None] * _d(scene.velocity).reshape(-1, 3)
    R, T = _d(cam.R).reshape(3, 3), _d(cam.T).reshape(3)
    X = m @ R.T + T
    Vc = _d(scene.velocity).reshape(-1, 3) @ R.T
    return np.stack([cam.fx * Vc[:, 0] / X[:, 2], cam.fy * Vc[:, 1] / X[:, 2]], axis=1)


def render_flow(scene, cam, t: float, pixels=None) -> dict:
    """The blended flow image (H, W, 2) (or (M, 2) at `pixels`), composited with the colour
    weights; the slack is the per-pixel bound of `render` with the flow as colour."""
    g = preprocess(scene, cam, t)
    f = flow_g2d(scene, cam, t)
    gf = dict(g)
    gf["rgb"] = np.column_stack([f, np.zeros(len(f))])
    out = render_g2d(gf, cam, pixels=pixels, bg=(0.0, 0.0, 0.0))
    # the slack bound takes non-negative values: evaluate it on |flow|
    gf["rgb"] = np.abs(gf["rgb"])
    mag = render_g2d(gf, cam, pixels=pixels, bg=(0.0, 0.0, 0.0))
    return dict(flow=out["rgb"][..., :2], slack=mag["slack"], T=out["T"])


def _sobel(img: np.ndarray):
    """Sobel x / y responses of an (H, W) image with replicated borders (kernel weights 1, 2, 1)."""
    p = np.pad(img, 1, mode="edge")
    H, W = img.shape
    s = lambda dy, dx: p[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
    gx = (s(-1, 1) + 2 * s(0, 1) + s(1, 1)) - (s(-1, -1) + 2 * s(0, -1) + s(1, -1))
    gy = (s(1, -1) + 2 * s(1, 0) + s(1, 1)) - (s(-1, -1) + 2 * s(-1, 0) + s(-1, 1))
    return gx, gy


def image_edge_weight(rgb: np.ndarray) -> np.ndarray:
    """1 - |grad I| / max |grad I| (the fixed guide of Eq. 18); 1 where the image is flat."""
    rgb = _d(rgb)
    g2 = np.zeros(rgb.shape[:2])
    for c in range(3):
        gx, gy = _sobel(rgb[..., c])
        g2 += gx * gx + gy * gy
    g = np.sqrt(g2)
    mx = g.max()
    return 1.0 - (g / mx if mx > 0 else np.zeros_like(g))


def flow_gradient_loss(flow: np.ndarray, weight: np.ndarray, lam: float = 1.0, eps: float = 1e-6) -> float:
    """Eq. 17-18: lambda / N * sum |grad M| * weight with M = sqrt(u^2 + v^2 + eps)."""
    flow = _d(flow)
    M = np.sqrt(flow[..., 0] ** 2 + flow[..., 1] ** 2 + eps)
    gx, gy = _sobel(M)
    nrm = np.sqrt(gx * gx + gy * gy) / 8.0
    return float(lam * np.mean(nrm * _d(weight)))


# ---------------------------------------------------------------------------
# Temporal / spatial splitting (Sec. III-C), plain numpy.  Readings: per
# Gaussian the training loop accumulates |dL/d mean| (the 3-vector norm) and
# |dL/d t_mean| over the steps that gave it a nonzero gradient; the averages
# decide, in float32 (the same rounded operations as the device), whether it
# splits in space (g_xyz > tau_xyz and max log-scale > log_min_xyz) and / or in
# time (g_t > tau_t and log s_t > log_min_t).  A split Gaussian becomes two:
# child 1 keeps its index, child 2 is appended after the kept ones in index
# order; the children's means are mu +- R(q) diag(s) n_xyz (a draw of
# N(mu, Sigma3D) and its mirror) and their spatial log-scales drop by
# log(factor) when splitting in space; t_mean +- s_t n_t and log s_t -
# log(factor) when splitting in time; everything else is copied.  n are
# standard normal samples passed in (N x 4: three spatial, one temporal).

def split_decisions(stats, log_scales, log_t_scale, tau_xyz, tau_t, log_min_xyz, log_min_t):
    """(split_space, split_time) boolean arrays; stats (N, 3) = (sum |dL/dmu|, sum |dL/dmu_t|, count)."""
    st = np.asarray(stats, np.float32).reshape(-1, 3)
    cnt = np.maximum(st[:, 2], np.float32(1.0))
    g_xyz = st[:, 0] / cnt
    g_t = st[:, 1] / cnt
    ls = np.asarray(log_scales, np.float32).reshape(-1, 3)
    ss = (g_xyz > np.float32(tau_xyz)) & (ls.max(axis=1) > np.float32(log_min_xyz))
    tt = (g_t > np.float32(tau_t)) & (np.asarray(log_t_scale, np.float32) > np.float32(log_min_t))
    return ss, tt


def split_scene(scene, stats, normals, tau_xyz, tau_t, log_min_xyz, log_min_t, factor=1.6):
    """The scene after splitting (FP64 arrays), and the two decision masks."""
    import synth
    ss, tt = split_decisions(stats, scene.log_scales, scene.log_t_scale, tau_xyz, tau_t, log_min_xyz, log_min_t)
    a = {k: _d(v).copy() for k, v in scene.arrays().items()}
    n = scene.n
    nrm = _d(normals).reshape(n, 4)
    q = a["quats"].reshape(n, 4)
    Rm = np.array([quat_to_rot(x / np.linalg.norm(x)) for x in q])
    d = np.einsum("nij,nj->ni", Rm, np.exp(a["log_scales"].reshape(n, 3)) * nrm[:, :3]) * ss[:, None]
    dt = np.exp(a["log_t_scale"]) * nrm[:, 3] * tt
    lf = math.log(factor)
    child1, child2 = dict(a), {k: v.copy() for k, v in a.items()}
    child1["means"] = a["means"].reshape(n, 3) + d
    child2["means"] = a["means"].reshape(n, 3) - d
    child1["t_mean"] = a["t_mean"] + dt
    child2["t_mean"] = a["t_mean"] - dt
    for c in (child1, child2):
        c["log_scales"] = a["log_scales"].reshape(n, 3) - lf * ss[:, None]
        c["log_t_scale"] = a["log_t_scale"] - lf * tt
    extra = ss | tt
    out = {k: np.concatenate([child1[k], child2[k][extra]], axis=0) for k in a}
    return synth.Scene(**out, sh_degree=scene.sh_degree), ss, tt
