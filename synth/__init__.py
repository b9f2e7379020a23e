"""Seeded synthetic inputs for the disentangled 4D Gaussian renderer.

This module only *draws* inputs: scenes (per-Gaussian raw parameters in the
disentangled form of the paper's Eq. 8: 4D scale, 4D mean, quaternion and 3D
velocity, plus 3DGS opacity and spherical-harmonic colour) and pinhole cameras.
It holds none of the rendering arithmetic, so both the CUDA path and the CPU
oracle can be fed from it without sharing any method code.

Workload recipes (the paper's datasets are not available; these stand in):

* ``tiny``   -- 1,000 Gaussians, means x,y ~ U[-1,1], z ~ U[2,6], log-scales
  N(-3, 0.5), unit quaternions, opacity logit N(0,1), SH degree 0 with
  rgb ~ U[0,1], velocity N(0, 0.1), temporal centre U[0,1], log temporal scale
  N(-1.5, 0.3); camera at the origin, 60 deg horizontal FoV, 128x128, t=0.5.
* ``scene``  -- the same distributions scaled to a 20-unit box (means
  U[-10,10]^3, log-scales N(-3+ln 10, 0.5), velocity N(0,1)), SH degree 3 with
  all 48 coefficients N(0, 0.2); 1352x1014 (the Plenoptic Video resolution,
  Sec. IV-A) on a seeded smooth orbit of radius 30 with 300 timestamps in [0,1]
  (10-second videos at 30 fps).
* ``large``  -- as ``scene`` with 1M Gaussians at 2704x2028.

Draw order inside one scene is fixed: means, log-scales, quaternions, opacity
logits, colour/SH, velocity, temporal centre, log temporal scale.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SH_C0 = 0.28209479177387814  # 1 / (2 sqrt(pi)), used only to store a degree-0 colour


@dataclass
class Scene:
    """Raw (pre-activation) parameters of N dynamic Gaussians, float32, SoA.

    means (N,3), t_mean (N,), velocity (N,3), log_scales (N,3), log_t_scale (N,),
    quats (N,4) in (w,x,y,z) order and not necessarily unit, opacity_logit (N,),
    sh (N, (deg+1)^2, 3).
    """

    means: np.ndarray
    t_mean: np.ndarray
    velocity: np.ndarray
    log_scales: np.ndarray
    log_t_scale: np.ndarray
    quats: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self):
        return dict(means=self.means, t_mean=self.t_mean, velocity=self.velocity,
                    log_scales=self.log_scales, log_t_scale=self.log_t_scale,
                    quats=self.quats, opacity_logit=self.opacity_logit, sh=self.sh)

    def subset(self, idx) -> "Scene":
        a = {k: np.ascontiguousarray(v[idx]) for k, v in self.arrays().items()}
        return Scene(sh_degree=self.sh_degree, **a)

    def nbytes(self) -> int:
        return int(sum(v.nbytes for v in self.arrays().values()))


@dataclass
class Scene4D:
    """Raw parameters of N 4D Gaussians in the slicing-first form (Eq. 5: a 4D
    mean, 4D scales and a 4D rotation), float32, SoA.

    means4 (N,4) as (x,y,z,t), log_scales4 (N,4), quat_l and quat_r (N,4) in
    (w,x,y,z) order and not necessarily unit -- the left and right quaternions
    of the rotation -- opacity_logit (N,), sh (N, (deg+1)^2, 3).
    """

    means4: np.ndarray
    log_scales4: np.ndarray
    quat_l: np.ndarray
    quat_r: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means4.shape[0])

    def arrays(self):
        return dict(means4=self.means4, log_scales4=self.log_scales4, quat_l=self.quat_l, quat_r=self.quat_r,
                    opacity_logit=self.opacity_logit, sh=self.sh)


@dataclass
class Camera:
    """Pinhole camera. World->camera: X_cam = R @ X_world + T (row-major R).

    The camera looks along +z with x to the right and y down; pixel (x, y) has
    its centre at (x + 0.5, y + 0.5); u = fx X/Z + cx, v = fy Y/Z + cy.
    """

    R: np.ndarray
    T: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2     # near plane on camera z (the renderer's config near)

    def __post_init__(self):
        self.R = np.ascontiguousarray(self.R, dtype=np.float32).reshape(3, 3)
        self.T = np.ascontiguousarray(self.T, dtype=np.float32).reshape(3)
        self.fx = float(np.float32(self.fx))
        self.fy = float(np.float32(self.fy))
        self.cx = float(np.float32(self.cx))
        self.cy = float(np.float32(self.cy))


def pinhole(width: int, height: int, hfov_deg: float = 60.0, R=None, T=None) -> Camera:
    """Camera with horizontal field of view ``hfov_deg``; fx = fy = (W/2)/tan(hfov/2)."""
    f = (0.5 * width) / math.tan(math.radians(hfov_deg) * 0.5)
    R = np.eye(3) if R is None else R
    T = np.zeros(3) if T is None else T
    return Camera(R=R, T=T, fx=f, fy=f, cx=0.5 * width, cy=0.5 * height,
                  width=width, height=height)


def look_at(position, target, width: int, height: int, hfov_deg: float = 60.0) -> Camera:
    """Camera at ``position`` looking at ``target``; world 'down' is +y."""
    p = np.asarray(position, np.float64)
    f = np.asarray(target, np.float64) - p
    f /= np.linalg.norm(f)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    T = -R @ p
    return pinhole(width, height, hfov_deg, R=R, T=T)


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def make_scene(n: int, seed: int, kind: str = "tiny", sh_degree: int | None = None) -> Scene:
    """Draw a seeded scene. ``kind`` is 'tiny' (unit box in front of the origin)
    or 'box20' (20-unit box centred at the origin, scales and speeds x10)."""
    rng = np.random.default_rng(seed)
    if kind == "tiny":
        deg = 0 if sh_degree is None else sh_degree
        xy = rng.uniform(-1.0, 1.0, (n, 2))
        z = rng.uniform(2.0, 6.0, (n, 1))
        means = np.concatenate([xy, z], axis=1)
        log_scales = rng.normal(-3.0, 0.5, (n, 3))
        vel_sd = 0.1
    elif kind == "box20":
        deg = 3 if sh_degree is None else sh_degree
        means = rng.uniform(-10.0, 10.0, (n, 3))
        log_scales = rng.normal(-3.0 + math.log(10.0), 0.5, (n, 3))
        vel_sd = 1.0
    else:
        raise ValueError(kind)
    quats = _unit_quats(rng, n)
    opacity_logit = rng.normal(0.0, 1.0, n)
    ncoef = (deg + 1) ** 2
    if deg == 0:
        rgb = rng.uniform(0.0, 1.0, (n, 3))
        sh = ((rgb - 0.5) / SH_C0).reshape(n, 1, 3)
    else:
        sh = rng.normal(0.0, 0.2, (n, ncoef, 3))
    velocity = rng.normal(0.0, vel_sd, (n, 3))
    t_mean = rng.uniform(0.0, 1.0, n)
    log_t_scale = rng.normal(-1.5, 0.3, n)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(means=f32(means), t_mean=f32(t_mean), velocity=f32(velocity),
                 log_scales=f32(log_scales), log_t_scale=f32(log_t_scale),
                 quats=f32(quats), opacity_logit=f32(opacity_logit), sh=f32(sh),
                 sh_degree=deg)


def make_scene4d(n: int, seed: int, kind: str = "box20", sh_degree: int | None = None, mix: float = 0.12) -> Scene4D:
    """Draw a seeded slicing-first scene shaped like ``make_scene``: means in the box,
    t_mean ~ U[0,1], spatial log-scales as make_scene's, temporal log-scale N(-1.5, 0.3);
    quat_l = q + noise and quat_r = conj(q) + noise for a random unit q, noise N(0, mix)
    per component (q with its conjugate alone leaves time untouched; the noise mixes
    space and time)."""
    rng = np.random.default_rng(seed)
    if kind == "tiny":
        deg = 0 if sh_degree is None else sh_degree
        xyz = np.concatenate([rng.uniform(-1.0, 1.0, (n, 2)), rng.uniform(2.0, 6.0, (n, 1))], axis=1)
        ls_xyz = rng.normal(-3.0, 0.5, (n, 3))
    elif kind == "box20":
        deg = 3 if sh_degree is None else sh_degree
        xyz = rng.uniform(-10.0, 10.0, (n, 3))
        ls_xyz = rng.normal(-3.0 + math.log(10.0), 0.5, (n, 3))
    else:
        raise ValueError(kind)
    t_mean = rng.uniform(0.0, 1.0, (n, 1))
    ls_t = rng.normal(-1.5, 0.3, (n, 1))
    q = _unit_quats(rng, n)
    ql = q + rng.normal(0.0, mix, (n, 4))
    qr = q * np.array([1.0, -1.0, -1.0, -1.0]) + rng.normal(0.0, mix, (n, 4))
    opacity_logit = rng.normal(0.0, 1.0, n)
    ncoef = (deg + 1) ** 2
    if deg == 0:
        sh = ((rng.uniform(0.0, 1.0, (n, 3)) - 0.5) / SH_C0).reshape(n, 1, 3)
    else:
        sh = rng.normal(0.0, 0.2, (n, ncoef, 3))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene4D(means4=f32(np.concatenate([xyz, t_mean], 1)), log_scales4=f32(np.concatenate([ls_xyz, ls_t], 1)),
                   quat_l=f32(ql), quat_r=f32(qr), opacity_logit=f32(opacity_logit), sh=f32(sh), sh_degree=deg)


def orbit(seed: int, width: int, height: int, n_frames: int = 300, radius: float = 30.0):
    """Seeded smooth orbit about the origin: frame k has azimuth
    theta0 + 0.5*pi*k/(n-1), elevation 0.2*sin(2*pi*k/(n-1) + phi0), and
    timestamp t_k = k/(n-1). Returns a list of (Camera, t)."""
    rng = np.random.default_rng(seed)
    theta0, phi0 = rng.uniform(0.0, 2.0 * math.pi, 2)
    out = []
    denom = max(n_frames - 1, 1)
    for k in range(n_frames):
        az = theta0 + 0.5 * math.pi * k / denom
        el = 0.2 * math.sin(2.0 * math.pi * k / denom + phi0)
        pos = radius * np.array([math.cos(el) * math.sin(az), -math.sin(el),
                                 math.cos(el) * math.cos(az)])
        out.append((look_at(pos, np.zeros(3), width, height), float(np.float32(k / denom))))
    return out


@dataclass
class Workload:
    name: str
    scene: Scene
    frames: list = field(default_factory=list)  # list of (Camera, t)
    tile: int = 16


def tiny_workload(n: int = 1000, seed: int = 0) -> Workload:
    """1,000 Gaussians, 128x128, camera at the origin, t = 0.5, 16x16 tiles."""
    scene = make_scene(n, seed, "tiny")
    return Workload("tiny-1k-128x128", scene, [(pinhole(128, 128), 0.5)], 16)


def scene_workload(n: int = 300_000, width: int = 1352, height: int = 1014,
                   n_frames: int = 300, seed: int = 0, orbit_seed: int = 1,
                   sh_degree: int = 3) -> Workload:
    """300k SH-3 Gaussians in a 20-unit box, 1352x1014, 300 orbit frames."""
    scene = make_scene(n, seed, "box20", sh_degree=sh_degree)
    frames = orbit(orbit_seed, width, height, n_frames)
    return Workload(f"scene-{n}-{width}x{height}", scene, frames, 16)


def large_workload(n: int = 1_000_000, n_frames: int = 300) -> Workload:
    return scene_workload(n=n, width=2704, height=2028, n_frames=n_frames)
