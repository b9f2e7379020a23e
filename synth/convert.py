"""Host-side conversion of slicing-first 4D Gaussians to the disentangled form.

A 4D Gaussian with mean (mu, mu_t), scales s4 and rotation R4 (the quaternion
pair (q_l, q_r) acting as p -> q_l p q_r on p = t + x i + y j + z k) has
Sigma4D = R4 diag(s4^2) R4^T = [[U, V], [V^T, W]] (Eq. 5).  Its decomposition
(Sec. III-B-1) is the velocity of the mean V3D = V / W, the temporal scale
s_t = sqrt(W) and the 3D covariance Sigma3D = U - V V^T / W, which is stored
as 3D scales and a unit quaternion (its eigen-decomposition).  Both forms
give the same 3D Gaussian and opacity at every time (Eq. 7).  FP64 numpy.

An input converter, kept beside the generators: the tests and the benchmark
use it to build the disentangled form of a slicing-first scene.  The CUDA
library does not import it, and neither does the oracle (which slices in its
own code).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class DisentangledArrays:
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


def _left_right(ql: np.ndarray, qr: np.ndarray) -> np.ndarray:
    """(N, 4, 4) matrices of p -> ql p qr in the quaternion basis (1, i, j, k)."""
    a0, a1, a2, a3 = ql.T
    b0, b1, b2, b3 = qr.T
    L = np.stack([np.stack([a0, -a1, -a2, -a3], -1), np.stack([a1, a0, -a3, a2], -1),
                  np.stack([a2, a3, a0, -a1], -1), np.stack([a3, -a2, a1, a0], -1)], 1)
    Rm = np.stack([np.stack([b0, -b1, -b2, -b3], -1), np.stack([b1, b0, b3, -b2], -1),
                   np.stack([b2, -b3, b0, b1], -1), np.stack([b3, b2, -b1, b0], -1)], 1)
    return L @ Rm


def rotation4(quat_l, quat_r) -> np.ndarray:
    """4D rotations in (x, y, z, t) order from the (normalised) quaternion pairs."""
    ql = np.asarray(quat_l, np.float64).reshape(-1, 4)
    qr = np.asarray(quat_r, np.float64).reshape(-1, 4)
    ql = ql / np.linalg.norm(ql, axis=1, keepdims=True)
    qr = qr / np.linalg.norm(qr, axis=1, keepdims=True)
    perm = [1, 2, 3, 0]   # x, y, z, t are the quaternion components i, j, k, 1
    return _left_right(ql, qr)[:, perm][:, :, perm]


def _rot_to_quat(Rm: np.ndarray) -> np.ndarray:
    """Unit quaternions (w, x, y, z) of (N, 3, 3) proper rotations (largest-component branch)."""
    n = len(Rm)
    q = np.zeros((n, 4))
    tr = np.trace(Rm, axis1=1, axis2=2)
    diag = np.stack([tr, Rm[:, 0, 0], Rm[:, 1, 1], Rm[:, 2, 2]], 1)
    k = np.argmax(diag, axis=1)
    for i in range(n):
        R = Rm[i]
        if k[i] == 0:
            w = 0.5 * np.sqrt(1.0 + tr[i])
            q[i] = [w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w), (R[1, 0] - R[0, 1]) / (4 * w)]
        elif k[i] == 1:
            x = 0.5 * np.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2])
            q[i] = [(R[2, 1] - R[1, 2]) / (4 * x), x, (R[0, 1] + R[1, 0]) / (4 * x), (R[0, 2] + R[2, 0]) / (4 * x)]
        elif k[i] == 2:
            y = 0.5 * np.sqrt(1.0 - R[0, 0] + R[1, 1] - R[2, 2])
            q[i] = [(R[0, 2] - R[2, 0]) / (4 * y), (R[0, 1] + R[1, 0]) / (4 * y), y, (R[1, 2] + R[2, 1]) / (4 * y)]
        else:
            z = 0.5 * np.sqrt(1.0 - R[0, 0] - R[1, 1] + R[2, 2])
            q[i] = [(R[1, 0] - R[0, 1]) / (4 * z), (R[0, 2] + R[2, 0]) / (4 * z), (R[1, 2] + R[2, 1]) / (4 * z), z]
    return q


def disentangle(scene4d) -> DisentangledArrays:
    """The disentangled parameters of a slicing-first scene (float32 arrays)."""
    m4 = np.asarray(scene4d.means4, np.float64).reshape(-1, 4)
    s4 = np.exp(np.asarray(scene4d.log_scales4, np.float64).reshape(-1, 4))
    R4 = rotation4(scene4d.quat_l, scene4d.quat_r)
    S4 = np.einsum("nik,nk,njk->nij", R4, s4 * s4, R4)
    U, V, W = S4[:, :3, :3], S4[:, :3, 3], S4[:, 3, 3]
    S3 = U - np.einsum("ni,nj->nij", V, V) / W[:, None, None]
    evals, evecs = np.linalg.eigh(S3)
    evecs[np.linalg.det(evecs) < 0, :, 0] *= -1.0   # proper rotations
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return DisentangledArrays(means=f32(m4[:, :3]), t_mean=f32(m4[:, 3]), velocity=f32(V / W[:, None]),
                              log_scales=f32(0.5 * np.log(np.maximum(evals, 1e-30))),
                              log_t_scale=f32(0.5 * np.log(W)), quats=f32(_rot_to_quat(evecs)),
                              opacity_logit=f32(scene4d.opacity_logit), sh=f32(scene4d.sh),
                              sh_degree=int(scene4d.sh_degree))
