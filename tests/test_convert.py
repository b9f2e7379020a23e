"""The host conversion of slicing-first 4D Gaussians to the disentangled form
(velocity V/W, temporal scale sqrt(W), Sigma3D = U - V V^T / W as scales and a
quaternion) gives, at every time, the mean, 3D covariance and opacity that the
oracle's slice of the 4D Gaussian gives (Eq. 7).  No GPU."""
import numpy as np

import oracle
import synth
from synth import convert


def test_disentangle_matches_the_oracle_slice():
    sc = synth.make_scene4d(300, 31, "box20", sh_degree=1)
    d = convert.disentangle(sc)
    q = d.quats.astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    Rq = np.array([oracle.quat_to_rot(x) for x in q])
    s2 = np.exp(2.0 * d.log_scales.astype(np.float64))
    S3 = np.einsum("nik,nk,njk->nij", Rq, s2, Rq)
    cov6 = S3[:, [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
    for t in (0.0, 0.31, 0.77, 1.0):
        static, ref6 = oracle.slice4d(sc, t)
        tau = t - d.t_mean.astype(np.float64)
        mean = d.means.astype(np.float64) + tau[:, None] * d.velocity.astype(np.float64)
        np.testing.assert_allclose(mean, static.means, rtol=1e-5, atol=1e-5)
        scale = np.abs(ref6).max(axis=1, keepdims=True)
        np.testing.assert_allclose(cov6 / scale, ref6 / scale, atol=2e-5)
        op = 1 / (1 + np.exp(-d.opacity_logit.astype(np.float64))) * np.exp(
            -0.5 * tau ** 2 / np.exp(2.0 * d.log_t_scale.astype(np.float64)))
        np.testing.assert_allclose(op, 1 / (1 + np.exp(-static.opacity_logit)), rtol=2e-5, atol=1e-7)


def test_rotation4_matches_the_oracle():
    sc = synth.make_scene4d(50, 32, "tiny", mix=0.5)
    np.testing.assert_allclose(convert.rotation4(sc.quat_l, sc.quat_r), oracle.rot4(sc.quat_l, sc.quat_r), atol=1e-13)
