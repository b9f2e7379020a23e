"""Pin of the oracle's FP64 adjoint against central finite differences of the
oracle's own forward (the adjoint is hand-derived; the forward is pinned in
test_oracle_pins.py).  L = sum(G * image) for a fixed random G.  A parameter is
compared only where the step does not change any pixel's blended list (the
image is piecewise smooth; the fingerprint detects a crossed discontinuity)."""
import math

import numpy as np
import pytest

import oracle
import synth

FIELDS = ("means", "t_mean", "velocity", "log_scales", "log_t_scale", "quats", "opacity_logit", "sh")


def fd_scene(n=200, seed=41, deg=0, size=32):
    sc = synth.make_scene(n, seed, "tiny", sh_degree=deg)
    sc = synth.Scene(**{k: np.asarray(v, np.float64).copy() for k, v in sc.arrays().items()}, sh_degree=deg)
    sc.opacity_logit = np.clip(sc.opacity_logit, -3.0, 3.0)          # keep alpha away from the 0.99 clamp
    sc.log_scales += 0.8                                                # a few pixels per Gaussian at 32x32
    if deg > 0:
        sc.sh[:, 0, :] = (np.random.default_rng(seed).uniform(0.3, 0.7, (n, 3)) - 0.5) / synth.SH_C0
        sc.sh[:, 1:, :] *= 0.3                                          # colours stay positive
    cam = synth.pinhole(size, size)
    return sc, cam


def loss(sc, cam, t, G):
    return float((oracle.render(sc, cam, t)["rgb"] * G).sum())


@pytest.mark.parametrize("deg", [0, 3])
def test_adjoint_matches_central_differences(deg):
    sc, cam = fd_scene(deg=deg)
    t = 0.5
    G = np.random.default_rng(7).standard_normal((cam.height, cam.width, 3))
    grads = oracle.backward(sc, cam, t, G)
    base_fp = oracle.fingerprint(sc, cam, t)
    rng = np.random.default_rng(11 + deg)
    checked = skipped = 0
    worst = 0.0
    for field in FIELDS:
        arr = getattr(sc, field)
        flat = arr.reshape(-1)
        picks = rng.choice(flat.size, size=min(flat.size, 60), replace=False)
        for j in picks:
            x0 = flat[j]
            h = 1e-6 * max(1.0, abs(x0))
            flat[j] = x0 + h
            fp_p = oracle.fingerprint(sc, cam, t)
            lp = loss(sc, cam, t, G)
            flat[j] = x0 - h
            fp_m = oracle.fingerprint(sc, cam, t)
            lm = loss(sc, cam, t, G)
            flat[j] = x0
            if not (np.array_equal(fp_p, base_fp) and np.array_equal(fp_m, base_fp)):
                skipped += 1
                continue
            fd = (lp - lm) / (2 * h)
            ad = grads[field].reshape(-1)[j]
            err = abs(fd - ad)
            tol = 1e-6 * max(abs(fd), abs(ad)) + 1e-8
            worst = max(worst, err / (abs(ad) + 1e-8))
            assert err <= tol, (field, int(j), fd, ad)
            checked += 1
    assert checked > 300 and skipped < 0.1 * (checked + skipped), (checked, skipped)


def test_adjoint_nonzero_for_every_parameter_kind():
    sc, cam = fd_scene(deg=3)
    G = np.ones((cam.height, cam.width, 3))
    grads = oracle.backward(sc, cam, 0.5, G)
    for f in FIELDS:
        assert np.abs(grads[f]).max() > 0, f
