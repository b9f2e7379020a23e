"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these checks re-types the oracle's general formula: each compares it
with a closed form of a special case, a library routine (scipy spherical
harmonics and rotations, numpy inverse / eigenvalues), the definition of a 4D
Gaussian (Eq. 5-7), or an invariant that must hold for any input.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C0 = 0.5 / math.sqrt(math.pi)


def scene64(means, rgb=None, opacity=None, log_scales=None, quats=None, velocity=None, t_mean=None,
            log_t_scale=None, sh=None, sh_degree=0):
    """A float64 scene for exact oracle pins (opacity given as a probability)."""
    means = np.asarray(means, np.float64).reshape(-1, 3)
    n = len(means)
    if sh is None:
        rgb = np.full((n, 3), 0.5) if rgb is None else np.asarray(rgb, np.float64).reshape(n, 3)
        sh = ((rgb - 0.5) / C0).reshape(n, 1, 3)
        sh_degree = 0
    op = np.full(n, 0.5) if opacity is None else np.asarray(opacity, np.float64)
    with np.errstate(divide="ignore"):
        logit = np.where(op >= 1.0, 60.0, np.log(op / (1.0 - op)))
    return synth.Scene(
        means=means,
        t_mean=np.zeros(n) if t_mean is None else np.asarray(t_mean, np.float64),
        velocity=np.zeros((n, 3)) if velocity is None else np.asarray(velocity, np.float64).reshape(n, 3),
        log_scales=np.full((n, 3), math.log(0.05)) if log_scales is None else np.asarray(log_scales, np.float64).reshape(n, 3),
        log_t_scale=np.full(n, 30.0) if log_t_scale is None else np.asarray(log_t_scale, np.float64),
        quats=np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None else np.asarray(quats, np.float64).reshape(n, 4),
        opacity_logit=logit, sh=np.asarray(sh, np.float64), sh_degree=sh_degree)


def camera(width=64, height=48, fx=60.0, fy=45.0, cx=None, cy=None, R=None, T=None):
    """A camera kept in float64 (the synth container rounds to float32 for the GPU)."""
    cam = synth.Camera(R=np.eye(3), T=np.zeros(3), fx=fx, fy=fy, cx=0.0, cy=0.0, width=width, height=height)
    cam.R = np.eye(3) if R is None else np.asarray(R, np.float64)
    cam.T = np.zeros(3) if T is None else np.asarray(T, np.float64)
    cam.fx, cam.fy = float(fx), float(fy)
    cam.cx = width / 2 + 0.5 if cx is None else float(cx)
    cam.cy = height / 2 + 0.5 if cy is None else float(cy)
    return cam


def rot_y(th):
    c, s = math.cos(th), math.sin(th)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


# ---------------------------------------------------------------------------
# library pins
# ---------------------------------------------------------------------------

def test_sh_basis_matches_scipy():
    """Real SH (Condon-Shortley phase, sqrt2 Re/Im) against scipy's complex harmonics."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(3)
    for _ in range(20):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        ours = oracle.sh_basis(d, 3)
        for l in range(4):
            for m in range(-l, l + 1):
                Y = complex(sph_harm_y(l, abs(m), theta, phi))
                ref = Y.real if m == 0 else math.sqrt(2) * (Y.imag if m < 0 else Y.real)
                assert ours[l * l + l + m] == pytest.approx(ref, abs=1e-12), (l, m)


def test_sh_basis_orthonormal():
    """Gauss-Legendre x uniform-phi quadrature of Y_i Y_j over the sphere is the identity."""
    xs, ws = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for z, w in zip(xs, ws):
        r = math.sqrt(1 - z * z)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = oracle.sh_basis([r * math.cos(ph), r * math.sin(ph), z], 3)
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_quat_to_rot_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(4)
    for _ in range(20):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is scalar-last
        np.testing.assert_allclose(oracle.quat_to_rot(q), ref, atol=1e-14)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("rotated", [False, True])
def test_single_gaussian_on_axis_closed_form(rotated):
    """On the optical axis, axis-aligned: Sigma' = diag(fx^2 sx^2/Z^2 + 0.3, fy^2 sy^2/Z^2 + 0.3)
    (Eq. 14, 16), and every pixel is min(0.99, o e^p) c (Eq. 1, 4)."""
    Z, sx, sy, o, c = 4.0, 0.07, 0.03, 0.7, np.array([0.9, 0.3, 0.6])
    R = rot_y(0.4) if rotated else np.eye(3)
    mu = R.T @ np.array([0.0, 0.0, Z])          # camera-space (0, 0, Z)
    # rotated camera: isotropic Gaussian so that Sigma_cam does not depend on R
    ls = [math.log(sx), math.log(sx if rotated else sy), math.log(0.05)]
    sy_eff = sx if rotated else sy
    sc = scene64([mu], rgb=[c], opacity=[o], log_scales=[ls])
    if rotated:
        sc.log_scales[0, 2] = math.log(sx)
    cam = camera(R=R)
    out = oracle.render(sc, cam, 0.0)
    g = out["g2d"]
    s00 = cam.fx ** 2 * sx ** 2 / Z ** 2 + 0.3
    s11 = cam.fy ** 2 * sy_eff ** 2 / Z ** 2 + 0.3
    assert g["u"][0] == pytest.approx(cam.cx, abs=1e-12)
    assert g["v"][0] == pytest.approx(cam.cy, abs=1e-12)
    np.testing.assert_allclose(g["cov2d"][0], [s00, 0.0, s11], atol=1e-12)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    dx, dy = xs + 0.5 - cam.cx, ys + 0.5 - cam.cy
    a = np.minimum(0.99, o * np.exp(-0.5 * (dx ** 2 / s00 + dy ** 2 / s11)))
    a = np.where(a >= 1 / 255, a, 0.0)
    np.testing.assert_allclose(out["rgb"], a[..., None] * c, atol=1e-12)
    np.testing.assert_allclose(out["T"], 1.0 - a, atol=1e-12)


def test_negative_colour_is_clamped():
    """The 3DGS colour model clamps SH . Y + 0.5 at zero per channel: a Gaussian whose
    degree-0 colour is (-0.4, 0.5, 1.2) renders (0, 0.5 alpha, 1.2 alpha)."""
    sc = scene64([[0.0, 0.0, 3.0]], rgb=[[-0.4, 0.5, 1.2]], opacity=[0.6])
    cam = camera()
    out = oracle.render(sc, cam, 0.0, pixels=[[cam.width // 2, cam.height // 2]])
    np.testing.assert_allclose(out["rgb"][0], [0.0, 0.3, 0.72], atol=1e-12)


def test_single_gaussian_off_axis_closed_form():
    """Off axis at (X, Y, Z), axis-aligned Sigma = diag(sx^2, sy^2, sz^2): from Eq. 14/16
    Sigma'_00 = fx^2 (sx^2/Z^2 + X^2 sz^2/Z^4) + 0.3, Sigma'_01 = fx fy X Y sz^2 / Z^4,
    Sigma'_11 = fy^2 (sy^2/Z^2 + Y^2 sz^2/Z^4) + 0.3."""
    X, Y, Z = 0.6, -0.4, 3.0
    sx, sy, sz = 0.05, 0.08, 0.2
    sc = scene64([[X, Y, Z]], log_scales=[[math.log(sx), math.log(sy), math.log(sz)]])
    cam = camera(width=96, height=80, fx=70.0, fy=55.0)
    g = oracle.preprocess(sc, cam, 0.0)
    fx, fy = cam.fx, cam.fy
    expect = [fx ** 2 * (sx ** 2 / Z ** 2 + X ** 2 * sz ** 2 / Z ** 4) + 0.3,
              fx * fy * X * Y * sz ** 2 / Z ** 4,
              fy ** 2 * (sy ** 2 / Z ** 2 + Y ** 2 * sz ** 2 / Z ** 4) + 0.3]
    np.testing.assert_allclose(g["cov2d"][0], expect, rtol=1e-12)
    assert g["u"][0] == pytest.approx(fx * X / Z + cam.cx, abs=1e-12)
    assert g["v"][0] == pytest.approx(fy * Y / Z + cam.cy, abs=1e-12)
    np.testing.assert_allclose(g["conic"][0], np.linalg.inv([[expect[0], expect[1]], [expect[1], expect[2]]])
                               .reshape(4)[[0, 1, 3]], rtol=1e-12)


def test_moving_gaussian_closed_form():
    """Time-shifted mean mu + (t - mu_t) V (Eq. 7) projects to u(t) = fx (X + tau Vx)/(Z + tau Vz) + cx,
    and the temporal factor is 1 at tau = 0 and e^{-1/2} at tau = +-s_t (Eq. 6)."""
    X, Y, Z = 0.3, 0.2, 3.0
    V = np.array([0.5, -0.25, 1.0])
    mu_t, s_t, o = 0.4, 0.15, 0.8
    sc = scene64([[X, Y, Z]], velocity=[V], opacity=[o], t_mean=[mu_t], log_t_scale=[math.log(s_t)])
    cam = camera()
    for t in (mu_t, mu_t + s_t, mu_t - s_t, 0.9):
        tau = t - mu_t
        g = oracle.preprocess(sc, cam, t, temporal_cull=False)
        assert g["u"][0] == pytest.approx(cam.fx * (X + tau * V[0]) / (Z + tau * V[2]) + cam.cx, abs=1e-12)
        assert g["v"][0] == pytest.approx(cam.fy * (Y + tau * V[1]) / (Z + tau * V[2]) + cam.cy, abs=1e-12)
        assert g["depth"][0] == pytest.approx(Z + tau * V[2], abs=1e-14)
    assert oracle.preprocess(sc, cam, mu_t)["opacity_t"][0] == pytest.approx(o, abs=1e-15)
    for t in (mu_t + s_t, mu_t - s_t):
        assert oracle.preprocess(sc, cam, t)["opacity_t"][0] == pytest.approx(o * math.exp(-0.5), abs=1e-15)


def test_projection_jacobian_matches_finite_differences():
    """Sigma' - 0.3 I equals J_fd W Sigma3D W^T J_fd^T with J_fd the central difference of the
    pinhole map (u, v)(X) (Eq. 14, 16), away from the Jacobian clamp."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(5)
    R = Rotation.from_rotvec([0.2, -0.3, 0.1]).as_matrix()
    cam = camera(width=200, height=160, fx=150.0, fy=140.0, R=R, T=[0.1, -0.2, 0.3])
    n = 30
    means = np.column_stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n), rng.uniform(2.5, 5.0, n)])
    means = (R.T @ (means - cam.T).T).T  # place them in front of the camera
    q = rng.standard_normal((n, 4))
    ls = rng.normal(-2.5, 0.4, (n, 3))
    sc = scene64(means, quats=q, log_scales=ls)
    g = oracle.preprocess(sc, cam, 0.0)
    Rc, Tc = cam.R.astype(np.float64), cam.T.astype(np.float64)

    def uv(Xc):
        return np.array([cam.fx * Xc[0] / Xc[2] + cam.cx, cam.fy * Xc[1] / Xc[2] + cam.cy])

    for i in range(n):
        Xc = Rc @ means[i] + Tc
        h = 1e-5
        J = np.column_stack([(uv(Xc + h * e) - uv(Xc - h * e)) / (2 * h) for e in np.eye(3)])
        Rq = Rotation.from_quat(np.roll(q[i] / np.linalg.norm(q[i]), -1)).as_matrix()
        S3 = Rq @ np.diag(np.exp(2 * ls[i])) @ Rq.T
        ref = J @ Rc @ S3 @ Rc.T @ J.T
        got = g["cov2d"][i]
        np.testing.assert_allclose([got[0] - 0.3, got[1], got[2] - 0.3], [ref[0, 0], ref[0, 1], ref[1, 1]],
                                   rtol=1e-7, atol=1e-9)
        inv = np.linalg.inv([[got[0], got[1]], [got[1], got[2]]])
        np.testing.assert_allclose(g["conic"][i], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-12)
        assert g["lambda_max"][i] >= np.linalg.eigvalsh([[got[0], got[1]], [got[1], got[2]]]).max() - 1e-12


def test_composite_golden():
    """Eq. 4 worked by hand (tests/golden/eq4_composite.json)."""
    data = json.load(open(os.path.join(GOLDEN, "eq4_composite.json")))
    cam = camera(width=8, height=8, fx=10.0, fy=10.0, cx=4.5, cy=4.5)
    for case in data["cases"]:
        L = case["layers"]
        sc = scene64([[0.0, 0.0, l["depth"]] for l in L], rgb=[l["rgb"] for l in L],
                     opacity=[l["opacity"] for l in L])
        out = oracle.render(sc, cam, 0.0, pixels=[[4, 4]])
        np.testing.assert_allclose(out["rgb"][0], case["expect_rgb"], atol=1e-12, err_msg=case["name"])
        assert out["T"][0] == pytest.approx(case["expect_T"], abs=1e-12), case["name"]
        assert out["ncontrib"][0] == case["expect_ncontrib"], case["name"]


def test_radius_factor_covers_alpha_threshold():
    """3.33^2 > 2 ln 255, so alpha >= 1/255 implies |d| < 3.33 sqrt(lambda_max)."""
    assert 3.33 ** 2 > 2 * math.log(255.0)
    assert 3.32 ** 2 < 2 * math.log(255.0)


# ---------------------------------------------------------------------------
# the paper's structural identities
# ---------------------------------------------------------------------------

def _random_4d(rng, n):
    """Random SPD 4D covariances R4 S4^2 R4^T (Eq. 5) with R4 from a QR factorisation."""
    out = []
    for _ in range(n):
        Q, Rr = np.linalg.qr(rng.standard_normal((4, 4)))
        Q = Q * np.sign(np.diag(Rr))
        s = np.exp(rng.normal([-3.0, -3.0, -3.0, -1.5], 0.3))
        out.append(Q @ np.diag(s ** 2) @ Q.T)
    return np.array(out)


def test_conditional_slice_identity():
    """The 4D Gaussian density factorises into the temporal marginal times the conditional 3D
    Gaussian with Sigma3D = U - V V^T / W and mean mu + (t - mu_t) V / W (Eq. 6-7)."""
    rng = np.random.default_rng(6)
    for S4 in _random_4d(rng, 10):
        mu4 = rng.standard_normal(4)
        U, V, W = S4[:3, :3], S4[:3, 3], S4[3, 3]
        inv4 = np.linalg.inv(S4)
        S3 = U - np.outer(V, V) / W
        inv3 = np.linalg.inv(S3)
        for _ in range(5):
            x, t = mu4[:3] + 0.1 * rng.standard_normal(3), mu4[3] + 0.3 * rng.standard_normal()
            d4 = np.append(x - mu4[:3], t - mu4[3])
            lhs = -0.5 * d4 @ inv4 @ d4
            m3 = mu4[:3] + (t - mu4[3]) * V / W
            rhs = -0.5 * (t - mu4[3]) ** 2 / W - 0.5 * (x - m3) @ inv3 @ (x - m3)
            assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-9)


def test_disentangled_equals_slicing_first():
    """Rendering the disentangled parameters (V3D = V/W, s_t = sqrt W, Sigma3D = U - VV^T/W)
    equals slicing each 4D Gaussian at t first (Eq. 7) and rendering the static 3D result."""
    rng = np.random.default_rng(7)
    n = 60
    S4 = _random_4d(rng, n)
    mu = np.column_stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n), rng.uniform(2.5, 4.0, n)])
    mu_t = rng.uniform(0, 1, n)
    op = 1 / (1 + np.exp(-rng.normal(0, 1, n)))
    rgb = rng.uniform(0, 1, (n, 3))
    U, V, W = S4[:, :3, :3], S4[:, :3, 3], S4[:, 3, 3]
    S3 = U - np.einsum("ni,nj->nij", V, V) / W[:, None, None]
    cov6 = S3[:, [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
    cam = camera(width=48, height=40, fx=40.0, fy=40.0)
    for t in (0.1, 0.5, 0.85):
        dis = scene64(mu, rgb=rgb, opacity=op, velocity=V / W[:, None], t_mean=mu_t,
                      log_t_scale=0.5 * np.log(W))
        a = oracle.render(dis, cam, t, cov3d=cov6, temporal_cull=False)
        m3 = mu + (t - mu_t)[:, None] * V / W[:, None]
        op_t = op * np.exp(-0.5 * (t - mu_t) ** 2 / W)
        sl = scene64(m3, rgb=rgb, opacity=op_t, t_mean=np.full(n, t))
        b = oracle.render(sl, cam, t, cov3d=cov6, temporal_cull=False)
        np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-12)
        assert np.abs(a["rgb"]).max() > 0.05


def test_static_reduction_time_invariant():
    """V = 0 and s_t -> infinity reduce to static 3DGS: the same image at every t."""
    w = synth.tiny_workload(200)
    sc = w.scene
    st = synth.Scene(**{k: v.copy() for k, v in sc.arrays().items()}, sh_degree=sc.sh_degree)
    st.velocity[:] = 0
    st.log_t_scale[:] = 30.0
    cam = synth.pinhole(64, 64)
    imgs = [oracle.render(st, cam, t)["rgb"] for t in (0.0, 0.37, 1.0)]
    assert np.abs(imgs[0]).max() > 0.05
    for im in imgs[1:]:
        assert np.array_equal(im, imgs[0])


def test_time_shift_equivalence():
    """Rendering at t equals a static scene whose means are pre-shifted to mu + tau V and whose
    opacity is pre-multiplied by the temporal factor (Algorithm 1's deferred slice); SH degree 3
    so the view direction of the shifted mean matters."""
    sc = synth.make_scene(150, 11, "tiny", sh_degree=3)
    cam = synth.pinhole(64, 64)
    t = 0.3
    a = oracle.render(sc, cam, t, temporal_cull=False)
    g = a["g2d"]
    tau = t - sc.t_mean.astype(np.float64)
    st = synth.Scene(**{k: np.asarray(v, np.float64).copy() for k, v in sc.arrays().items()}, sh_degree=3)
    st.means = sc.means.astype(np.float64) + tau[:, None] * sc.velocity.astype(np.float64)
    st.velocity[:] = 0
    oh = g["opacity_t"]
    st.opacity_logit = np.log(oh / (1 - oh))
    st.log_t_scale[:] = 30.0
    st.t_mean[:] = t
    b = oracle.render(st, cam, t, temporal_cull=False)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-12)
    # with the view direction of the *static* mean the images would differ
    assert np.abs(a["rgb"]).max() > 0.05


def test_temporal_cull_is_lossless():
    """Dropping Gaussians with o_hat < 1/255 cannot change any pixel (alpha < 1/255 everywhere)."""
    sc = synth.make_scene(400, 12, "tiny")
    cam = synth.pinhole(64, 64)
    for t in (0.0, 0.5, 1.0):
        a = oracle.render(sc, cam, t, temporal_cull=True)
        b = oracle.render(sc, cam, t, temporal_cull=False)
        assert a["g2d"]["drawn"].sum() < b["g2d"]["drawn"].sum() or t == 0.5
        assert np.array_equal(a["rgb"], b["rgb"])


def test_transmittance_and_colour_bounds():
    """1e-4 <= T <= 1 (stop-before-blend), and 0 <= C <= (1 - T) max c (Eq. 4 is a
    sub-convex combination of the colours)."""
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    out = oracle.render(w.scene, cam, t)
    T, rgb = out["T"], out["rgb"]
    assert T.min() >= 1e-4 and T.max() <= 1.0
    cmax = out["g2d"]["rgb"][out["g2d"]["drawn"]].max()
    assert rgb.min() >= 0.0
    assert np.all(rgb <= (1 - T)[..., None] * cmax + 1e-12)


def test_transmittance_monotone_in_added_layers():
    """Adding a Gaussian in front never increases T at any pixel."""
    sc = synth.make_scene(120, 13, "tiny")
    cam = synth.pinhole(48, 48)
    base = oracle.render(sc, cam, 0.5, temporal_cull=False)
    extra = scene64([[0.05, -0.02, 1.5]], opacity=[0.9], log_scales=[[math.log(0.1)] * 3], t_mean=[0.5])
    both = synth.Scene(**{k: np.concatenate([np.asarray(getattr(sc, k), np.float64), getattr(extra, k)])
                          for k in sc.arrays()}, sh_degree=0)
    more = oracle.render(both, cam, 0.5, temporal_cull=False)
    assert np.all(more["T"] <= base["T"] + 1e-15)
    assert (more["T"] < base["T"] - 1e-6).sum() > 10


# ---------------------------------------------------------------------------
# FP32 binning mirror
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("trim", [False, True])
def test_bin_f32_agrees_with_fp64(trim):
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    b = oracle.bin_f32(w.scene, cam, t, 16, trim=trim)
    g = oracle.preprocess(w.scene, cam, t)
    ok = b["tiles_touched"] > 0
    assert ok.sum() > 900
    assert np.all(g["drawn"][ok])
    np.testing.assert_allclose(b["uv"][ok, 0], g["u"][ok], atol=1e-3)
    np.testing.assert_allclose(b["uv"][ok, 1], g["v"][ok], atol=1e-3)
    depth = b["depth_key"][ok].view(np.float32).astype(np.float64)
    np.testing.assert_allclose(depth, g["depth"][ok], rtol=1e-6)
    x64 = 3.33 * np.sqrt(g["lambda_max"][ok])
    r64 = np.ceil(x64)
    # FP32 and FP64 may round a radius within FP32 reach of an integer differently
    clear = np.abs(x64 - np.round(x64)) > 1e-5 * x64
    assert clear.mean() > 0.99
    assert np.array_equal(b["radius"][ok][clear], r64[clear].astype(np.int32))
    rect = b["rect"][ok]
    area = (rect[:, 1] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 2] + 1)
    kept = np.array([kept_tiles(b, i).sum() for i in np.nonzero(ok)[0]])
    assert np.array_equal(b["tiles_touched"][ok], kept)
    if trim:
        assert np.all(kept <= area) and kept.sum() < area.sum()
    else:
        assert np.array_equal(kept, area) and not b["trims"].any()


def kept_tiles(b, i):
    """Boolean (rows x columns) mask of the rectangle tiles Gaussian i keeps after its column cuts
    (trims byte j: rows cut at the top of column x0 + j in the low nibble, at the bottom in the high)."""
    x0, x1, y0, y1 = (int(z) for z in b["rect"][i])
    h, w = y1 - y0 + 1, x1 - x0 + 1
    m = np.ones((h, w), bool)
    for j in range(min(w, 8)):
        byte = (int(b["trims"][i]) >> (8 * j)) & 0xFF
        top, bot = byte & 15, byte >> 4
        m[:top, j] = False
        m[h - bot:, j] = False
    return m


def box_min_quadratic(A00, A01, A11, xa, xb, ya, yb):
    """min of A00 x^2 + 2 A01 x y + A11 y^2 (positive definite) over the box [xa, xb] x [ya, yb]:
    0 if the origin is inside, else the least of the four edge minima (each a clamped 1D parabola)."""
    best = np.inf
    if xa <= 0.0 <= xb and ya <= 0.0 <= yb:
        return 0.0
    for x in (xa, xb):
        y = min(max(-A01 * x / A11, ya), yb)
        best = min(best, A00 * x * x + 2 * A01 * x * y + A11 * y * y)
    for y in (ya, yb):
        x = min(max(-A01 * y / A00, xa), xb)
        best = min(best, A00 * x * x + 2 * A01 * x * y + A11 * y * y)
    return best


@pytest.mark.parametrize("tile,frame", [(16, 0), (32, 150)])
def test_column_trims_match_fp64_box_test(tile, frame):
    """The FP32 column cuts keep exactly the tiles whose pixel-centre box (rows widened by 1/64 px)
    meets the binning ellipse d^T Sigma'^-1 d <= k2 (k2 = 2 ln(255 o_hat) 1.0008 + 0.0008), decided
    here independently in FP64 by minimising the quadratic form over each box; tiles within 1e-4
    relative of the ellipse, cuts saturated at 15 rows and flagged Gaussians are left out."""
    scene = synth.make_scene(3000, 21, "box20", sh_degree=0)
    cam, t = synth.orbit(4, 320, 240, 300)[frame]
    b = oracle.bin_f32(scene, cam, t, tile, trim=True)
    g = oracle.preprocess(scene, cam, t)
    checked = cut = 0
    for i in np.nonzero(b["tiles_touched"] > 0)[0]:
        s00, s01, s11 = g["cov2d"][i]
        det = s00 * s11 - s01 * s01
        A00, A01, A11 = s11 / det, -s01 / det, s00 / det
        k2 = 2.0 * np.log(255.0 * g["opacity_t"][i]) * 1.0008 + 0.0008
        u, v = g["u"][i], g["v"][i]
        x0, x1, y0, y1 = (int(z) for z in b["rect"][i])
        m = kept_tiles(b, i)
        for j in range(min(x1 - x0 + 1, 8)):
            byte = (int(b["trims"][i]) >> (8 * j)) & 0xFF
            if (byte & 15) == 15 or (byte >> 4) == 15:
                continue
            c = x0 + j
            xa, xb = c * tile + 0.5 - u, min(c * tile + tile - 0.5, cam.width - 0.5) - u
            for r in range(y0, y1 + 1):
                ya, yb = r * tile + 0.5 - 1 / 64 - v, r * tile + tile - 0.5 + 1 / 64 - v
                qmin = box_min_quadratic(A00, A01, A11, xa, xb, ya, yb)
                if abs(qmin - k2) <= 1e-4 * k2:
                    continue
                assert m[r - y0, j] == (qmin <= k2), (i, r, c, qmin, k2)
                checked += 1
                cut += qmin > k2
    assert checked > 2000 and cut > 100, (checked, cut)


@pytest.mark.parametrize("trim", [False, True])
def test_tile_rect_covers_alpha_support(trim):
    """Every pixel where a Gaussian's FP64 alpha reaches 1/255 lies in a tile its FP32 binning keeps
    (its rectangle, less the column cuts when they are on)."""
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    tile = 16
    b = oracle.bin_f32(w.scene, cam, t, tile, trim=trim)
    g = oracle.preprocess(w.scene, cam, t)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    px, py = xs.ravel() + 0.5, ys.ravel() + 0.5
    tx, ty = xs.ravel() // tile, ys.ravel() // tile
    checked = 0
    for i in np.nonzero(g["drawn"])[0]:
        a, bb, c = g["conic"][i]
        dx, dy = g["u"][i] - px, g["v"][i] - py
        p = -0.5 * (a * dx * dx + c * dy * dy) - bb * dx * dy
        alpha = np.minimum(0.99, g["opacity_t"][i] * np.exp(np.minimum(p, 0)))
        hit = (p <= 0) & (alpha >= 1 / 255)
        if not hit.any():
            continue
        assert b["tiles_touched"][i] > 0
        x0, x1, y0, y1 = b["rect"][i]
        assert np.all((tx[hit] >= x0) & (tx[hit] <= x1) & (ty[hit] >= y0) & (ty[hit] <= y1)), i
        assert np.all(kept_tiles(b, i)[ty[hit] - y0, tx[hit] - x0]), i
        checked += 1
    assert checked > 900


def test_tile_list_sorted_and_ranges():
    w = synth.tiny_workload()
    cam, t = w.frames[0]
    b = oracle.bin_f32(w.scene, cam, t, 16, trim=True)
    L = oracle.tile_list(b)
    key = (L["tile"].astype(np.uint64) << np.uint64(32)) | L["depth"].astype(np.uint64)
    assert np.all(np.diff(key.astype(np.float64)) >= 0) or np.all(key[1:] >= key[:-1])
    assert len(L["tile"]) == int(b["tiles_touched"].sum())
    r = L["ranges"]
    assert r[0, 0] == 0 and r[-1, 1] == len(L["tile"])
    assert np.all(r[1:, 0] == r[:-1, 1])
    for tid in range(len(r)):
        assert np.all(L["tile"][r[tid, 0]:r[tid, 1]] == tid)


# ---------------------------------------------------------------------------
# slicing-first form (Eq. 5-7 with the 4D rotation p -> q_l p q_r)

def test_rot4_conjugate_pair_is_the_3d_rotation():
    """q_r = conj(q_l): time is untouched and space turns by the 3D rotation of q_l."""
    rng = np.random.default_rng(21)
    q = rng.standard_normal((8, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)   # quat_to_rot takes unit quaternions
    R = oracle.rot4(q, q * np.array([1.0, -1, -1, -1]))
    for k in range(8):
        expect = np.eye(4)
        expect[:3, :3] = oracle.quat_to_rot(q[k])
        np.testing.assert_allclose(R[k], expect, atol=1e-14)


def test_rot4_equal_pair_turns_one_space_time_plane():
    """q_l = q_r = cos(phi/2) + u sin(phi/2): rotation by phi in the plane of t and u, identity on u's
    orthogonal complement in space."""
    rng = np.random.default_rng(22)
    for _ in range(5):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        phi = rng.uniform(-2, 2)
        q = np.append(math.cos(phi / 2), math.sin(phi / 2) * u)
        R = oracle.rot4(q, q)[0]
        et = np.array([0, 0, 0, 1.0])
        eu = np.append(u, 0.0)
        np.testing.assert_allclose(R @ et, math.cos(phi) * et + math.sin(phi) * eu, atol=1e-14)
        np.testing.assert_allclose(R @ eu, math.cos(phi) * eu - math.sin(phi) * et, atol=1e-14)
        w = np.cross(u, rng.standard_normal(3))
        w = np.append(w / np.linalg.norm(w), 0.0)
        np.testing.assert_allclose(R @ w, w, atol=1e-14)


def test_rot4_is_a_rotation():
    rng = np.random.default_rng(23)
    R = oracle.rot4(rng.standard_normal((50, 4)), rng.standard_normal((50, 4)))
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", R, R), np.broadcast_to(np.eye(4), R.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-13)


def test_slice4d_is_the_conditional_gaussian():
    """Sigma3D and the mean at t equal the conditional of the 4D Gaussian computed from the
    precision matrix (inverse of the spatial block of Sigma4D^-1; mean mu - P_xx^-1 P_xt (t - mu_t)),
    and the opacity factor is the temporal marginal exp(-(t - mu_t)^2 / (2 Sigma4D_tt))."""
    sc = synth.make_scene4d(40, 24, "tiny", mix=0.4)
    t = 0.37
    static, cov6 = oracle.slice4d(sc, t)
    R = oracle.rot4(sc.quat_l, sc.quat_r)
    s4 = np.exp(sc.log_scales4.astype(np.float64))
    for k in range(sc.n):
        S4 = R[k] @ np.diag(s4[k] ** 2) @ R[k].T
        P = np.linalg.inv(S4)
        S3 = np.linalg.inv(P[:3, :3])
        m4 = sc.means4[k].astype(np.float64)
        mean = m4[:3] - S3 @ P[:3, 3] * (t - m4[3])
        np.testing.assert_allclose(cov6[k], S3[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(static.means[k], mean, rtol=1e-10, atol=1e-12)
        o = 1 / (1 + np.exp(-float(sc.opacity_logit[k]))) * np.exp(-0.5 * (t - m4[3]) ** 2 / S4[3, 3])
        assert 1 / (1 + np.exp(-static.opacity_logit[k])) == pytest.approx(o, rel=1e-12)


def test_slicing_without_space_time_mixing_equals_the_disentangled_render():
    """Identity rotations: Sigma4D is diagonal, V = 0, so slicing-first equals the disentangled render
    with zero velocity, the same spatial scales and s_t = the fourth scale."""
    sc = synth.make_scene4d(80, 25, "tiny")
    n = sc.n
    ident = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    sc.quat_l, sc.quat_r = ident.astype(np.float32), ident.astype(np.float32)
    dis = synth.Scene(means=sc.means4[:, :3], t_mean=sc.means4[:, 3], velocity=np.zeros((n, 3), np.float32),
                      log_scales=sc.log_scales4[:, :3], log_t_scale=sc.log_scales4[:, 3], quats=ident,
                      opacity_logit=sc.opacity_logit, sh=sc.sh, sh_degree=sc.sh_degree)
    cam = camera(width=48, height=40, fx=40.0, fy=40.0)
    for t in (0.2, 0.6):
        a = oracle.render_slicing(sc, cam, t)
        b = oracle.render(dis, cam, t)
        np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-12)
        assert np.abs(a["rgb"]).max() > 0.05


# ---------------------------------------------------------------------------
# optical-flow channel and flow-gradient loss (Eq. 13, 17-18)

def test_flow_single_gaussian_closed_form():
    """One Gaussian on the optical axis moving along x: its flow is fx V_x / Z (Eq. 13 in pixels), and
    the blended flow at a pixel is alpha times that (a single contributor, background 0)."""
    Z, vx, fx = 4.0, 0.3, 60.0
    sc = scene64([[0.0, 0.0, Z]], velocity=[[vx, 0.0, 0.0]], t_mean=[0.5], opacity=[0.8],
                 log_scales=[[math.log(0.05)] * 3])
    cam = camera(width=32, height=24, fx=fx, fy=fx)
    f = oracle.flow_g2d(sc, cam, 0.5)
    assert f[0, 0] == pytest.approx(fx * vx / Z, rel=1e-14) and f[0, 1] == 0.0
    out = oracle.render_flow(sc, cam, 0.5)
    img = oracle.render(sc, cam, 0.5)
    alpha = 1.0 - img["T"]            # one Gaussian: T = 1 - alpha where it is blended
    np.testing.assert_allclose(out["flow"][..., 0], alpha * fx * vx / Z, atol=1e-14)
    assert np.abs(out["flow"][..., 1]).max() == 0.0 and alpha.max() > 0.3


def test_flow_of_a_moving_mean_matches_the_finite_difference_of_its_projection():
    """d u / dt of the projected time-shifted mean, minus the depth-change term that Eq. 13 leaves out,
    equals the flow: (u(t+h) - u(t-h)) / 2h = fx V_x / Z - fx X V_z / Z^2."""
    rng = np.random.default_rng(26)
    sc = scene64(rng.uniform(-0.5, 0.5, (5, 3)) + [0, 0, 3.0], velocity=rng.normal(0, 0.4, (5, 3)),
                 t_mean=rng.uniform(0, 1, 5))
    cam = camera(width=40, height=30, fx=50.0, fy=45.0)
    t, h = 0.4, 1e-6
    f = oracle.flow_g2d(sc, cam, t)
    gp, gm = oracle.preprocess(sc, cam, t + h, temporal_cull=False), oracle.preprocess(sc, cam, t - h, temporal_cull=False)
    du = (gp["u"] - gm["u"]) / (2 * h)
    m = sc.means + (t - sc.t_mean)[:, None] * sc.velocity
    Z = m[:, 2]
    np.testing.assert_allclose(du, f[:, 0] - cam.fx * m[:, 0] * sc.velocity[:, 2] / Z ** 2, rtol=1e-6, atol=1e-6)


def test_flow_gradient_loss_closed_forms():
    """A constant flow gives 0; a flow ramp u = a x + b on a flat image gives lambda a (W - 1) / W with
    replicated borders (the two border columns see half the ramp)."""
    H, W = 12, 17
    flat = np.full((H, W, 3), 0.4)
    wgt = oracle.image_edge_weight(flat)
    assert np.all(wgt == 1.0)
    const = np.zeros((H, W, 2)); const[..., 0] = 3.0
    assert oracle.flow_gradient_loss(const, wgt, lam=2.0) == pytest.approx(0.0, abs=1e-12)
    a, b = 0.25, 50.0
    ramp = np.zeros((H, W, 2)); ramp[..., 0] = a * np.arange(W)[None, :] + b
    L = oracle.flow_gradient_loss(ramp, wgt, lam=2.0, eps=0.0)
    assert L == pytest.approx(2.0 * a * (W - 1) / W, rel=1e-12)


def test_image_edge_weight_is_one_minus_normalised_sobel():
    """A vertical step edge: the weight is 0 on the two columns next to the step, 1 elsewhere."""
    img = np.zeros((8, 10, 3)); img[:, 5:, :] = 1.0
    w = oracle.image_edge_weight(img)
    np.testing.assert_allclose(w[:, [4, 5]], 0.0, atol=1e-15)
    np.testing.assert_allclose(np.delete(w, [4, 5], axis=1), 1.0)


# ---------------------------------------------------------------------------
# temporal / spatial splitting (Sec. III-C)

def test_split_children_straddle_the_parent():
    """The two children of a spatial split lie at mu +- R diag(s) n, so their midpoint is the parent's
    mean, their offset has Mahalanobis length |n| under the parent's Sigma3D, and their scales are the
    parent's divided by the factor; a temporal split does the same along t with s_t."""
    sc = synth.make_scene(50, 71, "tiny")
    rng = np.random.default_rng(72)
    normals = rng.standard_normal((50, 4))
    stats = np.column_stack([rng.uniform(0, 2, 50), rng.uniform(0, 2, 50), np.full(50, 2.0)])
    out, ss, tt = oracle.split_scene(sc, stats, normals, tau_xyz=0.5, tau_t=0.5, log_min_xyz=-10, log_min_t=-10)
    assert 0 < ss.sum() < 50 and 0 < tt.sum() < 50
    extra = np.nonzero(ss | tt)[0]
    assert out.n == 50 + len(extra)
    m64 = sc.means.astype(np.float64)
    for j, i in enumerate(extra):
        c1, c2 = out.means[i], out.means[50 + j]
        np.testing.assert_allclose((c1 + c2) / 2, m64[i], atol=1e-12)
        if ss[i]:
            q = sc.quats[i].astype(np.float64)
            R = oracle.quat_to_rot(q / np.linalg.norm(q))
            S2 = R @ np.diag(np.exp(2 * sc.log_scales[i].astype(np.float64))) @ R.T
            dv = c1 - m64[i]
            assert dv @ np.linalg.solve(S2, dv) == pytest.approx(np.sum(normals[i, :3] ** 2), rel=1e-9)
            np.testing.assert_allclose(np.exp(out.log_scales[i]), np.exp(sc.log_scales[i].astype(np.float64)) / 1.6, rtol=1e-12)
        else:
            np.testing.assert_allclose(c1, m64[i], atol=0)
        if tt[i]:
            st = math.exp(float(sc.log_t_scale[i]))
            assert out.t_mean[i] - sc.t_mean[i] == pytest.approx(st * normals[i, 3], rel=1e-9)
            assert out.t_mean[50 + j] - sc.t_mean[i] == pytest.approx(-st * normals[i, 3], rel=1e-9)


def test_split_nothing_below_thresholds():
    sc = synth.make_scene(30, 73, "tiny")
    stats = np.column_stack([np.full(30, 0.1), np.full(30, 0.1), np.ones(30)])
    out, ss, tt = oracle.split_scene(sc, stats, np.zeros((30, 4)), 0.5, 0.5, -10, -10)
    assert not ss.any() and not tt.any() and out.n == 30
    np.testing.assert_array_equal(out.means, sc.means.astype(np.float64))


def test_colour_static_mode_reduces_to_the_definition_without_motion():
    """The colour-cache mode evaluates SH towards the static mean: identical to the definition when
    no Gaussian moves (mu(t) = mu), different once they do (the approximation is real)."""
    sc = synth.make_scene(300, 61, "tiny", sh_degree=3)
    cam = synth.pinhole(48, 40)
    moving = oracle.render(sc, cam, 0.8)
    moving_c = oracle.render(sc, cam, 0.8, colour_static=True)
    assert np.abs(moving["rgb"] - moving_c["rgb"]).max() > 1e-4
    sc.velocity[:] = 0.0
    still = oracle.render(sc, cam, 0.8)
    still_c = oracle.render(sc, cam, 0.8, colour_static=True)
    assert np.array_equal(still["rgb"], still_c["rgb"])
