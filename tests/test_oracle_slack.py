"""Pins of the oracle's per-pixel slack (oracle.c, orc_render_pixels): the
allowance an FP32 renderer gets on a pixel where one of its discrete decisions
(alpha against 1/255, the stop rule, the depth order, the near plane) may go
the other way.  The slack rests on three things, and each is checked here
against something other than itself:

  * the binary32 footprint of each Gaussian (the projection evaluated in
    binary32 in the fixed operation order, exp and log included): its exp and
    log against numpy's double-precision functions, the footprint against the
    FP64 definition;
  * the window an FP32 blend's own rounding gets around that footprint's alpha
    (pair_window): it must cover an FP32 blend written here independently
    (numpy float32, two operation orders) on thin, rotated splats, and must not
    be loose (some pair comes within a factor 10 of it); in cov3d mode the
    a-priori bounds must cover a numpy float32 evaluation of the slicing-first
    form (Eq. 5-7);
  * the order of the binary32 depth keys: a constructed pair whose keys swap
    the FP64 order gets at least the colour change of the swap (Eq. 4).

And on whole images: a pixel whose FP64 decisions all lie far from their
thresholds has slack 0; no pixel's slack exceeds what flips near its
thresholds can do (twice alpha T max c per flip, Eq. 4).
"""
import math

import numpy as np
import pytest

import oracle
import synth

F32 = np.float32
LOG2E = 1.4426950408889634
AMIN = 1.0 / 255.0


def stress_scene(n=400, seed=3, spread=1.8):
    """Thin, rotated splats at several depths in front of the camera: log-scales
    N(-3, spread) per axis, so that conditioning numbers of 10^3-10^5 occur."""
    sc = synth.make_scene(n, seed, "tiny")
    rng = np.random.default_rng(seed + 100)
    sc.log_scales = rng.normal(-3.0, spread, (n, 3)).astype(np.float32)
    return sc


def pair_sample(g, b, cam, seed=0, per=48):
    """(Gaussian, pixel) pairs around every Gaussian both the binary32 footprint and the
    definition draw: pixels on rays from its mean at 0.2-1.15 times the radius where its
    alpha crosses 1/255 (the decision the window guards), the ray's direction random."""
    rng = np.random.default_rng(seed)
    ids = np.nonzero(g["drawn"] & (b["tiles_touched"] > 0))[0]
    gid, pix = [], []
    for i in ids:
        a, bb, c = g["conic"][i]
        k2 = 2.0 * math.log(255.0 * g["opacity_t"][i])
        if k2 <= 0:
            continue
        th = rng.uniform(0, 2 * math.pi, per)
        e = np.stack([np.cos(th), np.sin(th)], 1)
        qf = a * e[:, 0] ** 2 + 2 * bb * e[:, 0] * e[:, 1] + c * e[:, 1] ** 2
        r = np.sqrt(k2 / qf) * rng.uniform(0.2, 1.15, per)
        x = np.floor(g["u"][i] + r * e[:, 0]).astype(np.int64)
        y = np.floor(g["v"][i] + r * e[:, 1]).astype(np.int64)
        ok = (x >= 0) & (x < cam.width) & (y >= 0) & (y < cam.height)
        gid.append(np.full(ok.sum(), i))
        pix.append(np.stack([x[ok], y[ok]], 1))
    return np.concatenate(gid).astype(np.int32), np.concatenate(pix).astype(np.int32)


def _fma(a, b, c):
    """a b + c with one rounding to binary32 (the double product of two floats is exact)."""
    return F32(a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64))


def blend_alpha_f32(uv, foot, pix, order):
    """An FP32 blend's alpha 2^q of (Gaussian footprint, pixel) pairs, written independently:
    the conic from the binary32 Sigma' (determinant rounded once, float32 quotients), the base-2
    exponent form, q evaluated either with FMAs as (C dy + B dx) dy + A dx dx or as a plain sum
    of products, then + log2(o_hat) and exp2, all in numpy float32."""
    oh, s00, s01, s11 = (foot[:, k] for k in range(4))
    det = F32(s00.astype(np.float64) * s11 - s01.astype(np.float64) * s01)
    a, b, c = s11 / det, -s01 / det, s00 / det
    h = F32(-0.5) * F32(LOG2E)
    A, B, C = h * a, F32(-LOG2E) * b, h * c
    dx = uv[:, 0] - (pix[:, 0].astype(F32) + F32(0.5))
    dy = uv[:, 1] - (pix[:, 1].astype(F32) + F32(0.5))
    if order == "fma":
        p = _fma(_fma(C, dy, B * dx), dy, (A * dx) * dx)
    else:
        p = (A * (dx * dx) + B * (dx * dy)) + C * (dy * dy)
    q = p + np.log2(oh)
    return np.exp2(q).astype(np.float64)


def window_ratios(sc, cam, t, seed=0):
    g = oracle.preprocess(sc, cam, t)
    b = oracle.bin_f32(sc, cam, t, 16)
    gid, pix = pair_sample(g, b, cam, seed)
    pw = oracle.pair_windows(g, gid, pix)
    ratios = []
    for order in ("fma", "plain"):
        a32 = blend_alpha_f32(b["uv"][gid], b["foot"][gid], pix, order)
        ratios.append(np.abs(a32 / pw["alpha_f"] - 1.0) / pw["w"])
    return np.max(ratios, axis=0), pw, g, gid


# ---------------------------------------------------------------------------
# exp and log of the binary32 footprint
# ---------------------------------------------------------------------------

def test_expf32_and_logf32_within_an_ulp_or_two():
    x = np.linspace(-86.9, 88.4, 40001, dtype=np.float32)
    e = oracle.expf32(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    assert np.max(np.abs(e - ref) / np.spacing(ref.astype(np.float32)).astype(np.float64)) <= 1.0
    y = np.exp(np.linspace(-80.0, 80.0, 40001)).astype(np.float32)
    y = np.concatenate([y, np.linspace(0.5, 2.0, 20001, dtype=np.float32), np.float32([1e-40, 3e-39])])
    l = oracle.logf32(y).astype(np.float64)
    ref = np.log(y.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(l - ref) / np.maximum(ulp, 2.0 ** -149)) <= 2.0
    assert oracle.logf32(np.float32([1.0]))[0] == 0.0 and oracle.expf32(np.float32([0.0]))[0] == 1.0
    assert oracle.expf32(np.float32([-90.0]))[0] == 0.0 and np.isinf(oracle.expf32(np.float32([89.0]))[0])


def test_binary32_footprint_agrees_with_fp64():
    """u, v, depth, o_hat and the conic of the binary32 footprint against the FP64 definition,
    within what binary32 rounding allows (closer for the mean than the conic of thin splats)."""
    sc = stress_scene()
    cam = synth.pinhole(160, 120)
    g = oracle.preprocess(sc, cam, 0.5)
    e = g["err"]
    d = g["drawn"] & (e[:, 15] == 1)
    assert d.sum() > 300
    np.testing.assert_allclose(e[d, 0], g["u"][d], rtol=0, atol=2e-4)
    np.testing.assert_allclose(e[d, 1], g["v"][d], rtol=0, atol=2e-4)
    np.testing.assert_allclose(e[d, 2], g["depth"][d], rtol=3e-7)
    np.testing.assert_allclose(e[d, 3], g["opacity_t"][d], rtol=2e-6)
    c = g["cov2d"][d]
    lmax = g["lambda_max"][d]
    kappa = lmax * lmax / (c[:, 0] * c[:, 2] - c[:, 1] ** 2)   # condition number of Sigma'
    scale = np.abs(g["conic"][d]).max(axis=1)
    for k in range(3):
        # first order: |d Sigma'^-1| <= |Sigma'^-1|^2 |d Sigma'|, |d Sigma'| ~ 8u lambda_max
        assert np.all(np.abs(e[d, 4 + k] - g["conic"][d, k]) <= 1e-6 * scale * kappa)


# ---------------------------------------------------------------------------
# the blend window
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["stress", "tiny", "scene"])
def test_blend_window_covers_fp32_and_is_tight(kind):
    if kind == "stress":
        sc, cam, t = stress_scene(), synth.pinhole(160, 120), 0.5
    elif kind == "tiny":
        w = synth.tiny_workload()
        sc, (cam, t) = w.scene, w.frames[0]
    else:
        sc = synth.make_scene(3000, 21, "box20", sh_degree=0)
        cam, t = synth.orbit(4, 320, 240, 300)[150]
    ratio, pw, g, gid = window_ratios(sc, cam, t)
    assert len(ratio) > 5000
    # sound: an independent FP32 blend never leaves the window
    assert ratio.max() <= 1.0, f"FP32 alpha outside the window: {ratio.max():.3g}"
    # tight: some pair comes within a factor 10 of it
    assert ratio.max() >= 0.1, f"window loose: best pair at {ratio.max():.3g} of it"


# ---------------------------------------------------------------------------
# the a-priori bounds (cov3d mode: slicing first)
# ---------------------------------------------------------------------------

def slicing_footprint_f32(sc4, cam, t):
    """The slicing-first footprint (Eq. 5-7, then the projection) in numpy float32, written
    independently of the oracle: R4 from the normalised quaternion pair, M4 = R4 diag(e^s),
    Sigma4D = M4 M4^T, V/W, Sigma3D = U - V (V/W)^T, mean at t, o_hat, (u, v), J W, Sigma'."""
    f = lambda a: np.asarray(a, np.float32)
    ql, qr = f(sc4.quat_l), f(sc4.quat_r)
    ql = ql / np.sqrt((ql * ql).sum(1, keepdims=True))
    qr = qr / np.sqrt((qr * qr).sum(1, keepdims=True))
    R4 = oracle.rot4(ql.astype(np.float64), qr.astype(np.float64)).astype(np.float32)
    s4 = np.exp(f(sc4.log_scales4))
    M4 = R4 * s4[:, None, :]
    S4 = np.einsum("nik,njk->nij", M4, M4)
    V, W = S4[:, :3, 3], S4[:, 3, 3]
    v = V / W[:, None]
    S3 = S4[:, :3, :3] - V[:, :, None] * v[:, None, :]
    m4 = f(sc4.means4)
    tau = F32(t) - m4[:, 3]
    m = m4[:, :3] + tau[:, None] * v
    R, T = f(cam.R), f(cam.T)
    X = m @ R.T + T
    o = F32(1) / (F32(1) + np.exp(-f(sc4.opacity_logit)))
    oh = o * np.exp((F32(-0.5) * tau * tau) / W)
    Z = X[:, 2]
    u = F32(cam.fx) * (X[:, 0] / Z) + F32(cam.cx)
    vv = F32(cam.fy) * (X[:, 1] / Z) + F32(cam.cy)
    limx = F32(1.3) * (F32(0.5 * cam.width) / F32(cam.fx))
    limy = F32(1.3) * (F32(0.5 * cam.height) / F32(cam.fy))
    xzc = np.clip(X[:, 0] / Z, -limx, limx)
    yzc = np.clip(X[:, 1] / Z, -limy, limy)
    n = len(Z)
    J = np.zeros((n, 2, 3), np.float32)
    J[:, 0, 0] = F32(cam.fx) / Z
    J[:, 0, 2] = -(F32(cam.fx) * xzc) / Z
    J[:, 1, 1] = F32(cam.fy) / Z
    J[:, 1, 2] = -(F32(cam.fy) * yzc) / Z
    JW = J @ R
    S2 = JW @ S3 @ np.swapaxes(JW, 1, 2) + F32(0.3) * np.eye(2, dtype=np.float32)
    return dict(u=u, v=vv, Z=Z, oh=oh, s00=S2[:, 0, 0], s01=S2[:, 0, 1], s11=S2[:, 1, 1])


def test_apriori_bounds_cover_fp32_slicing():
    """In cov3d mode the oracle bounds, a priori, how far an FP32 evaluation of the slicing-first
    form lands from FP64: the mean, depth, opacity and Sigma' of an independent numpy float32
    evaluation stay within them, and so does its alpha (windowed per pair)."""
    sc4 = synth.make_scene4d(600, 41, "tiny", mix=0.3)
    sc4.log_scales4[:, :3] = np.random.default_rng(7).normal(-3.0, 1.5, (600, 3)).astype(np.float32)   # thin splats
    cam, t = synth.pinhole(128, 128), 0.4
    static, cov6 = oracle.slice4d(sc4, t)
    g = oracle.preprocess(static, cam, t, cov3d=cov6, in_err=oracle.slice4d_fp32_bounds(sc4, t))
    f = slicing_footprint_f32(sc4, cam, t)
    e = g["err"]
    d = g["drawn"] & (f["Z"] > 0.2) & (f["oh"] >= F32(AMIN))
    assert d.sum() > 200 and np.all(e[d, 15] == 0)
    assert np.all(np.abs(f["u"][d] - g["u"][d]) <= e[d, 8])
    assert np.all(np.abs(f["v"][d] - g["v"][d]) <= e[d, 9])
    assert np.all(np.abs(f["Z"][d] - g["depth"][d]) <= e[d, 10])
    assert np.all(np.abs(f["oh"][d] / g["opacity_t"][d] - 1) <= e[d, 11])
    for k, name in enumerate(("s00", "s01", "s11")):
        assert np.all(np.abs(f[name][d] - g["cov2d"][d, k]) <= e[d, 12 + k]), name
    # the windowed alpha: the footprint's alpha within the pair's window of the FP64 alpha
    b = dict(tiles_touched=np.where(d, 1, 0))
    gid, pix = pair_sample(g, b, cam)
    pw = oracle.pair_windows(g, gid, pix)
    uv = np.stack([f["u"], f["v"]], 1)[gid]
    foot = np.stack([f["oh"], f["s00"], f["s01"], f["s11"]], 1)[gid]
    for order in ("fma", "plain"):
        a32 = blend_alpha_f32(uv, foot, pix, order)
        assert np.all(np.abs(a32 / pw["alpha_f"] - 1) <= pw["w"]), order


# ---------------------------------------------------------------------------
# the slack on whole images
# ---------------------------------------------------------------------------

def pixel_walks(g, cam, keys):
    """Per pixel, independently in numpy from the FP64 2D Gaussians: the kept candidates in
    (depth, index) order up to the one that stops the pixel, their alphas, T before each and
    the stop tests; also the Gaussians near the alpha threshold anywhere before the stop."""
    ids = np.nonzero(g["drawn"])[0]
    H, W = cam.height, cam.width
    out = []
    for y in range(H):
        px = np.arange(W) + 0.5
        dx = g["u"][ids][None, :] - px[:, None]
        dy = g["v"][ids][None, :] - (y + 0.5)
        a, b, c = (g["conic"][ids, k][None, :] for k in range(3))
        p = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        al = np.minimum(0.99, g["opacity_t"][ids][None, :] * np.exp(np.minimum(p, 0.0)))
        for x in range(W):
            row = al[x]
            kept = np.nonzero(row >= AMIN)[0]
            order = np.lexsort((ids[kept], g["depth"][ids[kept]]))
            seq = ids[kept][order]
            als = row[kept][order]
            T = 1.0
            Ts, tests, n_bl = [], [], 0
            for k in range(len(seq)):
                test = T * (1 - als[k])
                Ts.append(T)
                tests.append(test)
                if test < 1e-4:
                    break
                T = test
                n_bl += 1
            reach = len(Ts)                      # candidates up to and including the stopper
            zmax = g["depth"][seq[reach - 1]] if reach else np.inf
            near_ids = np.nonzero(np.abs(row / AMIN - 1.0) <= 1e-2)[0]
            out.append(dict(seq=seq[:reach], alpha=als[:reach], T=np.array(Ts), tests=np.array(tests),
                            nblend=n_bl, zmax=zmax, near=ids[near_ids], near_alpha=row[near_ids],
                            cmax=float(g["rgb"][seq].max()) if len(seq) else 0.0))
    return out


@pytest.mark.parametrize("kind", ["tiny", "stress"])
def test_slack_zero_away_from_thresholds(kind):
    """A pixel has slack 0 when, with R = 1e-3: every Gaussian's FP64 alpha at it before the stop
    is more than R (relative) from 1/255, every stop test more than R from 1e-4, no two of its
    kept Gaussians up to the stop are within 1e-5 relative in depth, and the binary32 footprint's
    alphas are within R/10 of the FP64 ones there."""
    if kind == "tiny":
        w = synth.tiny_workload()
        sc, (cam, t) = w.scene, w.frames[0]
        cam = synth.pinhole(64, 64)
    else:
        sc, cam, t = stress_scene(spread=1.3), synth.pinhole(48, 40), 0.5
    ref = oracle.render(sc, cam, t)
    g = ref["g2d"]
    walks = pixel_walks(g, cam, None)
    R = 1e-3
    slack = ref["slack"].reshape(-1)
    clear_count = 0
    for q, wk in enumerate(walks):
        before = wk["near"][g["depth"][wk["near"]] <= wk["zmax"]] if len(wk["seq"]) else wk["near"]
        if len(before):
            continue
        if np.any(np.abs(wk["tests"] / 1e-4 - 1.0) <= R):
            continue
        z = np.sort(g["depth"][wk["seq"]])
        if len(z) > 1 and np.any(np.diff(z) <= 1e-5 * z[1:]):
            continue
        x, y = q % cam.width + 0.5, q // cam.width + 0.5
        e = g["err"][wk["seq"]]
        pf = -0.5 * (e[:, 4] * (e[:, 0] - x) ** 2 + e[:, 6] * (e[:, 1] - y) ** 2) - e[:, 5] * (e[:, 0] - x) * (e[:, 1] - y)
        af = np.minimum(0.99, e[:, 3] * np.exp(np.minimum(pf, 0)))
        if len(af) and np.max(np.abs(af / wk["alpha"] - 1)) > R / 10:
            continue
        clear_count += 1
        assert slack[q] == 0.0, f"pixel {q}: slack {slack[q]:.3g} far from every threshold"
    assert clear_count >= 0.8 * len(walks)


@pytest.mark.parametrize("kind", ["tiny", "stress", "box"])
def test_slack_within_flip_bound(kind):
    """No pixel's slack exceeds what flips near its thresholds can move it (Eq. 4): for each
    Gaussian before the stop within 1% of 1/255, 2 (1.01) alpha T max c; for each stop test
    within 1% of 1e-4, T alpha max c + 2e-4 max c; for each pair of kept Gaussians up to the
    stop within 1e-5 in relative depth, 2 alpha_i alpha_j max c; plus 1e-7 per decision."""
    if kind == "tiny":
        w = synth.tiny_workload()
        sc, (cam, t) = w.scene, w.frames[0]
        cam = synth.pinhole(64, 64)
    elif kind == "stress":
        sc, cam, t = stress_scene(spread=1.3), synth.pinhole(48, 40), 0.5
    else:   # dense enough that some pixels carry slack
        sc = synth.make_scene(30000, 21, "box20", sh_degree=3)
        cam, t = synth.orbit(4, 96, 72, 300)[150]
    ref = oracle.render(sc, cam, t)
    g = ref["g2d"]
    walks = pixel_walks(g, cam, None)
    slack = ref["slack"].reshape(-1)
    flagged = 0
    for q, wk in enumerate(walks):
        cmax = max(wk["cmax"], float(g["rgb"][wk["near"]].max()) if len(wk["near"]) else 0.0)
        bound = 0.0
        for i, a in zip(wk["near"], wk["near_alpha"]):
            if len(wk["seq"]) and g["depth"][i] > wk["zmax"]:
                continue
            pos = np.searchsorted(g["depth"][wk["seq"]], g["depth"][i])
            Tb = wk["T"][pos] if pos < len(wk["T"]) else (wk["T"][-1] if len(wk["T"]) else 1.0)
            bound += 2.02 * a * Tb * cmax + 1e-7
        for k in range(len(wk["tests"])):
            if abs(wk["tests"][k] / 1e-4 - 1.0) <= 1e-2:
                bound += wk["T"][k] * wk["alpha"][k] * cmax + 2e-4 * cmax
        z = g["depth"][wk["seq"]]
        for i in range(len(z)):
            for j in range(i + 1, len(z)):
                if abs(z[i] - z[j]) <= 1e-5 * max(z[i], z[j]):
                    bound += 2.0 * wk["alpha"][i] * wk["alpha"][j] * cmax * wk["T"][i] + 1e-7
        flagged += slack[q] > 0
        assert slack[q] <= bound + 1e-12, f"pixel {q}: slack {slack[q]:.3g} above the flip bound {bound:.3g}"
    assert flagged >= 5 or kind != "box"


def test_slack_covers_depth_key_swap():
    """Two overlapping splats 2e-7 apart in depth at z = 5 (the first moves 4e-7 per unit time,
    half a unit from its temporal centre): their binary32 depths round to the same key, so a
    renderer ordering the tile lists by (key, index) blends the deeper one (lower index) first;
    the slack covers the colour change of the swap, alpha_1 alpha_2 |c_1 - c_2|."""
    cam = synth.pinhole(32, 32)
    sc = synth.make_scene(2, 0, "tiny")
    sc.means[:] = np.float32([[0.0, 0.0, 5.0], [0.0, 0.0, 5.0]])
    sc.velocity[:] = np.float32([[0.0, 0.0, 4e-7], [0.0, 0.0, 0.0]])
    sc.t_mean[:] = np.float32(0.0)
    sc.log_scales[:] = np.float32(math.log(0.3))
    sc.quats[:] = np.float32([1, 0, 0, 0])
    sc.opacity_logit[:] = np.float32(0.0)
    sc.log_t_scale[:] = np.float32(30.0)
    sc.sh[:, 0, :] = np.float32([[(0.9 - 0.5) / synth.SH_C0] * 3, [(0.1 - 0.5) / synth.SH_C0] * 3])
    ref = oracle.render(sc, cam, 0.5, pixels=np.array([[16, 16]]))
    g = ref["g2d"]
    assert g["err"][0, 2] == g["err"][1, 2] and g["depth"][0] > g["depth"][1]
    ap = oracle.pair_windows(g, np.int32([0, 1]), np.int32([[16, 16], [16, 16]]))["alpha"]
    a0, a1 = np.minimum(0.99, ap)
    swap = a0 * a1 * abs(g["rgb"][0, 0] - g["rgb"][1, 0])
    assert swap > 0.05
    assert ref["slack"][0] >= swap * (1 - 1e-9)


def test_near_plane_straddle_is_flagged():
    """A splat at z = float32(0.2) = 0.2 + 3e-9: the definition (z > 0.2) draws it, binary32
    (z > 0.2f) culls it.  Its pixels carry at least the colour it adds (alpha T c)."""
    cam = synth.pinhole(32, 32)
    sc = synth.make_scene(1, 0, "tiny")
    sc.means[:] = np.float32([[0.0, 0.0, 0.2]])
    sc.velocity[:] = 0
    sc.log_scales[:] = np.float32(math.log(0.002))
    sc.quats[:] = np.float32([1, 0, 0, 0])
    sc.opacity_logit[:] = np.float32(2.0)
    sc.log_t_scale[:] = np.float32(30.0)
    ref = oracle.render(sc, cam, 0.5, pixels=np.array([[16, 16]]))
    g = ref["g2d"]
    assert g["drawn"][0] and g["err"][0, 7] == 1
    assert ref["rgb"][0].max() > 0.05
    assert ref["slack"][0] >= ref["rgb"][0].max()


# ---------------------------------------------------------------------------
# the gradient slack (oracle.backward with_slack)
# ---------------------------------------------------------------------------

def test_gradient_slack_zero_for_gaussians_away_from_near_decisions():
    """Only a Gaussian that takes part in a pixel carrying image slack (alpha there at least
    1/510 in FP64) can carry gradient slack: every other element's slack is exactly 0."""
    sc = synth.make_scene(30000, 21, "box20", sh_degree=1)
    cam, t = synth.orbit(4, 96, 72, 300)[150]
    ref = oracle.render(sc, cam, t)
    G = np.random.default_rng(1).standard_normal((cam.height, cam.width, 3))
    _, slack = oracle.backward(sc, cam, t, G, with_slack=True)
    g = ref["g2d"]
    flagged = np.argwhere(ref["slack"] > 0)
    assert len(flagged) >= 3
    touch = np.zeros(sc.n, bool)
    ids = np.nonzero(g["drawn"] | (g["err"][:, 7] == 2))[0]
    for y, x in flagged:
        dx, dy = g["u"][ids] - (x + 0.5), g["v"][ids] - (y + 0.5)
        a, b, c = (g["conic"][ids, k] for k in range(3))
        p = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        touch[ids[g["opacity_t"][ids] * np.exp(np.minimum(p, 0)) >= AMIN / 2]] = True
    any_slack = np.zeros(sc.n, bool)
    for f, v in slack.items():
        per = np.abs(v.reshape(sc.n, -1)).max(axis=1)
        assert np.all(per[~touch] == 0.0), f
        any_slack |= per > 0
    assert any_slack.sum() >= 3


def test_gradient_slack_covers_a_threshold_jump():
    """Two splats on the optical axis, the front one's alpha at the four pixels around the axis
    set 1e-9 above 1/255: a renderer that drops it there changes the back splat's gradients by
    the jump between the FP64 gradients just above and just below the threshold; the slack at
    the threshold covers that jump."""
    cam = synth.pinhole(32, 32)

    def scene(logit_a):
        sc = synth.make_scene(2, 0, "tiny", sh_degree=0)
        sc = synth.Scene(**{k: np.asarray(v, np.float64).copy() for k, v in sc.arrays().items()}, sh_degree=0)
        sc.means[:] = [[0.0, 0.0, 2.0], [0.01, -0.02, 3.0]]
        sc.velocity[:] = 0.0
        sc.t_mean[:] = 0.5
        sc.log_t_scale[:] = 30.0
        sc.log_scales[:] = np.log(0.02)
        sc.quats[:] = [1.0, 0.0, 0.0, 0.0]
        sc.opacity_logit[:] = [logit_a, 0.5]
        sc.sh[:, 0, :] = (np.array([[0.9, 0.2, 0.4], [0.1, 0.7, 0.3]]) - 0.5) / synth.SH_C0
        return sc

    g = oracle.preprocess(scene(0.0), cam, 0.5)
    dx, dy = g["u"][0] - 16.5, g["v"][0] - 16.5
    a, b, c = g["conic"][0]
    p = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
    logit = lambda oh: math.log(oh / (1.0 - oh))
    oh0 = AMIN * (1 + 1e-9) / math.exp(p)
    G = np.ones((32, 32, 3))
    base, slack = oracle.backward(scene(logit(oh0)), cam, 0.5, G, with_slack=True)
    hi = oracle.backward(scene(logit(oh0 * (1 + 1e-7))), cam, 0.5, G)
    lo = oracle.backward(scene(logit(oh0 * (1 - 1e-7))), cam, 0.5, G)
    for f in ("sh", "opacity_logit", "means", "log_scales"):
        jump = np.abs(hi[f][1] - lo[f][1]).max()
        assert jump > 1e-6, f
        assert slack[f][1].max() >= 0.99 * jump, (f, slack[f][1].max(), jump)
