"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of ``oracle/oracle.c`` (on the
CPU; the real oracle is untouched; every occurrence of the anchor is changed),
builds it, points the pin tests at the mutant, and requires at least one of the
named pins to fail.
"""
import importlib.util
import os
import shutil

import pytest

import tests.test_oracle_adjoint as adjoint_pins
import tests.test_oracle_pins as pins
import tests.test_oracle_slack as slack_pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    ("dropped dilation", "#define ORC_DILATION 0.3", "#define ORC_DILATION 0.0",
     ["test_single_gaussian_on_axis_closed_form"]),
    ("time shift sign (Eq. 7 vs Alg. 1)",
     "m[j] = sc->means[3 * (size_t)i + j] + tau * sc->velocity", "m[j] = sc->means[3 * (size_t)i + j] - tau * sc->velocity",
     ["test_moving_gaussian_closed_form", "test_disentangled_equals_slicing_first"]),
    ("temporal factor without the 1/2", "double oh = o * exp(-0.5 * tau * tau / (st * st));",
     "double oh = o * exp(-tau * tau / (st * st));", ["test_moving_gaussian_closed_form"]),
    ("Jacobian off-diagonal sign", "-cam->fx * xzc / Z, 0.0, cam->fy / Z, -cam->fy * yzc / Z",
     "cam->fx * xzc / Z, 0.0, cam->fy / Z, -cam->fy * yzc / Z", ["test_single_gaussian_off_axis_closed_form"]),
    ("fx / fy swapped in the Jacobian", "double J[6] = {cam->fx / Z, 0.0,", "double J[6] = {cam->fy / Z, 0.0,",
     ["test_single_gaussian_on_axis_closed_form"]),
    ("camera rotation transposed", "X[r] = cam->R[3 * r + 0] * m[0] + cam->R[3 * r + 1] * m[1] + cam->R[3 * r + 2] * m[2]",
     "X[r] = cam->R[0 + r] * m[0] + cam->R[3 + r] * m[1] + cam->R[6 + r] * m[2]",
     ["test_single_gaussian_on_axis_closed_form"]),
    ("conic off-diagonal sign", "out->conic[3 * (size_t)i + 1] = -c01 / det;", "out->conic[3 * (size_t)i + 1] = c01 / det;",
     ["test_single_gaussian_off_axis_closed_form"]),
    ("pixel centre without +0.5", "double x = (px ? px[q] : (int32_t)(q % W)) + 0.5;",
     "double x = (px ? px[q] : (int32_t)(q % W));", ["test_single_gaussian_on_axis_closed_form"]),
    ("blend after the stop test", "const int stop = test < ORC_T_MIN;", "const int stop = test < 0.0;", ["test_composite_golden"]),
    ("no alpha clamp", "double alpha = fmin(ORC_ALPHA_MAX,", "double alpha = fmin(1.0,", ["test_composite_golden"]),
    ("back-to-front order", "if (a->depth < b->depth) return -1;\n    if (a->depth > b->depth) return 1;",
     "if (a->depth < b->depth) return 1;\n    if (a->depth > b->depth) return -1;", ["test_composite_golden"]),
    ("quaternion order xyzw", "double w = q[0], x = q[1], y = q[2], z = q[3];",
     "double x = q[0], y = q[1], z = q[2], w = q[3];", ["test_quat_to_rot_matches_scipy"]),
    ("SH degree-1 sign", "Y[1] = -c1 * y;", "Y[1] = c1 * y;", ["test_sh_basis_matches_scipy"]),
    ("SH direction of the static mean",
     "const double *cm = sc->colour_static ? sc->means + 3 * (size_t)i : m;",
     "const double *cm = sc->means + 3 * (size_t)i;",
     ["test_time_shift_equivalence"]),
    ("colour not clamped at zero", "out->rgb[3 * (size_t)i + ch] = fmax(0.0, s + 0.5);",
     "out->rgb[3 * (size_t)i + ch] = s + 0.5;", ["test_negative_colour_is_clamped"]),
    ("FP32 radius factor 3.0", "float rf = ceilf(3.33f * sqrtf(lam));", "float rf = ceilf(3.0f * sqrtf(lam));",
     ["test_bin_f32_agrees_with_fp64"]),
    ("FP32 binning ellipse without the factor 2", "float k2 = ((2.0f * orc_logf(255.0f * oh)) * 1.0008f) + 0.0008f;",
     "float k2 = ((1.0f * orc_logf(255.0f * oh)) * 1.0008f) + 0.0008f;", ["test_tile_rect_covers_alpha_support"]),
    ("FP32 binning ellipse with the wrong axis", "float ex = sqrtf(k2 * s00), ey = sqrtf(k2 * s11);",
     "float ex = sqrtf(k2 * s11), ey = sqrtf(k2 * s00);", ["test_tile_rect_covers_alpha_support"]),
    ("FP32 rect with truncation", "float fx0 = floorf((u - rx) / tilef)", "float fx0 = floorf((u - rx) / tilef) + 1.0f",
     ["test_tile_rect_covers_alpha_support"]),
    ("column cuts on the wrong branch", "((v + ((s01 * xt) - sqrtf(", "((v + ((s01 * xt) + sqrtf(",
     ["test_column_trims_match_fp64_box_test", "test_tile_rect_covers_alpha_support"]),
    ("column cuts at the bottom point's abscissa", "const float xt = fminf(fmaxf(-xl, a), b)",
     "const float xt = fminf(fmaxf(xl, a), b)", ["test_column_trims_match_fp64_box_test"]),
    ("column cuts counted from the rectangle's last row", "cut_t = (int32_t)fminf(fmaxf(ceilf(flo) - (float)y0",
     "cut_t = (int32_t)fminf(fmaxf(ceilf(flo) - (float)(y0 + 1)", ["test_column_trims_match_fp64_box_test"]),
    # the per-pixel slack (tests/test_oracle_slack.py)
    ("slack window 10 times too wide", "    return ORC_SAFETY * w;\n}", "    return 10.0 * ORC_SAFETY * w;\n}",
     ["test_blend_window_covers_fp32_and_is_tight"]),
    ("slack window without the quadratic form's rounding (thin splats)",
     "const double dp_eval = 13.0 * u * Q + u * fabs(p);", "const double dp_eval = u * fabs(p);",
     ["test_blend_window_covers_fp32_and_is_tight"]),
    ("a-priori camera-space bound without the mean's own error (cov3d mode)", "dX[r] = prop + 4.0 * u * mag;",
     "dX[r] = 4.0 * u * mag;", ["test_apriori_bounds_cover_fp32_slicing"]),
    ("a-priori bound of Sigma' without the propagated factor error", "dv += dF[3 * r + k] * fabs(G[3 * q2 + k]) + fabs(F[3 * r + k]) * dG[3 * q2 + k];",
     "dv += 0.0;", ["test_apriori_bounds_cover_fp32_slicing"]),
    ("depth-key order ignored", "if (!sorted) {", "if (0) {", ["test_slack_covers_depth_key_swap"]),
    ("near-plane straddle ignored", "} else if (f32_draws == 0) {\n            mode = 1;", "} else if (0) {\n            mode = 1;",
     ["test_near_plane_straddle_is_flagged"]),
    ("slack of an alpha flip four times too big",
     "slack += 2.0 * fmax(fabs(alpha), af) * (1.0 + cand[k].w) * cmax * T + 1e-7;",
     "slack += 8.0 * fmax(fabs(alpha), af) * (1.0 + cand[k].w) * cmax * T + 1e-7;", ["test_slack_within_flip_bound"]),
    ("slack on every pixel", "if (out_slack) out_slack[q] = slack;", "if (out_slack) out_slack[q] = slack + 1e-6;",
     ["test_slack_zero_away_from_thresholds"]),
    ("gradient slack without the alpha flips", "if (cand[k].near_alpha) near_pos[nn++] = (int64_t)k;",
     "if (0) near_pos[nn++] = (int64_t)k;", ["test_gradient_slack_covers_a_threshold_jump"]),
    ("gradient slack through the signed Jacobian", "if (accumulate_abs) dst[f][j] += fabs(r[o]) * *w;",
     "if (accumulate_abs) dst[f][j] += r[o] * *w;", ["test_gradient_slack_covers_a_threshold_jump"]),
    # adjoint (caught by the finite-difference pin)
    ("adjoint: colour behind ignored", "dalpha += Ti * G[ch] * (c[ch] - B[ch]);", "dalpha += Ti * G[ch] * c[ch];",
     ["test_adjoint_matches_central_differences"]),
    ("adjoint: conic off-diagonal", "gi[3] = -dp * dx * dy;", "gi[3] = -0.5 * dp * dx * dy;",
     ["test_adjoint_matches_central_differences"]),
    ("adjoint: velocity dropped from dtau", "dtau += sc->velocity[3 * (size_t)i + j] * dm[j];", "dtau += 0.0 * dm[j];",
     ["test_adjoint_matches_central_differences"]),
    ("adjoint: quaternion normalisation", "gq[j] = (dqn[j] - qn[j] * dot) / nq;", "gq[j] = dqn[j] / nq;",
     ["test_adjoint_matches_central_differences"]),
]

ARGSETS = {
    "test_blend_window_covers_fp32_and_is_tight": [dict(kind="stress")],
    "test_slack_within_flip_bound": [dict(kind="box")],
    "test_slack_zero_away_from_thresholds": [dict(kind="tiny")],
    "test_single_gaussian_on_axis_closed_form": [dict(rotated=False), dict(rotated=True)],
    "test_column_trims_match_fp64_box_test": [dict(tile=16, frame=0), dict(tile=32, frame=150)],
    "test_tile_rect_covers_alpha_support": [dict(trim=True)],
    "test_bin_f32_agrees_with_fp64": [dict(trim=False), dict(trim=True)],
    "test_adjoint_matches_central_differences": [dict(deg=0), dict(deg=3)],
}


def _load_mutant(tmp, name, old, new):
    d = tmp / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), d, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    src = (d / "oracle.c").read_text()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"   # every occurrence is mutated
    (d / "oracle.c").write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{abs(hash(name))}", d / "__init__.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


@pytest.mark.parametrize("name,old,new,tests", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, monkeypatch, name, old, new, tests):
    mod = _load_mutant(tmp_path, name, old, new)
    monkeypatch.setattr(pins, "oracle", mod)
    monkeypatch.setattr(adjoint_pins, "oracle", mod)
    monkeypatch.setattr(slack_pins, "oracle", mod)
    caught = []
    for tname in tests:
        fn = getattr(pins, tname, None) or getattr(slack_pins, tname, None) or getattr(adjoint_pins, tname)
        argsets = ARGSETS.get(tname, [{}])
        for kw in argsets:
            try:
                fn(**kw)
            except (AssertionError, FloatingPointError, ValueError, ZeroDivisionError):
                caught.append(tname)
    assert caught, f"no pin caught the mutant '{name}'"
