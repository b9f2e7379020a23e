"""Temporal and spatial splitting on the GPU (needs a GPU): the statistics
accumulation and the split against the oracle (decisions bit-exact, children
in the same order, values within FP32 rounding)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def test_accumulate_sums_gradient_norms():
    m = gu.d4()
    rng = np.random.default_rng(81)
    n = 1000
    g = {k: torch.zeros(s, device="cuda") for k, s in (("means", (n, 3)), ("t_mean", (n,)), ("velocity", (n, 3)),
                                                      ("log_scales", (n, 3)), ("log_t_scale", (n,)),
                                                      ("quats", (n, 4)), ("opacity_logit", (n,)), ("sh", (n, 1, 3)))}
    stats = torch.zeros((n, 3), device="cuda")
    ref = np.zeros((n, 3))
    for step in range(3):
        gm = rng.normal(0, 1, (n, 3)) * (rng.uniform(0, 1, (n, 1)) > 0.3)
        gt = rng.normal(0, 1, n) * (gm[:, 0] != 0)
        g["means"].copy_(torch.tensor(gm, dtype=torch.float32))
        g["t_mean"].copy_(torch.tensor(gt, dtype=torch.float32))
        m.d4dgs_split_accumulate(g, stats)
        gm32, gt32 = gm.astype(np.float32).astype(np.float64), gt.astype(np.float32).astype(np.float64)
        nz = (np.abs(gm32).sum(1) > 0) | (gt32 != 0)
        ref[:, 0] += np.linalg.norm(gm32, axis=1) * nz
        ref[:, 1] += np.abs(gt32) * nz
        ref[:, 2] += nz
    np.testing.assert_allclose(stats.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("deg", [0, 3])
def test_split_matches_oracle(deg):
    m = gu.d4()
    sc = synth.make_scene(5000, 82, "box20", sh_degree=deg)
    rng = np.random.default_rng(83)
    stats = np.column_stack([rng.uniform(0, 1, sc.n), rng.uniform(0, 1, sc.n), rng.integers(0, 4, sc.n)]).astype(np.float32)
    normals = rng.standard_normal((sc.n, 4)).astype(np.float32)
    prm = dict(tau_xyz=0.6, tau_t=0.7, log_min_xyz=float(np.float32(-0.2)), log_min_t=float(np.float32(-1.6)))
    ds = m.DeviceScene.from_host(sc)
    out, cnt = m.d4dgs_split(ds, torch.tensor(stats, device="cuda"), torch.tensor(normals, device="cuda"), **prm)
    ref, ss, tt = oracle.split_scene(sc, stats, normals, **prm)
    assert 0 < ss.sum() < sc.n and 0 < tt.sum() < sc.n and (ss & tt).any()
    assert cnt == ref.n
    for k, v in out.t.items():
        got = v.cpu().numpy().astype(np.float64)
        exp = getattr(ref, k).reshape(got.shape)
        np.testing.assert_allclose(got, exp, rtol=2e-6, atol=2e-6 * max(1.0, np.abs(exp).max()), err_msg=k)
