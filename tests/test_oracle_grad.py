"""Pins of the oracle's sigma gradient (Sec. 4: trainable sigmas): the analytic
derivative of the mean squared depth error against central finite differences
of the plain oracle pipeline, for the single stage and through the two-stage
restore chain."""
import numpy as np
import pytest


def _loss(oracle_mod, v, gt, num_stages, stages):
    r = oracle_mod.densify_view(v, num_stages=num_stages, stages=stages, emit_points=False)
    m = r["valid"].astype(bool) & (gt > 0)
    return float(((r["depth"][m] - gt[m]) ** 2).sum() / m.sum())


@pytest.mark.parametrize("num_stages,stages", [
    (1, ((3, 2.5, 18.0),)),
    (2, ((4, 5.0, 20.0), (2, 5.0, 20.0))),
])
def test_gradient_matches_finite_differences(oracle_mod, small_view, num_stages, stages):
    v = small_view
    gt = v.gt_depth.astype(np.float64)
    gt[~np.isfinite(gt)] = 0.0
    loss, grad, n = oracle_mod.sigma_loss_grad(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], gt,
                                               num_stages=num_stages, stages=stages)
    assert n > 1000
    assert loss == pytest.approx(_loss(oracle_mod, v, gt, num_stages, stages), rel=1e-12)
    flat = [x for st in stages for x in st[1:]]
    for k in range(len(flat)):
        h = 1e-4 * flat[k]
        vals = []
        for sgn in (+1, -1):
            f = list(flat)
            f[k] += sgn * h
            st = tuple((stages[i][0], f[2 * i], f[2 * i + 1]) for i in range(len(stages)))
            vals.append(_loss(oracle_mod, v, gt, num_stages, st))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, abs(fd))), (k, grad[k], fd)
    if num_stages == 1:
        assert np.all(grad[2:] == 0)


def test_grad_forward_equals_filter(oracle_mod):
    rng = np.random.default_rng(21)
    H, W = 17, 23
    guide = rng.integers(0, 256, (H, W, 3)).astype(float)
    beta = (rng.random((H, W)) < 0.3).astype(float)
    bd = beta * rng.uniform(1, 5, (H, W))
    out, valid, _ = oracle_mod.jbf_grad(guide, beta, bd, 3, 2.0, 15.0)
    ref, rv = oracle_mod.jbf_gather(guide, beta, bd, 3, 2.0, 15.0)
    assert np.array_equal(valid, rv)
    np.testing.assert_allclose(out, ref, rtol=1e-13)
