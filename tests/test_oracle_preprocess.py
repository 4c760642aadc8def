"""Pins of the oracle's preprocessing and post-filtering steps (Sec. 4.1
afterimage and occluded-point removal, Sec. 5 contour removal), against
hand-built cases, scipy morphology and an independent numpy float32
evaluation of the stated arithmetic."""
import numpy as np
import pytest

EMPTY = 0x7F800000


def _zb(depth):
    d = np.asarray(depth, np.float32)
    z = d.view(np.uint32).copy()
    z[~np.isfinite(d)] = EMPTY
    return z


# ---------------------------------------------------------------------------
# occluded-point removal
# ---------------------------------------------------------------------------
def test_occlusion_removes_the_point_behind_a_surface(oracle_mod):
    H, W = 9, 11
    d = np.full((H, W), np.inf, np.float32)
    d[::2, ::2] = 2.0                  # sparse foreground surface at 2 m
    d[4, 5] = 6.0                      # a background point seen through it
    d[3, 3] = 2.2                      # slightly behind: kept with margin 0.3
    z, n = oracle_mod.occlusion(_zb(d).ravel(), W, H, 2, 0.3)
    z = z.reshape(H, W)
    assert n == 1 and z[4, 5] == EMPTY and z[3, 3] != EMPTY
    keep = np.isfinite(d)
    keep[4, 5] = False
    assert np.array_equal(z[keep], _zb(d)[keep])


def test_occlusion_matches_numpy_float32(oracle_mod):
    rng = np.random.default_rng(3)
    H, W, rho, margin = 23, 31, 3, np.float32(0.25)
    d = rng.uniform(1, 4, (H, W)).astype(np.float32)
    d[rng.random((H, W)) < 0.7] = np.inf
    z, n = oracle_mod.occlusion(_zb(d).ravel(), W, H, rho, float(margin))
    ref = _zb(d).copy()
    removed = 0
    for y in range(H):
        for x in range(W):
            if not np.isfinite(d[y, x]):
                continue
            s, c = np.float32(0), 0
            for dy in range(-rho, rho + 1):
                row = np.float32(0)
                for dx in range(-rho, rho + 1):
                    qy, qx = y + dy, x + dx
                    if 0 <= qy < H and 0 <= qx < W and np.isfinite(d[qy, qx]):
                        row = np.float32(row + d[qy, qx])
                        c += 1
                s = np.float32(s + row)
            if d[y, x] > np.float32(np.float32(s / np.float32(c)) + margin):
                ref[y, x] = EMPTY
                removed += 1
    assert n == removed > 0
    assert np.array_equal(z, ref.ravel())


# ---------------------------------------------------------------------------
# afterimage removal
# ---------------------------------------------------------------------------
def test_motion_mask_is_threshold_then_closing(oracle_mod):
    from scipy.ndimage import binary_dilation, binary_erosion
    rng = np.random.default_rng(4)
    H, W = 29, 37
    prev = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    cur = prev.copy()
    moving = rng.random((H, W)) < 0.08
    cur[moving] = rng.integers(0, 256, (int(moving.sum()), 3), dtype=np.uint8)
    tau, c = 30.0, 2
    m = oracle_mod.motion_mask(cur, prev, tau, c)
    d2 = ((cur.astype(np.int64) - prev.astype(np.int64)) ** 2).sum(-1)
    raw = d2 > tau * tau
    se = np.ones((2 * c + 1, 2 * c + 1), bool)
    ref = binary_erosion(binary_dilation(raw, se, border_value=0), se, border_value=1)
    assert np.array_equal(m.astype(bool), ref)


def test_masked_projection_drops_old_scans_in_motion(oracle_mod):
    W, H, f, cx, cy = 16, 12, 64.0, 8.0, 6.0
    I = np.eye(4)
    _, M = oracle_mod.compose(I, I)
    p = np.array([[(3 + 0.5 - cx) * 4 / f, (5 + 0.5 - cy) * 4 / f, 4.0]], np.float32)
    mask = np.zeros((H, W), np.uint8)
    mask[5, 3] = 1
    for newest, kept in ((False, 0), (True, 1)):
        zb = np.full(W * H, EMPTY, np.uint32)
        _, k = oracle_mod.project_masked(M, p, W, H, f, f, cx, cy, mask, newest, zb)
        assert k == kept and (zb != EMPTY).sum() == kept
    zb = np.full(W * H, EMPTY, np.uint32)
    mask[5, 3] = 0
    _, k = oracle_mod.project_masked(M, p, W, H, f, f, cx, cy, mask, False, zb)
    assert k == 1


# ---------------------------------------------------------------------------
# contour removal
# ---------------------------------------------------------------------------
def test_contour_drops_both_sides_of_a_step_only(oracle_mod):
    H, W = 6, 10
    d = np.where(np.arange(W)[None, :] < 5, 2.0, 4.0).astype(np.float32) * np.ones((H, 1), np.float32)
    d[:, :5] += np.linspace(0, 0.01, 5, dtype=np.float32)[None, :]   # a gentle ramp is kept
    v = np.ones((H, W), np.uint8)
    v[0, 0] = 0
    do, vo, n = oracle_mod.contour(d, v, 0.1)
    dropped = (v == 1) & (vo == 0)
    assert np.array_equal(np.nonzero(dropped.any(0))[0], [4, 5])
    assert n == 2 * H and np.all(do[vo == 0][1:] == 0)
    assert vo[0, 0] == 0


def test_contour_matches_numpy_float32(oracle_mod):
    rng = np.random.default_rng(5)
    H, W, t = 17, 23, np.float32(0.05)
    d = rng.uniform(1, 3, (H, W)).astype(np.float32)
    v = (rng.random((H, W)) < 0.8).astype(np.uint8)
    do, vo, n = oracle_mod.contour(d, v, float(t))
    ref = v.copy()
    for y in range(H):
        for x in range(W):
            if not v[y, x]:
                continue
            lim = np.float32(t * d[y, x])
            for qy, qx in ((y, x - 1), (y, x + 1), (y - 1, x), (y + 1, x)):
                if 0 <= qy < H and 0 <= qx < W and v[qy, qx] and abs(np.float32(d[qy, qx] - d[y, x])) > lim:
                    ref[y, x] = 0
    assert np.array_equal(vo, ref) and n == int((v != ref).sum()) > 0


def test_pipeline_hooks(oracle_mod, small_view):
    v = small_view
    base = oracle_mod.densify_view(v)
    pre = oracle_mod.densify_view(v, occlusion_radius=4, occlusion_margin=0.3, contour_threshold=0.05)
    assert pre["occluded"] >= 0 and pre["contour_dropped"] > 0
    assert np.array_equal(pre["zbuf_merged"], base["zbuf"])
    assert (pre["valid"] <= pre["valid_filtered"]).all()
    prev = v.rgb.copy()
    prev[100:140, 100:160] = 0                              # something moved there
    mot = oracle_mod.densify_view(v, prev_rgb=prev, motion_threshold=40.0, motion_close_radius=2)
    assert mot["motion"][100:140, 100:160].mean() > 0.5
    assert mot["in_image"] <= base["in_image"]
