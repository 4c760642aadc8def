"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these checks re-types the oracle's own loops: they use closed forms
(uniform guide -> normalised Gaussian convolution, constant depth, lone
point), an independent formulation (Algorithm 1's scatter form against the
gather form of Eq. (1)), library routines (numpy float32 arithmetic, matrix
inverse, scipy correlation, np.kron), hand-worked values (tests/golden) and
brute force on tiny images.
"""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EMPTY = 0x7F800000


def _rng(seed=0):
    return np.random.default_rng(seed)


def _rigid(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = rng.uniform(-3, 3, size=3)
    return T


# ---------------------------------------------------------------------------
# calibration
# ---------------------------------------------------------------------------
def test_compose_matches_matrix_inverse(oracle_mod):
    rng = _rng(1)
    for _ in range(20):
        C, L = _rigid(rng), _rigid(rng)
        M64, M32 = oracle_mod.compose(C, L)
        ref = (np.linalg.inv(C) @ L)[:3]
        np.testing.assert_allclose(M64, ref, rtol=0, atol=1e-12)
        assert np.array_equal(M32, M64.astype(np.float32))


def test_compose_exact_permutation():
    """A 90-degree yaw camera at (1, 2, 3): inverse is [R^T, -R^T t] exactly."""
    import oracle
    C = np.eye(4)
    C[:3, :3] = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]
    C[:3, 3] = [1, 2, 3]
    M64, _ = oracle.compose(C, np.eye(4))
    assert np.array_equal(M64, np.array([[0, 1, 0, -2], [-1, 0, 0, 1], [0, 0, 1, -3]], dtype=float))


# ---------------------------------------------------------------------------
# projection and z-buffer
# ---------------------------------------------------------------------------
def _pixel_centre_points(ii, jj, z, fx, cx, cy):
    # x = (i + 1/2 - cx) z / fx is exact in binary for fx = 64, z = 2^k
    return np.stack([(ii + 0.5 - cx) * z / fx, (jj + 0.5 - cy) * z / fx, np.full(ii.shape, z)], 1).astype(np.float32)


def test_known_points_land_on_known_pixels(oracle_mod):
    W, H, f, cx, cy = 16, 12, 64.0, 8.0, 6.0
    jj, ii = np.mgrid[0:H, 0:W]
    ii, jj = ii.ravel().astype(float), jj.ravel().astype(float)
    pts = _pixel_centre_points(ii, jj, 4.0, f, cx, cy)
    I = np.eye(4)
    _, M32 = oracle_mod.compose(I, I)
    zbuf, kept = oracle_mod.project(M32, pts, W, H, f, f, cx, cy)
    assert kept == W * H
    assert np.all(zbuf == np.float32(4.0).view(np.uint32))
    # one point per pixel, in a shuffled order, lands where it was made
    order = _rng(3).permutation(W * H)[:40]
    for k in order:
        zb, kept = oracle_mod.project(M32, pts[k:k + 1], W, H, f, f, cx, cy)
        assert kept == 1
        hit = np.flatnonzero(zb != EMPTY)
        assert hit.tolist() == [int(jj[k]) * W + int(ii[k])]


def test_rotated_camera_known_pixel(oracle_mod):
    """Camera at (1, 2, 3) with a 90-degree yaw: world point -> known pixel."""
    C = np.eye(4)
    C[:3, :3] = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]
    C[:3, 3] = [1, 2, 3]
    W, H, f, cx, cy = 16, 12, 64.0, 8.0, 6.0
    # camera point (x, y, z) = ((i+.5-cx) z/f, (j+.5-cy) z/f, z) with i=11, j=2, z=8
    pc = np.array([(11.5 - cx) * 8 / f, (2.5 - cy) * 8 / f, 8.0])
    pw = C[:3, :3] @ pc + C[:3, 3]
    _, M32 = oracle_mod.compose(C, np.eye(4))
    zb, kept = oracle_mod.project(M32, pw[None].astype(np.float32), W, H, f, f, cx, cy)
    assert kept == 1
    assert np.flatnonzero(zb != EMPTY).tolist() == [2 * W + 11]
    assert zb[2 * W + 11] == np.float32(8.0).view(np.uint32)


def test_nearest_depth_wins_and_rejections(oracle_mod):
    W, H, f, cx, cy = 16, 12, 64.0, 8.0, 6.0
    I = np.eye(4)
    _, M32 = oracle_mod.compose(I, I)
    a = _pixel_centre_points(np.array([3.0]), np.array([5.0]), 4.0, f, cx, cy)
    b = _pixel_centre_points(np.array([3.0]), np.array([5.0]), 2.0, f, cx, cy)
    behind = np.array([[0.1, 0.1, -1.0]], np.float32)
    outside = np.array([[100.0, 0.0, 1.0]], np.float32)
    nan = np.array([[np.nan, 0.0, 1.0]], np.float32)
    on_plane = np.array([[0.0, 0.0, 0.0]], np.float32)
    for pts in (np.concatenate([a, b, behind, outside, nan, on_plane]),
                np.concatenate([on_plane, nan, b, outside, a, behind])):
        zb, kept = oracle_mod.project(M32, pts, W, H, f, f, cx, cy)
        assert kept == 2
        assert np.flatnonzero(zb != EMPTY).tolist() == [5 * W + 3]
        assert zb[5 * W + 3] == np.float32(2.0).view(np.uint32)


def test_projection_matches_numpy_float32(oracle_mod):
    """The FP32 contract, evaluated independently with numpy float32 ops."""
    rng = _rng(4)
    W, H = 96, 64
    fx, fy, cx, cy = np.float32(70.3), np.float32(69.1), np.float32(47.7), np.float32(31.2)
    C, L = _rigid(rng), _rigid(rng)
    _, M = oracle_mod.compose(C, L)
    pts_c = np.stack([rng.uniform(-2, 2, 5000), rng.uniform(-1.5, 1.5, 5000), rng.uniform(-1, 6, 5000)], 1)
    pts = ((np.linalg.inv(L) @ C @ np.c_[pts_c, np.ones(5000)].T).T[:, :3]).astype(np.float32)
    zb, kept = oracle_mod.project(M, pts, W, H, fx, fy, cx, cy)
    ref = np.full(W * H, EMPTY, np.uint32)
    n = 0
    with np.errstate(all="ignore"):
        for p in pts:
            c = [((M[i, 0] * p[0] + M[i, 1] * p[1]) + M[i, 2] * p[2]) + M[i, 3] for i in range(3)]
            if not (c[2] > 0 and np.isfinite(c[2])):
                continue
            u = fx * (c[0] / c[2]) + cx
            v = fy * (c[1] / c[2]) + cy
            assert u.dtype == np.float32
            if not (0 <= u < W and 0 <= v < H):
                continue
            k = int(np.floor(v)) * W + int(np.floor(u))
            ref[k] = min(ref[k], np.float32(c[2]).view(np.uint32))
            n += 1
    assert kept == n and n > 500
    assert np.array_equal(zb, ref)


def test_fp64_projection_known_pixels(oracle_mod):
    """Pure FP64 projection: points at pixel centres land on their pixels with their exact depth;
    a non-square image and distinct row and column targets catch a u/v swap."""
    W, H, f, cx, cy = 16, 12, 64.0, 8.0, 6.0
    jj, ii = np.mgrid[0:H, 0:W]
    ii, jj = ii.ravel().astype(float), jj.ravel().astype(float)
    pts = _pixel_centre_points(ii, jj, 4.0, f, cx, cy)
    I = np.eye(4)
    M64, _ = oracle_mod.compose(I, I)
    depth, kept = oracle_mod.project_fp64(M64, pts, W, H, f, f, cx, cy)
    assert kept == W * H and np.all(depth == 4.0)
    for k in _rng(5).permutation(W * H)[:40]:
        d, kept = oracle_mod.project_fp64(M64, pts[k:k + 1], W, H, f, f, cx, cy)
        assert kept == 1
        assert np.flatnonzero(np.isfinite(d)).tolist() == [int(jj[k]) * W + int(ii[k])]
    # nearest wins, rejections as in the FP32 contract
    a = _pixel_centre_points(np.array([3.0]), np.array([5.0]), 4.0, f, cx, cy)
    b = _pixel_centre_points(np.array([3.0]), np.array([5.0]), 2.0, f, cx, cy)
    junk = np.array([[0.1, 0.1, -1.0], [100.0, 0.0, 1.0], [np.nan, 0.0, 1.0], [0.0, 0.0, 0.0]], np.float32)
    d, kept = oracle_mod.project_fp64(M64, np.concatenate([a, junk, b]), W, H, f, f, cx, cy)
    assert kept == 2 and np.flatnonzero(np.isfinite(d)).tolist() == [5 * W + 3] and d[5 * W + 3] == 2.0


def test_fp64_projection_matches_numpy_float64(oracle_mod):
    """Pure FP64 projection re-evaluated with numpy float64 on random rigid poses."""
    rng = _rng(6)
    W, H = 96, 64
    fx, fy, cx, cy = 70.3, 69.1, 47.7, 31.2
    for _ in range(3):
        C, L = _rigid(rng), _rigid(rng)
        M64, _ = oracle_mod.compose(C, L)
        pts_c = np.stack([rng.uniform(-2, 2, 4000), rng.uniform(-1.5, 1.5, 4000), rng.uniform(-1, 6, 4000)], 1)
        pts = ((np.linalg.inv(L) @ C @ np.c_[pts_c, np.ones(4000)].T).T[:, :3]).astype(np.float32)
        depth, kept = oracle_mod.project_fp64(M64, pts, W, H, fx, fy, cx, cy)
        c = pts.astype(np.float64) @ M64[:, :3].T + M64[:, 3]
        with np.errstate(all="ignore"):
            u = fx * (c[:, 0] / c[:, 2]) + cx
            v = fy * (c[:, 1] / c[:, 2]) + cy
            ok = (c[:, 2] > 0) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
        ref = np.full(W * H, np.inf)
        np.minimum.at(ref, (np.floor(v[ok]) * W + np.floor(u[ok])).astype(np.int64), c[ok, 2])
        assert kept == int(ok.sum()) and kept > 400
        assert np.array_equal(np.isfinite(depth), np.isfinite(ref))
        m = np.isfinite(ref)
        np.testing.assert_allclose(depth[m], ref[m], rtol=1e-13, atol=0)


def test_fp64_projection_decides_edges_exactly(oracle_mod):
    """A point whose exact image coordinate lies one FP32 ulp below a pixel edge: the FP32 contract
    (numpy float32 agrees) rounds it onto the next pixel, the FP64 projection keeps it on the pixel
    the exact value lies in. With fx = z = 3 and cx = 0 the exact u is x itself."""
    I = np.eye(4)
    M64, M32 = oracle_mod.compose(I, I)
    three = np.float32(3.0)
    found = 0
    W, H = 4096, 8
    for k in range(1, W):
        x = np.nextafter(np.float32(k), np.float32(0))          # largest float32 below k
        u32 = three * (x / three)
        if u32 < k:
            continue                                            # FP32 keeps it below the edge too
        y = np.float32(4.5)                                     # row 4 in both precisions
        p = np.array([[x, y, 3.0]], np.float32)
        zb, _ = oracle_mod.project(M32, p, W, H, 3.0, 3.0, 0.0, 0.0)
        d, _ = oracle_mod.project_fp64(M64, p, W, H, 3.0, 3.0, 0.0, 0.0)
        assert np.flatnonzero(zb != EMPTY).tolist() == [4 * W + k]        # FP32: rounded onto pixel k
        assert np.flatnonzero(np.isfinite(d)).tolist() == [4 * W + k - 1]  # exact: pixel k - 1
        found += 1
    assert found > 100


def test_fp32_contract_against_fp64_projection_1080p(oracle_mod):
    """The FP32 projection contract against pure FP64 on the 1080p three-scan workload: the same
    observed pixels up to a handful moved across a pixel edge, the same nearest point elsewhere,
    depths within FP32 rounding."""
    import scene
    v = scene.make_view(1001, res="1080p", scene_kind="room", n_scans=3, beams=128, az_steps=1024,
                        view_index=0, n_views=7)
    rep = oracle_mod.projection_precision_report(v.camera, [(s.xyz, s.lidar_to_world) for s in v.scans])
    print(rep)
    assert rep["observed_fp32"] > 50000
    assert rep["pixels_assigned_differently"] <= 1e-3 * rep["observed_fp32"]
    assert rep["max_rel_depth_same_point"] < 1e-6


def test_merge_order_independent(oracle_mod, small_view):
    v = small_view
    cam = v.camera
    zs = []
    for order in ([0, 1, 2], [2, 0, 1]):
        zb = np.full(cam.width * cam.height, EMPTY, np.uint32)
        for s in order:
            _, M = oracle_mod.compose(cam.cam_to_world, v.scans[s].lidar_to_world)
            oracle_mod.project(M, v.scans[s].xyz, cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, zb)
        zs.append(zb)
    assert np.array_equal(zs[0], zs[1])


# ---------------------------------------------------------------------------
# pooling and restore
# ---------------------------------------------------------------------------
def test_pool_hand_example(oracle_mod):
    """4 x 5 image, f = 3 (ceil mode): coarse 2 x 2, partial edge blocks."""
    H, W = 4, 5
    d = np.full((H, W), np.inf, np.float32)
    d[0, 0], d[2, 2], d[3, 4], d[1, 3] = 1.5, 2.5, 4.0, 8.0
    zb = d.view(np.uint32).copy()
    zb[np.isinf(d)] = EMPTY
    rgb = np.zeros((H, W, 3), np.uint8)
    rgb[..., 0] = np.arange(W)[None, :] * 10
    rgb[..., 1] = np.arange(H)[:, None] * 20
    rgb[..., 2] = 7
    ssum, cnt, g = oracle_mod.pool(zb.ravel(), rgb, W, H, 3)
    assert ssum.tolist() == [[1.5 + 2.5, 8.0], [0.0, 4.0]]
    assert cnt.tolist() == [[2, 1], [0, 1]]
    # block (0,0): x 0..2, y 0..2 -> mean r = 10, mean g = 20
    assert g[0, 0].tolist() == [10.0, 20.0, 7.0]
    # block (0,1): x 3..4, y 0..2 -> r mean 35, g mean 20
    assert g[0, 1].tolist() == [35.0, 20.0, 7.0]
    # block (1,0): x 0..2, y 3 -> r mean 10, g 60; block (1,1): x 3..4, y 3
    assert g[1, 0].tolist() == [10.0, 60.0, 7.0]
    assert g[1, 1].tolist() == [35.0, 60.0, 7.0]


def test_pool_matches_reshape_sums(oracle_mod):
    rng = _rng(5)
    H, W = 27, 36
    d = rng.uniform(1, 9, (H, W)).astype(np.float32)
    obs = rng.random((H, W)) < 0.3
    zb = np.where(obs, d.view(np.uint32), np.uint32(EMPTY)).astype(np.uint32)
    rgb = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    ssum, cnt, g = oracle_mod.pool(zb.ravel(), rgb, W, H, 3)
    blk = lambda a: a.reshape(H // 3, 3, W // 3, 3, *a.shape[2:]).sum(axis=(1, 3))
    np.testing.assert_allclose(ssum, blk(np.where(obs, d.astype(float), 0.0)), rtol=1e-15)
    assert np.array_equal(cnt, blk(obs.astype(float)))
    np.testing.assert_allclose(g, blk(rgb.astype(float)) / 9.0, rtol=1e-15)


def test_upsample_is_kron(oracle_mod):
    rng = _rng(6)
    d1 = rng.uniform(1, 5, (4, 5))
    v1 = (rng.random((4, 5)) < 0.7).astype(np.uint8)
    beta, bd = oracle_mod.upsample(d1, v1, 3, 14, 11)
    big_v = np.kron(v1, np.ones((3, 3)))[:11, :14]
    big_d = np.kron(d1 * v1, np.ones((3, 3)))[:11, :14]
    assert np.array_equal(beta, big_v)
    assert np.array_equal(bd, big_d)
    # override reading: observed full-resolution pixels keep their own depth
    zb = np.full(11 * 14, EMPTY, np.uint32)
    zb[3 * 14 + 5] = np.float32(9.5).view(np.uint32)
    beta, bd = oracle_mod.upsample(d1, v1, 3, 14, 11, zbuf=zb, override=True)
    assert beta[3, 5] == 1.0 and bd[3, 5] == 9.5
    mask = np.ones((11, 14), bool)
    mask[3, 5] = False
    assert np.array_equal(bd[mask], big_d[mask])


# ---------------------------------------------------------------------------
# joint bilateral filter: Eq. (1)-(4) and Algorithm 1
# ---------------------------------------------------------------------------
def _random_jbf_inputs(rng, H, W, density=0.3, counts=False):
    guide = rng.integers(0, 256, (H, W, 3)).astype(float)
    if counts:
        beta = rng.integers(0, 10, (H, W)).astype(float) * (rng.random((H, W)) < density)
    else:
        beta = (rng.random((H, W)) < density).astype(float)
    depth = rng.uniform(0.5, 10, (H, W))
    return guide, beta, beta * depth if not counts else beta * depth


def test_golden_hand_example(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "jbf_hand_example.json")))
    guide = np.array(g["guide"], float).reshape(1, 3, 3)
    beta = np.array(g["beta"], float).reshape(1, 3)
    bd = beta * np.array(g["depth"], float).reshape(1, 3)
    for shifted in (False, True):
        out, valid = oracle_mod.jbf_gather(guide, beta, bd, g["radius"], g["sigma_p"], g["sigma_c"], shifted)
        np.testing.assert_allclose(out.ravel(), g["expected_depth"], rtol=1e-15)
        assert valid.ravel().tolist() == g["expected_valid"]


def test_uniform_guide_is_normalised_gaussian_convolution(oracle_mod):
    """Constant guide: w_c = 1, so Eq. (1) is the normalised convolution
    sum(G * BD) / sum(G * B) with the spatial Gaussian G (zero padding)."""
    from scipy.ndimage import correlate
    rng = _rng(7)
    H, W = 23, 31
    for r, sp in ((1, 0.7), (2, 1.3), (4, 2.5), (7, 5.0)):
        _, beta, bd = _random_jbf_inputs(rng, H, W, 0.25)
        guide = np.full((H, W, 3), 93.0)
        a = np.arange(-r, r + 1)
        G = np.exp(-(a[:, None] ** 2 + a[None, :] ** 2) / (2 * sp * sp))
        num = correlate(bd, G, mode="constant", cval=0.0)
        den = correlate(beta, G, mode="constant", cval=0.0)
        has = correlate(beta, np.ones_like(G), mode="constant", cval=0.0) > 0
        out, valid = oracle_mod.jbf_gather(guide, beta, bd, r, sp, 11.0)
        assert np.array_equal(valid.astype(bool), has)
        np.testing.assert_allclose(out[has], num[has] / den[has], rtol=1e-12)
        assert np.all(out[~has] == 0)
        # sigma_c -> infinity on a random guide gives the same result
        g2, _, _ = _random_jbf_inputs(rng, H, W)
        out2, _ = oracle_mod.jbf_gather(g2, beta, bd, r, sp, 1e12)
        np.testing.assert_allclose(out2[has], num[has] / den[has], rtol=1e-10)


def test_two_colour_guide_separates_regions(oracle_mod):
    """sigma_c small against a colour step: cross weights are below 1e-200, so
    each side is the normalised Gaussian convolution of its own depths."""
    from scipy.ndimage import correlate
    rng = _rng(8)
    H, W, r, sp = 17, 24, 3, 2.0
    left = np.zeros((H, W), bool)
    left[:, :11] = True
    guide = np.where(left[..., None], np.array([10.0, 200.0, 30.0]), np.array([240.0, 20.0, 130.0]))
    _, beta, bd = _random_jbf_inputs(rng, H, W, 0.3)
    out, valid = oracle_mod.jbf_gather(guide, beta, bd, r, sp, 5.0)
    a = np.arange(-r, r + 1)
    G = np.exp(-(a[:, None] ** 2 + a[None, :] ** 2) / (2 * sp * sp))
    for side in (left, ~left):
        num = correlate(bd * side, G, mode="constant")
        den = correlate(beta * side, G, mode="constant")
        m = side & (den > 0)
        np.testing.assert_allclose(out[m], num[m] / den[m], rtol=1e-12)


def test_constant_depth_reproduced_exactly(oracle_mod):
    rng = _rng(9)
    guide, beta, _ = _random_jbf_inputs(rng, 19, 26, 0.4)
    for c in (0.25, 4.0, 64.0):
        for shifted in (False, True):
            out, valid = oracle_mod.jbf_gather(guide, beta, beta * c, 3, 2.0, 20.0, shifted)
            assert np.all(out[valid.astype(bool)] == c)
    # pooled counts: beta in 0..9, beta_d = c * beta
    cnt = rng.integers(0, 10, (19, 26)).astype(float)
    out, valid = oracle_mod.jbf_gather(guide, cnt, cnt * 8.0, 4, 5.0, 20.0)
    assert np.all(out[valid.astype(bool)] == 8.0)


def test_lone_point_fills_exactly_its_window(oracle_mod):
    rng = _rng(10)
    H, W = 21, 30
    guide = rng.integers(0, 256, (H, W, 3)).astype(float)
    for r in (1, 2, 4, 7):
        beta = np.zeros((H, W))
        beta[9, 13] = 1.0
        d = 3.7
        out, valid = oracle_mod.jbf_gather(guide, beta, beta * d, r, 2.0, 20.0, shifted=True)
        win = np.zeros((H, W), bool)
        win[max(0, 9 - r):9 + r + 1, max(0, 13 - r):13 + r + 1] = True
        assert np.array_equal(valid.astype(bool), win)
        assert np.all(out[win] == d) and np.all(out[~win] == 0.0)
        out_p, _ = oracle_mod.jbf_gather(guide, beta, beta * d, r, 2.0, 20.0, shifted=False)
        np.testing.assert_allclose(out_p[win], d, rtol=2.3e-16)


def test_depth_scaling_commutes_exactly(oracle_mod):
    rng = _rng(11)
    guide, beta, bd = _random_jbf_inputs(rng, 15, 22, 0.3)
    out, valid = oracle_mod.jbf_gather(guide, beta, bd, 2, 1.5, 20.0)
    out8, valid8 = oracle_mod.jbf_gather(guide, beta, bd * 8.0, 2, 1.5, 20.0)
    assert np.array_equal(valid, valid8)
    assert np.array_equal(out * 8.0, out8)


def test_scatter_form_equals_gather_form(oracle_mod):
    """Algorithm 1 (transpose-convolution scatter) against Eq. (1) (gather)."""
    rng = _rng(12)
    for (H, W, r, sp, sc, counts) in ((13, 29, 1, 1.0, 20.0, False), (24, 17, 2, 5.0, 20.0, False),
                                      (31, 22, 4, 5.0, 20.0, True), (16, 16, 7, 3.0, 10.0, False)):
        guide, beta, bd = _random_jbf_inputs(rng, H, W, 0.2, counts)
        og, vg = oracle_mod.jbf_gather(guide, beta, bd, r, sp, sc)
        os_, vs = oracle_mod.jbf_scatter(guide, beta, bd, r, sp, sc)
        assert np.array_equal(vg, vs)
        np.testing.assert_allclose(og, os_, rtol=1e-12, atol=0)


def test_plain_and_shifted_forms_agree(oracle_mod):
    rng = _rng(13)
    guide, beta, bd = _random_jbf_inputs(rng, 28, 19, 0.1)
    a, va = oracle_mod.jbf_gather(guide, beta, bd, 4, 5.0, 20.0, shifted=False)
    b, vb = oracle_mod.jbf_gather(guide, beta, bd, 4, 5.0, 20.0, shifted=True)
    assert np.array_equal(va, vb)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_transpose_equivariance(oracle_mod):
    rng = _rng(14)
    guide, beta, bd = _random_jbf_inputs(rng, 14, 27, 0.3, counts=True)
    out, valid = oracle_mod.jbf_gather(guide, beta, bd, 3, 2.0, 15.0)
    outT, validT = oracle_mod.jbf_gather(guide.transpose(1, 0, 2).copy(), beta.T.copy(), bd.T.copy(), 3, 2.0, 15.0)
    assert np.array_equal(valid.T, validT)
    np.testing.assert_allclose(out.T, outT, rtol=1e-14)


def test_brute_force_tiny(oracle_mod):
    """Every pixel of tiny images by an independent offset-major loop."""
    rng = _rng(15)
    for (H, W, r) in ((5, 7, 1), (6, 4, 2), (7, 8, 3)):
        guide, beta, bd = _random_jbf_inputs(rng, H, W, 0.4, counts=True)
        sp, sc = 1.7, 23.0
        num = np.zeros((H, W))
        den = np.zeros((H, W))
        has = np.zeros((H, W), bool)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                for y in range(H):
                    for x in range(W):
                        qy, qx = y + dy, x + dx
                        if 0 <= qy < H and 0 <= qx < W and beta[qy, qx] > 0:
                            col = sum((guide[qy, qx, c] - guide[y, x, c]) ** 2 for c in range(3))
                            w = math.exp(-col / (2 * sc * sc)) * math.exp(-(dx * dx + dy * dy) / (2 * sp * sp))
                            num[y, x] += bd[qy, qx] * w
                            den[y, x] += beta[qy, qx] * w
                            has[y, x] = True
        out, valid = oracle_mod.jbf_gather(guide, beta, bd, r, sp, sc)
        assert np.array_equal(valid.astype(bool), has)
        np.testing.assert_allclose(out[has], num[has] / den[has], rtol=1e-13)


# ---------------------------------------------------------------------------
# back-projection
# ---------------------------------------------------------------------------
def test_backproject_closed_form_and_round_trip(oracle_mod):
    rng = _rng(16)
    H, W = 12, 16
    fx, fy, cx, cy = 64.0, 60.0, 8.0, 6.0
    depth = rng.uniform(1, 5, (H, W))
    valid = (rng.random((H, W)) < 0.5).astype(np.uint8)
    rgb = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    C = _rigid(rng)
    xyz, rgba = oracle_mod.backproject(depth, valid, rgb, fx, fy, cx, cy, C)
    jj, ii = np.nonzero(valid)          # row-major order
    assert xyz.shape == (len(ii), 3)
    Z = depth[jj, ii]
    pc = np.stack([(ii + 0.5 - cx) * Z / fx, (jj + 0.5 - cy) * Z / fy, Z], 1)
    np.testing.assert_allclose(xyz, pc @ C[:3, :3].T + C[:3, 3], rtol=1e-13, atol=1e-13)
    exp = rgb[jj, ii, 0].astype(np.uint32) | (rgb[jj, ii, 1].astype(np.uint32) << 8) | \
        (rgb[jj, ii, 2].astype(np.uint32) << 16) | np.uint32(255 << 24)
    assert np.array_equal(rgba, exp)
    # round trip: project the points back into the same camera -> same pixels
    M64, M32 = oracle_mod.compose(C, np.eye(4))
    for k in range(0, len(ii), 7):
        zb, kept = oracle_mod.project(M32, xyz[k:k + 1].astype(np.float32), W, H, fx, fy, cx, cy)
        assert kept == 1 and np.flatnonzero(zb != EMPTY).tolist() == [jj[k] * W + ii[k]]


# ---------------------------------------------------------------------------
# whole path invariants
# ---------------------------------------------------------------------------
class _Cam:
    def __init__(self, W, H, f, cx, cy, T=None):
        self.width, self.height, self.fx, self.fy, self.cx, self.cy = W, H, f, f, cx, cy
        self.cam_to_world = np.eye(4) if T is None else T


def test_golden_paper_parameters():
    import oracle
    g = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    p = oracle.PAPER_TWO_STAGE
    assert p["pool"] == g["pool_factor"]
    assert p["stages"][0][0] == g["stage1_radius"] and p["stages"][1][0] == g["stage2_radius"]
    assert (2 * g["stage1_radius"] + 1) ** 2 == g["window_taps_stage1"]
    assert (2 * g["stage2_radius"] + 1) ** 2 == g["window_taps_stage2"]


@pytest.mark.parametrize("stages", [1, 2])
def test_plane_reproduced_exactly(oracle_mod, stages):
    W, H, f, cx, cy = 40, 31, 64.0, 20.0, 15.5
    jj, ii = np.mgrid[0:H, 0:W]
    pts = _pixel_centre_points(ii.ravel().astype(float), jj.ravel().astype(float), 4.0, f, cx, cy)
    rng = _rng(17)
    rgb = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    res = oracle_mod.densify(_Cam(W, H, f, cx, cy), rgb, [(pts, np.eye(4))], num_stages=stages,
                             stages=((2, 3.0, 20.0),) if stages == 1 else ((4, 5.0, 20.0), (2, 5.0, 20.0)))
    assert res["valid"].all()
    assert np.all(res["depth"] == 4.0)
    np.testing.assert_allclose(res["xyz"][:, 2], 4.0, rtol=0, atol=0)


def test_lone_point_two_stage_support(oracle_mod):
    """One observation: stage 1 fills its coarse Chebyshev-4 window, the
    restore makes 3x3 blocks of it, stage 2 grows that by 2 pixels."""
    W, H, f, cx, cy = 60, 45, 64.0, 30.0, 22.5
    p = _pixel_centre_points(np.array([31.0]), np.array([20.0]), 2.0, f, cx, cy)
    rgb = _rng(18).integers(0, 256, (H, W, 3), dtype=np.uint8)
    res = oracle_mod.densify(_Cam(W, H, f, cx, cy), rgb, [(p, np.eye(4))], shifted=True)
    I, J = 31 // 3, 20 // 3
    v1 = np.zeros((15, 20), bool)
    v1[max(0, J - 4):J + 5, max(0, I - 4):I + 5] = True
    assert np.array_equal(res["v1"].astype(bool), v1)
    assert np.all(res["d1"][v1] == 2.0)
    big = np.kron(v1, np.ones((3, 3), bool))[:H, :W]
    from scipy.ndimage import binary_dilation
    grown = binary_dilation(big, np.ones((5, 5), bool))
    assert np.array_equal(res["valid"].astype(bool), grown)
    assert np.all(res["depth"][grown] == 2.0)


def test_coarse_shapes_ceil(oracle_mod):
    for (W, H) in ((1920, 1080), (1280, 720), (320, 240), (1281, 721)):
        zb = np.full(W * H, EMPTY, np.uint32)
        ssum, cnt, g = oracle_mod.pool(zb, np.zeros((H, W, 3), np.uint8), W, H, 3)
        assert ssum.shape == (-(-H // 3), -(-W // 3)) and g.shape == ssum.shape + (3,)
