"""Preprocessing (Sec. 4.1: afterimage and occluded-point removal) and
post-filtering (Sec. 5: contour removal) on the GPU against the oracle.

Integer decisions are bit-exact: the closed motion mask, the z-buffer after
afterimage and occlusion removal (the occlusion decision is fixed to FP32
row/column sums on both sides), the validity masks. The contour decision is
taken on the filtered FP32 map, so it is checked by running the oracle's
contour step on the GPU's own filtered map; against the all-oracle pipeline
only pixels whose decision is within rounding of the threshold may differ.
"""
import numpy as np
import pytest

import scene

pytestmark = pytest.mark.gpu

STAGES = ((4, 5.0, 20.0), (2, 5.0, 20.0))


def _run(v, torch, prev=None, **params):
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300.frames import FrameBuffers
    build.build()
    with Densifier(dict(num_stages=2, stages=STAGES, launch_policy=1, **params)) as d:
        b = FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], debug=True, prev_rgb=prev)
        assert d.poll(d.submit(b.frame), -1) == 0
        torch.cuda.synchronize()
        return b.results()


def _moved(v, seed=0):
    """A previous frame in which a block of the image differed (something moved)."""
    rng = np.random.default_rng(seed)
    prev = v.rgb.copy()
    H, W = prev.shape[:2]
    y0, x0 = H // 3, W // 3
    prev[y0:y0 + H // 4, x0:x0 + W // 4] = rng.integers(0, 256, 3, dtype=np.uint8)
    return prev


@pytest.fixture(scope="module")
def view():
    return scene.make_view(404, res="720p", scene_kind="room", n_scans=3, beams=128, az_steps=1024)


def test_occlusion_removal_bit_exact(view):
    import torch
    import oracle
    g = _run(view, torch, occlusion_radius=5, occlusion_margin=0.3)
    o = oracle.densify_view(view, num_stages=2, stages=STAGES, occlusion_radius=5, occlusion_margin=0.3)
    assert o["occluded"] > 0
    assert np.array_equal(g["zbuf"].reshape(-1), o["zbuf"].reshape(-1))
    assert np.array_equal(g["valid"], o["valid"])
    m = o["valid"].astype(bool)
    np.testing.assert_allclose(g["depth"][m], o["depth"][m], rtol=1e-4)


def test_afterimage_removal_bit_exact(view):
    import torch
    import oracle
    prev = _moved(view)
    kw = dict(motion_threshold=40.0, motion_close_radius=2)
    g = _run(view, torch, prev=prev, **kw)
    o = oracle.densify_view(view, num_stages=2, stages=STAGES, prev_rgb=prev, **kw)
    assert o["motion"].any()
    assert np.array_equal(g["motion"], o["motion"])
    assert np.array_equal(g["zbuf"].reshape(-1), o["zbuf"].reshape(-1))
    base = oracle.densify_view(view, num_stages=2, stages=STAGES)
    assert o["in_image"] < base["in_image"]          # older scans lost points inside the motion
    assert np.array_equal(g["valid"], o["valid"])


def test_contour_removal_on_the_filtered_map(view):
    import torch
    import oracle
    t = 0.05
    plain = _run(view, torch)
    g = _run(view, torch, contour_threshold=t)
    d, vmask, n = oracle.contour(plain["depth"], plain["valid"], t)
    assert n > 0
    assert np.array_equal(g["valid"], vmask)
    assert np.array_equal(g["depth"], d)
    assert g["n"] == int(vmask.sum())
    # against the all-oracle pipeline: differences only at decisions within rounding of the threshold
    o = oracle.densify_view(view, num_stages=2, stages=STAGES, contour_threshold=t)
    diff = g["valid"] != o["valid"]
    assert diff.mean() < 1e-4, int(diff.sum())


def test_all_three_together(view):
    import torch
    import oracle
    prev = _moved(view, 1)
    kw = dict(occlusion_radius=4, occlusion_margin=0.25, motion_threshold=30.0, motion_close_radius=1)
    g = _run(view, torch, prev=prev, contour_threshold=0.05, **kw)
    o = oracle.densify_view(view, num_stages=2, stages=STAGES, prev_rgb=prev, contour_threshold=0.05, **kw)
    assert np.array_equal(g["zbuf"].reshape(-1), o["zbuf"].reshape(-1))
    assert np.array_equal(g["motion"], o["motion"])
    assert (g["valid"] != o["valid"]).mean() < 1e-4


@pytest.mark.parametrize("res", [(1281, 721), (97, 250), (33, 17), (31, 40), (1, 1)])
@pytest.mark.parametrize("close_radius", [0, 2, 7])
def test_ragged_sizes(res, close_radius):
    """Widths that are not multiples of 32 or of 4 (the closing's bit-packed rows end in a partial
    word; the motion and contour kernels take their per-pixel paths), tiles cut by the image
    border, and the largest closing radii against the frame: motion mask and z-buffer bit-exact,
    the contour step exact on the GPU's own filtered map."""
    import torch
    import oracle
    W, H = res
    rng = np.random.default_rng(W * 13 + H + close_radius)
    sc = scene.make_scene(6, "room")
    f = 1400.0 * max(W, 8) / 1920.0
    cam = scene.make_camera(W, H, f, f, W / 2.0, H / 2.0, (0.0, 0.0, 1.5))
    rgb, gt = scene.render_rgb(sc, cam, rng)
    scans = []
    for s in range(3):
        pose = scene.make_lidar_pose(cam, (0.1 * s, 0.05, 0.02), 2.0 * s)
        scans.append(scene.Scan(scene.lidar_sweep(sc, pose, 48, 700 + s, rng), pose))
    v = scene.View(cam, rgb, scans, gt)
    prev = rgb.copy()
    prev[H // 3:H // 3 + max(1, H // 4), W // 3:W // 3 + max(1, W // 4)] = rng.integers(0, 256, 3, dtype=np.uint8)
    prev[0, 0] = 255 - prev[0, 0]   # a changed pixel at the corner (the closing's border)
    kw = dict(occlusion_radius=3, occlusion_margin=0.2, motion_threshold=30.0, motion_close_radius=close_radius)
    g = _run(v, torch, prev=prev, **kw)
    o = oracle.densify_view(v, num_stages=2, stages=STAGES, prev_rgb=prev, **kw)
    assert np.array_equal(g["motion"], o["motion"])
    assert np.array_equal(g["zbuf"].reshape(-1), o["zbuf"].reshape(-1))
    assert np.array_equal(g["valid"], o["valid"])
    m = o["valid"].astype(bool)
    np.testing.assert_allclose(g["depth"][m], o["depth"][m], rtol=1e-4)
    t = 0.05
    gc = _run(v, torch, prev=prev, contour_threshold=t, **kw)
    d, vmask, _ = oracle.contour(g["depth"], g["valid"], t)
    assert np.array_equal(gc["valid"], vmask)
    assert np.array_equal(gc["depth"], d)
