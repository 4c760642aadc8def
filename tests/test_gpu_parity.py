"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar (stated per step):
  * z-buffer, valid masks (coarse and final), point count and colours: bit-exact;
  * FP32 depth (coarse and final): |gpu - oracle| <= 1e-4 * oracle;
  * points: world position within 1e-4 of the camera distance plus 8 FP32
    ulps of the largest coordinate: a point is the depth times the pixel's
    ray, so the depth bar moves it by at most 1e-4 of its distance, and the
    FP32 ray and camera-to-world transform add a few roundings.
"""
import numpy as np
import pytest

import scene

pytestmark = pytest.mark.gpu

RTOL = 1e-4
EMPTY = 0x7F800000
QVGA_STAGES = ((4, 3.0, 20.0),)                       # 9x9 window, sigma_s 3 px, sigma_r 20
PAPER_STAGES = ((4, 5.0, 20.0), (2, 5.0, 20.0))       # r=4 at 1/3, r=2 at full (Sec. 5)
VARIANTS = [0, 1, 2]   # TMA kernels (expanded FP32 form where in range), plain kernels, TMA difference form


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2601_01210_gb300 import build
    build.build()
    return torch


def run_gpu(views, num_stages, stages, torch, stage2_input=0, memory=0, max_batch=16, xyzw=False,
            points_cap=None, policy=1, **extra):
    from paper_2601_01210_gb300 import Densifier
    from paper_2601_01210_gb300.frames import FrameBuffers
    params = dict(num_stages=num_stages, stages=stages, stage2_input=stage2_input, max_batch=max_batch,
                  max_inflight=max(16, len(views)), launch_policy=policy, **extra)
    with Densifier(params) as d:
        bufs = [FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], num_stages=num_stages,
                             debug=True, memory=memory, xyzw=xyzw, points_cap=points_cap) for v in views]
        tickets = [d.submit(b.frame) for b in bufs]
        d.flush()
        for t in tickets:
            assert d.poll(t, -1) == 0
        torch.cuda.synchronize()
        return [b.results() for b in bufs]


def run_oracle(v, num_stages, stages, stage2_input=0):
    import oracle
    return oracle.densify_view(v, num_stages=num_stages, stages=stages, stage2_input=stage2_input)


def compare(g, o, num_stages, label=""):
    H, W = o["depth"].shape
    assert np.array_equal(g["zbuf"].reshape(-1), o["zbuf"].reshape(-1)), f"{label}: z-buffer differs"
    if num_stages == 2:
        assert np.array_equal(g["coarse_valid"], o["v1"]), f"{label}: coarse valid differs"
        m1 = o["v1"].astype(bool)
        if m1.any():
            rel1 = np.abs(g["coarse"][m1] - o["d1"][m1]) / o["d1"][m1]
            assert rel1.max() <= RTOL, f"{label}: coarse depth rel err {rel1.max():.3g}"
        assert np.all(g["coarse"][~m1] == 0)
    assert np.array_equal(g["valid"], o["valid"]), f"{label}: valid differs ({(g['valid'] != o['valid']).sum()} px)"
    m = o["valid"].astype(bool)
    if m.any():
        rel = np.abs(g["depth"][m] - o["depth"][m]) / o["depth"][m]
        assert rel.max() <= RTOL, f"{label}: depth rel err {rel.max():.3g}"
    assert np.all(g["depth"][~m] == 0)
    if "xyz" in o:
        assert g["n"] == len(o["xyz"]) == int(m.sum())
        assert np.array_equal(g["rgba"], o["rgba"])
        return m
    return m


def check_points(g, o, cam):
    t = cam.cam_to_world[:3, 3]
    dist = np.linalg.norm(o["xyz"] - t, axis=1)
    err = np.linalg.norm(g["xyz"].astype(np.float64) - o["xyz"], axis=1)
    scale = np.maximum(np.abs(o["xyz"]).max(axis=1), dist).astype(np.float32)
    tol = RTOL * dist + 8 * np.spacing(scale).astype(np.float64)
    assert np.all(err <= tol), f"points: max err {err.max():.3g}, worst ratio {(err / tol).max():.3g}"


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("variant", VARIANTS)
def test_qvga_single_stage(torch_cuda, variant):
    v = scene.make_workload("qvga_1scan", 1000)
    g = run_gpu([v], 1, QVGA_STAGES, torch_cuda, kernel_variant=variant)[0]
    o = run_oracle(v, 1, QVGA_STAGES)
    compare(g, o, 1, "qvga")
    check_points(g, o, v.camera)
    assert o["valid"].mean() > 0.2


@pytest.mark.parametrize("variant", VARIANTS)
def test_1080p_three_scans_two_stage(torch_cuda, variant):
    v = scene.make_workload("1080p_3scan", 1001)
    g = run_gpu([v], 2, PAPER_STAGES, torch_cuda, kernel_variant=variant)[0]
    o = run_oracle(v, 2, PAPER_STAGES)
    compare(g, o, 2, "1080p two-stage")
    check_points(g, o, v.camera)
    assert o["in_image"] > 30000


@pytest.mark.parametrize("variant", VARIANTS)
def test_1080p_single_stage_15x15(torch_cuda, variant):
    v = scene.make_workload("1080p_3scan", 1002)
    st = ((7, 5.0, 20.0),)
    g = run_gpu([v], 1, st, torch_cuda, kernel_variant=variant)[0]
    o = run_oracle(v, 1, st)
    compare(g, o, 1, "1080p 15x15")
    check_points(g, o, v.camera)


def test_stage2_override_reading(torch_cuda):
    v = scene.make_view(77, res="qvga", scene_kind="room", n_scans=3, beams=64, az_steps=512)
    g = run_gpu([v], 2, PAPER_STAGES, torch_cuda, stage2_input=1)[0]
    o = run_oracle(v, 2, PAPER_STAGES, stage2_input=1)
    compare(g, o, 2, "override")


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("res", [(1281, 721), (33, 17), (97, 250), (1, 1)])
def test_ragged_sizes(torch_cuda, res, variant):
    W, H = res
    rng = np.random.default_rng(W * 7 + H)
    sc = scene.make_scene(5, "room")
    f = 1400.0 * max(W, 8) / 1920.0
    cam = scene.make_camera(W, H, f, f, W / 2.0, H / 2.0, (0.0, 0.0, 1.5))
    rgb, gt = scene.render_rgb(sc, cam, rng)
    scans = []
    for s in range(3):
        pose = scene.make_lidar_pose(cam, (0.1 * s, 0.05, 0.02), 2.0 * s)
        scans.append(scene.Scan(scene.lidar_sweep(sc, pose, 48, 700 + s, rng), pose))
    v = scene.View(cam, rgb, scans, gt)
    # (the single stage at r = 2, sigma_c = 20 runs the column-paired kernel by default)
    for stages, st in ((2, PAPER_STAGES), (1, ((3, 2.0, 15.0),)), (1, ((4, 3.0, 20.0),)), (1, ((2, 1.5, 10.0),)),
                       (1, ((2, 5.0, 20.0),))):
        g = run_gpu([v], stages, st, torch_cuda, kernel_variant=variant)[0]
        o = run_oracle(v, stages, st)
        compare(g, o, stages, f"{W}x{H} {stages}-stage")


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("res", [(16384, 64), (64, 16384)])
def test_largest_width_and_height(torch_cuda, res, variant):
    """Frames at the largest width and height the boundary accepts (16384), as strips: pixel
    indices, tile counts, pooled grids and compaction chunks at their largest per row or column.
    The intrinsics spread 90 x 40 degrees over the strip, so the sweeps cover it."""
    W, H = res
    rng = np.random.default_rng(W + 3 * H)
    sc = scene.make_scene(9, "room")
    fx = (W / 2.0) / np.tan(np.radians(45.0))
    fy = (H / 2.0) / np.tan(np.radians(20.0))
    cam = scene.make_camera(W, H, fx, fy, W / 2.0, H / 2.0, (0.0, 0.0, 1.5))
    rgb, gt = scene.render_rgb(sc, cam, rng)
    scans = []
    for s in range(2):
        pose = scene.make_lidar_pose(cam, (0.1 * s, 0.05, 0.02), 2.0 * s)
        scans.append(scene.Scan(scene.lidar_sweep(sc, pose, 64, 2048 + s, rng), pose))
    v = scene.View(cam, rgb, scans, gt)
    for stages, st in ((2, PAPER_STAGES), (1, ((2, 5.0, 20.0),))):
        g = run_gpu([v], stages, st, torch_cuda, kernel_variant=variant)[0]
        o = run_oracle(v, stages, st)
        m = compare(g, o, stages, f"{W}x{H} {stages}-stage")
        assert m.sum() > 1000, "the sweeps should cover the strip"
        check_points(g, o, cam)


def test_empty_and_degenerate_scans(torch_cuda):
    v = scene.make_view(3, res="qvga", scene_kind="room", n_scans=2, beams=16, az_steps=128)
    # no scans at all, an empty scan, and a scan entirely behind the camera
    rng = np.random.default_rng(0)
    behind = np.stack([rng.uniform(-2, 2, 500), rng.uniform(-2, 2, 500), rng.uniform(-5, -0.1, 500)], 1)
    cases = [[], [(np.zeros((0, 3), np.float32), v.scans[0].lidar_to_world)],
             [(behind.astype(np.float32), v.camera.cam_to_world)]]
    for scans in cases:
        vv = scene.View(v.camera, v.rgb, [scene.Scan(x, p) for x, p in scans], v.gt_depth)
        g = run_gpu([vv], 2, PAPER_STAGES, torch_cuda)[0]
        assert not g["valid"].any() and not g["depth"].any() and g["n"] == 0
        assert np.all(g["zbuf"] == EMPTY)


def test_xyzw_stride_and_host_memory(torch_cuda):
    v = scene.make_view(11, res="qvga", scene_kind="room", n_scans=3, beams=32, az_steps=333)
    o = run_oracle(v, 2, PAPER_STAGES)
    g16 = run_gpu([v], 2, PAPER_STAGES, torch_cuda, xyzw=True)[0]
    compare(g16, o, 2, "xyzw")
    gh = run_gpu([v], 2, PAPER_STAGES, torch_cuda, memory=1)[0]
    compare(gh, o, 2, "host memory")
    check_points(gh, o, v.camera)


def test_points_capacity_short(torch_cuda):
    v = scene.make_view(12, res="qvga", scene_kind="room", n_scans=1, beams=32, az_steps=256)
    o = run_oracle(v, 2, PAPER_STAGES)
    g = run_gpu([v], 2, PAPER_STAGES, torch_cuda, points_cap=100)[0]
    assert g["n"] == len(o["xyz"]) > 100
    assert np.array_equal(g["rgba"][:100], o["rgba"][:100])


@pytest.mark.parametrize("variant", VARIANTS)
def test_batched_equals_alone(torch_cuda, variant):
    """Uneven views in one launch give the same bits as each view alone."""
    views = [scene.make_batch_view(500, res, i, 6) for i, res in enumerate(["540p", "720p", "qvga", "540p"])]
    alone = [run_gpu([v], 2, PAPER_STAGES, torch_cuda, kernel_variant=variant)[0] for v in views]
    mixed = run_gpu(views, 2, PAPER_STAGES, torch_cuda, max_batch=8, kernel_variant=variant)
    for a, b in zip(alone, mixed):
        for k in ("zbuf", "valid", "depth", "coarse", "coarse_valid", "xyz", "rgba"):
            assert np.array_equal(a[k], b[k]), k
    o = run_oracle(views[1], 2, PAPER_STAGES)
    compare(mixed[1], o, 2, "batched 720p")


def test_variants_agree_bit_for_bit(torch_cuda):
    """The TMA-staged and the plain filter kernels in the difference form
    evaluate the same sums in the same order: identical outputs. The expanded
    form evaluates the same weights with other roundings: identical integer
    decisions, depths within FP32 rounding (the exponent's terms reach about
    2 * 88.6 in log2 units, so a few units of 2^-17 per exponent)."""
    v = scene.make_view(31, res="540p", scene_kind="room", n_scans=3, beams=64, az_steps=1024)
    e = run_gpu([v], 2, PAPER_STAGES, torch_cuda, kernel_variant=0)[0]
    b = run_gpu([v], 2, PAPER_STAGES, torch_cuda, kernel_variant=1)[0]
    a = run_gpu([v], 2, PAPER_STAGES, torch_cuda, kernel_variant=2)[0]
    for k in ("valid", "coarse_valid", "zbuf"):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(e[k], b[k]), k
    np.testing.assert_allclose(a["depth"], b["depth"], rtol=2e-6)
    np.testing.assert_allclose(a["coarse"], b["coarse"], rtol=2e-6)
    np.testing.assert_allclose(e["depth"], b["depth"], rtol=3e-5)
    np.testing.assert_allclose(e["coarse"], b["coarse"], rtol=3e-5)


def test_clean_zbuffer_pool_over_many_batches(torch_cuda):
    """Two-stage frames that do not ask for the z-buffer take it from the context's pool of clean
    z-buffers, and the pooling kernel empties the cells it found observed. Rounds of frames of
    different sizes through one context, each round's z-buffers on regions earlier rounds used: every
    frame matches the oracle, so no frame sees another frame's observations."""
    from paper_2601_01210_gb300 import Densifier
    from paper_2601_01210_gb300.frames import FrameBuffers
    res = ["1080p", "720p", "540p", "qvga", "540p", "720p"]
    views = [scene.make_batch_view(55, r, i, len(res)) for i, r in enumerate(res)]
    ref = {}
    with Densifier(dict(num_stages=2, stages=PAPER_STAGES, launch_policy=1, max_batch=4, max_inflight=8,
                        hbm_budget_bytes=512 << 20)) as d:
        for rnd in range(4):
            pick = [(rnd + k) % len(views) for k in range(4)]
            bufs = [FrameBuffers(views[i].camera, views[i].rgb,
                                 [(s.xyz, s.lidar_to_world) for s in views[i].scans]) for i in pick]
            ts = [d.submit(b.frame) for b in bufs]
            d.flush()
            for t in ts:
                assert d.poll(t, -1) == 0
            torch_cuda.cuda.synchronize()
            for i, b in zip(pick, bufs):
                if i not in ref:
                    ref[i] = run_oracle(views[i], 2, PAPER_STAGES)
                g, o = b.results(), ref[i]
                assert np.array_equal(g["valid"], o["valid"]), (rnd, i)
                m = o["valid"].astype(bool)
                rel = np.abs(g["depth"][m] - o["depth"][m]) / o["depth"][m]
                assert rel.max() <= RTOL, (rnd, i, rel.max())
                assert g["n"] == int(m.sum())
