"""densify_frame_noalloc: the entry point that allocates nothing, for callers
that cannot call cudaMalloc (a real-time loop with a frozen device-memory
footprint, or a plug-in inside an application that owns the GPU allocator).

Checks it through the C ABI against the context path (densify_create /
densify_submit / densify_poll) on two calls in a row with different frames,
so the second call runs on scratch the first one left behind. Same bar as
the parity tests: masks, z-buffer, point count and colours bit-exact, depth
and points within 1e-4 relative.
"""
import numpy as np
import pytest

import scene

pytestmark = pytest.mark.gpu

STAGES = ((4, 5.0, 20.0), (2, 5.0, 20.0))
QVGA_STAGES = ((4, 3.0, 20.0),)                       # single stage, 9x9 window


def _context_results(v, torch, stages=STAGES, emit_points=True):
    from paper_2601_01210_gb300 import Densifier
    from paper_2601_01210_gb300.frames import FrameBuffers
    ns = len(stages)
    with Densifier(dict(num_stages=ns, stages=stages, launch_policy=1, emit_points=int(emit_points))) as d:
        b = FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], debug=True, num_stages=ns,
                         emit_points=emit_points)
        t = d.submit(b.frame)
        assert d.poll(t, -1) == 0
        torch.cuda.synchronize()
        return b.results()


def _params(stages, emit_points=True):
    from paper_2601_01210_gb300 import densify as D
    p = D.densify_default_params()
    p.num_stages = len(stages)
    for i, st in enumerate(stages):
        p.stage[i] = D.densify_stage(*st)
    p.emit_points = int(emit_points)
    return p


def _noalloc_results(v, torch, stages=STAGES, emit_points=True):
    from paper_2601_01210_gb300 import densify as D
    from paper_2601_01210_gb300.frames import FrameBuffers
    b = FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], debug=True,
                     num_stages=len(stages), emit_points=emit_points)
    stream = torch.cuda.Stream()
    st = D.densify_frame_noalloc(_params(stages, emit_points), b.frame, stream.cuda_stream)
    assert st == D.DENSIFY_OK, D.densify_last_error(None)
    stream.synchronize()
    return b.results()


def _same(a, b, two_stage=True, points=True):
    for k in ("zbuf", "valid") + (("coarse_valid",) if two_stage else ()):
        assert np.array_equal(a[k], b[k]), k
    m = a["valid"].astype(bool)
    np.testing.assert_allclose(b["depth"][m], a["depth"][m], rtol=1e-4)
    assert not b["depth"][~m].any()
    if two_stage:
        np.testing.assert_allclose(b["coarse"], a["coarse"], rtol=1e-4, atol=0)
    if points:
        assert a["n"] == b["n"]
        assert np.array_equal(a["rgba"], b["rgba"])
        np.testing.assert_allclose(b["xyz"], a["xyz"], rtol=1e-4, atol=1e-5)


def test_noalloc_matches_context_twice_in_a_row():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_01210_gb300 import build
    build.build()
    views = [scene.make_workload("1080p_3scan", 1001),
             scene.make_view(61, res="720p", scene_kind="room", n_scans=2, beams=96, az_steps=1024)]
    for v in views:
        _same(_context_results(v, torch), _noalloc_results(v, torch))


def test_noalloc_rejects_oversized_frames():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_01210_gb300 import densify as D
    from paper_2601_01210_gb300.frames import FrameBuffers

    class Cam:
        width, height, fx, fy, cx, cy = 3840, 2160, 2800.0, 2800.0, 1920.0, 1080.0
        cam_to_world = np.eye(4)

    rgb = np.zeros((2160, 3840, 3), np.uint8)
    b = FrameBuffers(Cam, rgb, [], emit_points=False)
    p = D.densify_default_params()
    p.emit_points = 0
    st = D.densify_frame_noalloc(p, b.frame, None)
    assert st == D.DENSIFY_E_INVALID
    assert "bytes of scratch" in D.densify_last_error(None)


def test_noalloc_single_stage_and_depth_only():
    """The single-stage path (9x9 window at 320x240) and a call with points off, each against the
    context path."""
    import torch
    assert torch.cuda.is_available()
    from paper_2601_01210_gb300 import build
    build.build()
    v = scene.make_workload("qvga_1scan", 1000)
    _same(_context_results(v, torch, QVGA_STAGES), _noalloc_results(v, torch, QVGA_STAGES), two_stage=False)
    w = scene.make_view(62, res="540p", scene_kind="room", n_scans=3, beams=64, az_steps=1024)
    _same(_context_results(w, torch, emit_points=False), _noalloc_results(w, torch, emit_points=False), points=False)


def test_noalloc_allocates_nothing_after_the_first_call():
    """After one call on the device (it looks up the scratch array and may load the kernels' code),
    further calls leave the device's free memory unchanged."""
    import torch
    assert torch.cuda.is_available()
    from paper_2601_01210_gb300 import build
    from paper_2601_01210_gb300 import densify as D
    from paper_2601_01210_gb300.frames import FrameBuffers
    build.build()
    views = [scene.make_workload("qvga_1scan", 1000), scene.make_batch_view(77, "540p", 0, 1)]
    bufs = [FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans]) for v in views]
    stream = torch.cuda.Stream()
    calls = [(_params(STAGES), b) for b in bufs] + [(_params(QVGA_STAGES), bufs[0])]
    for p, b in calls:   # first calls: set-up
        assert D.densify_frame_noalloc(p, b.frame, stream.cuda_stream) == D.DENSIFY_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for p, b in calls:
            assert D.densify_frame_noalloc(p, b.frame, stream.cuda_stream) == D.DENSIFY_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
