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


def _context_results(v, torch):
    from paper_2601_01210_gb300 import Densifier
    from paper_2601_01210_gb300.frames import FrameBuffers
    with Densifier(dict(num_stages=2, stages=STAGES, launch_policy=1)) as d:
        b = FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], debug=True)
        t = d.submit(b.frame)
        assert d.poll(t, -1) == 0
        torch.cuda.synchronize()
        return b.results()


def _noalloc_results(v, torch):
    from paper_2601_01210_gb300 import densify as D
    from paper_2601_01210_gb300.frames import FrameBuffers
    p = D.densify_default_params()
    p.stage[0] = D.densify_stage(*STAGES[0])
    p.stage[1] = D.densify_stage(*STAGES[1])
    b = FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], debug=True)
    stream = torch.cuda.Stream()
    st = D.densify_frame_noalloc(p, b.frame, stream.cuda_stream)
    assert st == D.DENSIFY_OK, D.densify_last_error(None)
    stream.synchronize()
    return b.results()


def _same(a, b):
    for k in ("zbuf", "valid", "coarse_valid", "rgba"):
        assert np.array_equal(a[k], b[k]), k
    assert a["n"] == b["n"]
    m = a["valid"].astype(bool)
    np.testing.assert_allclose(b["depth"][m], a["depth"][m], rtol=1e-4)
    assert not b["depth"][~m].any()
    np.testing.assert_allclose(b["coarse"], a["coarse"], rtol=1e-4, atol=0)
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
