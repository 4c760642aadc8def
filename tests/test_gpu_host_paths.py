"""Host-memory frames: page-locked buffers (points written by the GPU straight
into host memory) and pageable buffers (staged copies) give the device path's
results; two batches in flight on the context's own streams give the same
results as one at a time."""
import numpy as np
import pytest

import scene

pytestmark = pytest.mark.gpu

STAGES = ((4, 5.0, 20.0), (2, 5.0, 20.0))


def _views():
    return [scene.make_batch_view(321, r, i, 4) for i, r in enumerate(["540p", "720p", "qvga", "540p"])]


def _run(views, torch, memory=0, pinned=True, depth_out=True, **params):
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300.frames import FrameBuffers
    build.build()
    with Densifier(dict(num_stages=2, stages=STAGES, launch_policy=1, max_batch=2, max_inflight=16, **params)) as d:
        bufs = [FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], memory=memory,
                             pinned=pinned, depth_out=depth_out) for v in views]
        ts = [d.submit(b.frame) for b in bufs]
        d.flush()
        for t in ts:
            assert d.poll(t, -1) == 0
        torch.cuda.synchronize()
        return [b.results() for b in bufs]


def _same(a, b, keys):
    for k in keys:
        assert np.array_equal(a[k], b[k]), k


def test_pinned_and_pageable_host_frames_match_device_frames():
    import torch
    views = _views()
    dev = _run(views, torch)
    pinned = _run(views, torch, memory=1)
    pageable = _run(views, torch, memory=1, pinned=False)
    points_only = _run(views, torch, memory=1, depth_out=False)
    for a, b, c, e in zip(dev, pinned, pageable, points_only):
        _same(a, b, ("depth", "valid", "xyz", "rgba", "n"))
        _same(a, c, ("depth", "valid", "xyz", "rgba", "n"))
        _same(a, e, ("xyz", "rgba", "n"))


def test_two_batches_in_flight_on_own_streams():
    import torch
    views = _views()
    one = _run(views, torch, batches_in_flight=1)
    two = _run(views, torch, memory=1, batches_in_flight=2)
    for a, b in zip(one, two):
        _same(a, b, ("depth", "valid", "xyz", "rgba", "n"))


def test_bounded_wait_failure_reaches_the_caller():
    """The error path of a kernel's bounded wait, injected on the host: the batch's status word is
    set (bit 0, as the kernels set it) and collecting its ticket returns DENSIFY_E_CUDA with the
    bounded-wait message; the context stays failed. No wait on the GPU runs out."""
    import torch
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300 import densify as D
    from paper_2601_01210_gb300.frames import FrameBuffers
    build.build()
    v = _views()[2]
    with Densifier(dict(num_stages=2, stages=STAGES, launch_policy=1, max_batch=2, max_inflight=4)) as d:
        b = FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans])
        t = d.submit(b.frame)
        d.flush()
        assert d.poll(t, -1) == 0                       # a healthy batch first
        assert D.densify_inject_wait_failure(d.ctx) == D.DENSIFY_OK
        t = d.submit(b.frame)
        d.flush()
        st = D.densify_poll(d.ctx, t, -1)
        assert st == D.DENSIFY_E_CUDA
        assert "bounded wait" in D.densify_last_error(d.ctx)
        st, _ = D.densify_submit(d.ctx, b.frame)
        assert st == D.DENSIFY_E_CUDA                   # the context stays failed
        torch.cuda.synchronize()
        assert D.densify_destroy(d.ctx) == D.DENSIFY_OK   # and still tears down cleanly
        d.ctx = None
