"""Serving on the GPU: frames from many viewpoints arrive while others are on
the device, are admitted as slots free up and go out in shared batches; each
result equals the same frame densified alone.

Both precisions and one or two batches in flight are covered. The comparison
is bit-exact in every case, which is stricter than the per-form tolerance (FP32:
1e-4 relative against the oracle; FP16: 1 mm or 1e-3 relative): a frame runs
the same kernels with the same sums whatever batch it shares, and with two
batches in flight on the context's own streams their work overlaps on the GPU
without touching each other's scratch."""
import numpy as np
import pytest

import scene

pytestmark = pytest.mark.gpu

STAGES = ((4, 5.0, 20.0), (2, 5.0, 20.0))


@pytest.mark.parametrize("batches_in_flight", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_results_in_the_mix_equal_results_alone(precision, batches_in_flight):
    import torch
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300.frames import FrameBuffers
    from paper_2601_01210_gb300.serve import ServeLoop, poisson_arrivals
    build.build()
    res = ["540p", "qvga", "720p", "540p", "qvga", "540p"]
    views = [scene.make_batch_view(900, r, i, len(res)) for i, r in enumerate(res)]

    def bufs(v):
        return FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans])

    # alone: one frame per launch
    alone = []
    with Densifier(dict(num_stages=2, stages=STAGES, max_batch=1, launch_policy=0, precision=precision)) as d:
        for v in views:
            b = bufs(v)
            assert d.poll(d.submit(b.frame), -1) == 0
            torch.cuda.synchronize()
            alone.append(b.results())
    # served: 2 output slots per view, frames every ~2 ms per view (with two batches in flight,
    # every ~0.5 ms, so that a second batch is launched while the first runs), admission limit 4
    ring = [[bufs(v) for _ in range(2)] for v in views]
    frames = [[b.frame for b in r] for r in ring]
    fps = 500.0 if batches_in_flight == 1 else 2000.0
    with Densifier(dict(num_stages=2, stages=STAGES, max_batch=16, max_inflight=4,
                        batches_in_flight=batches_in_flight, launch_policy=0, precision=precision)) as d:
        arr = poisson_arrivals(len(views), fps, 0.3, seed=5)
        st = ServeLoop(d, frames).run(arr, 0.3, drain_s=10.0)
        batches = d.describe()["batches"]
    torch.cuda.synchronize()
    assert st.completed == st.offered == len(arr)
    assert st.refused_again > 0                      # admission pushed back at least once
    assert batches["launched"] < st.completed        # frames shared batches
    if batches_in_flight == 2:
        assert batches["max_in_flight"] == 2         # a second batch went out while the first ran
    for v, r in enumerate(ring):
        for b in r:
            g = b.results()
            for k in ("valid", "depth", "xyz", "rgba"):
                assert np.array_equal(g[k], alone[v][k]), (v, k)
