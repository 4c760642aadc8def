"""Kernel timing modes and the kernel launch counter of the C ABI.

timing = 1 times every step of the batch, timing = 2
only the full-resolution filter kernel; densify_kernel_launches counts the
CUDA kernels of completed batches either way."""
import pytest

import scene

pytestmark = pytest.mark.gpu

STAGES = ((4, 5.0, 20.0), (2, 5.0, 20.0))


def _run(timing, batches=3):
    import torch
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300.frames import FrameBuffers
    build.build()
    v = scene.make_view(21, res="540p", scene_kind="room", n_scans=3, beams=64, az_steps=1024)
    with Densifier(dict(num_stages=2, stages=STAGES, launch_policy=1, timing=timing)) as d:
        b = FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans])
        for _ in range(batches):
            assert d.poll(d.submit(b.frame), -1) == 0
        torch.cuda.synchronize()
        return d.kernel_times(), d.kernel_launches(), d.describe()


def test_timing_modes_and_launch_count():
    t1, n1, desc = _run(1)
    tma = [s["chosen"]["kernel"] == "tma" for s in desc["stages"]]
    # prep, project, pool (which flags the first filter's tiles), the first filter, the second
    # filter (its tiles are flagged by the first filter), compaction count + scan + write
    assert tma[0]
    per_batch = 3 + 1 + 1 + 3
    assert n1 == 3 * per_batch
    steps = {"prep_compose_clear", "project_zbuf", "pool3", "jbf_stage1", "jbf_stage2", "bp_count", "bp_write"}
    assert set(t1) == steps
    assert all(n == 3 and us > 0.0 for us, n in t1.values())
    t2, n2, _ = _run(2)
    assert set(t2) == {"jbf_stage2"} and t2["jbf_stage2"][1] == 3 and n2 == n1
    t0, n0, _ = _run(0)
    assert t0 == {} and n0 == n1


def test_timing_value_checked():
    from paper_2601_01210_gb300 import Densifier
    from paper_2601_01210_gb300 import densify as D
    with pytest.raises(D.DensifyError):
        Densifier(dict(num_stages=2, stages=STAGES, timing=3))
