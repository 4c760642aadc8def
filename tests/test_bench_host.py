"""Host-side pieces of bench.py that the reported numbers rest on: the observed-tap
counts of both filter stages (the roofline's algorithmic work), each kernel's work for
the path roofline, and the DRAM-traffic lookup keyed on the captured kernel's sources.
Brute force on small random masks; no GPU."""
import json
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _brute_taps(obs, r):
    """Sum over output pixels of the observed pixels in the (2r+1)^2 window."""
    H, W = obs.shape
    n = 0
    for y in range(H):
        for x in range(W):
            n += int(obs[max(0, y - r):y + r + 1, max(0, x - r):x + r + 1].sum())
    return n


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_stage1_taps_brute_force(seed):
    rng = np.random.default_rng(seed)
    obs = rng.random((11, 17)) < 0.25
    assert bench.valid_taps_stage1(obs, r=4) == _brute_taps(obs, 4)


@pytest.mark.parametrize("W,H", [(20, 13), (9, 9), (7, 4)])
def test_stage2_taps_brute_force(W, H):
    rng = np.random.default_rng(W * H)
    Hc, Wc = -(-H // 3), -(-W // 3)
    cv = (rng.random((Hc, Wc)) < 0.5).astype(np.uint8)
    full = np.kron(cv, np.ones((3, 3), np.uint8))[:H, :W] > 0   # restored validity, cropped
    assert bench.valid_taps_stage2(cv, W, H) == _brute_taps(full, 2)


class _T:
    def __init__(self, a):
        self.a = a

    def cpu(self):
        return self

    def numpy(self):
        return self.a


def test_step_work_counts():
    W, H = 97, 50
    z = np.full((H, W), 0x7F800000, np.uint32)
    z[10, 10] = np.float32(1.0).view(np.uint32)
    z[49, 96] = np.float32(2.0).view(np.uint32)
    Hc, Wc = -(-H // 3), -(-W // 3)
    cv = np.zeros((Hc, Wc), np.uint8)
    cv[3, 3] = 1
    probe = types.SimpleNamespace(W=W, H=H, zbuf=_T(z.view(np.int32)), coarse_valid=_T(cv), n_points=lambda: 25)
    view = types.SimpleNamespace(scans=[types.SimpleNamespace(xyz=np.zeros((100, 3), np.float32))] * 2)
    w = bench.step_work(probe, view)
    assert w["prep_compose_clear"] == 4 * W * H
    assert w["project_zbuf"] == 12 * 200 + 4 * 2
    assert w["pool3"] == 7 * W * H + 20 * Wc * Hc
    assert w["bp_count"] == W * H
    assert w["bp_write"] == 8 * W * H + 16 * 25
    # pooled observations at (3, 3) and (16, 32): a full 9 x 9 reach clipped by the grid edge,
    # and the corner pixel's 5 x 5
    assert w["taps1"] == 8 * 8 + 5 * 5
    # the restored 3 x 3 block of pooled pixel (3, 3): 9 pixels, each in 25 windows
    assert w["taps2"] == 9 * 25


def test_traffic_record_follows_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cuh"
    src.write_text("kernel v1\n")
    import hashlib
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"kernel": "k", "variant": {"kp": 4, "warps": 8}, "dram_bytes_per_launch": 123,
           "sources": {"k.cuh": digest}}
    (prof / "traffic.json").write_text(json.dumps({"jbf_stage2": [rec]}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("jbf_stage2", {"kp": 4, "warps": 8}) == 123
    assert bench.profiled_traffic("jbf_stage2", {"kp": 4, "warps": 4}) is None   # another variant
    src.write_text("kernel v2\n")
    assert bench.profiled_traffic("jbf_stage2", {"kp": 4, "warps": 8}) is None   # sources changed


def test_host_link_bounds():
    link = {"h2d_GBps": 200.0, "d2h_GBps": 100.0}
    b = bench.host_link_bounds(link, h2d_bytes=2e9, d2h_bytes=4e9, frames=8, world=2)
    # 10 ms in, 40 ms out: both at once 40 ms a step, one after the other 50 ms
    assert b["bound_frames_per_s"] == round(8 / 0.040 * 2, 1)
    assert b["serial_frames_per_s"] == round(8 / 0.050 * 2, 1)
    assert b["h2d_GBps"] == 200.0 and b["d2h_GBps"] == 100.0


def test_tap_peaks_take_the_binding_bound():
    """The filter forms' tap peaks are the least of the issue, FMA-pipe and ex2 bounds of the
    measured per-SM-per-clock rates."""
    from paper_2601_01210_gb300 import alu_peaks
    rates = {"ffma": 128.0, "ffma2": 64.0, "ex2_f32": 32.0, "ex2_f16x2": 32.0, "tap_paired": 20.0, "dp4a": 64.0}
    p = alu_peaks.tap_peaks(rates)
    # paired: issue 128 / 3.5 = 36.6; FMA pipe shared by 1.5 two-lane FMA and 1 dp4a a tap:
    # 1 / (1.5 / 64 + 1 / 64) = 25.6; ex2 32 / 1 = 32
    assert p["fp32_expanded_pairs"]["binds"] == "fma_pipe"
    assert abs(p["fp32_expanded_pairs"]["taps_per_sm_clk"] - 25.6) < 1e-9
    assert p["fp32_expanded_pairs"]["thread_instructions_per_tap"] == 3.5
    # expanded: issue 128 / 6 = 21.3, FMA 128 / 5 = 25.6, ex2 32
    assert p["fp32_expanded"]["binds"] == "issue"
    rates["dp4a"] = 1e9
    assert abs(alu_peaks.tap_peaks(rates)["fp32_expanded_pairs"]["bounds_taps_per_sm_clk"]["fma_pipe"] -
               64.0 / 1.5) < 1e-3
    rates["ex2_f32"] = 16.0
    assert alu_peaks.tap_peaks(rates)["fp32_expanded_pairs"]["binds"] == "ex2"
    # without a measured dp4a rate the paired form has no peak
    del rates["dp4a"]
    assert "fp32_expanded_pairs" not in alu_peaks.tap_peaks(rates)


def test_alu_microbenchmark_library_builds():
    import subprocess
    from paper_2601_01210_gb300 import build
    lib = build.build_peaks()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    assert " T alu_peak_run" in out


def test_config_cpu_leg_reports_errors_against_the_oracle():
    """The CPU leg of the extra workloads: the oracle's own outputs score zero error and exact masks,
    a perturbed depth map is reported with its error."""
    import numpy as np

    import bench
    import oracle
    import scene
    oracle.build()
    views = [scene.make_workload("qvga_1scan", 1000 + i) for i in range(2)]
    cfg = bench.EXTRA_CONFIGS["qvga_1scan_single_stage_fp32"]
    outs = []
    for v in views:
        o = oracle.densify_view(v, num_stages=1, stages=cfg["stages"], emit_points=False)
        outs.append({"depth": o["depth"].astype(np.float32), "valid": o["valid"]})
    rep = bench.config_cpu_leg("qvga", cfg, views, outs, 2)
    e = rep["error_vs_oracle"]
    assert e["all_masks_exact"] and e["max_rel"] < 1e-7
    outs[1]["depth"] = outs[1]["depth"] * np.float32(1.001)
    e = bench.config_cpu_leg("qvga", cfg, views, outs, 2)["error_vs_oracle"]
    assert abs(e["max_rel"] - 1e-3) < 1e-5


def test_single_stage_work_counts_observed_taps():
    """Observed taps of the single-stage filter: a lone observation in a 9x9 window reaches 81 output
    pixels; at the image corner only 25."""
    import numpy as np
    import torch

    import bench

    class Buf:
        W, H = 20, 16

        def __init__(self, cells):
            z = np.full((16, 20), 0x7F800000, np.uint32)
            for (y, x) in cells:
                z[y, x] = np.float32(2.0).view(np.uint32)
            self.zbuf = torch.from_numpy(z.view(np.int32))

        def n_points(self):
            return 0

    class View:
        scans = []

    assert bench.step_work(Buf([(8, 10)]), View, single_radius=4)["taps1"] == 81
    assert bench.step_work(Buf([(0, 0)]), View, single_radius=4)["taps1"] == 25


def test_prepost_config_leg_runs_the_oracle_with_the_same_options():
    """The pre/post-filter workload's CPU leg: the oracle runs with the workload's preprocessing and
    post-filter options and each view's previous frame, so the oracle's own outputs for those options
    score exact masks and no error, and outputs without the options do not."""
    import numpy as np

    import bench
    import oracle
    import scene
    oracle.build()
    cfg = bench.EXTRA_CONFIGS["1080p_3scan_two_stage_prepost_fp32"]
    views = [scene.make_view(606 + i, res="qvga", scene_kind="room", n_scans=3, beams=64, az_steps=512)
             for i in range(2)]
    outs, plain = [], []
    for i, v in enumerate(views):
        o = oracle.densify_view(v, num_stages=2, stages=cfg["stages"], emit_points=False,
                                prev_rgb=bench.moved_frame(v, i), **cfg["prepost"])
        outs.append({"depth": o["depth"].astype(np.float32), "valid": o["valid"]})
        p = oracle.densify_view(v, num_stages=2, stages=cfg["stages"], emit_points=False)
        plain.append({"depth": p["depth"].astype(np.float32), "valid": p["valid"]})
    e = bench.config_cpu_leg("prepost", cfg, views, outs, 2)["error_vs_oracle"]
    assert e["all_masks_exact"] and e["max_rel"] < 1e-7 and "masks_note" in e
    e = bench.config_cpu_leg("prepost", cfg, views, plain, 2)["error_vs_oracle"]
    assert not e["all_masks_exact"]


def test_prepost_work_adds_the_preprocessing_kernels():
    import numpy as np
    import torch

    import bench

    class Buf:
        W, H = 20, 16
        zbuf = torch.from_numpy(np.full((16, 20), 0x7F800000, np.uint32).view(np.int32))

        def n_points(self):
            return 0

    class View:
        scans = []

    w = bench.step_work(Buf(), View, single_radius=2, prepost=dict(occlusion_radius=5, motion_threshold=40.0,
                                                                   contour_threshold=0.05))
    assert (w["motion_mask"], w["motion_dilate"], w["occlusion"], w["contour"]) == (7 * 320, 2 * 320, 8 * 320, 10 * 320)
    assert "occlusion" not in bench.step_work(Buf(), View, single_radius=2)
