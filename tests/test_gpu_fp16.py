"""FP16 form against the FP64 oracle.

The full-resolution filter stage keeps its RGB guide and weights in FP16 and
accumulates the numerator and weight sum in FP32; projection, pooling and the
first stage are FP32 as in the FP32 form. Bar: z-buffer and every validity
mask bit-exact (integer decisions); depth within 1 mm absolute or 1e-3
relative of the oracle at every valid pixel. The error statistics (max abs,
p99 abs, max rel) are printed for the record.
"""
import numpy as np
import pytest

import scene

pytestmark = pytest.mark.gpu

PAPER_STAGES = ((4, 5.0, 20.0), (2, 5.0, 20.0))


def _run(v, stages, precision, torch):
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300.frames import FrameBuffers
    build.build()
    with Densifier(dict(num_stages=len(stages), stages=stages, precision=precision, launch_policy=1)) as d:
        b = FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], debug=True,
                         num_stages=len(stages))
        assert d.poll(d.submit(b.frame), -1) == 0
        torch.cuda.synchronize()
        return b.results()


def _check(g, o, label):
    assert np.array_equal(g["zbuf"].reshape(-1), o["zbuf"].reshape(-1)), label
    if "v1" in o:
        assert np.array_equal(g["coarse_valid"], o["v1"]), label
    assert np.array_equal(g["valid"], o["valid"]), label
    m = o["valid"].astype(bool)
    err = np.abs(g["depth"][m].astype(np.float64) - o["depth"][m])
    rel = err / o["depth"][m]
    bound = np.maximum(1e-3, 1e-3 * o["depth"][m])
    stats = dict(max_abs_m=float(err.max()), p99_abs_m=float(np.percentile(err, 99)), max_rel=float(rel.max()),
                 over_bound=int((err > bound).sum()), pixels=int(m.sum()))
    print(f"\n{label} FP16 depth error vs FP64 oracle: {stats}")
    assert stats["over_bound"] == 0, stats
    assert g["n"] == int(m.sum())
    assert np.array_equal(g["rgba"], o["rgba"])
    return stats


def test_fp16_1080p_two_stage():
    import torch
    import oracle
    v = scene.make_workload("1080p_3scan", 1001)
    g = _run(v, PAPER_STAGES, 1, torch)
    o = oracle.densify_view(v, num_stages=2, stages=PAPER_STAGES)
    _check(g, o, "1080p two-stage")


def test_fp16_qvga_single_stage():
    """Sixteen views of the 320x240 workload (far ground at grazing angles, box edges: windows whose
    depths spread widely, where FP16 weight errors matter most)."""
    import torch
    import oracle
    st = ((4, 3.0, 20.0),)
    for seed in range(1000, 1016):
        v = scene.make_workload("qvga_1scan", seed)
        g = _run(v, st, 1, torch)
        o = oracle.densify_view(v, num_stages=1, stages=st)
        _check(g, o, f"qvga 9x9 seed {seed}")


@pytest.mark.parametrize("radius,sigma_p", [(4, 3.0), (7, 5.0), (2, 5.0)])
def test_fp16_single_stage_every_candidate(tmp_path, monkeypatch, radius, sigma_p):
    """Each FP16 kernel the tuner may pick for a single stage (the sparse form with FP16 weights and
    the gather form with FP16 weights), forced through a tuning-cache entry, holds the FP16 bar against
    the oracle (two 320x240 views and a 960x540 view in one batch: ragged tiles of every kind)."""
    import torch
    import oracle
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300.frames import FrameBuffers
    build.build()
    st = ((radius, sigma_p, 20.0),)
    views = [scene.make_workload("qvga_1scan", 1003), scene.make_workload("qvga_1scan", 1011),
             scene.make_batch_view(80, "540p", 0, 2)]

    def run(**params):
        with Densifier(dict(num_stages=1, stages=st, precision=1, launch_policy=1, max_batch=8, **params)) as d:
            bufs = [FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], debug=True,
                                 num_stages=1) for v in views]
            ts = [d.submit(b.frame) for b in bufs]
            d.flush()
            for t in ts:
                assert d.poll(t, -1) == 0
            torch.cuda.synchronize()
            return [b.results() for b in bufs], d.describe()

    _, desc = run()
    oracles = [oracle.densify_view(v, num_stages=1, stages=st) for v in views]
    px = sum(v.rgb.shape[0] * v.rgb.shape[1] for v in views)
    key = f"kind=0,r={radius},half=1,px=2^{px.bit_length() - 1}"
    tag = {"fp16": "fp16", "fp16_sparse": "sparse_fp16"}
    tried = set()
    for c in desc["stages"][0]["candidates"]:
        name = f"tma:kp{c['kp']}:nw{c['warps']}:{tag[c['form']]}"
        cache = tmp_path / f"{radius}_{name.replace(':', '_')}.txt"
        cache.write_text(f"{key} {name}\n")
        monkeypatch.setenv("DENSIFY_TUNE_CACHE", str(cache))
        got, d = run(autotune=1)
        ch = d["stages"][0]["chosen"]
        assert (ch["kp"], ch["warps"], ch["form"]) == (c["kp"], c["warps"], c["form"])
        for g, o, v in zip(got, oracles, views):
            _check(g, o, f"{name} {v.name}")
        tried.add(c["form"])
    assert tried == {"fp16", "fp16_sparse"}


def test_fp16_uneven_views_two_stage():
    import torch
    import oracle
    for i, res in enumerate(["1080p", "720p", "540p"]):
        v = scene.make_batch_view(1003, res, 4 * i, 12)
        g = _run(v, PAPER_STAGES, 1, torch)
        o = oracle.densify_view(v, num_stages=2, stages=PAPER_STAGES)
        _check(g, o, f"{res} two-stage")


def test_fp16_rejected_where_unavailable():
    from paper_2601_01210_gb300 import densify as D
    p = D.densify_default_params()
    p.precision = D.DENSIFY_FP16
    p.kernel_variant = 1
    with pytest.raises(D.DensifyError) as e:
        D.densify_create(p)
    assert e.value.status == D.DENSIFY_E_INVALID
