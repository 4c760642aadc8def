"""Autotuner: on the first batch every kernel able to run a filter stage is
timed on that batch and the fastest kept. Candidates of one arithmetic form
evaluate the same sums in the same order; the expanded and the difference FP32
forms round differently, so tuned and untuned contexts agree bit for bit on
every integer decision and within FP32 rounding on depth."""
import json
import os

import numpy as np
import pytest

import scene

pytestmark = pytest.mark.gpu

STAGES = ((4, 5.0, 20.0), (2, 5.0, 20.0))


def _run(views, torch, debug=False, **params):
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300.frames import FrameBuffers
    build.build()
    with Densifier(dict(num_stages=2, stages=STAGES, launch_policy=1, max_batch=8, **params)) as d:
        bufs = [FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], debug=debug)
                for v in views]
        ts = [d.submit(b.frame) for b in bufs]
        d.flush()
        for t in ts:
            assert d.poll(t, -1) == 0
        torch.cuda.synchronize()
        return [b.results() for b in bufs], d.describe()


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_equals_untuned_and_cache_is_reused(tmp_path, monkeypatch, precision):
    import torch
    views = [scene.make_batch_view(77, r, i, 3) for i, r in enumerate(["1080p", "720p", "540p"])]
    base, desc0 = _run(views, torch, precision=precision)
    assert desc0["tuned"] is False
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("DENSIFY_TUNE_CACHE", str(cache))
    tuned, desc = _run(views, torch, precision=precision, autotune=1)
    assert desc["tuned"] is True
    for st in desc["stages"]:
        timed = [c for c in st["candidates"] if "tuned_us" in c]
        if len(st["candidates"]) > 1:
            assert len(timed) == len(st["candidates"])
            best = min(timed, key=lambda c: c["tuned_us"])
            key = ("kernel", "kp", "warps", "form")
            assert tuple(best[k] for k in key) == tuple(st["chosen"][k] for k in key)
    for a, b in zip(base, tuned):
        for k in ("valid", "rgba"):
            assert np.array_equal(a[k], b[k]), k
        np.testing.assert_allclose(a["depth"], b["depth"], rtol=3e-5)
    lines = cache.read_text().splitlines()
    assert lines and all(" " in l for l in lines)
    # the key's pixel class is the batch's pixel count: 1920x1080 + 1280x720 + 960x540 -> 2^21
    px = sum(v.rgb.shape[0] * v.rgb.shape[1] for v in views)
    assert all(l.split(" ")[0].endswith(f",px=2^{px.bit_length() - 1}") for l in lines), lines
    # a second context with the same workload takes the choices from the cache without timing
    again, desc2 = _run(views, torch, precision=precision, autotune=1)
    assert cache.read_text().splitlines() == lines
    for s1, s2 in zip(desc["stages"], desc2["stages"]):
        assert all(s1["chosen"][k] == s2["chosen"][k] for k in ("kernel", "kp", "warps", "form"))


_FORM_TAG = {"fp32": "fp32", "fp16": "fp16", "fp32_expanded": "exp", "fp32_expanded_pairs": "exp_pairs",
             "fp32_sparse": "sparse", "fp16_sparse": "sparse_fp16"}


@pytest.mark.parametrize("stage", [0, 1])
def test_every_candidate_matches_the_plain_kernel(tmp_path, monkeypatch, stage):
    """Each kernel the tuner may pick for a stage, forced through a tuning-cache
    entry (the other stage runs the plain kernel), gives the plain kernel's
    integer decisions and its depths within FP32 rounding (frames of three
    sizes in one batch: tiles of every kind, ragged rows and columns)."""
    import torch
    views = [scene.make_batch_view(78, r, i, 3) for i, r in enumerate(["1080p", "720p", "540p"])]
    plain, _ = _run(views, torch, debug=True, kernel_variant=1)
    _, desc = _run(views, torch)
    px = sum(v.rgb.shape[0] * v.rgb.shape[1] for v in views)
    keys = [f"kind={k},r={STAGES[i][0]},half=0,px=2^{px.bit_length() - 1}" for i, k in enumerate((1, 2))]
    other = next(c for c in desc["stages"][1 - stage]["candidates"] if c["kernel"] == "plain")
    other_name = f"plain:kp{other['kp']}:nw{other['warps']}"
    tried = set()
    for c in desc["stages"][stage]["candidates"]:
        if c["kernel"] != "tma":
            continue
        name = f"tma:kp{c['kp']}:nw{c['warps']}:{_FORM_TAG[c['form']]}"
        cache = tmp_path / f"{stage}_{name.replace(':', '_')}.txt"
        cache.write_text(f"{keys[stage]} {name}\n{keys[1 - stage]} {other_name}\n")
        monkeypatch.setenv("DENSIFY_TUNE_CACHE", str(cache))
        got, d = _run(views, torch, debug=True, autotune=1)
        assert d["stages"][1 - stage]["chosen"]["kernel"] == "plain"
        ch = d["stages"][stage]["chosen"]
        assert (ch["kp"], ch["warps"], ch["form"]) == (c["kp"], c["warps"], c["form"])
        for a, b in zip(got, plain):
            for k in ("valid", "coarse_valid", "rgba"):
                assert np.array_equal(a[k], b[k]), (name, k)
            np.testing.assert_allclose(a["depth"], b["depth"], rtol=3e-5, err_msg=name)
            np.testing.assert_allclose(a["coarse"], b["coarse"], rtol=3e-5, err_msg=name)
        tried.add(c["form"])
    assert "fp32_expanded" in tried


@pytest.mark.parametrize("radius", [2, 4, 7])
def test_every_single_stage_candidate_matches_the_plain_kernel(tmp_path, monkeypatch, radius):
    """The single stage on the z-buffer: each candidate the tuner may pick (the sparse form and the
    gather forms), forced through a tuning-cache entry, gives the plain kernel's
    integer decisions and its depths within FP32 rounding (frames of three sizes, ragged edges)."""
    import torch
    from paper_2601_01210_gb300 import Densifier, build
    from paper_2601_01210_gb300.frames import FrameBuffers
    build.build()
    views = [scene.make_batch_view(79, r, i, 3) for i, r in enumerate(["720p", "540p", "qvga"])]
    st = ((radius, 5.0, 20.0),)

    def run(**params):
        with Densifier(dict(num_stages=1, stages=st, launch_policy=1, max_batch=8, **params)) as d:
            bufs = [FrameBuffers(v.camera, v.rgb, [(s.xyz, s.lidar_to_world) for s in v.scans], debug=True,
                                 num_stages=1) for v in views]
            ts = [d.submit(b.frame) for b in bufs]
            d.flush()
            for t in ts:
                assert d.poll(t, -1) == 0
            torch.cuda.synchronize()
            return [b.results() for b in bufs], d.describe()

    plain, _ = run(kernel_variant=1)
    _, desc = run()
    px = sum(v.rgb.shape[0] * v.rgb.shape[1] for v in views)
    key = f"kind=0,r={radius},half=0,px=2^{px.bit_length() - 1}"
    tried = set()
    for c in desc["stages"][0]["candidates"]:
        if c["kernel"] != "tma":
            continue
        name = f"tma:kp{c['kp']}:nw{c['warps']}:{_FORM_TAG[c['form']]}"
        cache = tmp_path / f"{radius}_{name.replace(':', '_')}.txt"
        cache.write_text(f"{key} {name}\n")
        monkeypatch.setenv("DENSIFY_TUNE_CACHE", str(cache))
        got, d = run(autotune=1)
        ch = d["stages"][0]["chosen"]
        assert (ch["kp"], ch["warps"], ch["form"]) == (c["kp"], c["warps"], c["form"])
        for a, b in zip(got, plain):
            for k in ("zbuf", "valid", "rgba"):
                assert np.array_equal(a[k], b[k]), (name, k)
            np.testing.assert_allclose(a["depth"], b["depth"], rtol=3e-5, err_msg=name)
        tried.add(c["form"])
    assert "fp32_sparse" in tried
