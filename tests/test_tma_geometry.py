"""Geometry of the TMA filter tiles, checked on the CPU for every instantiated
variant: a host-only program (tests/tma_geometry_check.cuh), compiled with nvcc
against the same TmaGeom constants the kernels use, walks every tile of a set of
grids and every index the kernels compute into the raw boxes, staged records and
observation bitmaps. The variant list is read from the instantiation lists of the
library's sources, so a new variant is checked before it first runs."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_01210_gb300", "csrc")


def variants():
    out = []
    for fn in ("k_jbf_tma.cu", "k_jbf_tma_exp.cu", "k_jbf_sparse.cu"):
        text = open(os.path.join(CSRC, fn)).read()
        out += re.findall(r"X\((SRC_\w+),\s*(\d+),\s*(\d+),\s*(FORM_\w+),\s*(\d+)\)", text)
    return out


def test_variant_lists_parse():
    v = variants()
    assert len(v) >= 20 and ("SRC_UP", "2", "4", "FORM_EXP_PAIRS", "4") in v
    assert ("SRC_ZBUF", "7", "4", "FORM_SPARSE", "8") in v


def test_every_variant_stays_in_bounds(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    calls = "\n".join(
        f'    bad += geomcheck::check<dz::{s}, {r}, {kp}, {nw}, dz::{f}>("{s} r={r} kp={kp} nw={nw} {f}");'
        for s, r, kp, f, nw in variants())
    src = tmp_path / "geom.cu"
    src.write_text('#include "tma_geometry_check.cuh"\n\nint main() {\n    int bad = 0;\n' + calls +
                   '\n    std::printf("violations: %d\\n", bad);\n    return bad != 0;\n}\n')
    exe = tmp_path / "geom"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "tests"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout[-3000:]
    assert "violations: 0" in run.stdout
