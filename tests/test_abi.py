"""CPU checks of the C ABI: the library builds and loads, exports exactly what
include/densify.h declares, and the ctypes structs match the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "densify.h")


@pytest.fixture(scope="module")
def built():
    from paper_2601_01210_gb300 import build
    return build.build()


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"DENSIFY_API\s+[\w\s\*]*?\b(densify_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("densify_create", "densify_submit", "densify_poll", "densify_destroy"):
        assert required in names


def _doc_comments():
    """Map each declared function to the comment block directly in front of its declaration."""
    src = open(HEADER).read()
    out = {}
    for m in re.finditer(r"/\*((?:[^*]|\*(?!/))*)\*/\s*DENSIFY_API\s+[\w\s\*]*?\b(densify_\w+)\s*\(", src):
        out[m.group(2)] = " ".join(m.group(1).replace("*", " ").split())
    return out


def test_every_declaration_cites_its_passage():
    """Each entry point's comment names the paper passage that defines what it runs (a section,
    equation, algorithm or table), or states that the paper has no counterpart."""
    docs = _doc_comments()
    assert sorted(docs) == _declared(), "every declaration needs a comment block in front of it"
    cite = re.compile(r"\b(Sec\. \d|Eq\. \(\d|Algorithm \d|Table \d)")
    for name, doc in docs.items():
        assert cite.search(doc) or "no counterpart" in doc.lower(), f"{name}: no passage cited"
    for name in ("densify_create", "densify_submit", "densify_flush", "densify_poll", "densify_destroy"):
        assert cite.search(docs[name]), f"{name}: the boundary call must cite a passage"


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = sorted(set(re.findall(r"\bT (densify_\w+)", out)))
    assert exported == _declared()
    lib = ctypes.CDLL(built)
    for name in _declared():
        assert getattr(lib, name) is not None


def test_binding_covers_every_symbol(built):
    from paper_2601_01210_gb300 import densify as D
    assert sorted(D.EXPORTED) == _declared()
    for name in _declared():
        assert callable(getattr(D, name))


def test_struct_layout_matches_c(tmp_path, built):
    from paper_2601_01210_gb300 import densify as D
    fields = {
        "densify_params": D.densify_params, "densify_frame": D.densify_frame, "densify_scan": D.densify_scan,
        "densify_intrinsics": D.densify_intrinsics, "densify_stage": D.densify_stage,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "densify.h"', "int main(void){"]
    for sname, cls in fields.items():
        lines.append(f'printf("{sname} %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname}.{fname} %zu\\n", offsetof({sname}, {fname}));')
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(c), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    for sname, cls in fields.items():
        assert int(got[sname]) == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert int(got[f"{sname}.{fname}"]) == getattr(cls, fname).offset, f"{sname}.{fname}"


def test_default_params_are_the_paper_two_stage(built):
    import json
    from paper_2601_01210_gb300 import densify as D
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))
    p = D.densify_default_params()
    assert p.num_stages == 2 and p.pool == g["pool_factor"]
    assert p.stage[0].radius == g["stage1_radius"] and p.stage[1].radius == g["stage2_radius"]


def test_create_without_gpu_fails_loudly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2601_01210_gb300 import densify as D
    with pytest.raises(D.DensifyError):
        D.densify_create(D.densify_default_params())


def test_invalid_params_rejected(built):
    from paper_2601_01210_gb300 import densify as D
    p = D.densify_default_params()
    p.stage[1].radius = 9
    with pytest.raises(D.DensifyError) as e:
        D.densify_create(p)
    assert e.value.status == D.DENSIFY_E_INVALID
    assert "radius" in D.densify_last_error(None)


def test_scratch_bytes_scale_with_frame(built):
    from paper_2601_01210_gb300 import densify as D
    p = D.densify_default_params()
    f = D.densify_frame()
    f.K.width, f.K.height = 1920, 1080
    big = D.densify_frame_scratch_bytes(p, f)
    f.K.width, f.K.height = 960, 540
    small = D.densify_frame_scratch_bytes(p, f)
    # z-buffer (4 B) + depth (4 B) + valid (1 B) per pixel at least
    assert big >= 1920 * 1080 * 9 and small >= 960 * 540 * 9
    assert 3.5 < big / small < 4.5
