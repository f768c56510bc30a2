"""C ABI library checks that need no GPU: it builds, loads, and exports every symbol the
header declares; configuration defaults; calls fail with a status instead of crashing
when no device is present."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pmbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmbs_[a-z0-9_]+)\s*\(", src)))


@pytest.mark.parametrize("checked", [False, True])
def test_library_exports_every_declared_symbol(checked):
    """Both the release library and its bounds-checked twin export every call."""
    from paper_2207_06649_b300 import pmbs
    lib = pmbs.load(checked=checked)
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(pmbs.EXPORTED) == names


def test_default_config_matches_documented_values():
    from paper_2207_06649_b300 import pmbs
    c = pmbs.default_config()
    assert c.substeps_per_push == 240 and c.pgs_iters == 10
    assert abs(c.dt - 1 / 240) < 1e-9 and abs(c.gamma - 0.8) < 1e-7
    assert abs(c.pusher_radius - 0.01) < 1e-9 and abs(c.grasp_opening - 0.085) < 1e-9
    assert c.contact_cap == 512 and c.grasp_angles == 16 and c.contour_points == 16


def test_config_struct_layout_matches_header():
    from paper_2207_06649_b300 import pmbs
    src = open(os.path.join(ROOT, "include", "pmbs.h")).read()
    body = src[src.index("typedef struct {"):src.index("} pmbs_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.replace("typedef struct {", "").strip()
        if not decl:
            continue
        parts = decl.split(None, 1)
        for name in parts[1].split(","):
            fields.append(re.sub(r"\[.*\]", "", name).strip())
    assert fields == [f[0] for f in pmbs.pmbs_config._fields_]


def test_create_without_gpu_returns_status():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2207_06649_b300 import pmbs
    lib = pmbs.load()
    cfg = pmbs.default_config(mem_budget_bytes=64 << 20)
    ctx = C.c_void_p()
    st = lib.pmbs_create(C.byref(cfg), None, C.byref(ctx))
    assert st in (pmbs.PMBS_E_CUDA, pmbs.PMBS_E_OOM)
    assert not ctx
    bad = pmbs.default_config(max_boxes_per_env=65)
    assert lib.pmbs_create(C.byref(bad), None, C.byref(ctx)) == pmbs.PMBS_E_INVALID
    lib.pmbs_destroy(None)


def test_binding_has_no_cpu_fallback():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2207_06649_b300")
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
