"""The C-ABI library builds, loads and exports every symbol include/gc.h
declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "gc.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(gc_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1407_6745_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = _declared()
    for must in ("gc_color", "gc_recolor", "gc_color_recolor", "gc_validate", "gc_check_graph",
                 "gc_status_string", "gc_version"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert missing == []


def test_host_only_entry_points(lib):
    lib.gc_status_string.restype = ctypes.c_char_p
    assert lib.gc_status_string(0) == b"ok"
    assert lib.gc_status_string(3) == b"input coloring is not proper"
    assert lib.gc_version() >= 100


def test_argument_checks_need_no_gpu():
    """Invalid arguments are rejected on the host before any CUDA call."""
    import torch
    import paper_1407_6745_gb300 as gc
    off = torch.tensor([0, 1, 2], dtype=torch.int64)
    idx = torch.tensor([1, 0], dtype=torch.int32)
    with pytest.raises(gc.GCError) as e:
        gc.gc_color(off, idx, "RXF", X=0)
    assert e.value.name == "GC_ERR_INVALID_ARG"
    with pytest.raises(gc.GCError) as e:
        gc.gc_recolor(off, idx, torch.ones(2, dtype=torch.int32), perm=7)
    assert e.value.name == "GC_ERR_INVALID_ARG"
    with pytest.raises(gc.GCError):
        gc.gc_set_tuning(g4_max_deg=9, g8_max_deg=8)
    gc.gc_set_tuning()
    t = gc.gc_get_tuning()
    assert t["warp_max_deg"] == 1024 and t["rc_warp_max_deg"] == 512
    assert t["g2_max_deg"] == 32 and t["rc_g2_max_deg"] == 16
    with pytest.raises(gc.GCError):
        gc.gc_set_tuning(rc_g2_max_deg=-1)
    gc.gc_set_tuning()
    for budget, max_batch, workers in ((0, 8, 2), (1 << 20, 0, 2), (1 << 20, 70000, 2), (1 << 20, 8, 0)):
        with pytest.raises(gc.GCError) as e:
            gc.gc_server_create(budget, max_batch, workers)
        assert e.value.name == "GC_ERR_INVALID_ARG"


def test_server_struct_layouts():
    """The binding's ctypes structs match the header's field order and sizes."""
    import ctypes
    import paper_1407_6745_gb300 as gc
    assert ctypes.sizeof(gc._Request) == 40 + 4 + 4 + 8 + 4 + 4 + 8
    assert ctypes.sizeof(gc._RequestResult) == 4 * 4 + 3 * 8
    assert ctypes.sizeof(gc._ServerInfo) == 4 * 8 + 4 * 8 + 2 * 8


def test_presets_are_the_papers_parameter_sets():
    """gc_preset_params returns the parameter sets named in Sec. 4.3 / Sec. 5
    (tests/golden/nd_rand_schedules.json)."""
    import json
    import paper_1407_6745_gb300 as gc
    with open(os.path.join(ROOT, "tests", "golden", "nd_rand_schedules.json")) as f:
        presets = json.load(f)["presets"]
    for name in ("speed", "quality", "quality10"):
        want = presets[name]
        assert gc.gc_preset_params(name) == want
    with pytest.raises(gc.GCError):
        gc.gc_preset_params(7)


def test_schedule_codes_match_the_oracle():
    """The binding's schedule names map to the codes the oracle uses."""
    import oracle
    import paper_1407_6745_gb300 as gc
    for name in ("RV", "NI", "ND", "RAND", "ND-RAND%5", "ND-RAND%10", "ND-RAND%2^i", "ND-RAND%1"):
        assert gc._perm(name) == oracle.perm_code(name)


def test_plans_are_host_objects():
    """gc_plan_create checks its arguments and keeps its settings and knobs
    without touching the GPU or the process-wide knobs."""
    import paper_1407_6745_gb300 as gc
    tun = ctypes.sizeof(gc._Tuning)
    assert tun == 4 * len(gc._Tuning._fields_)
    assert ctypes.sizeof(gc._PlanInfo) == (tun + 4 * 4 + 4 + 7) // 8 * 8 + 2 * 8  # int64 aligned
    gc.gc_set_tuning()
    before = gc.gc_get_tuning()
    with gc.gc_plan_create({"g4_max_deg": 8, "g8_max_deg": 16, "g16_max_deg": 32, "g2_max_deg": 4},
                           "RXF", 6, "ND-RAND%2^i", 9) as p:
        info = gc.gc_plan_get_info(p)
        assert info["strategy"] == gc.RANDOM_X_FIT and info["X"] == 6 and info["iterations"] == 9
        assert info["perm"] == gc._perm("ND-RAND%2^i")
        assert info["tuning"] == dict(before, g4_max_deg=8, g8_max_deg=16, g16_max_deg=32, g2_max_deg=4)
        assert info["tuned_ms"] == 0 and info["tuned_n"] == 0 and info["tuned_nnz"] == 0
    assert p.handle is None and gc.gc_get_tuning() == before
    with gc.gc_plan_create(None, "FF", 17, "RV", 0) as p:  # First Fit ignores X
        info = gc.gc_plan_get_info(p)
        assert info["X"] == 1 and info["tuning"] == before
    bad = [dict(tuning={"g4_max_deg": 65, "g8_max_deg": 64}), dict(strategy=5), dict(strategy="RXF", X=0),
           dict(perm=7), dict(iterations=-1), dict(tuning={"spin_limit": 0})]
    for kw in bad:
        with pytest.raises(gc.GCError) as e:
            gc.gc_plan_create(**kw)
        assert e.value.name == "GC_ERR_INVALID_ARG", kw
