"""gc_validate_noalloc: the validation entry point that allocates nothing.

It serves callers that cannot allocate device memory -- a process whose own
caching allocator has reserved the device's memory up front, a check right
after an out-of-memory error, a path that must not wait on the driver's
allocator -- by working in a fixed scratch array in the library's static
device memory.  These checks call it through the C ABI and compare it with
gc_validate (the allocating entry point) and with the CPU oracle's validation
on consecutive calls, so a result left in the shared array by one call cannot
leak into the next.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

gc = pytest.importorskip("paper_1407_6745_gb300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gc.load()


def _both(off, idx, colors):
    got = gc.gc_validate_noalloc(off, idx, colors)
    ref = gc.gc_validate(off, idx, colors)
    assert got == ref
    want = oracle.validate(off.cpu().numpy(), idx.cpu().numpy(), colors.cpu().numpy())
    assert got == want
    return got


def test_noalloc_matches_validate_on_consecutive_calls():
    g = gg.erdos_renyi(20000, 12.0, seed=21)
    off, idx = g.offsets.cuda(), g.idx.cuda()
    proper, _ = gc.gc_color(off, idx, "RXF", 5, 3)
    rng = np.random.default_rng(4)
    improper = torch.from_numpy(rng.integers(0, 9, size=g.n).astype(np.int32)).cuda()
    first = _both(off, idx, proper)        # call 1: a proper coloring
    second = _both(off, idx, improper)     # call 2: conflicts and uncolored vertices
    third = _both(off, idx, proper)        # call 3: the shared array was cleared
    assert first["n_conflicts"] == 0 and first["first_bad_vertex"] == -1
    assert second["n_conflicts"] > 0 and second["n_uncolored"] > 0
    assert third == first


def test_noalloc_heavy_rows_and_limits():
    g = gg.hubs([300, 700, 2500, 9000], 12000, seed=6)
    off, idx = g.offsets.cuda(), g.idx.cuda()
    col, _ = gc.gc_color(off, idx, "FF")
    bad = col.clone()
    bad[0] = bad[int(g.idx[int(g.offsets[0])])]  # hub 0 now shares a color with a neighbor
    _both(off, idx, col)
    r = _both(off, idx, bad)
    assert r["n_conflicts"] >= 2 and r["first_bad_vertex"] == 0
    # colors beyond the scratch's 65536-color bitmap are rejected, not miscounted
    big = col.clone()
    big[5] = 70000
    with pytest.raises(gc.GCError) as e:
        gc.gc_validate_noalloc(off, idx, big)
    assert e.value.name == "GC_ERR_INVALID_ARG"
    with pytest.raises(gc.GCError) as e:
        gc.gc_validate_noalloc(g.offsets, g.idx, col.cpu())
    assert e.value.name == "GC_ERR_INVALID_ARG"
    _both(off, idx, col)
