"""Failure detection without a GPU fault: the bounded waits of the dataflow
recoloring give up and report GC_ERR_TIMEOUT (no trap, no hang), and the
context stays usable; malformed inputs are reported as errors."""
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
    gc.gc_set_tuning()
    yield
    gc.gc_set_tuning()


def test_bounded_wait_times_out_and_the_context_survives():
    """K_n recolored in RV order is one chain of n classes of one vertex each:
    every class waits for the one before.  With a spin limit of one poll the
    first wait gives up, the launch drains, and the call reports the timeout."""
    g = gg.complete(1500)
    off, idx = g.offsets.cuda(), g.idx.cuda()
    start = torch.arange(1, 1501, dtype=torch.int32, device="cuda")
    statuses = []
    try:
        gc.gc_set_tuning(spin_limit=1, recolor_mode=0)
        for _ in range(3):
            try:
                gc.gc_recolor(off, idx, start, "RV", 1)
                statuses.append("GC_OK")
            except gc.GCError as e:
                statuses.append(e.name)
    finally:
        gc.gc_set_tuning()
    assert set(statuses) <= {"GC_OK", "GC_ERR_TIMEOUT"}
    assert "GC_ERR_TIMEOUT" in statuses
    # the same call with the default limit is correct afterwards
    out, nc, _ = gc.gc_recolor(off, idx, start, "RV", 2)
    o, i = g.numpy()
    ref, rnc = oracle.recolor(o, i, start.cpu().numpy(), "RV", 2)
    assert np.array_equal(out.cpu().numpy(), ref) and nc == rnc.tolist()


def test_bad_inputs_are_errors_not_faults():
    g = gg.erdos_renyi(2000, 8.0, seed=3)
    off, idx = g.offsets.cuda(), g.idx.cuda()
    bad = idx.clone()
    bad[17] = 5000  # out of range
    with pytest.raises(gc.GCError) as e:
        gc.gc_color(off, bad, "FF")
    assert e.value.name == "GC_ERR_BAD_GRAPH"
    bad = idx.clone()
    bad[int(g.offsets[3])] = 3  # self-loop in row 3
    with pytest.raises(gc.GCError) as e:
        gc.gc_color_recolor(off, bad, "RXF", 4, 1, "ND", 2)
    assert e.value.name == "GC_ERR_BAD_GRAPH"
    # the context is intact
    c, _ = gc.gc_color(off, idx, "FF", 1, 2)
    o, i = g.numpy()
    assert np.array_equal(c.cpu().numpy(), oracle.color(o, i, 1, 2)[0])


def _calls(g, off, idx):
    start = torch.from_numpy(oracle.color(*g.numpy(), 3, 1)[0]).cuda()
    u = gg.batch_union([g, gg.erdos_renyi(500, 6.0, seed=2)]).to("cuda")
    desc = [dict(n=g.n, seed=1, X=3, perm="NI", iterations=2), dict(n=500, seed=2, perm="RAND", iterations=1)]
    return [
        ("color_recolor", lambda: gc.gc_color_recolor(off, idx, "RXF", 3, 1, "NI", 2, 0, validate=True)[0]),
        ("recolor", lambda: gc.gc_recolor(off, idx, start, "RAND", 2, 5)[0]),
        ("color_host", lambda: gc.gc_color(off.cpu(), idx.cpu(), "FF", 1, 2)[0]),
        ("lf", lambda: gc.gc_color_ordered(off, idx, "FF", 1, 2, "LF")[0]),
        ("arc", lambda: gc.gc_recolor_async(off, idx, start, "ND", 2, 1)[0]),
        ("validate", lambda: gc.gc_validate(off, idx, start)),
        ("batch", lambda: gc.gc_color_recolor_batch(u.offsets, u.idx, desc)[0]),
    ]


def test_allocation_failures_are_reported_and_harmless():
    """Host-side fault injection: the k-th scratch allocation of a call fails.
    Every entry point returns GC_ERR_OOM (or succeeds when it allocates fewer
    than k times), and the next call gives the right answer."""
    g = gg.workload("rmat10")  # split rows and heavy rows on both phases
    off, idx = g.offsets.cuda(), g.idx.cuda()
    for name, call in _calls(g, off, idx):
        ref = call()
        ref = ref if isinstance(ref, dict) else ref.clone()
        for k in range(0, 40):
            gc.gc_inject_alloc_failure(k)
            try:
                call()
                failed = False
            except gc.GCError as e:
                assert e.name == "GC_ERR_OOM", (name, k, e.name)
                failed = True
            finally:
                gc.gc_inject_alloc_failure(-1)
            again = call()
            if isinstance(ref, dict):
                assert again == ref, (name, k)
            else:
                assert torch.equal(again, ref), (name, k)
            if not failed:
                break  # the call makes fewer than k + 1 allocations
