"""Batched coloring and recoloring: each graph of a batch gets exactly the
colors it gets alone (and from the oracle), whatever the mix of sizes,
strategies, permutations (schedules included) and iteration counts in the
batch."""
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


def _mixed_batch(count, seed):
    graphs = gg.batch_mix(count, seed, 30, 4000)
    graphs.append(gg.hubs([700, 2500], 3000, seed=seed))   # rows split into chunks when recoloring
    graphs.append(gg.empty(5))
    graphs.append(gg.workload("rmat12"))  # isolated vertices (722) beside split rows (13)
    rng = np.random.default_rng(seed)
    desc = []
    for i, g in enumerate(graphs):
        desc.append(dict(n=g.n, seed=int(rng.integers(1 << 40)), X=int(rng.choice([1, 1, 3, 8])),
                         perm=["RV", "NI", "ND", "RAND", "ND-RAND%2", "ND-RAND%2^i"][i % 6],
                         iterations=int(rng.integers(0, 6)),
                         perm_seed=int(rng.integers(1 << 40))))
    # the isolated vertices of a graph with no recoloring iteration keep their
    # Random-8 Fit colors (a finished graph, not color 1)
    desc[-2].update(X=8, iterations=0)
    return graphs, desc


def _slices(desc):
    base = 0
    for d in desc:
        yield base, base + d["n"]
        base += d["n"]


@pytest.mark.parametrize("knobs", [{}, dict(recolor_mode=1), dict(spec_graph=0, grid_blocks=5)])
def test_batch_equals_alone(knobs):
    graphs, desc = _mixed_batch(40, 7)
    u = gg.batch_union(graphs).to("cuda")
    try:
        gc.gc_set_tuning(**knobs) if knobs else gc.gc_set_tuning()
        col, rounds, maxc, _ = gc.gc_color_batch(u.offsets, u.idx, desc)
        rc, rmax, _ = gc.gc_recolor_batch(u.offsets, u.idx, desc, col)
        pc, prounds, pmax, _ = gc.gc_color_recolor_batch(u.offsets, u.idx, desc)
    finally:
        gc.gc_set_tuning()
    assert torch.equal(pc, rc) and prounds == rounds and pmax == rmax
    col, rc = col.cpu().numpy(), rc.cpu().numpy()
    for i, ((lo, hi), g, d) in enumerate(zip(_slices(desc), graphs, desc)):
        do, di = g.offsets.cuda(), g.idx.cuda()
        strategy = "RXF" if d["X"] > 1 else "FF"
        alone, st = gc.gc_color(do, di, strategy, d["X"], d["seed"])
        assert np.array_equal(col[lo:hi], alone.cpu().numpy()), f"graph {i} coloring"
        assert rounds[i] == st["rounds"] and maxc[i] == (st["max_color"] if g.n else 0)
        if g.n:
            ralone, nc, _ = gc.gc_recolor(do, di, alone, d["perm"], d["iterations"], d["perm_seed"])
            assert np.array_equal(rc[lo:hi], ralone.cpu().numpy()), f"graph {i} recoloring"
            assert rmax[i] == nc[-1]
        if (i % 9 == 0 or i >= len(graphs) - 3) and g.n:  # the oracle on a sample and the special graphs
            off, idx = g.numpy()
            oc, _ = oracle.color(off, idx, d["X"], d["seed"])
            orc, _ = oracle.recolor(off, idx, oc, d["perm"], d["iterations"], d["perm_seed"])
            assert np.array_equal(rc[lo:hi], orc)


def test_batch_host_memory_and_errors():
    graphs, desc = _mixed_batch(10, 3)
    u = gg.batch_union(graphs)
    hc, hr, hm, _ = gc.gc_color_recolor_batch(u.offsets, u.idx, desc)
    du = u.to("cuda")
    dc, dr, dm, _ = gc.gc_color_recolor_batch(du.offsets, du.idx, desc)
    assert torch.equal(hc, dc.cpu()) and hr == dr and hm == dm
    bad = [dict(d) for d in desc]
    bad[1]["n"] += 1  # no longer tiles the vertices
    with pytest.raises((gc.GCError, ValueError)):
        gc.gc_color_batch(du.offsets, du.idx, bad)
    with pytest.raises(gc.GCError) as e:
        gc.gc_recolor_batch(du.offsets, du.idx, desc, torch.ones(du.n, dtype=torch.int32, device="cuda"))
    assert e.value.name == "GC_ERR_IMPROPER_INPUT"


def test_autotune_returns_valid_knobs_and_caches(tmp_path, monkeypatch):
    from paper_1407_6745_gb300 import autotune
    monkeypatch.setenv("GC_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    g = gg.workload("rmat12").to("cuda")
    before = gc.gc_get_tuning()
    knobs, ms = autotune.autotune(g.offsets, g.idx, "RXF", 4, 3, "RAND", 3)
    assert ms > 0 and gc.gc_get_tuning() == before
    ref, _ = gc.gc_color(g.offsets, g.idx, "RXF", 4, 3)
    try:
        applied = autotune.apply(g.offsets, g.idx, "RXF", 4, 3, "RAND", 3)
        assert (tmp_path / "tune.json").exists() and gc.gc_get_tuning() == applied
        again, _ = gc.gc_color(g.offsets, g.idx, "RXF", 4, 3)
        assert torch.equal(ref, again)
    finally:
        gc.gc_set_tuning()
