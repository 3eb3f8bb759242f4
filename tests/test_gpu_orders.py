"""Vertex-visit orders as conflict priorities, against the oracle: Largest
First (Sec. 2.2.1) and asynchronous recoloring aRC (Sec. 3)."""
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


def _lf(g, X, seed):
    off, idx = g.numpy()
    oc, ost = oracle.color_lf(off, idx, X, seed)
    c, st = gc.gc_color_ordered(g.offsets.cuda(), g.idx.cuda(), "RXF" if X > 1 else "FF", X, seed, "LF")
    c = c.cpu().numpy()
    assert np.array_equal(c, oc), f"{g.name}: first mismatch at {np.nonzero(c != oc)[0][:5]}"
    for k in ("rounds", "max_color", "edges_examined", "conflicts"):
        assert st[k] == ost[k], (k, st[k], ost[k])
    return oc


GRAPHS = {
    "er": lambda: gg.erdos_renyi(8000, 18.0, seed=31),
    "st27": lambda: gg.workload("st27-20"),
    "rmat12": lambda: gg.workload("rmat12"),
    "rmat14": lambda: gg.workload("rmat14"),
    "hubs": lambda: gg.hubs([0, 3, 63, 64, 65, 600, 2048, 2049, 5000], 12000, seed=8),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("X", [1, 6, 90])
def test_largest_first_matches_oracle(name, X):
    _lf(GRAPHS[name](), X, 5)


@pytest.mark.parametrize("knobs", [dict(warp_max_deg=0), dict(spec_graph=0), dict(grid_blocks=3)])
def test_largest_first_scheduling_independent(knobs):
    g = gg.workload("rmat12")
    try:
        gc.gc_set_tuning(**knobs)
        _lf(g, 1, 9)
        _lf(g, 7, 9)
    finally:
        gc.gc_set_tuning()


def test_largest_first_closed_forms_on_gpu():
    star = gg.star(300)
    c, _ = gc.gc_color_ordered(star.offsets.cuda(), star.idx.cuda(), "FF", 1, 2, "LF")
    c = c.cpu().numpy()
    assert c[0] == 1 and np.all(c[1:] == 2)
    kpq = gg.complete_bipartite(4, 9)
    c, _ = gc.gc_color_ordered(kpq.offsets.cuda(), kpq.idx.cuda(), "FF", 1, 2, "LF")
    deg = np.diff(kpq.offsets.numpy())
    assert np.all(c.cpu().numpy()[deg == 9] == 1) and np.all(c.cpu().numpy()[deg == 4] == 2)
    # the random order through the same entry point is gc_color
    g = gg.erdos_renyi(3000, 9.0, seed=2)
    a, _ = gc.gc_color_ordered(g.offsets.cuda(), g.idx.cuda(), "RXF", 4, 8, "random")
    b, _ = gc.gc_color(g.offsets.cuda(), g.idx.cuda(), "RXF", 4, 8)
    assert torch.equal(a, b)


def _arc(g, colors, perm, iters, seed, device="cuda"):
    off, idx = g.numpy()
    orc, onc, orounds = oracle.recolor_async(off, idx, colors, perm, iters, seed)
    out, nc, st = gc.gc_recolor_async(g.offsets.to(device), g.idx.to(device),
                                      torch.from_numpy(colors).to(device), perm, iters, seed)
    got = out.cpu().numpy()
    assert np.array_equal(got, orc), f"{g.name}/{perm}: first mismatch at {np.nonzero(got != orc)[0][:5]}"
    assert nc == onc.tolist() and st["rounds"] == int(orounds.sum())
    return orc


@pytest.mark.parametrize("name", ["er", "st27", "rmat12", "hubs"])
@pytest.mark.parametrize("perm", ["RV", "NI", "ND", "RAND", "ND-RAND%2"])
def test_arc_matches_oracle(name, perm):
    g = GRAPHS[name]()
    off, idx = g.numpy()
    c, _ = oracle.color(off, idx, 5, 3)
    _arc(g, c, perm, 3, 11)


def test_arc_host_memory_in_place_and_errors():
    g = gg.erdos_renyi(5000, 12.0, seed=4)
    off, idx = g.numpy()
    c, _ = oracle.color(off, idx, 3, 1)
    _arc(g, c, "ND", 2, 0, device="cpu")
    # in place on the device
    dc = torch.from_numpy(c).cuda()
    out, nc, _ = gc.gc_recolor_async(g.offsets.cuda(), g.idx.cuda(), dc, "RV", 2, 0, out=dc)
    orc, onc, _ = oracle.recolor_async(off, idx, c, "RV", 2, 0)
    assert np.array_equal(dc.cpu().numpy(), orc)
    # iterations = 0 copies; an improper input is rejected
    out, nc, _ = gc.gc_recolor_async(g.offsets.cuda(), g.idx.cuda(), torch.from_numpy(c).cuda(), "RV", 0)
    assert np.array_equal(out.cpu().numpy(), c) and nc == [int(c.max())]
    bad = c.copy()
    bad[idx[off[0]]] = bad[0]
    with pytest.raises(gc.GCError) as e:
        gc.gc_recolor_async(g.offsets.cuda(), g.idx.cuda(), torch.from_numpy(bad).cuda(), "RV", 1)
    assert e.value.name == "GC_ERR_IMPROPER_INPUT"


def test_arc_complete_graph_equals_rc():
    g = gg.complete(40)
    rng = np.random.default_rng(5)
    start = (rng.permutation(40) + 1).astype(np.int32)
    a, nc, st = gc.gc_recolor_async(g.offsets.cuda(), g.idx.cuda(), torch.from_numpy(start).cuda(), "RAND", 2, 3)
    r, rnc, _ = gc.gc_recolor(g.offsets.cuda(), g.idx.cuda(), torch.from_numpy(start).cuda(), "RAND", 2, 3)
    assert torch.equal(a, r) and nc == rnc and st["rounds"] == 80
