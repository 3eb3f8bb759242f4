"""Element-wise parity on R-MAT graphs large enough to reach the long-run
logic of the speculative rounds.

Graph500 R-MAT (0.57, 0.19, 0.19, 0.05), edge factor 16, at scale 20 and 22
runs the coloring of the full-size R-MAT workload (First Fit and Random-4
Fit, each followed by 20 RAND recoloring iterations, Sec. 4.1) for hundreds
of rounds with thousands of rows above the block threshold: the marking form
of the heavy rows, its probes of the list heads and its periodic compaction
are all exercised.  The three R-MAT classes of Sec. 4.1 / Table 2 (RMAT-ER,
RMAT-Good, RMAT-Bad; edge factor 8) are run at scale 20 with First Fit + 10
ND iterations, the paper's setting; RMAT-Good and RMAT-Bad take the pulling
form (no row above 12,288 entries: every heavy row a warp row).  Every
comparison is bit-exact against the CPU oracle: colors, round counts,
conflict counts, examined entries and the color count after each iteration.
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
    gc.gc_set_tuning()


_GRAPHS = {}


def _graph(name):
    if name not in _GRAPHS:
        _GRAPHS.clear()  # one graph held at a time
        g = gg.workload(name, device="cuda")
        _GRAPHS[name] = (g, g.numpy())
    return _GRAPHS[name]


def _heavy_form(g, X):
    deg = (g.offsets[1:] - g.offsets[:-1]).to(torch.int64)
    heavy = deg + X > 64
    if not bool(heavy.any()):
        return "none"
    if int(deg.max()) <= 12288:
        return "pull-all"  # every heavy row a warp row
    block_entries = int(deg[heavy & (deg > 1024)].sum())
    return "pull-near" if block_entries * 16 < g.nnz else "marks"


def _check(name, strategy, X, seed, perm, iters, perm_seed, min_rounds, form):
    g, (off, idx) = _graph(name)
    assert _heavy_form(g, X) == form
    oc, ost = oracle.color(off, idx, X, seed)
    assert ost["rounds"] >= min_rounds
    # the coloring alone, with its statistics
    c, st = gc.gc_color(g.offsets, g.idx, strategy, X, seed)
    got = c.cpu().numpy()
    assert np.array_equal(got, oc), f"{name}: first mismatch at {np.nonzero(got != oc)[0][:5]}"
    for k in ("rounds", "max_color", "edges_examined", "conflicts"):
        assert st[k] == ost[k], (k, st[k], ost[k])
    # the recoloring alone
    orc, onc = oracle.recolor(off, idx, oc, perm, iters, perm_seed)
    r, nc, _ = gc.gc_recolor(g.offsets, g.idx, c, perm, iters, perm_seed)
    got = r.cpu().numpy()
    assert np.array_equal(got, orc), f"{name}/{perm}: first mismatch at {np.nonzero(got != orc)[0][:5]}"
    assert nc == onc.tolist()
    # the whole path in one call, validated on the device, as the benchmark runs it
    p, pnc, pst, val = gc.gc_color_recolor(g.offsets, g.idx, strategy, X, seed, perm, iters,
                                           perm_seed, validate=True)
    assert torch.equal(p, r) and pnc == nc and pst["rounds"] == ost["rounds"]
    assert val == oracle.validate(off, idx, orc)
    assert val["n_conflicts"] == 0 and val["n_uncolored"] == 0


@pytest.mark.parametrize("strategy,X,min_rounds", [("FF", 1, 200), ("RXF", 4, 60)])
def test_graph500_rmat20(strategy, X, min_rounds):
    """Scale 20 (1.05 M vertices, 31.4 M entries, max degree 64,470):
    FF (240 rounds) or Random-4 Fit (75 rounds), then 20 RAND iterations."""
    _check("rmat20", strategy, X, 7, "RAND", 20, 5, min_rounds, "marks")


def test_graph500_rmat22_first_fit():
    """Scale 22 (4.2 M vertices, about 130 M entries): First Fit + 20 RAND,
    the largest R-MAT the oracle colors in about a minute."""
    _check("rmat22", "FF", 1, 7, "RAND", 20, 5, 300, "marks")


@pytest.mark.parametrize("cls,form,min_rounds", [("er", "none", 8), ("good", "pull-all", 16),
                                                 ("bad", "pull-all", 60)])
def test_paper_rmat_classes(cls, form, min_rounds):
    """RMAT-ER / RMAT-Good / RMAT-Bad (Sec. 4.1, Table 2) at scale 20, edge
    factor 8: First Fit + 10 ND iterations."""
    _check(f"rmat-{cls}20", "FF", 1, 7, "ND", 10, 0, min_rounds, form)


def test_paper_rmat_bad_random_x_fit():
    """RMAT-Bad at scale 20 with Random-4 Fit + 10 RAND iterations."""
    _check("rmat-bad20", "RXF", 4, 11, "RAND", 10, 3, 20, "pull-all")
