"""GPU path (C ABI -> CUDA kernels) against the CPU oracle, element by element.

Every comparison is bit-exact: the method is integer throughout, so colors,
round counts, conflict counts and per-iteration color counts must match the
oracle exactly on the same seeded inputs.
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
    yield
    gc.gc_set_tuning()


def _dev(g):
    return g.offsets.cuda(), g.idx.cuda()


def _spec(g, strategy, X, seed):
    off, idx = g.numpy()
    oc, ost = oracle.color(off, idx, X if strategy == "RXF" else 1, seed)
    do, di = _dev(g)
    c, st = gc.gc_color(do, di, strategy, X, seed)
    c = c.cpu().numpy()
    assert np.array_equal(c, oc), f"{g.name}: first mismatch at {np.nonzero(c != oc)[0][:5]}"
    for k in ("rounds", "max_color", "edges_examined", "conflicts"):
        assert st[k] == ost[k], (k, st[k], ost[k])
    return oc


def _recolor(g, colors, perm, iters, seed):
    off, idx = g.numpy()
    orc, onc = oracle.recolor(off, idx, colors, perm, iters, seed)
    do, di = _dev(g)
    r, nc, st = gc.gc_recolor(do, di, torch.from_numpy(colors).cuda(), perm, iters, seed)
    r = r.cpu().numpy()
    assert np.array_equal(r, orc), f"{g.name}/{perm}: first mismatch at {np.nonzero(r != orc)[0][:5]}"
    assert nc == onc.tolist()
    return orc


def _pipeline(g, strategy, X, seed, perm, iters, perm_seed, expect):
    do, di = _dev(g)
    r, nc, st, val = gc.gc_color_recolor(do, di, strategy, X, seed, perm, iters, perm_seed,
                                         validate=True)
    assert np.array_equal(r.cpu().numpy(), expect)
    off, idx = g.numpy()
    assert val == oracle.validate(off, idx, expect)
    return nc


# --------------------------------------------------------------------------
# The workload shapes, at sizes the oracle finishes in seconds
# --------------------------------------------------------------------------

def test_erdos_renyi_first_fit_reverse():
    """G(10,000, mean degree 16): FF, then 2 recoloring iterations RV."""
    g = gg.workload("er10k")
    c = _spec(g, "FF", 1, 1)
    r = _recolor(g, c, "RV", 2, 0)
    off, idx = g.numpy()
    _, onc = oracle.recolor(off, idx, c, "RV", 2, 0)
    assert _pipeline(g, "FF", 1, 1, "RV", 2, 0, r) == onc.tolist()


@pytest.mark.parametrize("side", [16, 40])
def test_stencil_random_x_fit_noninc(side):
    """27-point stencil, shuffled ids: Random-8 Fit, then 10 iterations NI."""
    g = gg.workload(f"st27-{side}")
    c = _spec(g, "RXF", 8, 3)
    r = _recolor(g, c, "NI", 10, 0)
    _pipeline(g, "RXF", 8, 3, "NI", 10, 0, r)


@pytest.mark.parametrize("scale", [10, 14])
@pytest.mark.parametrize("strategy,X", [("FF", 1), ("RXF", 4)])
def test_rmat_random_perm(scale, strategy, X):
    """R-MAT (0.57, 0.19, 0.19, 0.05), edge factor 16: FF or Random-4 Fit,
    then 20 iterations RAND."""
    g = gg.workload(f"rmat{scale}")
    c = _spec(g, strategy, X, 7)
    r = _recolor(g, c, "RAND", 20, 5)
    _pipeline(g, strategy, X, 7, "RAND", 20, 5, r)


@pytest.mark.parametrize("perm", ["RV", "NI", "ND", "RAND"])
def test_every_permutation(perm):
    g = gg.erdos_renyi(5000, 24.0, seed=9)
    c = _spec(g, "RXF", 5, 2)
    _recolor(g, c, perm, 4, 13)


@pytest.mark.parametrize("schedule,iters", [("ND-RAND%3", 7), ("ND-RAND%2^i", 9), ("ND-RAND%1", 3),
                                             ("ND-RAND%10", 12)])
def test_nd_rand_schedules(schedule, iters):
    """Sec. 4.2.1 schedules: ND at most iterations, RAND at the scheduled ones."""
    for g in (gg.erdos_renyi(6000, 20.0, seed=12), gg.workload("rmat12"), gg.workload("st27-16")):
        c = _spec(g, "RXF", 6, 4)
        _recolor(g, c, schedule, iters, 21)


@pytest.mark.parametrize("preset", ["speed", "quality", "quality10"])
def test_presets(preset):
    """The "speed" and "quality" parameter sets of Sec. 4.3, end to end."""
    p = gc.gc_preset_params(preset)
    g = gg.workload("st27-24")
    off, idx = g.numpy()
    oc, _ = oracle.color(off, idx, p["X"], 17)
    orc, onc = oracle.recolor(off, idx, oc, p["perm"], p["iterations"], 0)
    nc = _pipeline(g, p["strategy"], p["X"], 17, p["perm"], p["iterations"], 0, orc)
    assert nc == onc.tolist()


# --------------------------------------------------------------------------
# Scheduling thresholds and bitmap windows
# --------------------------------------------------------------------------

THRESHOLD_DEGREES = [0, 1, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 47, 48, 56, 57, 62, 63, 64,
                     65, 100, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 2047, 2048, 2049, 2050,
                     4000, 20000]


@pytest.mark.parametrize("strategy,X", [("FF", 1), ("RXF", 2), ("RXF", 8), ("RXF", 60),
                                        ("RXF", 3000)])
def test_degree_thresholds(strategy, X):
    """Vertices exactly on every bucket boundary (4/8/16 lanes, deg + X = 64,
    the warp thresholds of coloring (1024) and recoloring (512), the 256-entry
    recoloring chunks) and Random-X draws beyond the 64-color register window
    and the 2048-color warp bitmap."""
    g = gg.hubs(THRESHOLD_DEGREES, 30000, seed=3)
    c = _spec(g, strategy, X, 11)
    for perm in ("RV", "NI", "ND", "RAND"):
        _recolor(g, c, perm, 2, 3)


def test_pull_form_with_a_marked_block_row():
    """Warp rows that pull next to one block row (degree 13,000) whose
    neighbors mark it: the form of a graph with one row above 12,288 entries
    holding under 1/16 of the entries."""
    from test_forms import pull_near_graph
    g = pull_near_graph()
    for strategy, X in (("FF", 1), ("RXF", 5)):
        c = _spec(g, strategy, X, 21)
        _recolor(g, c, "RAND", 2, 4)


def test_block_bitmap_window():
    """Random-X draws far past a heavy row's marked bitmap (about degree + 128
    colors): its tentative color comes from the full-row fallback, in 2048-color
    windows, up to colors above 131072 (hubs of degree > 2048 are block-bucket
    rows)."""
    g = gg.hubs([3000, 5000, 2100], 8000, seed=4)
    c = _spec(g, "RXF", 140000, 5)
    assert c.max() > 131072
    _recolor(g, c, "RV", 1, 0)


def test_complete_graph_crosses_register_window():
    """K_70: 70 colors, above the 64-bit register mask."""
    g = gg.complete(70)
    c = _spec(g, "FF", 1, 4)
    assert sorted(c.tolist()) == list(range(1, 71))
    _recolor(g, c, "ND", 2, 0)


@pytest.mark.parametrize("knobs", [
    dict(recolor_mode=1),
    dict(g2_max_deg=0, g4_max_deg=0, g8_max_deg=0, g16_max_deg=0),
    dict(g2_max_deg=0),
    dict(g4_max_deg=64, g8_max_deg=64, g16_max_deg=64),
    dict(warp_max_deg=0),
    dict(warp_max_deg=1 << 30),
    dict(grid_blocks=7),
    dict(grid_blocks=1, recolor_mode=1),
    dict(spec_graph=0),
    dict(spec_graph=0, grid_blocks=3, recolor_mode=1),
    dict(g2_max_deg=8),
    dict(g2_max_deg=64, g4_max_deg=64, g8_max_deg=64, g16_max_deg=64),
    dict(g2_max_deg=4, recolor_mode=1),
    dict(rc_warp_max_deg=0),
    dict(rc_warp_max_deg=1 << 30),
    dict(rc_g2_max_deg=0),
    dict(rc_g2_max_deg=8),    # the value a chain-bound launch takes by default
    dict(rc_g2_max_deg=15),   # about the default of a launch not bound by its chain
    dict(rc_g2_max_deg=64, g2_max_deg=0),
    dict(g2_max_deg=16, rc_g2_max_deg=32),
])
def test_results_do_not_depend_on_scheduling(knobs):
    g = gg.hubs(THRESHOLD_DEGREES[:-1], 6000, seed=8)
    try:
        gc.gc_set_tuning(**knobs)
        c = _spec(g, "RXF", 6, 1)
        _recolor(g, c, "RAND", 3, 2)
        c = _spec(g, "FF", 1, 1)
        _recolor(g, c, "NI", 3, 2)
    finally:
        gc.gc_set_tuning()


# --------------------------------------------------------------------------
# Degenerate inputs, host memory, errors
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 33])
def test_empty_graphs(n):
    g = gg.empty(n)
    c = _spec(g, "RXF", 3, 9)
    if n:
        _recolor(g, c, "RV", 2, 0)


def test_host_memory_matches_device():
    g = gg.workload("rmat12")
    off, idx = g.offsets.cpu(), g.idx.cpu()
    ch, sh = gc.gc_color(off, idx, "RXF", 4, 6)
    do, di = _dev(g)
    cd, sd = gc.gc_color(do, di, "RXF", 4, 6)
    assert torch.equal(ch, cd.cpu()) and sh["rounds"] == sd["rounds"]
    rh, nch, _ = gc.gc_recolor(off, idx, ch, "ND", 3, 1)
    rd, ncd, _ = gc.gc_recolor(do, di, cd, "ND", 3, 1)
    assert torch.equal(rh, rd.cpu()) and nch == ncd
    ph, _, _, _ = gc.gc_color_recolor(off, idx, "RXF", 4, 6, "ND", 3, 1)
    assert torch.equal(ph, rh)
    assert gc.gc_validate(off, idx, rh)["n_conflicts"] == 0


def test_recolor_in_place():
    g = gg.workload("rmat12")
    do, di = _dev(g)
    c, _ = gc.gc_color(do, di, "FF", 1, 3)
    ref, _, _ = gc.gc_recolor(do, di, c, "RAND", 3, 4)
    gc.gc_recolor(do, di, c, "RAND", 3, 4, out=c)
    assert torch.equal(c, ref)


def test_priorities_match_oracle_philox():
    n, seed = 1 << 20, 0x1234_5678_9ABC
    p = gc.gc_priorities(seed, n).cpu().numpy().astype(np.uint32)
    sample = np.random.default_rng(0).integers(0, n, size=4000)
    assert all(int(p[v]) == oracle.priority(seed, int(v)) for v in sample)
    assert p[:64].tolist() == [oracle.priority(seed, v) for v in range(64)]


def test_validate_matches_oracle():
    g = gg.erdos_renyi(3000, 10.0, seed=2)
    off, idx = g.numpy()
    do, di = _dev(g)
    rng = np.random.default_rng(5)
    for trial in range(5):
        col = rng.integers(0 if trial == 0 else 1, 12, size=g.n).astype(np.int32)
        assert gc.gc_validate(do, di, torch.from_numpy(col).cuda()) == oracle.validate(off, idx, col)


def test_bad_graph_is_an_error_not_a_fault():
    """Neighbor ids out of range and broken offsets are caught by the kernels'
    own bounds checks and reported; nothing reads out of bounds."""
    g = gg.path(50)
    do, di = _dev(g)
    bad = di.clone()
    bad[3] = 1000
    for call in (lambda: gc.gc_color(do, bad, "FF"),
                 lambda: gc.gc_recolor(do, bad, torch.ones(50, dtype=torch.int32, device="cuda"))):
        with pytest.raises(gc.GCError) as e:
            call()
        assert e.value.name in ("GC_ERR_BAD_GRAPH", "GC_ERR_IMPROPER_INPUT")
    boff = do.clone()
    boff[10] = boff[11] + 5
    with pytest.raises(gc.GCError) as e:
        gc.gc_color(boff, di, "FF")
    assert e.value.name == "GC_ERR_BAD_GRAPH"
    assert gc.gc_check_graph(do, di) == -1
    assert gc.gc_check_graph(do, bad) == 2  # entry 3 belongs to row 2
    loops = gg.path(4)
    lo = loops.idx.clone()
    lo[0] = 0  # row 0 now holds a self-loop
    assert gc.gc_check_graph(loops.offsets.cuda(), lo.cuda()) == 0


def test_improper_recolor_input():
    g = gg.cycle(9)
    do, di = _dev(g)
    for col in ([1] * 9, [1, 2] * 4 + [1], [0] + [1, 2] * 4):
        with pytest.raises(gc.GCError) as e:
            gc.gc_recolor(do, di, torch.tensor(col, dtype=torch.int32, device="cuda"), "RV", 1)
        assert e.value.name == "GC_ERR_IMPROPER_INPUT"


def test_misaligned_adjacency_uses_scalar_reads():
    """An idx view that is not 16-byte aligned takes the scalar read path;
    results are identical to the aligned (4-id chunk) path and the oracle."""
    g = gg.workload("rmat12")
    do, di = _dev(g)
    buf = torch.empty(di.numel() + 1, dtype=torch.int32, device="cuda")
    buf[1:] = di
    mis = buf[1:]
    assert mis.data_ptr() % 16 != 0
    a, _ = gc.gc_color(do, di, "RXF", 3, 5)
    b, _ = gc.gc_color(do, mis, "RXF", 3, 5)
    assert torch.equal(a, b)
    ra, nca, _ = gc.gc_recolor(do, di, a, "ND", 3, 1)
    rb, ncb, _ = gc.gc_recolor(do, mis, b, "ND", 3, 1)
    assert torch.equal(ra, rb) and nca == ncb
    assert gc.gc_validate(do, mis, rb) == gc.gc_validate(do, di, ra)
    off, idx = g.numpy()
    oc, _ = oracle.color(off, idx, 3, 5)
    assert np.array_equal(a.cpu().numpy(), oc)
