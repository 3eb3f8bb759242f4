"""Plans: knobs tuned for one graph shape, applied to a plan's own calls
only.  A plan's run gives the oracle's coloring whatever its knobs, the
process-wide knobs never move, and plans with different knobs run side by
side on several threads."""
import threading

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


def _expect(g, X, seed, perm, iters, perm_seed):
    off, idx = g.numpy()
    c, _ = oracle.color(off, idx, X, seed)
    r, nc = oracle.recolor(off, idx, c, perm, iters, perm_seed)
    return r, nc.tolist()


def test_plan_autotune_runs_the_oracles_coloring():
    g = gg.workload("rmat12")
    off, idx = g.offsets.cuda(), g.idx.cuda()
    before = gc.gc_get_tuning()
    with gc.gc_plan_autotune(off, idx, "RXF", 4, 3, "ND-RAND%2^i", 4, repeats=1) as p:
        assert gc.gc_get_tuning() == before  # tuning ran on this thread's own knobs
        info = gc.gc_plan_get_info(p)
        assert info["tuned_ms"] > 0 and info["tuned_n"] == g.n and info["tuned_nnz"] == g.nnz
        assert info["X"] == 4 and info["iterations"] == 4
        # the plan runs on any graph: the one it was tuned on and another shape
        for graph, seed, perm_seed in ((g, 3, 0), (g, 11, 7), (gg.workload("st27-16"), 5, 2)):
            exp, enc = _expect(graph, 4, seed, "ND-RAND%2^i", 4, perm_seed)
            r, nc, st, val = gc.gc_plan_color_recolor(p, graph.offsets.cuda(), graph.idx.cuda(), seed,
                                                      perm_seed, validate=True)
            assert np.array_equal(r.cpu().numpy(), exp) and nc == enc
            assert val["n_conflicts"] == 0 and st["iterations"] == 4
            # host tensors too
            rh, nch, _, _ = gc.gc_plan_color_recolor(p, graph.offsets, graph.idx, seed, perm_seed)
            assert np.array_equal(rh.numpy(), exp) and nch == enc
    assert gc.gc_get_tuning() == before


EXTREMES = [
    {"g4_max_deg": 0, "g8_max_deg": 0, "g16_max_deg": 0, "g2_max_deg": 0, "warp_max_deg": 0,
     "rc_warp_max_deg": 0, "recolor_mode": 1, "spec_graph": 0, "grid_blocks": 7},
    {"g4_max_deg": 64, "g8_max_deg": 64, "g16_max_deg": 64, "g2_max_deg": 64, "warp_max_deg": 100000,
     "rc_warp_max_deg": 100000, "recolor_mode": 0, "spec_graph": 1},
    None,
]


def test_plans_with_different_knobs_run_side_by_side():
    """Three threads, each with a plan of very different knobs, on their own
    streams at once, several times over; the process-wide knobs are set to a
    fourth setting meanwhile and stay untouched."""
    graphs = [gg.workload("rmat11"), gg.hubs([700, 2500], 3000, seed=4), gg.workload("st27-16")]
    exp = {i: _expect(g, 3, 20 + i, "NI", 3, 0) for i, g in enumerate(graphs)}
    plans = [gc.gc_plan_create(k, "RXF", 3, "NI", 3) for k in EXTREMES]
    gc.gc_set_tuning(g4_max_deg=8, g8_max_deg=16, g16_max_deg=32, g2_max_deg=4)
    process_wide = gc.gc_get_tuning()
    errors = []

    def run(t):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for rep in range(4):
                    i = (t + rep) % len(graphs)
                    g = graphs[i]
                    r, nc, _, _ = gc.gc_plan_color_recolor(plans[t], g.offsets.cuda(), g.idx.cuda(),
                                                           20 + i, 0)
                    s.synchronize()
                    if not (np.array_equal(r.cpu().numpy(), exp[i][0]) and nc == exp[i][1]):
                        errors.append((t, rep, i))
        except Exception as e:  # surfaced below
            errors.append((t, repr(e)))

    try:
        threads = [threading.Thread(target=run, args=(t,)) for t in range(len(plans))]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert errors == []
        assert gc.gc_get_tuning() == process_wide
    finally:
        for p in plans:
            gc.gc_plan_free(p)
        gc.gc_set_tuning()


def test_plan_errors():
    g = gg.erdos_renyi(500, 6.0, seed=1)
    with gc.gc_plan_create(None, "FF", 1, "RV", 1) as p:
        bad = g.idx.cuda().clone()
        bad[3] = 900
        with pytest.raises(gc.GCError) as e:
            gc.gc_plan_color_recolor(p, g.offsets.cuda(), bad, 1)
        assert e.value.name == "GC_ERR_BAD_GRAPH"
    with pytest.raises(ValueError):
        gc.gc_plan_color_recolor(p, g.offsets.cuda(), g.idx.cuda(), 1)
    with pytest.raises(gc.GCError) as e:  # tuning needs the graph on the device
        gc.gc_plan_autotune(g.offsets, g.idx, "FF")
    assert e.value.name == "GC_ERR_INVALID_ARG"


def test_cached_plan_reuses_the_tuned_knobs(tmp_path, monkeypatch):
    from paper_1407_6745_gb300 import autotune
    monkeypatch.setenv("GC_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    g = gg.workload("rmat10")
    off, idx = g.offsets.cuda(), g.idx.cuda()
    before = gc.gc_get_tuning()
    with autotune.plan(off, idx, "FF", 1, 3, "NI", 2) as p1, \
            autotune.plan(off, idx, "FF", 1, 3, "NI", 2) as p2:  # the second from the cache
        assert (tmp_path / "tune.json").exists() and gc.gc_get_tuning() == before
        assert gc.gc_plan_get_info(p1)["tuning"] == gc.gc_plan_get_info(p2)["tuning"]
        exp, enc = _expect(g, 1, 3, "NI", 2, 0)
        r, nc, _, _ = gc.gc_plan_color_recolor(p2, off, idx, 3, 0)
        assert np.array_equal(r.cpu().numpy(), exp) and nc == enc
