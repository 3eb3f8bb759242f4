"""The serving loop (gc_server_*): every request's colors, round count and
final max color equal what gc_color_recolor gives the same graph alone, for
requests submitted concurrently and batched however the load falls; requests
admitted while others run and retiring with their own iterations; budget
admission, host-side rejection of bad requests, and the counters."""
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


def _mix(seed):
    """A request mix: graph families and sizes of the served workload, scaled
    down, plus the degenerate cases (no vertices, no edges, one hub)."""
    rng = np.random.default_rng(seed)
    graphs = [
        gg.erdos_renyi(3000, 12.0, seed=1),
        gg.erdos_renyi(20000, 25.0, seed=2),
        gg.shuffle_ids(gg.stencil_3d(16, 16, 16, 27), seed=3),
        gg.stencil_3d(20, 18, 9, 7),
        gg.rmat(12, 16, 0.57, 0.19, 0.19, seed=4),
        gg.rmat(14, 16, 0.57, 0.19, 0.19, seed=5),
        gg.hubs([300, 1500, 6000], 8000, seed=6),
        gg.star(2000),
        gg.complete(60),
        gg.cycle(1001),
        gg.path(2),
        gg.empty(0),
        gg.empty(17),
        gg.grid_2d(50, 40),
    ]
    reqs = []
    for i, g in enumerate(graphs * 2):
        strategy = "FF" if rng.random() < 0.5 else "RXF"
        reqs.append(dict(graph=g, strategy=strategy, X=1 if strategy == "FF" else int(rng.integers(2, 40)),
                         seed=int(rng.integers(0, 2**63)),
                         perm=["RV", "NI", "ND", "RAND", "ND-RAND%3", "ND-RAND%2^i"][i % 6],
                         iterations=int(rng.integers(0, 21)), perm_seed=int(rng.integers(0, 2**32))))
    return reqs


def _alone(r, device="cuda"):
    g = r["graph"]
    off, idx = g.offsets.to(device), g.idx.to(device)
    col, nc, st, _ = gc.gc_color_recolor(off, idx, r["strategy"], r["X"], r["seed"], r["perm"],
                                         r["iterations"], r["perm_seed"])
    return col.cpu().numpy(), nc[-1] if nc else 0, st["rounds"]


def _submit(server, r, device):
    g = r["graph"]
    return gc.gc_server_submit(server, g.offsets.to(device), g.idx.to(device), r["strategy"], r["X"],
                               r["seed"], r["perm"], r["iterations"], r["perm_seed"])


@pytest.mark.parametrize("workers,max_batch,device", [(2, 8, "cuda"), (3, 4, "cpu"), (1, 16, "cpu")])
def test_served_results_equal_alone(workers, max_batch, device):
    reqs = _mix(7 + workers)
    expect = [_alone(r) for r in reqs]
    results = [None] * len(reqs)
    with gc.gc_server_create(2 << 30, max_batch, workers) as srv:
        tickets = [None] * len(reqs)

        def client(part):  # two client threads submit interleaved halves
            for i in range(part, len(reqs), 2):
                tickets[i] = _submit(srv, reqs[i], device)

        th = [threading.Thread(target=client, args=(p,)) for p in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for i, t in enumerate(tickets):
            results[i] = gc.gc_server_wait(srv, t, timeout_ms=120_000)
            assert results[i] is not None, f"request {i} still pending"
        info = gc.gc_server_stats(srv)
    sizes = set()
    for i, ((col, res), (ecol, emax, erounds)) in enumerate(zip(results, expect)):
        assert np.array_equal(col.numpy(), ecol), f"request {i}: colors differ from the graph alone"
        assert res["max_color"] == emax and res["rounds"] == erounds, (i, res, emax, erounds)
        assert res["submit_ms"] <= res["start_ms"] <= res["done_ms"]
        sizes.add(res["batch_size"])
    assert info["submitted"] == info["completed"] == len(reqs) and info["rejected"] == 0
    assert info["bytes_in_use"] == 0 and 0 < info["bytes_peak"] <= 2 << 30
    assert 0 <= info["p50_ms"] <= info["p99_ms"] and info["graphs_per_s"] > 0
    assert max(sizes) <= max_batch


def test_served_results_match_the_oracle():
    """Two small requests checked against the oracle itself."""
    cases = [(gg.erdos_renyi(2000, 10.0, seed=31), "RXF", 6, 17, "ND", 5, 0),
             (gg.shuffle_ids(gg.stencil_3d(10, 10, 10, 27), seed=2), "FF", 1, 3, "RAND", 7, 99)]
    with gc.gc_server_create(1 << 30, 8, 2) as srv:
        tickets = [gc.gc_server_submit(srv, g.offsets, g.idx, s, X, seed, p, it, ps)
                   for g, s, X, seed, p, it, ps in cases]
        out = [gc.gc_server_wait(srv, t) for t in tickets]
    for (g, s, X, seed, p, it, ps), (col, res) in zip(cases, out):
        off, idx = g.numpy()
        oc, ost = oracle.color(off, idx, X, seed)
        orc, onc = oracle.recolor(off, idx, oc, p, it, ps)
        assert np.array_equal(col.numpy(), orc)
        assert res["rounds"] == ost["rounds"] and res["max_color"] == onc[-1]


def test_budget_admission_and_rejections():
    small = gg.erdos_renyi(500, 8.0, seed=3)
    big = gg.rmat(16, 16, 0.57, 0.19, 0.19, seed=4)
    # a budget that holds the small graph but never the big one
    with gc.gc_server_create(4 << 20, 8, 2) as srv:
        with pytest.raises(gc.GCError) as e:
            gc.gc_server_submit(srv, big.offsets, big.idx, "FF")
        assert e.value.name == "GC_ERR_BUDGET"
        ts = [gc.gc_server_submit(srv, small.offsets, small.idx, "RXF", 3, k, "NI", 4) for k in range(12)]
        outs = [gc.gc_server_wait(srv, t) for t in ts]
        info = gc.gc_server_stats(srv)
        assert info["rejected"] == 1 and info["completed"] == 12
        assert info["bytes_peak"] <= 4 << 20
        for k, (col, res) in enumerate(outs):
            ecol, emax, _ = _alone(dict(graph=small, strategy="RXF", X=3, seed=k, perm="NI",
                                        iterations=4, perm_seed=0))
            assert np.array_equal(col.numpy(), ecol) and res["max_color"] == emax
        # a result is handed out once; unknown tickets are rejected
        with pytest.raises(gc.GCError) as e:
            gc.gc_server_poll(srv, ts[0])
        assert e.value.name == "GC_ERR_INVALID_ARG"
        # malformed offsets and arguments are rejected at submit
        loop = gg.path(4)
        bad_off = loop.offsets.clone()
        bad_off[2] = 7  # beyond nnz
        with pytest.raises(gc.GCError) as e:
            gc.gc_server_submit(srv, bad_off, loop.idx, "FF")
        assert e.value.name == "GC_ERR_BAD_GRAPH"
        with pytest.raises(gc.GCError) as e:
            gc.gc_server_submit(srv, small.offsets, small.idx, "RXF", 0)
        assert e.value.name == "GC_ERR_INVALID_ARG"
        with pytest.raises(gc.GCError) as e:
            gc.gc_server_submit(srv, small.offsets, small.idx, "FF", 1, 0, perm=9)
        assert e.value.name == "GC_ERR_INVALID_ARG"


def test_poll_until_done_and_destroy_with_unclaimed_results():
    g = gg.erdos_renyi(50000, 16.0, seed=9)
    srv = gc.gc_server_create(1 << 30, 4, 2)
    t = gc.gc_server_submit(srv, g.offsets, g.idx, "FF", 1, 5, "RV", 20)
    unclaimed = [gc.gc_server_submit(srv, g.offsets, g.idx, "RXF", 4, k, "RAND", 3, k) for k in range(5)]
    got = None
    for _ in range(200000):
        got = gc.gc_server_poll(srv, t)
        if got is not None:
            break
    if got is None:
        got = gc.gc_server_wait(srv, t, timeout_ms=120_000)
    col, res = got
    ecol, emax, _ = _alone(dict(graph=g, strategy="FF", X=1, seed=5, perm="RV", iterations=20, perm_seed=0))
    assert np.array_equal(col.numpy(), ecol) and res["max_color"] == emax
    assert len(unclaimed) == 5
    gc.gc_server_destroy(srv)  # finishes the queue, frees the unclaimed results
    assert srv.handle is None


@pytest.mark.parametrize("device", ["cpu", "cuda"])
def test_malformed_ids_fail_alone_in_their_batch(device):
    """Ids are checked when the cohort is staged on the device: the request
    with a bad row finishes with GC_ERR_BAD_GRAPH, the others of its cohort
    are colored as if it had not been there."""
    good = [gg.erdos_renyi(4000, 9.0, seed=40 + k) for k in range(5)]
    p = gg.path(6)
    self_loop = p.idx.clone()
    self_loop[3] = 2  # row 2 lists itself
    out_of_range = p.idx.clone()
    out_of_range[0] = 6
    bad = [(p.offsets, self_loop), (p.offsets, out_of_range)]
    with gc.gc_server_create(1 << 30, 16, 1) as srv:
        order = ["g0", "b0", "g1", "g2", "b1", "g3", "g4"]
        tickets = {}
        for name in order:
            if name[0] == "g":
                g = good[int(name[1])]
                tickets[name] = gc.gc_server_submit(srv, g.offsets.to(device), g.idx.to(device), "RXF", 5,
                                                    int(name[1]), "RAND", 6, 1)
            else:
                off, idx = bad[int(name[1])]
                tickets[name] = gc.gc_server_submit(srv, off.to(device), idx.to(device), "FF")
        for name in order:
            if name[0] == "b":
                with pytest.raises(gc.GCError) as e:
                    gc.gc_server_wait(srv, tickets[name])
                assert e.value.name == "GC_ERR_BAD_GRAPH"
            else:
                k = int(name[1])
                col, res = gc.gc_server_wait(srv, tickets[name])
                ecol, emax, erounds = _alone(dict(graph=good[k], strategy="RXF", X=5, seed=k, perm="RAND",
                                                  iterations=6, perm_seed=1))
                assert np.array_equal(col.numpy(), ecol) and res["max_color"] == emax
                assert res["rounds"] == erounds


def _wait_admitted(srv, cohorts, timeout_s=60.0):
    """Blocks until the server has admitted `cohorts` cohorts."""
    import time
    t0 = time.time()
    while gc.gc_server_stats(srv)["batches"] < cohorts:
        assert time.time() - t0 < timeout_s, "the server admitted nothing"
        time.sleep(0.001)


def test_request_admitted_while_another_runs():
    """Continuous batching: a request that arrives while a long one is on the
    GPU is admitted at the next step boundary (its own cohort, later start),
    finishes long before the long one, and both get their colors alone."""
    long_g = gg.rmat(17, 16, 0.57, 0.19, 0.19, seed=11)
    short_g = gg.erdos_renyi(3000, 10.0, seed=12)
    long_r = dict(graph=long_g, strategy="FF", X=1, seed=5, perm="RAND", iterations=400, perm_seed=9)
    short_r = dict(graph=short_g, strategy="RXF", X=3, seed=6, perm="NI", iterations=2, perm_seed=0)
    with gc.gc_server_create(4 << 30, 8, 1) as srv:
        tl = _submit(srv, long_r, "cuda")
        _wait_admitted(srv, 1)
        ts = _submit(srv, short_r, "cuda")
        s_col, s_res = gc.gc_server_wait(srv, ts, timeout_ms=120_000)
        l_col, l_res = gc.gc_server_wait(srv, tl, timeout_ms=300_000)
        info = gc.gc_server_stats(srv)
    assert info["batches"] == 2
    assert s_res["start_ms"] > l_res["start_ms"] and s_res["batch_size"] == 1
    assert s_res["done_ms"] < l_res["done_ms"], (s_res, l_res)
    for r, col, res in ((long_r, l_col, l_res), (short_r, s_col, s_res)):
        ecol, emax, erounds = _alone(r)
        assert np.array_equal(col.numpy(), ecol) and res["max_color"] == emax and res["rounds"] == erounds
    # the short request was served by the oracle's rules too
    off, idx = short_g.numpy()
    oc, _ = oracle.color(off, idx, 3, 6)
    orc, _ = oracle.recolor(off, idx, oc, "NI", 2, 0)
    assert np.array_equal(s_col.numpy(), orc)


def test_requests_retire_with_their_own_iterations():
    """Requests of one cohort retire in the order of their iteration counts,
    each as soon as its own iterations are done; once most of the cohort has
    retired it is compacted, and the request still running gets its colors
    alone all the same (checked against the oracle)."""
    graphs = [gg.erdos_renyi(40000, 12.0, seed=20 + k) for k in range(4)]
    iters = [0, 1, 3, 60]
    reqs = [dict(graph=g, strategy="RXF", X=4, seed=k, perm="RAND", iterations=it, perm_seed=3 + k)
            for k, (g, it) in enumerate(zip(graphs, iters))]
    with gc.gc_server_create(4 << 30, 16, 1) as srv:
        blocker = _submit(srv, dict(graph=graphs[0], strategy="FF", X=1, seed=1, perm="RV", iterations=1,
                                    perm_seed=0), "cuda")
        tickets = [_submit(srv, r, "cuda") for r in reqs]  # queued while the blocker runs: one cohort
        gc.gc_server_wait(srv, blocker, timeout_ms=120_000)
        out = [gc.gc_server_wait(srv, t, timeout_ms=300_000) for t in tickets]
        info = gc.gc_server_stats(srv)
    starts = {res["start_ms"] for _, res in out}
    done = [res["done_ms"] for _, res in out]
    for (col, res), r in zip(out, reqs):
        ecol, emax, erounds = _alone(r)
        assert np.array_equal(col.numpy(), ecol) and res["max_color"] == emax and res["rounds"] == erounds
    if len(starts) == 1:  # they formed one cohort (the usual case): retirement order follows iterations
        assert done == sorted(done) and done[0] < done[-1]
    off, idx = graphs[3].numpy()
    oc, _ = oracle.color(off, idx, 4, 3)
    orc, _ = oracle.recolor(off, idx, oc, "RAND", 60, 6)
    assert np.array_equal(out[3][0].numpy(), orc)
    assert info["bytes_in_use"] == 0 and info["completed"] == 5
