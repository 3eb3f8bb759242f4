"""Pins of the CPU oracle to what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
hand trace of the paper's rules (tests/golden), a closed form, a theorem the
paper states (Delta+1 bound, Culberson's non-increase, RC sequential ==
class-parallel), brute force on tiny graphs, or a statistical property.
"""
import itertools
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _np(g):
    return g.numpy()


def _deg(off):
    return np.diff(off)


def _adj(off, idx, v):
    return idx[off[v]:off[v + 1]]


def _brute_chromatic(n, off, idx):
    """Smallest k admitting a proper coloring, by exhaustive search."""
    if n == 0:
        return 0
    edges = [(v, int(u)) for v in range(n) for u in _adj(off, idx, v) if v < u]
    for k in range(1, n + 1):
        for assign in itertools.product(range(k), repeat=n):
            if all(assign[a] != assign[b] for a, b in edges):
                return k
    return n


# --------------------------------------------------------------------------
# Hand traces (tests/golden)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", _load("speculative_hand_traces.json")["cases"],
                         ids=lambda c: c["name"])
def test_speculative_hand_traces(case):
    g = gg.from_edge_list(case["n"], case["edges"])
    off, idx = _np(g)
    draws = None if case["draws"] is None else np.array(case["draws"], dtype=np.uint32)
    colors, st = oracle.color_tables(off, idx, case["X"], np.array(case["prio"], np.uint32), draws)
    assert colors.tolist() == case["expected_colors"]
    assert st["rounds"] == case["expected_rounds"]
    assert st["conflicts"] == case["expected_conflicts"]


@pytest.mark.parametrize("case", _load("recolor_hand_traces.json")["recolor_cases"],
                         ids=lambda c: c["name"])
def test_recolor_hand_traces(case):
    g = gg.from_edge_list(case["n"], case["edges"])
    off, idx = _np(g)
    out, nc = oracle.recolor(off, idx, np.array(case["colors_in"]), case["perm"], 1)
    assert out.tolist() == case["expected_colors"]
    assert nc.tolist() == [max(case["colors_in"]), max(case["expected_colors"])]


@pytest.mark.parametrize("case", _load("recolor_hand_traces.json")["class_order_cases"])
def test_class_order_hand_cases(case):
    draws = case.get("draws")
    order = oracle.class_order(np.array(case["sizes"]), case["perm"],
                               draws=None if draws is None else np.array(draws, np.uint32))
    assert order.tolist() == case["expected"]


@pytest.mark.parametrize("case", _load("validate_hand_cases.json")["cases"],
                         ids=lambda c: c["name"])
def test_validate_hand_cases(case):
    g = gg.from_edge_list(case["n"], case["edges"])
    off, idx = _np(g)
    assert oracle.validate(off, idx, np.array(case["colors"])) == case["expected"]


# --------------------------------------------------------------------------
# Closed forms and special cases
# --------------------------------------------------------------------------

def test_empty_and_single_vertex():
    for n in (0, 1):
        g = gg.empty(n)
        off, idx = _np(g)
        c, st = oracle.color(off, idx, 1, 5)
        assert c.tolist() == [1] * n
        assert st["rounds"] == (1 if n else 0)
        out, nc = oracle.recolor(off, idx, c, "RV", 3)
        assert out.tolist() == [1] * n


@pytest.mark.parametrize("X", [1, 2, 5, 17])
def test_isolated_vertices_closed_form(X):
    """No neighbor is ever colored: the j-th permissible color is j+1, so
    Random-X Fit gives floor(w * X / 2^32) + 1, decided in round 0."""
    n, seed = 200, 99
    off, idx = _np(gg.empty(n))
    c, st = oracle.color(off, idx, X, seed)
    expect = [((oracle.rxf_draw(seed, v, 0) * X) >> 32) + 1 if X > 1 else 1 for v in range(n)]
    assert c.tolist() == expect
    assert st["rounds"] == 1 and st["conflicts"] == 0


@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_complete_graph_needs_n(n):
    off, idx = _np(gg.complete(n))
    c, st = oracle.color(off, idx, 1, 3)
    assert sorted(c.tolist()) == list(range(1, n + 1))
    for perm in ("RV", "NI", "ND", "RAND"):
        out, nc = oracle.recolor(off, idx, c, perm, 2, seed=4)
        assert sorted(out.tolist()) == list(range(1, n + 1))
        assert nc.tolist() == [n, n, n]


def test_complete_graph_first_fit_rounds():
    """On K_n all vertices stay in conflict but one per round: FF colors the
    (prio, id)-largest with 1 in round 0, the next with 2 in round 1, ..."""
    n, seed = 9, 11
    off, idx = _np(gg.complete(n))
    c, st = oracle.color(off, idx, 1, seed)
    rank = sorted(range(n), key=lambda v: (oracle.priority(seed, v), v), reverse=True)
    assert [c[v] for v in rank] == list(range(1, n + 1))
    assert st["rounds"] == n


@pytest.mark.parametrize("m", [1, 2, 3, 10, 50])
def test_odd_cycle_three_colors(m):
    off, idx = _np(gg.cycle(2 * m + 1))
    for X, seed in ((1, 1), (1, 2), (2, 3)):
        c, _ = oracle.color(off, idx, X, seed)
        if X == 1:
            assert c.max() == 3
        assert oracle.validate(off, idx, c)["n_conflicts"] == 0
        out, nc = oracle.recolor(off, idx, c, "ND", 3)
        assert nc[-1] == 3


@pytest.mark.parametrize("n", [4, 6, 20])
def test_even_cycle(n):
    off, idx = _np(gg.cycle(n))
    c, _ = oracle.color(off, idx, 1, 8)
    assert 2 <= c.max() <= 3


@pytest.mark.parametrize("leaves", [1, 2, 7, 40])
def test_star_two_colors(leaves):
    """FF on a star: the center and the leaves that beat it win color 1 in
    round 0 unless the center wins; either way two colors suffice."""
    off, idx = _np(gg.star(leaves))
    for seed in range(5):
        c, _ = oracle.color(off, idx, 1, seed)
        assert c.max() == 2 and oracle.validate(off, idx, c)["n_conflicts"] == 0


def test_first_fit_round0_winners_are_local_maxima():
    """FF round 0 gives everybody 1; exactly the local maxima of (prio, id)
    keep it, and nothing can take color 1 later next to them."""
    g = gg.erdos_renyi(3000, 6.0, seed=5)
    off, idx = _np(g)
    seed = 21
    c, _ = oracle.color(off, idx, 1, seed)
    prio = np.array([oracle.priority(seed, v) for v in range(g.n)], dtype=np.uint64)
    key = prio * np.uint64(1 << 32) + np.arange(g.n, dtype=np.uint64)
    for v in range(g.n):
        nb = _adj(off, idx, v)
        if nb.size == 0 or key[v] > key[nb].max():
            assert c[v] == 1


def test_random_x_fit_with_x1_is_first_fit():
    g = gg.erdos_renyi(2000, 10.0, seed=3)
    off, idx = _np(g)
    a, sa = oracle.color(off, idx, 1, 77)
    # an explicit draw table: X = 1 makes j = 0 whatever the draw
    prio = np.array([oracle.priority(77, v) for v in range(g.n)], dtype=np.uint32)
    draws = np.random.default_rng(0).integers(0, 2**32, size=(sa["rounds"], g.n), dtype=np.uint32)
    b, sb = oracle.color_tables(off, idx, 1, prio, draws)
    assert np.array_equal(a, b) and sa == sb


def test_bipartite_two_coloring_stays_two():
    """Culberson: recoloring never increases the color count; a proper
    2-coloring of a bipartite graph therefore stays a 2-coloring."""
    for g, side in ((gg.complete_bipartite(4, 7), None), (gg.grid_2d(9, 6), (9, 6))):
        off, idx = _np(g)
        if side is None:
            c = np.array([1] * 4 + [2] * 7, dtype=np.int32)
        else:
            X, Y = side
            c = np.array([1 + ((v % X) + (v // X)) % 2 for v in range(g.n)], dtype=np.int32)
        assert oracle.validate(off, idx, c)["n_conflicts"] == 0
        for perm in ("RV", "NI", "ND", "RAND"):
            out, nc = oracle.recolor(off, idx, c, perm, 3, seed=2)
            assert nc.tolist() == [2, 2, 2, 2]
            assert oracle.validate(off, idx, out)["n_conflicts"] == 0


# --------------------------------------------------------------------------
# Theorems the paper states, on random graphs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_bounds_and_properness(seed):
    """Proper coloring (Sec. 1); FF color(v) <= deg(v)+1, hence <= Delta+1
    (Sec. 2.1); Random-X Fit color(v) <= deg(v)+X."""
    g = gg.erdos_renyi(1500, 4.0 + 3 * seed, seed=seed)
    off, idx = _np(g)
    deg = _deg(off)
    for X in (1, 3, 8):
        c, st = oracle.color(off, idx, X, seed + 100)
        val = oracle.validate(off, idx, c)
        assert val["n_conflicts"] == 0 and val["n_uncolored"] == 0
        assert np.all(c <= deg + X)
        assert st["rounds"] <= g.n
        assert st["max_color"] == c.max()


@pytest.mark.parametrize("seed", range(6))
def test_recolor_never_increases(seed):
    g = gg.erdos_renyi(1200, 12.0, seed=10 + seed)
    off, idx = _np(g)
    c, _ = oracle.color(off, idx, 5, seed)
    for perm in ("RV", "NI", "ND", "RAND"):
        out, nc = oracle.recolor(off, idx, c, perm, 6, seed=seed)
        assert np.all(np.diff(nc) <= 0)
        val = oracle.validate(off, idx, out)
        assert val["n_conflicts"] == 0 and val["max_color"] == nc[-1]
        # First Fit output is dense: every color 1..max is used
        assert val["n_distinct"] == val["max_color"]
        assert np.all(out <= _deg(off) + 1)


def _class_parallel_recolor(off, idx, colors, order):
    """RC of Sec. 3: one step per class, all vertices of the class choose at
    once against the new colors of the classes already done."""
    n = len(off) - 1
    new = np.zeros(n, dtype=np.int64)
    for c in order:
        members = np.nonzero(colors == c)[0]
        choice = {}
        for v in members:
            used = {int(new[u]) for u in _adj(off, idx, v) if new[u] > 0}
            k = 1
            while k in used:
                k += 1
            choice[v] = k
        for v, k in choice.items():
            new[v] = k
    return new


@pytest.mark.parametrize("perm", ["RV", "NI", "ND", "RAND"])
def test_recolor_sequential_equals_class_parallel(perm):
    """Sec. 3: coloring a class's vertices all at once creates no conflict
    and gives exactly the sequential result."""
    for seed in range(4):
        g = gg.erdos_renyi(400, 9.0, seed=40 + seed)
        off, idx = _np(g)
        c, _ = oracle.color(off, idx, 4, seed)
        sizes = np.bincount(c, minlength=c.max() + 1)
        order = oracle.class_order(sizes, perm, seed=seed, iteration=0)
        expect = _class_parallel_recolor(off, idx, c, order)
        out, _ = oracle.recolor(off, idx, c, perm, 1, seed=seed)
        assert np.array_equal(out, expect)


@pytest.mark.parametrize("seed", range(25))
def test_brute_force_chromatic_lower_bound(seed):
    n = 4 + seed % 7
    g = gg.random_small(n, 0.45, seed)
    off, idx = _np(g)
    chi = _brute_chromatic(n, off, idx)
    for X in (1, 2, 4):
        c, _ = oracle.color(off, idx, X, seed)
        assert c.max() >= chi
        out, nc = oracle.recolor(off, idx, c, "ND", 2)
        assert nc[-1] >= chi


# --------------------------------------------------------------------------
# ND-RAND permutation schedules (Sec. 4.2.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", _load("nd_rand_schedules.json")["cases"], ids=lambda c: c["schedule"])
def test_schedule_rand_iterations_match_the_paper(case):
    perms = [oracle.perm_of_iteration(case["schedule"], t) for t in range(case["iterations"])]
    assert [t + 1 for t, p in enumerate(perms) if p == oracle.PERM_RANDOM] == case["rand_at"]
    assert all(p in (oracle.PERM_RANDOM, oracle.PERM_NONDEC) for p in perms)


@pytest.mark.parametrize("schedule,iters", [("ND-RAND%3", 7), ("ND-RAND%2^i", 9), ("ND-RAND%1", 3)])
def test_schedule_recolor_is_the_iterations_composed(schedule, iters):
    """Each iteration is one RC pass (computed here class by class, outside
    the oracle) in the order ND, or RAND drawn with that iteration's number."""
    rand_at = {t for t in range(1, iters + 1)
               if oracle.perm_of_iteration(schedule, t - 1) == oracle.PERM_RANDOM}
    for seed in range(3):
        g = gg.erdos_renyi(300, 10.0, seed=70 + seed)
        off, idx = _np(g)
        c, _ = oracle.color(off, idx, 6, seed)
        cur = c.astype(np.int64)
        for t in range(1, iters + 1):
            sizes = np.bincount(cur, minlength=cur.max() + 1)
            if t in rand_at:
                order = oracle.class_order(sizes, "RAND", seed=seed + 9, iteration=t - 1)
            else:
                order = oracle.class_order(sizes, "ND")
            cur = _class_parallel_recolor(off, idx, cur, order)
        out, nc = oracle.recolor(off, idx, c, schedule, iters, seed=seed + 9)
        assert np.array_equal(out, cur)
        assert np.all(np.diff(nc) <= 0)


def test_schedule_without_a_rand_iteration_is_nd():
    g = gg.erdos_renyi(500, 14.0, seed=5)
    off, idx = _np(g)
    c, _ = oracle.color(off, idx, 3, 2)
    nd, _ = oracle.recolor(off, idx, c, "ND", 4)
    assert np.array_equal(oracle.recolor(off, idx, c, "ND-RAND%5", 4, seed=1)[0], nd)
    assert np.array_equal(oracle.recolor(off, idx, c, "ND-RAND%2^i", 1, seed=1)[0],
                          oracle.recolor(off, idx, c, "ND", 1)[0])


def test_schedule_codes_out_of_range():
    g = gg.path(3)
    off, idx = _np(g)
    c = np.array([1, 2, 1], dtype=np.int32)
    for bad in (oracle.SCHED_EVERY_BASE, oracle.SCHED_EVERY_BASE + 65536, 5, -1):
        with pytest.raises(oracle.OracleError):
            oracle.recolor(off, idx, c, bad, 1)
        assert oracle.perm_of_iteration(bad, 0) == -1


# --------------------------------------------------------------------------
# Largest First (Sec. 2.2.1) and asynchronous recoloring (aRC, Sec. 3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("leaves", [2, 5, 40])
def test_lf_star_hub_keeps_first_color(leaves):
    """The hub has the largest degree, so it wins round 0 with color 1 and
    every leaf takes 2 in round 1 (a random order usually loses the hub)."""
    g = gg.star(leaves)
    off, idx = _np(g)
    c, st = oracle.color_lf(off, idx, 1, 3)
    hub = int(np.argmax(_deg(off)))
    assert c[hub] == 1 and np.all(np.delete(c, hub) == 2) and st["rounds"] == 2


@pytest.mark.parametrize("p,q", [(2, 5), (3, 7), (1, 4)])
def test_lf_complete_bipartite_closed_form(p, q):
    """K_{p,q}, p < q: the p side (degree q) beats the q side (degree p)."""
    g = gg.complete_bipartite(p, q)
    off, idx = _np(g)
    c, _ = oracle.color_lf(off, idx, 1, 0)
    deg = _deg(off)
    assert np.all(c[deg == q] == 1) and np.all(c[deg == p] == 2)


def test_lf_priority_definition_and_path_ends():
    g = gg.path(5)
    off, idx = _np(g)
    for v in range(5):
        d = int(_deg(off)[v])
        assert oracle.ordered_priority(d, 9, v) == (d << 16) | (oracle.priority(9, v) >> 16)
    assert oracle.ordered_priority(70000, 9, 1) >> 16 == 65535
    # interior vertices (degree 2) beat the ends: round 0 keeps 1 on a maximal
    # independent subset of the interior
    c, _ = oracle.color_lf(off, idx, 1, 9)
    assert oracle.validate(off, idx, c)["n_conflicts"] == 0 and c.max() <= 3


@pytest.mark.parametrize("seed", range(3))
def test_lf_bounds_and_regular_graphs(seed):
    g = gg.erdos_renyi(800, 10.0, seed=seed)
    off, idx = _np(g)
    for X in (1, 4):
        c, st = oracle.color_lf(off, idx, X, seed)
        assert oracle.validate(off, idx, c)["n_conflicts"] == 0
        assert np.all(c <= _deg(off) + X)
    # on a regular graph every degree is equal: LF is the random order with
    # a 16-bit priority (the same winners as whenever no two upper halves tie)
    cyc = gg.cycle(101)
    off, idx = _np(cyc)
    c, _ = oracle.color_lf(off, idx, 1, seed)
    assert c.max() == 3


@pytest.mark.parametrize("perm", ["RV", "NI", "ND", "RAND"])
def test_arc_on_complete_graph_equals_rc(perm):
    """K_n: only the vertex of the earliest class can win each round, so the
    class of rank r takes color r + 1, exactly as in RC."""
    g = gg.complete(9)
    off, idx = _np(g)
    rng = np.random.default_rng(3)
    start = (rng.permutation(9) + 1).astype(np.int32)
    out, nc, rounds = oracle.recolor_async(off, idx, start, perm, 2, seed=4)
    rc, rnc = oracle.recolor(off, idx, start, perm, 2, seed=4)
    assert np.array_equal(out, rc) and list(nc) == list(rnc) and list(rounds) == [9, 9]


@pytest.mark.parametrize("name", ["grid", "cycle", "kpq"])
def test_arc_bipartite_two_coloring(name):
    """A connected bipartite graph with a proper 2-coloring: the earlier class
    wins round 0 with color 1, the other class takes 2 in round 1."""
    g = {"grid": gg.grid_2d(9, 7), "cycle": gg.cycle(40), "kpq": gg.complete_bipartite(3, 6)}[name]
    off, idx = _np(g)
    # 2-coloring by BFS parity
    n = len(off) - 1
    side = np.full(n, -1)
    side[0] = 0
    todo = [0]
    while todo:
        v = todo.pop()
        for u in _adj(off, idx, v):
            if side[u] < 0:
                side[u] = 1 - side[v]
                todo.append(u)
    start = (side + 1).astype(np.int32)
    for perm in ("RV", "NI", "RAND"):
        out, nc, rounds = oracle.recolor_async(off, idx, start, perm, 1, seed=1)
        sizes = np.bincount(start, minlength=3)
        order = oracle.class_order(sizes, perm, seed=1, iteration=0)
        assert np.all(out[start == order[0]] == 1) and np.all(out[start == order[1]] == 2)
        assert rounds[0] == 2


@pytest.mark.parametrize("seed", range(4))
def test_arc_properness_bounds_and_rounds(seed):
    g = gg.erdos_renyi(700, 12.0, seed=30 + seed)
    off, idx = _np(g)
    c, _ = oracle.color(off, idx, 5, seed)
    out, nc, rounds = oracle.recolor_async(off, idx, c, "ND-RAND%2", 5, seed=seed)
    assert oracle.validate(off, idx, out)["n_conflicts"] == 0
    assert np.all(out <= _deg(off) + 1)
    assert nc[-1] == out.max()
    # a class of rank r is fixed by round r, so an iteration takes at most
    # as many rounds as the previous coloring has classes
    cur = c
    for it in range(5):
        nxt, _, r = oracle.recolor_async(off, idx, cur, oracle.perm_of_iteration("ND-RAND%2", it), 1, seed=seed)
        assert r[0] <= len(np.unique(cur))
        cur = nxt
    # an edgeless graph keeps one class
    e = gg.empty(6)
    eo, ei = _np(e)
    out, nc, rounds = oracle.recolor_async(eo, ei, np.ones(6, dtype=np.int32), "ND", 2)
    assert np.all(out == 1) and list(rounds) == [1, 1]
    with pytest.raises(oracle.OracleError):
        oracle.recolor_async(off, idx, np.ones(len(off) - 1, dtype=np.int32), "RV", 1)


# --------------------------------------------------------------------------
# Sequential greedy in the NAT and LF orders (Alg. 1; Tables 1-2 columns)
# --------------------------------------------------------------------------

def _crown(k):
    """K_{k,k} minus a perfect matching, sides interleaved u1, v1, u2, v2, ...:
    the classic graph on which natural-order greedy uses k colors (chi = 2)."""
    edges = [(2 * i, 2 * j + 1) for i in range(k) for j in range(k) if i != j]
    return gg.from_edge_list(2 * k, edges)


@pytest.mark.parametrize("k", [3, 5, 9])
def test_greedy_natural_order_on_crown_graph(k):
    off, idx = _np(_crown(k))
    c = oracle.greedy_sequential(off, idx, "NAT")
    assert c.max() == k and list(c[0::2]) == list(range(1, k + 1))
    assert oracle.greedy_sequential(off, idx, "LF").max() == k  # all degrees equal: id order


def test_greedy_closed_forms():
    off, idx = _np(gg.star(30))
    assert list(oracle.greedy_sequential(off, idx, "NAT")[:3]) == [1, 2, 2]
    off, idx = _np(gg.complete(12))
    assert sorted(oracle.greedy_sequential(off, idx, "LF")) == list(range(1, 13))
    off, idx = _np(gg.path(7))
    assert list(oracle.greedy_sequential(off, idx, "NAT")) == [1, 2, 1, 2, 1, 2, 1]
    # LF on a path: the interior (degree 2) first, in id order, then the ends
    assert list(oracle.greedy_sequential(off, idx, "LF")) == [2, 1, 2, 1, 2, 1, 2]


@pytest.mark.parametrize("seed", range(20))
def test_greedy_bounds(seed):
    n = 4 + seed % 7
    g = gg.random_small(n, 0.5, seed)
    off, idx = _np(g)
    chi = _brute_chromatic(n, off, idx)
    for order in ("NAT", "LF"):
        c = oracle.greedy_sequential(off, idx, order)
        assert oracle.validate(off, idx, c)["n_conflicts"] == 0
        assert chi <= c.max() <= _deg(off).max(initial=0) + 1


# --------------------------------------------------------------------------
# Class orders and the generator
# --------------------------------------------------------------------------

def test_class_order_is_permutation_of_present():
    rng = np.random.default_rng(1)
    for _ in range(50):
        sizes = rng.integers(0, 4, size=rng.integers(2, 30))
        sizes[0] = 0
        present = [c for c in range(1, len(sizes)) if sizes[c] > 0]
        for perm in ("RV", "NI", "ND", "RAND"):
            o = oracle.class_order(sizes, perm, seed=int(rng.integers(1 << 30)))
            assert sorted(o.tolist()) == present
        ni = oracle.class_order(sizes, "NI").tolist()
        assert all(sizes[a] >= sizes[b] for a, b in zip(ni, ni[1:]))
        nd = oracle.class_order(sizes, "ND").tolist()
        assert all(sizes[a] <= sizes[b] for a, b in zip(nd, nd[1:]))


def test_random_class_order_uniform():
    """Knuth's shuffle with independent uniform draws gives every one of the
    k! orders with probability 1/k! (chi-square, k = 3, 6000 seeds)."""
    counts = {}
    trials = 6000
    for s in range(trials):
        o = tuple(oracle.class_order(np.array([0, 1, 1, 1]), "RAND", seed=s).tolist())
        counts[o] = counts.get(o, 0) + 1
    assert len(counts) == 6
    exp = trials / 6
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 20.5  # p ~ 0.001 at 5 degrees of freedom


def test_philox_statistics():
    """Philox w0 over consecutive counters: uniform bytes (chi-square over 256
    bins) and about half the output bits flip when one counter bit flips."""
    seed = 12345
    w = np.array([oracle.priority(seed, v) for v in range(1 << 14)], dtype=np.uint64)
    counts = np.bincount((w >> np.uint64(24)).astype(np.int64), minlength=256)
    exp = len(w) / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 340  # 255 dof, p ~ 3e-4
    flips = []
    for v in range(512):
        a = oracle.philox4x32_10([v, 0, 0, 1], [seed & 0xFFFFFFFF, 0])
        b = oracle.philox4x32_10([v ^ 1, 0, 0, 1], [seed & 0xFFFFFFFF, 0])
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 60 < np.mean(flips) < 68  # 128 bits, half expected
    # the tags separate the three streams
    assert oracle.priority(seed, 5) != oracle.rxf_draw(seed, 5, 0)


def test_rxf_draw_index_mapping():
    """j = floor(w X / 2^32) is in [0, X) and each index is hit about
    equally often."""
    X = 7
    js = np.array([(oracle.rxf_draw(3, v, 1) * X) >> 32 for v in range(14000)])
    assert js.min() == 0 and js.max() == X - 1
    counts = np.bincount(js, minlength=X)
    assert np.all(np.abs(counts - 2000) < 200)


# --------------------------------------------------------------------------
# Error behaviour
# --------------------------------------------------------------------------

def test_self_loop_is_a_malformed_graph():
    """C(u) != C(v) on every edge cannot hold on a loop (Sec. 1)."""
    g = gg.path(4)
    off, idx = _np(g)
    idx = idx.copy()
    idx[0] = 0  # row 0 lists itself
    for call in (lambda: oracle.color(off, idx, 1, 0), lambda: oracle.color_lf(off, idx, 1, 0),
                 lambda: oracle.greedy_sequential(off, idx, "NAT")):
        with pytest.raises(oracle.OracleError) as e:
            call()
        assert e.value.code == oracle.ERR_BAD_GRAPH
    # as a coloring to recolor it is improper: the loop is a conflict
    with pytest.raises(oracle.OracleError) as e:
        oracle.recolor(off, idx, np.array([1, 2, 1, 2], dtype=np.int32), "RV", 1)
    assert e.value.code == oracle.ERR_IMPROPER_INPUT


def test_errors():
    off, idx = _np(gg.path(4))
    with pytest.raises(oracle.OracleError) as e:
        oracle.color(off, idx, 0, 1)
    assert e.value.code == oracle.ERR_INVALID_ARG
    bad = idx.copy()
    bad[0] = 9
    with pytest.raises(oracle.OracleError) as e:
        oracle.color(off, bad, 1, 1)
    assert e.value.code == oracle.ERR_BAD_GRAPH
    with pytest.raises(oracle.OracleError) as e:
        oracle.recolor(off, idx, np.array([1, 1, 2, 1]), "RV", 1)
    assert e.value.code == oracle.ERR_IMPROPER_INPUT
    with pytest.raises(oracle.OracleError) as e:
        oracle.recolor(off, idx, np.array([1, 0, 1, 2]), "RV", 1)
    assert e.value.code == oracle.ERR_IMPROPER_INPUT
    out, nc = oracle.recolor(off, idx, np.array([3, 1, 3, 1]), "RV", 0)
    assert out.tolist() == [3, 1, 3, 1] and nc.tolist() == [3]
