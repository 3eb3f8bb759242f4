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
