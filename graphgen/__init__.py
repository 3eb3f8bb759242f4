"""Seeded synthetic graph generators (input data only).

This module builds undirected simple graphs as symmetric CSR arrays
(``offsets`` int64[n+1], ``idx`` int32[nnz]) and holds none of the coloring
method's arithmetic.  It is the one module shared by the CPU oracle side
(tests, CPU baseline) and the CUDA side (tests, benchmark): every graph is
produced here once and handed to both.

Every generator is deterministic for a given (parameters, seed, device type):
the random draws come from a ``torch.Generator`` seeded with ``seed`` on the
device the graph is built on.  Large graphs are built on the GPU (sorting and
deduplicating half a billion entries is a device job); small ones on the CPU.

Workload shapes (the paper's real-world matrices are not available, so these
stand in for them): the 27-point stencil mimics the finite-element meshes of
Table 1 (average degree 15-52), R-MAT (Chakrabarti et al., Sec. 4.1) the
RMAT-ER/Good/Bad graphs of Table 2, Erdos-Renyi G(n, p) the ER class.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch


@dataclass
class CSRGraph:
    """Symmetric CSR of an undirected simple graph."""
    offsets: torch.Tensor   # int64[n+1]
    idx: torch.Tensor       # int32[nnz]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.offsets.numel()) - 1

    @property
    def nnz(self) -> int:
        return int(self.idx.numel())

    def to(self, device) -> "CSRGraph":
        return CSRGraph(self.offsets.to(device), self.idx.to(device), self.name)

    def numpy(self):
        return self.offsets.cpu().numpy(), self.idx.cpu().numpy()

    def max_degree(self) -> int:
        if self.n == 0:
            return 0
        return int((self.offsets[1:] - self.offsets[:-1]).max().item())


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def csr_from_edges(n: int, src: torch.Tensor, dst: torch.Tensor, *, symmetrize: bool = True,
                   name: str = "") -> CSRGraph:
    """CSR from an edge list: drops self-loops, optionally adds reversed
    edges, removes duplicates, sorts every row by neighbor id."""
    device = src.device
    src = src.to(torch.int64)
    dst = dst.to(torch.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    if symmetrize:
        src, dst = torch.cat([src, dst]), torch.cat([dst, src])
    key = src * n + dst
    del src, dst
    key = torch.unique(key, sorted=True)
    row = torch.div(key, n, rounding_mode="floor")
    idx = (key - row * n).to(torch.int32)
    del key
    counts = torch.bincount(row, minlength=n)
    del row
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=offsets[1:])
    return CSRGraph(offsets, idx, name)


def relabel(g: CSRGraph, perm: torch.Tensor, name: str | None = None) -> CSRGraph:
    """Rename vertex v to perm[v] and rebuild sorted rows."""
    n = g.n
    device = g.offsets.device
    deg = g.offsets[1:] - g.offsets[:-1]
    src = torch.repeat_interleave(torch.arange(n, device=device), deg)
    perm = perm.to(device)
    return csr_from_edges(n, perm[src], perm[g.idx.to(torch.int64)], symmetrize=False,
                          name=name if name is not None else g.name)


def shuffle_ids(g: CSRGraph, seed: int) -> CSRGraph:
    perm = torch.randperm(g.n, generator=_gen(seed, g.offsets.device), device=g.offsets.device)
    return relabel(g, perm, name=g.name + f"-shuffled{seed}")


# ---------------------------------------------------------------------------
# Erdos-Renyi G(n, p) by geometric skipping over the n(n-1)/2 vertex pairs
# ---------------------------------------------------------------------------

def _pair_from_index(k: torch.Tensor, n: int):
    """Strict upper-triangle pair (i, j), i < j, of row-major index k."""
    kf = k.to(torch.float64)
    b = 2.0 * n - 1.0
    i = torch.floor((b - torch.sqrt(torch.clamp(b * b - 8.0 * kf, min=0.0))) / 2.0).to(torch.int64)
    i = torch.clamp(i, 0, n - 2)

    def row_start(r):
        return r * (2 * n - r - 1) // 2
    for _ in range(3):  # exact integer correction of the float estimate
        i = torch.where(row_start(i + 1) <= k, i + 1, i)
        i = torch.where(row_start(i) > k, i - 1, i)
    j = k - row_start(i) + i + 1
    return i, j


def erdos_renyi(n: int, mean_degree: float, seed: int, device="cpu") -> CSRGraph:
    """G(n, p) with p = mean_degree / (n - 1): every pair is an edge
    independently with probability p."""
    name = f"er-n{n}-d{mean_degree:g}-s{seed}"
    if n < 2:
        return CSRGraph(torch.zeros(n + 1, dtype=torch.int64, device=device),
                        torch.zeros(0, dtype=torch.int32, device=device), name)
    p = min(1.0, mean_degree / (n - 1))
    total = n * (n - 1) // 2
    g = _gen(seed, device)
    if p <= 0.0:
        return csr_from_edges(n, torch.zeros(0, dtype=torch.int64, device=device),
                              torch.zeros(0, dtype=torch.int64, device=device), name=name)
    expected = total * p
    chunk = int(expected + 6.0 * math.sqrt(expected) + 1024)
    picks = []
    base = torch.full((1,), -1, dtype=torch.int64, device=device)
    while True:
        gaps = torch.empty(chunk, dtype=torch.float64, device=device).geometric_(p, generator=g)
        pos = base + torch.cumsum(gaps.to(torch.int64), 0)
        inside = pos < total
        picks.append(pos[inside])
        if not bool(inside.all()):
            break
        base = pos[-1:].clone()
    k = torch.cat(picks)
    i, j = _pair_from_index(k, n)
    return csr_from_edges(n, i, j, symmetrize=True, name=name)


# ---------------------------------------------------------------------------
# Structured meshes
# ---------------------------------------------------------------------------

def stencil_3d(side_x: int, side_y: int, side_z: int, points: int = 27, device="cpu") -> CSRGraph:
    """3D box mesh with the 7-point (faces) or 27-point (faces, edges,
    corners) neighborhood; vertex (x, y, z) has id x + X (y + Y z)."""
    assert points in (7, 27)
    X, Y, Z = side_x, side_y, side_z
    n = X * Y * Z
    ids = torch.arange(n, dtype=torch.int64, device=device)
    x = ids % X
    y = (ids // X) % Y
    z = ids // (X * Y)
    srcs, dsts = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == dy == dz == 0:
                    continue
                if points == 7 and abs(dx) + abs(dy) + abs(dz) != 1:
                    continue
                ok = ((x + dx >= 0) & (x + dx < X) & (y + dy >= 0) & (y + dy < Y)
                      & (z + dz >= 0) & (z + dz < Z))
                s = ids[ok]
                srcs.append(s)
                dsts.append(s + dx + X * (dy + Y * dz))
    return csr_from_edges(n, torch.cat(srcs), torch.cat(dsts), symmetrize=False,
                          name=f"stencil{points}-{X}x{Y}x{Z}")


def grid_2d(side_x: int, side_y: int, device="cpu") -> CSRGraph:
    """2D 5-point grid."""
    g = stencil_3d(side_x, side_y, 1, points=7, device=device)
    g.name = f"grid5-{side_x}x{side_y}"
    return g


# ---------------------------------------------------------------------------
# R-MAT (Chakrabarti, Zhan, Faloutsos)
# ---------------------------------------------------------------------------

def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         device="cpu", chunk: int = 1 << 25) -> CSRGraph:
    """R-MAT with 2^scale vertices and edge_factor * 2^scale generated edges:
    at every level of the recursion each edge falls in one of the four
    quadrants with probabilities (a, b, c, d = 1 - a - b - c).  No noise,
    natural ids; self-loops dropped, symmetrized, deduplicated."""
    n = 1 << scale
    m = edge_factor * n
    g = _gen(seed, device)
    ab = a + b
    a_ab = a / ab
    c_cd = c / (1.0 - ab)
    srcs, dsts = [], []
    for start in range(0, m, chunk):
        cnt = min(chunk, m - start)
        u = torch.zeros(cnt, dtype=torch.int64, device=device)
        v = torch.zeros(cnt, dtype=torch.int64, device=device)
        for level in range(scale):
            r1 = torch.rand(cnt, generator=g, device=device, dtype=torch.float32)
            r2 = torch.rand(cnt, generator=g, device=device, dtype=torch.float32)
            down = r1 >= ab                                   # lower half: c or d
            right = torch.where(down, r2 >= c_cd, r2 >= a_ab)  # right half: b or d
            bit = 1 << (scale - 1 - level)
            u += down.to(torch.int64) * bit
            v += right.to(torch.int64) * bit
        srcs.append(u)
        dsts.append(v)
    return csr_from_edges(n, torch.cat(srcs), torch.cat(dsts), symmetrize=True,
                          name=f"rmat-s{scale}-ef{edge_factor}-{a:g},{b:g},{c:g}-s{seed}")


# ---------------------------------------------------------------------------
# Small named graphs (tests and edge cases)
# ---------------------------------------------------------------------------

def from_edge_list(n: int, edges, name: str = "") -> CSRGraph:
    if len(edges) == 0:
        e = torch.zeros((0, 2), dtype=torch.int64)
    else:
        e = torch.tensor(edges, dtype=torch.int64)
    return csr_from_edges(n, e[:, 0], e[:, 1], symmetrize=True, name=name)


def complete(n: int) -> CSRGraph:
    return from_edge_list(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def cycle(n: int) -> CSRGraph:
    return from_edge_list(n, [(i, (i + 1) % n) for i in range(n)], f"C{n}")


def path(n: int) -> CSRGraph:
    return from_edge_list(n, [(i, i + 1) for i in range(n - 1)], f"P{n}")


def star(leaves: int) -> CSRGraph:
    return from_edge_list(leaves + 1, [(0, i) for i in range(1, leaves + 1)], f"star{leaves}")


def empty(n: int) -> CSRGraph:
    return from_edge_list(n, [], f"empty{n}")


def complete_bipartite(p: int, q: int) -> CSRGraph:
    return from_edge_list(p + q, [(i, p + j) for i in range(p) for j in range(q)], f"K{p},{q}")


def random_small(n: int, p: float, seed: int) -> CSRGraph:
    """Tiny G(n, p) drawn pair by pair (for brute-force checks)."""
    rng = np.random.default_rng(seed)
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    return from_edge_list(n, edges, f"small-n{n}-p{p:g}-s{seed}")


def hubs(degrees, base_n: int, seed: int, device="cpu") -> CSRGraph:
    """Graph whose first len(degrees) vertices have exactly the given degrees
    (distinct random neighbors among the other base_n vertices), plus a sparse
    random background among those base_n vertices.  Used to put vertices
    exactly on every scheduling threshold."""
    rng = np.random.default_rng(seed)
    h = len(degrees)
    n = h + base_n
    src, dst = [], []
    for i, d in enumerate(degrees):
        d = min(int(d), base_n)
        nb = rng.choice(base_n, size=d, replace=False) + h
        src.append(np.full(d, i, dtype=np.int64))
        dst.append(nb.astype(np.int64))
    m = 2 * base_n
    src.append(rng.integers(h, n, size=m))
    dst.append(rng.integers(h, n, size=m))
    s = torch.from_numpy(np.concatenate(src)).to(device)
    t = torch.from_numpy(np.concatenate(dst)).to(device)
    # hub-to-hub edges would change the hubs' degrees: the background avoids
    # ids < h, and hub neighbors are all >= h, so every hub keeps its degree.
    return csr_from_edges(n, s, t, symmetrize=True, name=f"hubs-{len(degrees)}-s{seed}")


# ---------------------------------------------------------------------------
# Batches of graphs
# ---------------------------------------------------------------------------

def batch_union(graphs, device=None) -> CSRGraph:
    """Disjoint union of graphs as one CSR: graph i's vertices follow graph
    i-1's, ids shifted accordingly."""
    device = device if device is not None else graphs[0].offsets.device
    offs, idxs = [torch.zeros(1, dtype=torch.int64, device=device)], []
    vbase, ebase = 0, 0
    for g in graphs:
        offs.append(g.offsets[1:].to(device) + ebase)
        idxs.append((g.idx.to(device).to(torch.int64) + vbase).to(torch.int32))
        vbase += g.n
        ebase += g.nnz
    return CSRGraph(torch.cat(offs), torch.cat(idxs) if idxs else torch.zeros(0, dtype=torch.int32),
                    f"batch{len(graphs)}")


def batch_mix_plan(count: int, seed: int, n_lo: float, n_hi: float):
    """The graphs of batch_mix as specifications, with their expected
    adjacency entries (to place them before building them): a list of
    (kind, size parameter, mean degree or None, generator seed, est. entries)."""
    rng = np.random.default_rng(seed)
    plan = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        if i % 2 == 0:
            n = max(n, 2)
            d = float(rng.uniform(8.0, 32.0))
            plan.append(("er", n, d, seed * 100003 + i, int(n * d)))
        elif rng.random() < 0.5:
            side = max(2, int(round(math.sqrt(n))))
            plan.append(("grid2d", side, None, 0, 4 * side * side))
        else:
            side = max(2, int(round(n ** (1.0 / 3.0))))
            plan.append(("st7", side, None, 0, 6 * side ** 3))
    return plan


def build_planned(spec, device="cpu") -> CSRGraph:
    kind, size, d, gseed, _ = spec
    if kind == "er":
        return erdos_renyi(size, d, seed=gseed, device=device)
    if kind == "grid2d":
        return grid_2d(size, size, device=device)
    return stencil_3d(size, size, size, points=7, device=device)


def batch_mix(count: int, seed: int, n_lo: float, n_hi: float, device="cpu", only=None):
    """The batch workload: `count` graphs, half G(n, p) with mean degree drawn
    from U[8, 32], half 2D 5-point or 3D 7-point grids; n log-uniform in
    [n_lo, n_hi].  Returns the graphs (each with its own ids); with `only`,
    just the graphs of those indices (in that order), the same as in the
    full list."""
    plan = batch_mix_plan(count, seed, n_lo, n_hi)
    pick = range(count) if only is None else only
    return [build_planned(plan[i], device) for i in pick]


# ---------------------------------------------------------------------------
# The benchmark workloads
# ---------------------------------------------------------------------------

# The (a, b, c) quadrant probabilities of the paper's R-MAT graphs (Sec. 4.1).
PAPER_RMAT = {"er": (0.25, 0.25, 0.25), "good": (0.45, 0.15, 0.15), "bad": (0.55, 0.15, 0.15)}


def workload(name: str, device="cpu") -> CSRGraph:
    """The named synthetic workloads:
    er10k    -- G(n=10,000, mean degree 16), seed 1
    st27-128 -- 27-point stencil 128^3, ids shuffled by a seed-2 permutation
    rmat24   -- R-MAT scale 24, edge factor 16, (0.57, 0.19, 0.19, 0.05), seed 4
    rmat-er / rmat-good / rmat-bad -- the R-MAT classes of Sec. 4.1 (Table 2):
                (0.25, 0.25, 0.25, 0.25), (0.45, 0.15, 0.15, 0.25) and
                (0.55, 0.15, 0.15, 0.15), scale 24, edge factor 8, seed 4
    Smaller variants for tests: st27-<side>, rmat<scale>, rmat-er<scale>, ..."""
    if name == "er10k":
        return erdos_renyi(10_000, 16.0, seed=1, device=device)
    if name.startswith("st27-"):
        s = int(name.split("-")[1])
        return shuffle_ids(stencil_3d(s, s, s, 27, device=device), seed=2)
    for cls, (a, b, c) in PAPER_RMAT.items():
        if name.startswith(f"rmat-{cls}"):
            rest = name[len(f"rmat-{cls}"):]
            return rmat(int(rest) if rest else 24, 8, a, b, c, seed=4, device=device)
    if name.startswith("rmat"):
        scale = int(name[4:])
        return rmat(scale, 16, 0.57, 0.19, 0.19, seed=4, device=device)
    raise KeyError(name)
