"""Sharding of independent graphs over ranks: the bin packing, and a
world-size-2 run over the gloo backend on CPU (one process per rank) in which
each rank colors its share of a batch and rank 0 gathers the results.  The
coloring inside the ranks is the oracle's (no GPU here); the point is the
host logic around it: every graph colored exactly once, by one rank, with the
result it gets when the whole batch runs in one process."""
import json
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import graphgen as gg
import oracle
from paper_1407_6745_gb300 import shard


def test_partition_covers_every_item_once_and_balances():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        for n in (0, 1, 5, 37, 200):
            w = rng.integers(1, 10_000, size=n).tolist()
            parts = shard.partition(w, world)
            assert len(parts) == world
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            if n:
                ld = shard.loads(w, parts)
                # greedy list scheduling: no rank exceeds the mean by more than one item
                assert max(ld) <= sum(w) / world + max(w)
            assert shard.partition(w, world) == parts  # deterministic


def test_partition_lpt_example():
    # heaviest first to the lightest rank: 7 -> r0, 5 -> r1, 4 -> r1 (5 < 7), 3 -> r0, 1 -> r1
    assert shard.partition([3, 7, 1, 5, 4], 2) == [[0, 1], [2, 3, 4]]
    with pytest.raises(ValueError):
        shard.partition([1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graphs():
    return gg.batch_mix(9, 11, 30, 600)


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        graphs = _graphs()
        parts = shard.partition([g.nnz for g in graphs], world)
        mine = {}
        for i in parts[rank]:
            off, idx = graphs[i].numpy()
            c, _ = oracle.color(off, idx, 3, 100 + i)
            r, _ = oracle.recolor(off, idx, c, "ND", 2, 0)
            mine[i] = r.tolist()
        slowest = shard.max_over_ranks(10.0 + rank)
        got = shard.gather({"rank": rank, "parts": parts, "colors": mine})
        if rank == 0:
            with open(out_path, "w") as f:
                json.dump({"slowest": slowest, "gathered": got}, f)
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo(tmp_path):
    out = str(tmp_path / "rank0.json")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    with open(out) as f:
        res = json.load(f)
    assert res["slowest"] == 11.0
    gathered = res["gathered"]
    assert [g["rank"] for g in gathered] == [0, 1]
    assert gathered[0]["parts"] == gathered[1]["parts"]  # the same assignment on both ranks
    colors = {}
    for g in gathered:
        for i, c in g["colors"].items():
            assert int(i) not in colors
            colors[int(i)] = c
    graphs = _graphs()
    assert sorted(colors) == list(range(len(graphs)))
    for i, g in enumerate(graphs):  # each graph as the whole batch in one process gives it
        off, idx = g.numpy()
        c, _ = oracle.color(off, idx, 3, 100 + i)
        r, _ = oracle.recolor(off, idx, c, "ND", 2, 0)
        assert colors[i] == r.tolist()


def test_single_process_fallbacks():
    assert shard.max_over_ranks(3.5) == 3.5
    assert shard.gather({"a": 1}) == [{"a": 1}]
