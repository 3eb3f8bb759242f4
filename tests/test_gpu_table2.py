"""The paper's R-MAT classes (Sec. 4.1), regenerated at full size (scale 24,
edge factor 8) and checked against Table 2: edge count, maximum degree and
the colors of sequential greedy in the Natural and Largest-First orders
(oracle).  Generation runs on the GPU; the greedy runs on the host."""
import json
import os

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TABLE2 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_rmat.json")))["graphs"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("cls", ["er", "good", "bad"])
def test_regenerated_rmat_matches_table2(cls):
    want = TABLE2[cls]
    g = gg.workload(f"rmat-{cls}", device="cuda")
    off, idx = g.numpy()
    del g
    torch.cuda.empty_cache()
    assert len(off) - 1 == want["V"]
    # |E| (undirected, after dropping loops and duplicates): within 0.01 %
    assert abs(len(idx) // 2 - want["E"]) <= 1e-4 * want["E"]
    # the maximum degree and the sequential color counts: within 5 %
    assert abs(int(np.diff(off).max()) - want["max_degree"]) <= 0.05 * want["max_degree"]
    for order in ("NAT", "LF"):
        c = oracle.greedy_sequential(off, idx, order)
        assert abs(int(c.max()) - want[order]) <= max(1, 0.05 * want[order]), (order, int(c.max()))
