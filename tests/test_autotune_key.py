"""The autotuner's cache key (host logic, no GPU): the same for the same
graph shape and settings, different when the degree histogram, the size or a
setting changes."""
import graphgen as gg
from paper_1407_6745_gb300 import autotune


def test_shape_key():
    a = gg.workload("rmat10")
    b = gg.workload("rmat10")
    k = autotune.shape_key(a.offsets, "FF", 1, "NI", 2)
    assert k == autotune.shape_key(b.offsets, "FF", 1, "NI", 2)
    others = [autotune.shape_key(a.offsets, "RXF", 1, "NI", 2),
              autotune.shape_key(a.offsets, "FF", 2, "NI", 2),
              autotune.shape_key(a.offsets, "FF", 1, "ND", 2),
              autotune.shape_key(a.offsets, "FF", 1, "NI", 3),
              autotune.shape_key(gg.workload("st27-16").offsets, "FF", 1, "NI", 2),
              autotune.shape_key(gg.workload("rmat12").offsets, "FF", 1, "NI", 2)]
    assert k not in others and len(set(others)) == len(others)
