"""The GPU parity graphs exercise every form the speculative rounds take for
heavy rows (rows with degree + X > 64): none at all, warp-bucket rows that
keep lists of all their unfixed neighbors (no row longer than 12288
entries, when every heavy row is a warp row, or the block-bucket rows hold
under 1/16 of the entries), and marked bitmaps for both heavy buckets.  The
rule is restated here from the library's documented defaults (warp_max_deg
1024) so that a change of the test graphs cannot silently drop a form."""
import torch

import graphgen as gg

THRESHOLD_DEGREES = [0, 1, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 47, 48, 56, 57, 62, 63, 64,
                     65, 100, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 2047, 2048, 2049, 2050,
                     4000, 20000]


def _form(g, X=1, warp_max_deg=1024):
    deg = (g.offsets[1:] - g.offsets[:-1]).to(torch.int64)
    heavy = deg + X > 64
    if not bool(heavy.any()):
        return "none"
    if int(deg.max()) <= 12288:
        return "pull-all"  # every heavy row a warp row
    block_entries = int(deg[heavy & (deg > warp_max_deg)].sum())
    return "pull-near" if block_entries * 16 < g.nnz else "marks"


# One block-bucket row (degree 13,000, above the 12,288 of the warp-row form)
# among 100 warp rows: the warp rows pull and only the block row's neighbors mark.
def pull_near_graph():
    return gg.hubs([13000] + [300] * 100, 40000, seed=5)


def test_parity_graphs_cover_every_heavy_row_form():
    forms = {
        "er10k": _form(gg.workload("er10k")),
        "st27-16": _form(gg.workload("st27-16")),
        "rmat10": _form(gg.workload("rmat10")),
        "rmat12": _form(gg.workload("rmat12")),
        "rmat14": _form(gg.workload("rmat14")),
        "hubs": _form(gg.hubs(THRESHOLD_DEGREES, 30000, seed=3)),
        "pull-near": _form(pull_near_graph()),
    }
    assert set(forms.values()) == {"none", "pull-all", "pull-near", "marks"}, forms
    assert forms["rmat12"] == "pull-all"
    assert forms["pull-near"] == "pull-near"
    assert forms["hubs"] == "marks"
