"""Pin of the oracle's Philox4x32-10 against an independent implementation.

Every random choice of the method goes through one generator: the random
total order of the speculative rounds (Sec. 2.2), the Random-X Fit draws
(Sec. 3.2) and the RAND class shuffle (Sec. 3).  The oracle writes
Philox4x32-10 (Salmon et al., SC'11) from its definition; here it is held
against PyTorch's open-source engine (ATen/core/PhiloxRNGEngine.h,
at::Philox4_32), compiled with g++ from the header into a temporary directory
by this test.  The helper is test-only: neither the oracle nor the CUDA
library links it.

Counter layout: at::Philox4_32(seed, subsequence, offset) starts at counter
(offset_lo, offset_hi, subsequence_lo, subsequence_hi), so the oracle's
counter (a, b, c, tag) is offset = a | b << 32, subsequence = c | tag << 32.
Its first draw is word 0 of that block.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "helpers", "at_philox.cpp")
TAG_PRIO, TAG_RXF, TAG_PERM = 1, 2, 3


@pytest.fixture(scope="module")
def at_philox(tmp_path_factory):
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PyTorch's Philox header is not installed")
    so = str(tmp_path_factory.mktemp("at_philox") / "at_philox.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I" + inc, SRC,
                           "-o", so])
    lib = ctypes.CDLL(so)
    P = ctypes.c_void_p
    lib.at_philox_w0.argtypes = [P, P, ctypes.c_int64, P]
    lib.at_philox_block.argtypes = [P, ctypes.c_uint64, P]

    def w0(ctr, seeds):
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        out = np.zeros(len(ctr), dtype=np.uint32)
        lib.at_philox_w0(ctr.ctypes.data_as(P), seeds.ctypes.data_as(P), len(ctr),
                         out.ctypes.data_as(P))
        return out

    def block(ctr, seed):
        c = np.ascontiguousarray(ctr, dtype=np.uint32)
        out = np.zeros(4, dtype=np.uint32)
        lib.at_philox_block(c.ctypes.data_as(P), seed, out.ctypes.data_as(P))
        return out

    return w0, block


def _seeds(rng, m):
    # full 64-bit keys, including both halves' extremes
    s = rng.integers(0, 2**64, size=m, dtype=np.uint64)
    s[:4] = np.array([0, 1, 2**32 - 1, 2**64 - 1], dtype=np.uint64)
    return s


def test_whole_block_matches(at_philox):
    """All four output words of a block, for counters and keys with every
    word exercised (a swapped multiplier, a missed key bump or a key bump
    before the first round changes them)."""
    _, block = at_philox
    rng = np.random.default_rng(2024)
    for t in range(2000):
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        seed = int(rng.integers(0, 2**64, dtype=np.uint64))
        if t < 4:
            ctr[:] = [0, 0xFFFFFFFF, 0x12345678, 0x9ABCDEF0][t]
        want = block(ctr, seed)
        got = oracle.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert np.array_equal(got, want), (ctr.tolist(), seed)


def test_priority_layout(at_philox):
    """prio(v) = word 0 at counter (v_lo, v_hi, 0, PRIO) (Sec. 2.2)."""
    w0, _ = at_philox
    rng = np.random.default_rng(1)
    m = 4000
    seeds = _seeds(rng, m)
    vs = rng.integers(0, 2**40, size=m, dtype=np.int64)
    vs[:1000] = np.arange(1000)
    ctr = np.stack([vs & 0xFFFFFFFF, vs >> 32, np.zeros(m, np.int64), np.full(m, TAG_PRIO)], 1)
    want = w0(ctr, seeds)
    got = np.array([oracle.priority(int(s), int(v)) for s, v in zip(seeds, vs)], dtype=np.uint32)
    assert np.array_equal(got, want)


def test_random_x_fit_draw_layout(at_philox):
    """Random-X Fit draw of vertex v in round r = word 0 at counter
    (v_lo, v_hi, r, RXF) (Sec. 3.2)."""
    w0, _ = at_philox
    rng = np.random.default_rng(2)
    m = 4000
    seeds = _seeds(rng, m)
    vs = rng.integers(0, 2**36, size=m, dtype=np.int64)
    rs = rng.integers(0, 1000, size=m, dtype=np.int64)
    ctr = np.stack([vs & 0xFFFFFFFF, vs >> 32, rs, np.full(m, TAG_RXF)], 1)
    want = w0(ctr, seeds)
    got = np.array([oracle.rxf_draw(int(s), int(v), int(r)) for s, v, r in zip(seeds, vs, rs)],
                   dtype=np.uint32)
    assert np.array_equal(got, want)


def test_shuffle_draw_layout(at_philox):
    """Knuth-shuffle draw i of recoloring iteration it = word 0 at counter
    (i, it, 0, PERM) (Sec. 3, RAND)."""
    w0, _ = at_philox
    rng = np.random.default_rng(3)
    m = 4000
    seeds = _seeds(rng, m)
    i_s = rng.integers(0, 1 << 20, size=m, dtype=np.int64)
    its = rng.integers(0, 64, size=m, dtype=np.int64)
    ctr = np.stack([i_s, its, np.zeros(m, np.int64), np.full(m, TAG_PERM)], 1)
    want = w0(ctr, seeds)
    got = np.array([oracle.perm_draw(int(s), int(i), int(it)) for s, i, it in zip(seeds, i_s, its)],
                   dtype=np.uint32)
    assert np.array_equal(got, want)
