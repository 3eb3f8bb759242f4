"""CPU oracle for speculative graph coloring with iterative recoloring.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The product library never
imports, links or calls anything here, and this package imports nothing from
the product package.

The arithmetic lives in ``gc_oracle.c`` (plain single-threaded C, compiled
with gcc into ``liboracle.so`` next to it); this module only marshals numpy
arrays.  Passages followed: Alg. 1 and First Fit (Sec. 2.1), the speculative
rounds of Sec. 2.2, Random-X Fit (Sec. 3.2), recoloring and the class
permutations RV/NI/ND/RAND (Sec. 2.1, Sec. 3) and their ND-RAND schedules
(Sec. 4.2.1), Largest-First priorities (Sec. 2.2.1) and asynchronous
recoloring (aRC, Sec. 3).  The readings taken where the
paper is silent are listed at the top of ``gc_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_BAD_GRAPH, ERR_IMPROPER_INPUT, ERR_OOM = 0, 1, 2, 3, 4
ERR_ROUND_LIMIT = 7
PERM_REVERSE, PERM_NONINC, PERM_NONDEC, PERM_RANDOM = 0, 1, 2, 3
PERMS = {"RV": PERM_REVERSE, "NI": PERM_NONINC, "ND": PERM_NONDEC, "RAND": PERM_RANDOM}
SCHED_POW2, SCHED_EVERY_BASE = 4, 256


def perm_code(perm) -> int:
    """A permutation name (RV, NI, ND, RAND) or schedule name (ND-RAND%x,
    ND-RAND%2^i; Sec. 4.2.1) as the oracle's integer code; ints pass through."""
    if not isinstance(perm, str):
        return int(perm)
    p = perm.upper()
    if p in PERMS:
        return PERMS[p]
    if p == "ND-RAND%2^I":
        return SCHED_POW2
    if p.startswith("ND-RAND%"):
        return SCHED_EVERY_BASE + int(p[len("ND-RAND%"):])
    raise KeyError(perm)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


class ColorStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("max_color", ctypes.c_int32),
                ("edges_examined", ctypes.c_int64), ("conflicts", ctypes.c_int64)]


class Validation(ctypes.Structure):
    _fields_ = [("n_conflicts", ctypes.c_int64), ("n_uncolored", ctypes.c_int64),
                ("max_color", ctypes.c_int32), ("n_distinct", ctypes.c_int32),
                ("first_bad_vertex", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile gc_oracle.c with gcc (plain -O2, no vector or arch flags)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC",
                                   _SRC, "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.oracle_philox4x32_10.argtypes = [P, P, P]
        lib.oracle_priority.argtypes = [ctypes.c_uint64, ctypes.c_int64]
        lib.oracle_priority.restype = ctypes.c_uint32
        lib.oracle_rxf_draw.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32]
        lib.oracle_rxf_draw.restype = ctypes.c_uint32
        lib.oracle_perm_draw.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32]
        lib.oracle_perm_draw.restype = ctypes.c_uint32
        lib.oracle_color.argtypes = [ctypes.c_int64, P, P, ctypes.c_int32, ctypes.c_uint64,
                                     P, ctypes.POINTER(ColorStats)]
        lib.oracle_color_tables.argtypes = [ctypes.c_int64, P, P, ctypes.c_int32, P, P,
                                            ctypes.c_int32, P, ctypes.POINTER(ColorStats)]
        lib.oracle_validate.argtypes = [ctypes.c_int64, P, P, P, ctypes.POINTER(Validation)]
        lib.oracle_class_order.argtypes = [ctypes.c_int32, P, ctypes.c_int32, ctypes.c_uint64,
                                           ctypes.c_int32, P, P]
        lib.oracle_class_order.restype = ctypes.c_int32
        lib.oracle_recolor.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_uint64, P, P]
        lib.oracle_color_lf.argtypes = [ctypes.c_int64, P, P, ctypes.c_int32, ctypes.c_uint64,
                                        P, ctypes.POINTER(ColorStats)]
        lib.oracle_color_lf.restype = ctypes.c_int
        lib.oracle_recolor_async.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_uint64, P, P, P]
        lib.oracle_recolor_async.restype = ctypes.c_int
        lib.oracle_ordered_priority.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64]
        lib.oracle_ordered_priority.restype = ctypes.c_uint32
        lib.oracle_greedy_sequential.argtypes = [ctypes.c_int64, P, P, ctypes.c_int32, P]
        lib.oracle_greedy_sequential.restype = ctypes.c_int
        lib.oracle_perm_of_iteration.argtypes = [ctypes.c_int32, ctypes.c_int32]
        lib.oracle_perm_of_iteration.restype = ctypes.c_int32
        for f in (lib.oracle_color, lib.oracle_color_tables, lib.oracle_validate,
                  lib.oracle_recolor):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _graph(off, idx):
    off = np.ascontiguousarray(off, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    return off, idx, len(off) - 1


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ctr = 4 uint32 words, key = 2 uint32 words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def priority(seed: int, v: int) -> int:
    return int(_load().oracle_priority(seed, v))


def rxf_draw(seed: int, v: int, r: int) -> int:
    return int(_load().oracle_rxf_draw(seed, v, r))


def perm_draw(seed: int, i: int, it: int) -> int:
    return int(_load().oracle_perm_draw(seed, i, it))


def perm_of_iteration(perm, it: int) -> int:
    """The permutation (0..3) recoloring iteration `it` (0-based) uses under a
    permutation or schedule; -1 for an unknown code."""
    return int(_load().oracle_perm_of_iteration(perm_code(perm), it))


def color(off, idx, X: int = 1, seed: int = 0):
    """Speculative coloring to convergence; X = 1 is First Fit, X > 1 is
    Random-X Fit.  Returns (colors int32[n], stats dict)."""
    lib = _load()
    off, idx, n = _graph(off, idx)
    out = np.zeros(n, dtype=np.int32)
    st = ColorStats()
    rc = lib.oracle_color(n, _ptr(off), _ptr(idx), X, seed, _ptr(out), ctypes.byref(st))
    if rc != OK:
        raise OracleError(rc, "color")
    return out, {"rounds": st.rounds, "max_color": st.max_color,
                 "edges_examined": st.edges_examined, "conflicts": st.conflicts}


def color_tables(off, idx, X, prio, draws=None):
    """Speculative rounds with explicit priorities (uint32[n]) and draws
    (uint32[rounds, n], row r used in round r)."""
    lib = _load()
    off, idx, n = _graph(off, idx)
    prio = np.ascontiguousarray(prio, dtype=np.uint32)
    rounds = 0
    if draws is not None:
        draws = np.ascontiguousarray(draws, dtype=np.uint32)
        rounds = draws.shape[0]
    out = np.zeros(n, dtype=np.int32)
    st = ColorStats()
    rc = lib.oracle_color_tables(n, _ptr(off), _ptr(idx), X, _ptr(prio), _ptr(draws), rounds,
                                 _ptr(out), ctypes.byref(st))
    if rc != OK:
        raise OracleError(rc, "color_tables")
    return out, {"rounds": st.rounds, "max_color": st.max_color,
                 "edges_examined": st.edges_examined, "conflicts": st.conflicts}


def validate(off, idx, colors):
    lib = _load()
    off, idx, n = _graph(off, idx)
    colors = np.ascontiguousarray(colors, dtype=np.int32)
    v = Validation()
    rc = lib.oracle_validate(n, _ptr(off), _ptr(idx), _ptr(colors), ctypes.byref(v))
    if rc != OK:
        raise OracleError(rc, "validate")
    return {"n_conflicts": v.n_conflicts, "n_uncolored": v.n_uncolored,
            "max_color": v.max_color, "n_distinct": v.n_distinct,
            "first_bad_vertex": v.first_bad_vertex}


def class_order(sizes, perm, seed: int = 0, iteration: int = 0, draws=None):
    """Order in which the present classes are recolored.  sizes[c] is the size
    of class c (index 0 unused)."""
    lib = _load()
    sizes = np.ascontiguousarray(sizes, dtype=np.int64)
    maxc = len(sizes) - 1
    order = np.zeros(max(maxc, 1), dtype=np.int32)
    if draws is not None:
        draws = np.ascontiguousarray(draws, dtype=np.uint32)
    k = lib.oracle_class_order(maxc, _ptr(sizes), PERMS.get(perm, perm), seed, iteration,
                               _ptr(draws), _ptr(order))
    if k < 0:
        raise OracleError(k, "class_order")
    return order[:k].copy()


def ordered_priority(first_key: int, seed: int, v: int) -> int:
    """Conflict priority with a vertex-visit key first (LF degree, aRC rank)."""
    return int(_load().oracle_ordered_priority(first_key, seed, v))


def color_lf(off, idx, X: int = 1, seed: int = 0):
    """Speculative coloring where the larger degree wins a conflict (Largest
    First, Sec. 2.2.1).  Returns (colors, stats) as color()."""
    lib = _load()
    off, idx, n = _graph(off, idx)
    out = np.zeros(n, dtype=np.int32)
    st = ColorStats()
    rc = lib.oracle_color_lf(n, _ptr(off), _ptr(idx), X, seed, _ptr(out), ctypes.byref(st))
    if rc != OK:
        raise OracleError(rc, "color_lf")
    return out, {"rounds": st.rounds, "max_color": st.max_color,
                 "edges_examined": st.edges_examined, "conflicts": st.conflicts}


def recolor_async(off, idx, colors_in, perm="RV", iterations: int = 1, seed: int = 0):
    """Asynchronous recoloring (aRC, Sec. 3).  Returns (colors,
    ncolors int32[iterations+1], rounds int32[iterations])."""
    lib = _load()
    off, idx, n = _graph(off, idx)
    cin = np.ascontiguousarray(colors_in, dtype=np.int32)
    out = np.zeros(n, dtype=np.int32)
    nc = np.zeros(iterations + 1, dtype=np.int32)
    rounds = np.zeros(max(iterations, 1), dtype=np.int32)
    rc = lib.oracle_recolor_async(n, _ptr(off), _ptr(idx), _ptr(cin), perm_code(perm), iterations,
                                  seed, _ptr(out), _ptr(nc), _ptr(rounds))
    if rc != OK:
        raise OracleError(rc, "recolor_async")
    return out, nc, rounds[:iterations]


def greedy_sequential(off, idx, order="NAT"):
    """Sequential Alg. 1 in the Natural ("NAT", id) or Largest-First ("LF",
    non-increasing degree, ties by id) vertex-visit order."""
    lib = _load()
    off, idx, n = _graph(off, idx)
    out = np.zeros(n, dtype=np.int32)
    rc = lib.oracle_greedy_sequential(n, _ptr(off), _ptr(idx), {"NAT": 0, "LF": 1}[order.upper()], _ptr(out))
    if rc != OK:
        raise OracleError(rc, "greedy_sequential")
    return out


def recolor(off, idx, colors_in, perm="RV", iterations: int = 1, seed: int = 0):
    """Iterative recoloring; returns (colors int32[n], ncolors int32[iterations+1])."""
    lib = _load()
    off, idx, n = _graph(off, idx)
    cin = np.ascontiguousarray(colors_in, dtype=np.int32)
    out = np.zeros(n, dtype=np.int32)
    nc = np.zeros(iterations + 1, dtype=np.int32)
    rc = lib.oracle_recolor(n, _ptr(off), _ptr(idx), _ptr(cin), perm_code(perm),
                            iterations, seed, _ptr(out), _ptr(nc))
    if rc != OK:
        raise OracleError(rc, "recolor")
    return out, nc
