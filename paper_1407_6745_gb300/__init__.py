"""GB300 speculative distance-1 graph coloring with iterative recoloring.

Thin Python binding of the C ABI in ``include/gc.h`` (``libgc.so``).  The
functions carry the C names and only marshal arguments: every step of the
method runs in the library's CUDA kernels.  Graph and color arrays are torch
tensors; CUDA tensors are passed as device pointers (``GC_MEM_DEVICE``, on the
current torch stream), CPU tensors as host pointers (``GC_MEM_HOST``: the
library copies them to the GPU and back).

There is no CPU fallback: if ``libgc.so`` has not been built (``python -m
paper_1407_6745_gb300.build``) every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

__all__ = [
    "GCError", "FIRST_FIT", "RANDOM_X_FIT", "PERM", "library_path", "load",
    "gc_color", "gc_recolor", "gc_color_recolor", "gc_color_batch", "gc_recolor_batch",
    "gc_color_recolor_batch", "gc_validate", "gc_validate_noalloc",
    "gc_check_graph", "gc_server_create", "gc_server_submit", "gc_server_poll", "gc_server_wait",
    "gc_server_stats", "gc_server_destroy",
    "gc_priorities", "gc_set_tuning", "gc_get_tuning", "gc_profile_enable", "gc_profile_read",
    "gc_kernel_launches", "gc_status_string", "gc_version", "gc_preset_params",
    "gc_color_ordered", "gc_recolor_async", "gc_inject_alloc_failure",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libgc.so")
_lock = threading.Lock()
_lib = None

FIRST_FIT, RANDOM_X_FIT = 0, 1
PERM = {"RV": 0, "NI": 1, "ND": 2, "RAND": 3}
GC_MEM_DEVICE, GC_MEM_HOST = 0, 1
STATUS = {0: "GC_OK", 1: "GC_ERR_INVALID_ARG", 2: "GC_ERR_BAD_GRAPH", 3: "GC_ERR_IMPROPER_INPUT",
          4: "GC_ERR_OOM", 5: "GC_ERR_CUDA", 6: "GC_ERR_TIMEOUT", 7: "GC_ERR_ROUND_LIMIT",
          8: "GC_ERR_BUDGET", 9: "GC_PENDING"}


class GCError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__(f"{where}: {self.name} ({gc_status_string(code)})")


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("mem", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("max_color", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("edges_examined", ctypes.c_int64), ("conflicts", ctypes.c_int64),
                ("ms_color", ctypes.c_float), ("ms_recolor", ctypes.c_float)]


class _Validation(ctypes.Structure):
    _fields_ = [("n_conflicts", ctypes.c_int64), ("n_uncolored", ctypes.c_int64),
                ("max_color", ctypes.c_int32), ("n_distinct", ctypes.c_int32),
                ("first_bad_vertex", ctypes.c_int64)]


class _BatchGraph(ctypes.Structure):
    _fields_ = [("vertex_base", ctypes.c_int64), ("n", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("X", ctypes.c_int32), ("perm", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("perm_seed", ctypes.c_uint64)]


class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


class _Tuning(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("g4_max_deg", "g8_max_deg", "g16_max_deg",
                                               "warp_max_deg", "grid_blocks", "recolor_mode",
                                               "spin_limit", "spec_graph", "rc_warp_max_deg",
                                               "g2_max_deg", "rc_g2_max_deg")]


class _PlanInfo(ctypes.Structure):
    _fields_ = [("tuning", _Tuning), ("strategy", ctypes.c_int32), ("X", ctypes.c_int32),
                ("perm", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("tuned_ms", ctypes.c_float), ("tuned_n", ctypes.c_int64),
                ("tuned_nnz", ctypes.c_int64)]


class _Request(ctypes.Structure):
    _fields_ = [("graph", _Graph), ("strategy", ctypes.c_int32), ("X", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("perm", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("perm_seed", ctypes.c_uint64)]


class _RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("rounds", ctypes.c_int32), ("max_color", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("submit_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


class _ServerInfo(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("graphs_per_s", ctypes.c_double), ("bytes_in_use", ctypes.c_int64),
                ("bytes_peak", ctypes.c_int64)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libgc.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing; build it with "
                               "`python -m paper_1407_6745_gb300.build`")
        lib = ctypes.CDLL(_LIB_PATH)
        P, G = ctypes.c_void_p, ctypes.POINTER(_Graph)
        S = ctypes.POINTER(_Stats)
        lib.gc_color.argtypes = [G, ctypes.c_int, ctypes.c_int32, ctypes.c_uint64, P, S, P]
        lib.gc_recolor.argtypes = [G, P, ctypes.c_int, ctypes.c_int32, ctypes.c_uint64, P, P, S, P]
        lib.gc_color_recolor.argtypes = [G, ctypes.c_int, ctypes.c_int32, ctypes.c_uint64,
                                         ctypes.c_int, ctypes.c_int32, ctypes.c_uint64, P, P, S,
                                         ctypes.POINTER(_Validation), P]
        lib.gc_validate.argtypes = [G, P, ctypes.POINTER(_Validation), P]
        lib.gc_validate_noalloc.argtypes = [G, P, ctypes.POINTER(_Validation), P]
        lib.gc_validate_noalloc.restype = ctypes.c_int
        lib.gc_check_graph.argtypes = [G, ctypes.POINTER(ctypes.c_int64), P]
        B = ctypes.POINTER(_BatchGraph)
        lib.gc_color_batch.argtypes = [G, B, ctypes.c_int32, P, P, P, S, P]
        lib.gc_recolor_batch.argtypes = [G, B, ctypes.c_int32, P, P, P, S, P]
        lib.gc_color_recolor_batch.argtypes = [G, B, ctypes.c_int32, P, P, P, S, P]
        for f in ("gc_color_batch", "gc_recolor_batch", "gc_color_recolor_batch"):
            getattr(lib, f).restype = ctypes.c_int
        lib.gc_priorities.argtypes = [ctypes.c_uint64, ctypes.c_int64, P, P]
        lib.gc_priorities.restype = ctypes.c_int
        lib.gc_set_tuning.argtypes = [ctypes.POINTER(_Tuning)]
        lib.gc_get_tuning.argtypes = [ctypes.POINTER(_Tuning)]
        H = ctypes.c_void_p
        lib.gc_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(H)]
        lib.gc_server_submit.argtypes = [H, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]
        lib.gc_server_poll.argtypes = [H, ctypes.c_uint64, P, ctypes.POINTER(_RequestResult)]
        lib.gc_server_wait.argtypes = [H, ctypes.c_uint64, P, ctypes.POINTER(_RequestResult),
                                       ctypes.c_int32]
        lib.gc_server_stats.argtypes = [H, ctypes.POINTER(_ServerInfo)]
        lib.gc_color_ordered.argtypes = [G, ctypes.c_int, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int,
                                         P, S, P]
        lib.gc_recolor_async.argtypes = [G, P, ctypes.c_int, ctypes.c_int32, ctypes.c_uint64, P, P, S, P]
        for f in ("gc_color_ordered", "gc_recolor_async"):
            getattr(lib, f).restype = ctypes.c_int
        lib.gc_inject_alloc_failure.argtypes = [ctypes.c_int64]
        lib.gc_inject_alloc_failure.restype = None
        lib.gc_preset_params.argtypes = [ctypes.c_int, P, P, P, P]
        lib.gc_preset_params.restype = ctypes.c_int
        lib.gc_server_destroy.argtypes = [H]
        lib.gc_server_destroy.restype = None
        T = ctypes.POINTER(_Tuning)
        lib.gc_autotune.argtypes = [G, ctypes.c_int, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int,
                                    ctypes.c_int32, ctypes.c_int32, T,
                                    ctypes.POINTER(ctypes.c_float), P]
        lib.gc_plan_create.argtypes = [T, ctypes.c_int, ctypes.c_int32, ctypes.c_int, ctypes.c_int32,
                                       ctypes.POINTER(H)]
        lib.gc_plan_autotune.argtypes = [G, ctypes.c_int, ctypes.c_int32, ctypes.c_uint64,
                                         ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(H), P]
        lib.gc_plan_get_info.argtypes = [H, ctypes.POINTER(_PlanInfo)]
        lib.gc_plan_color_recolor.argtypes = [H, G, ctypes.c_uint64, ctypes.c_uint64, P, P, S,
                                              ctypes.POINTER(_Validation), P]
        for f in ("gc_autotune", "gc_plan_create", "gc_plan_autotune", "gc_plan_get_info",
                  "gc_plan_color_recolor"):
            getattr(lib, f).restype = ctypes.c_int
        lib.gc_plan_free.argtypes = [H]
        lib.gc_plan_free.restype = None
        for f in ("gc_color", "gc_recolor", "gc_color_recolor", "gc_validate", "gc_validate_noalloc",
                  "gc_check_graph", "gc_priorities", "gc_set_tuning", "gc_get_tuning",
                  "gc_server_create", "gc_server_submit", "gc_server_poll", "gc_server_wait",
                  "gc_server_stats"):
            getattr(lib, f).restype = ctypes.c_int
        lib.gc_kernel_launches.restype = ctypes.c_int64
        lib.gc_profile_enable.argtypes = [ctypes.c_int32]
        lib.gc_profile_read.argtypes = [ctypes.POINTER(_KernelTime), ctypes.c_int32]
        lib.gc_profile_read.restype = ctypes.c_int32
        lib.gc_status_string.argtypes = [ctypes.c_int]
        lib.gc_status_string.restype = ctypes.c_char_p
        lib.gc_version.restype = ctypes.c_int32
        _lib = lib
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise GCError(rc, where)


def _ptr(t):
    return None if t is None or t.numel() == 0 else ctypes.c_void_p(t.data_ptr())


def _graph(offsets: torch.Tensor, idx: torch.Tensor):
    if offsets.dtype != torch.int64 or idx.dtype != torch.int32:
        raise TypeError("offsets must be int64 and idx int32")
    if offsets.device != idx.device:
        raise ValueError("offsets and idx must be on the same device")
    offsets = offsets.contiguous()
    idx = idx.contiguous()
    g = _Graph()
    g.n = offsets.numel() - 1
    g.nnz = idx.numel()
    g.offsets = _ptr(offsets)
    g.idx = _ptr(idx)
    g.mem = GC_MEM_DEVICE if offsets.is_cuda else GC_MEM_HOST
    return g, (offsets, idx)


def _stream(device: torch.device, stream):
    if device.type != "cuda":
        return None
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _stats_dict(st: _Stats):
    return {k: getattr(st, k) for k, _ in _Stats._fields_ if k != "reserved"}


def _strategy(s):
    if isinstance(s, str):
        return {"FF": FIRST_FIT, "RXF": RANDOM_X_FIT}[s.upper()]
    return int(s)


PERM_ND_RAND_POW2 = 4


def PERM_ND_RAND_EVERY(x: int) -> int:
    """gc_perm code of the ND-RAND%x schedule (Sec. 4.2.1)."""
    return 256 + int(x)


def _perm(p):
    """A gc_perm code from RV/NI/ND/RAND, ND-RAND%x or ND-RAND%2^i (ints pass through)."""
    if not isinstance(p, str):
        return int(p)
    u = p.upper()
    if u in PERM:
        return PERM[u]
    if u == "ND-RAND%2^I":
        return PERM_ND_RAND_POW2
    if u.startswith("ND-RAND%"):
        return PERM_ND_RAND_EVERY(int(u[len("ND-RAND%"):]))
    raise KeyError(p)


def _check_colors(t: torch.Tensor, n: int, device, name: str):
    if t.dtype != torch.int32 or t.numel() != n or t.device != device or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous int32 tensor of {n} entries on {device}")


def gc_color(offsets, idx, strategy="FF", X: int = 1, seed: int = 0, out=None, stream=None):
    """Speculative coloring (Sec. 2.2 rounds; First Fit or Random-X Fit).
    Returns (colors int32[n], stats dict)."""
    lib = load()
    g, keep = _graph(offsets, idx)
    dev = keep[0].device
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
    _check_colors(out, g.n, dev, "out")
    st = _Stats()
    _check(lib.gc_color(ctypes.byref(g), _strategy(strategy), int(X), int(seed) & (2**64 - 1),
                        _ptr(out), ctypes.byref(st), _stream(dev, stream)), "gc_color")
    return out, _stats_dict(st)


ORDER = {"RANDOM": 0, "LF": 1, "LARGEST_FIRST": 1}


def gc_color_ordered(offsets, idx, strategy="FF", X: int = 1, seed: int = 0, order="LF", out=None,
                     stream=None):
    """Speculative coloring with a vertex-visit order as the conflict priority
    (Sec. 2.2.1): "LF" (largest degree wins) or "random" (= gc_color).
    Returns (colors int32[n], stats dict)."""
    lib = load()
    g, keep = _graph(offsets, idx)
    dev = keep[0].device
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
    _check_colors(out, g.n, dev, "out")
    st = _Stats()
    code = ORDER[order.upper()] if isinstance(order, str) else int(order)
    _check(lib.gc_color_ordered(ctypes.byref(g), _strategy(strategy), int(X), int(seed) & (2**64 - 1),
                                code, _ptr(out), ctypes.byref(st), _stream(dev, stream)),
           "gc_color_ordered")
    return out, _stats_dict(st)


def gc_recolor_async(offsets, idx, colors_in, perm="RV", iterations: int = 1, seed: int = 0, out=None,
                     stream=None):
    """Asynchronous recoloring aRC (Sec. 3).  Returns (colors, ncolors list,
    stats dict); stats["rounds"] sums the rounds of all iterations."""
    lib = load()
    g, keep = _graph(offsets, idx)
    dev = keep[0].device
    _check_colors(colors_in, g.n, dev, "colors_in")
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
    _check_colors(out, g.n, dev, "out")
    nc = (ctypes.c_int32 * (iterations + 1))()
    st = _Stats()
    _check(lib.gc_recolor_async(ctypes.byref(g), _ptr(colors_in), _perm(perm), int(iterations),
                                int(seed) & (2**64 - 1), _ptr(out), nc, ctypes.byref(st),
                                _stream(dev, stream)), "gc_recolor_async")
    return out, list(nc), _stats_dict(st)


def gc_recolor(offsets, idx, colors_in, perm="RV", iterations: int = 1, seed: int = 0, out=None,
               stream=None):
    """Iterative recoloring (Sec. 2.1 / Sec. 3).  Returns (colors, ncolors
    list of iterations + 1 max colors, stats dict)."""
    lib = load()
    g, keep = _graph(offsets, idx)
    dev = keep[0].device
    _check_colors(colors_in, g.n, dev, "colors_in")
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
    _check_colors(out, g.n, dev, "out")
    nc = (ctypes.c_int32 * (iterations + 1))()
    st = _Stats()
    _check(lib.gc_recolor(ctypes.byref(g), _ptr(colors_in), _perm(perm), int(iterations),
                          int(seed) & (2**64 - 1), _ptr(out), nc, ctypes.byref(st),
                          _stream(dev, stream)), "gc_recolor")
    return out, list(nc), _stats_dict(st)


def gc_color_recolor(offsets, idx, strategy="FF", X: int = 1, seed: int = 0, perm="RV",
                     iterations: int = 0, perm_seed: int = 0, out=None, validate: bool = False,
                     stream=None):
    """Speculative coloring followed by recoloring iterations, in one call.
    Returns (colors, ncolors list, stats dict, validation dict or None)."""
    lib = load()
    g, keep = _graph(offsets, idx)
    dev = keep[0].device
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
    _check_colors(out, g.n, dev, "out")
    nc = (ctypes.c_int32 * (iterations + 1))()
    st = _Stats()
    val = _Validation() if validate else None
    _check(lib.gc_color_recolor(ctypes.byref(g), _strategy(strategy), int(X),
                                int(seed) & (2**64 - 1), _perm(perm), int(iterations),
                                int(perm_seed) & (2**64 - 1), _ptr(out), nc, ctypes.byref(st),
                                ctypes.byref(val) if validate else None, _stream(dev, stream)),
           "gc_color_recolor")
    vd = {k: getattr(val, k) for k, _ in _Validation._fields_} if validate else None
    return out, list(nc), _stats_dict(st), vd


def _batch(graphs):
    """graphs: list of dicts with n, seed, X (default 1), perm ('RV'...),
    iterations (default 0), perm_seed (default 0); bases are laid out in order."""
    arr = (_BatchGraph * len(graphs))()
    base = 0
    for i, d in enumerate(graphs):
        arr[i].vertex_base = base
        arr[i].n = int(d["n"])
        arr[i].seed = int(d.get("seed", 0)) & (2**64 - 1)
        arr[i].X = int(d.get("X", 1))
        arr[i].perm = _perm(d.get("perm", "RV"))
        arr[i].iterations = int(d.get("iterations", 0))
        arr[i].perm_seed = int(d.get("perm_seed", 0)) & (2**64 - 1)
        base += int(d["n"])
    return arr, base


def _batch_call(fn, where, offsets, idx, graphs, colors_in=None, out=None, stream=None):
    lib = load()
    g, keep = _graph(offsets, idx)
    dev = keep[0].device
    arr, total = _batch(graphs)
    if total != g.n:
        raise ValueError(f"graphs cover {total} vertices, the batch CSR has {g.n}")
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
    _check_colors(out, g.n, dev, "out")
    ng = len(graphs)
    rounds = (ctypes.c_int32 * ng)()
    maxc = (ctypes.c_int32 * ng)()
    st = _Stats()
    if colors_in is None:
        rc = getattr(lib, fn)(ctypes.byref(g), arr, ng, _ptr(out), rounds, maxc, ctypes.byref(st),
                              _stream(dev, stream))
    else:
        _check_colors(colors_in, g.n, dev, "colors_in")
        rc = getattr(lib, fn)(ctypes.byref(g), arr, ng, _ptr(colors_in), _ptr(out), maxc,
                              ctypes.byref(st), _stream(dev, stream))
    _check(rc, where)
    return out, list(rounds), list(maxc), _stats_dict(st)


def gc_color_batch(offsets, idx, graphs, out=None, stream=None):
    """Speculative coloring of a batch of graphs laid out in one CSR.
    Returns (colors, rounds per graph, max color per graph, stats)."""
    return _batch_call("gc_color_batch", "gc_color_batch", offsets, idx, graphs, out=out, stream=stream)


def gc_recolor_batch(offsets, idx, graphs, colors_in, out=None, stream=None):
    """Recoloring of a batch (each graph's perm, perm_seed, iterations).
    Returns (colors, max color per graph, stats)."""
    out, _, maxc, st = _batch_call("gc_recolor_batch", "gc_recolor_batch", offsets, idx, graphs,
                                   colors_in=colors_in, out=out, stream=stream)
    return out, maxc, st


def gc_color_recolor_batch(offsets, idx, graphs, out=None, stream=None):
    """Coloring then recoloring of a batch, in one call.
    Returns (colors, rounds per graph, final max color per graph, stats)."""
    return _batch_call("gc_color_recolor_batch", "gc_color_recolor_batch", offsets, idx, graphs,
                       out=out, stream=stream)


def gc_validate(offsets, idx, colors, stream=None):
    """The definition of Sec. 1 checked on the device."""
    lib = load()
    g, keep = _graph(offsets, idx)
    dev = keep[0].device
    _check_colors(colors, g.n, dev, "colors")
    v = _Validation()
    _check(lib.gc_validate(ctypes.byref(g), _ptr(colors), ctypes.byref(v), _stream(dev, stream)),
           "gc_validate")
    return {k: getattr(v, k) for k, _ in _Validation._fields_}


def gc_validate_noalloc(offsets, idx, colors, stream=None):
    """gc_validate without any device allocation (fixed scratch in the
    library's static device memory; device tensors only, colors < 65536;
    concurrent calls on the GPU must be serialised by the caller)."""
    lib = load()
    g, keep = _graph(offsets, idx)
    dev = keep[0].device
    _check_colors(colors, g.n, dev, "colors")
    v = _Validation()
    _check(lib.gc_validate_noalloc(ctypes.byref(g), _ptr(colors), ctypes.byref(v),
                                   _stream(dev, stream)), "gc_validate_noalloc")
    return {k: getattr(v, k) for k, _ in _Validation._fields_}


def gc_check_graph(offsets, idx, stream=None):
    """Returns -1 for a well-formed CSR, else the first bad row."""
    lib = load()
    g, keep = _graph(offsets, idx)
    first = ctypes.c_int64(-1)
    rc = lib.gc_check_graph(ctypes.byref(g), ctypes.byref(first), _stream(keep[0].device, stream))
    if rc not in (0, 2):
        _check(rc, "gc_check_graph")
    return int(first.value)


def gc_priorities(seed: int, n: int, device="cuda", stream=None):
    """prio(v) for v in [0, n): the random total order of Sec. 2.2 (uint32
    values returned in an int64 tensor)."""
    lib = load()
    dev = torch.device(device)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    _check(lib.gc_priorities(int(seed) & (2**64 - 1), int(n), _ptr(out), _stream(dev, stream)),
           "gc_priorities")
    return out.to(torch.int64) & 0xFFFFFFFF


GC_PENDING = 9


class GCServer:
    """Handle of a gc_server (the serving loop); use the gc_server_* functions.
    Holds each pending request's graph tensors (the server reads them in
    place) and vertex count until its result is claimed."""

    def __init__(self, handle):
        self.handle = handle
        self.pending = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        gc_server_destroy(self)


def gc_server_create(mem_budget: int, max_batch: int = 64, workers: int = 2) -> GCServer:
    """Start a server on the current CUDA device: admission by a device-memory
    budget (bytes), batches of at most max_batch requests, `workers`
    concurrent batches."""
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.gc_server_create(int(mem_budget), int(max_batch), int(workers), ctypes.byref(h)),
           "gc_server_create")
    return GCServer(h)


def gc_server_submit(server: GCServer, offsets, idx, strategy="FF", X: int = 1, seed: int = 0,
                     perm="RV", iterations: int = 0, perm_seed: int = 0) -> int:
    """Queue one request; returns its ticket.  The tensors are kept alive by
    the handle until the result is claimed (the server reads them in place);
    do not modify them meanwhile."""
    lib = load()
    g, keep = _graph(offsets, idx)
    if keep[0].is_cuda:
        torch.cuda.current_stream(keep[0].device).synchronize()
    q = _Request()
    q.graph = g
    q.strategy = _strategy(strategy)
    q.X = int(X)
    q.seed = int(seed) & (2**64 - 1)
    q.perm = _perm(perm)
    q.iterations = int(iterations)
    q.perm_seed = int(perm_seed) & (2**64 - 1)
    t = ctypes.c_uint64()
    _check(lib.gc_server_submit(server.handle, ctypes.byref(q), ctypes.byref(t)), "gc_server_submit")
    server.pending[t.value] = (g.n, keep)
    return t.value


def _server_result(server, ticket, rc, out, res, where):
    if rc == GC_PENDING:
        return None
    server.pending.pop(ticket, None)
    _check(rc, where)
    return out, {k: getattr(res, k) for k, _ in _RequestResult._fields_}


def gc_server_poll(server: GCServer, ticket: int):
    """None while pending, else (colors int32[n] on the CPU, result dict);
    raises GCError if the request failed.  A result is handed out once."""
    lib = load()
    n = server.pending.get(ticket, (0, None))[0]
    out = torch.empty(n, dtype=torch.int32)
    res = _RequestResult()
    rc = lib.gc_server_poll(server.handle, ctypes.c_uint64(ticket), _ptr(out), ctypes.byref(res))
    return _server_result(server, ticket, rc, out, res, "gc_server_poll")


def gc_server_wait(server: GCServer, ticket: int, timeout_ms: int = -1):
    """As gc_server_poll, blocking up to timeout_ms (< 0: until done)."""
    lib = load()
    n = server.pending.get(ticket, (0, None))[0]
    out = torch.empty(n, dtype=torch.int32)
    res = _RequestResult()
    rc = lib.gc_server_wait(server.handle, ctypes.c_uint64(ticket), _ptr(out), ctypes.byref(res),
                            int(timeout_ms))
    return _server_result(server, ticket, rc, out, res, "gc_server_wait")


def gc_server_stats(server: GCServer):
    """Counts, p50/p99/mean submit-to-done latency (ms), graphs/s, memory in use."""
    lib = load()
    info = _ServerInfo()
    _check(lib.gc_server_stats(server.handle, ctypes.byref(info)), "gc_server_stats")
    return {k: getattr(info, k) for k, _ in _ServerInfo._fields_}


def gc_server_destroy(server: GCServer):
    """Finish the queued requests, stop the workers and free the server."""
    if server.handle:
        load().gc_server_destroy(server.handle)
        server.handle = None
        server.pending.clear()


class GCPlan:
    """Handle of a gc_plan: run settings plus the knobs to run them with.
    Use gc_plan_color_recolor / gc_plan_get_info; freed by gc_plan_free, at
    the end of a ``with`` block, or when the handle is collected."""

    def __init__(self, handle):
        self.handle = handle

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        gc_plan_free(self)

    def __del__(self):
        try:
            gc_plan_free(self)
        except Exception:
            pass


def _tuning_struct(knobs):
    t = _Tuning()
    _check(load().gc_get_tuning(ctypes.byref(t)), "gc_get_tuning")
    for k, v in (knobs or {}).items():
        setattr(t, k, int(v))
    return t


def gc_plan_create(tuning=None, strategy="FF", X: int = 1, perm="RV", iterations: int = 0) -> GCPlan:
    """A plan from knobs (dict of gc_tuning fields over the knobs in force;
    None: the library defaults) and run settings."""
    lib = load()
    h = ctypes.c_void_p()
    t = _tuning_struct(tuning) if tuning is not None else None
    _check(lib.gc_plan_create(ctypes.byref(t) if t is not None else None, _strategy(strategy),
                              int(X), _perm(perm), int(iterations), ctypes.byref(h)),
           "gc_plan_create")
    return GCPlan(h)


def gc_plan_autotune(offsets, idx, strategy="FF", X: int = 1, seed: int = 0, perm="RV",
                     iterations: int = 0, repeats: int = 2, stream=None) -> GCPlan:
    """Tune the knobs for these settings on this graph (device tensors) and
    return a plan holding them."""
    lib = load()
    g, keep = _graph(offsets, idx)
    h = ctypes.c_void_p()
    _check(lib.gc_plan_autotune(ctypes.byref(g), _strategy(strategy), int(X),
                                int(seed) & (2**64 - 1), _perm(perm), int(iterations),
                                int(repeats), ctypes.byref(h), _stream(keep[0].device, stream)),
           "gc_plan_autotune")
    return GCPlan(h)


def gc_plan_get_info(plan: GCPlan):
    """The plan's knobs (dict), settings and tuned time / shape."""
    info = _PlanInfo()
    _check(load().gc_plan_get_info(plan.handle, ctypes.byref(info)), "gc_plan_get_info")
    d = {k: getattr(info, k) for k, _ in _PlanInfo._fields_ if k != "tuning"}
    d["tuning"] = {k: getattr(info.tuning, k) for k, _ in _Tuning._fields_}
    return d


def gc_plan_color_recolor(plan: GCPlan, offsets, idx, seed: int = 0, perm_seed: int = 0, out=None,
                          validate: bool = False, stream=None):
    """gc_color_recolor with the plan's settings and knobs.  Returns (colors,
    ncolors list, stats dict, validation dict or None)."""
    lib = load()
    if not plan.handle:
        raise ValueError("plan was freed")
    info = _PlanInfo()
    _check(lib.gc_plan_get_info(plan.handle, ctypes.byref(info)), "gc_plan_get_info")
    g, keep = _graph(offsets, idx)
    dev = keep[0].device
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
    _check_colors(out, g.n, dev, "out")
    nc = (ctypes.c_int32 * (info.iterations + 1))()
    st = _Stats()
    val = _Validation() if validate else None
    _check(lib.gc_plan_color_recolor(plan.handle, ctypes.byref(g), int(seed) & (2**64 - 1),
                                     int(perm_seed) & (2**64 - 1), _ptr(out), nc, ctypes.byref(st),
                                     ctypes.byref(val) if validate else None, _stream(dev, stream)),
           "gc_plan_color_recolor")
    vd = {k: getattr(val, k) for k, _ in _Validation._fields_} if validate else None
    return out, list(nc), _stats_dict(st), vd


def gc_plan_free(plan: GCPlan):
    """Release the plan (idempotent)."""
    if plan.handle:
        load().gc_plan_free(plan.handle)
        plan.handle = None


def gc_set_tuning(**knobs):
    """Set scheduling knobs (see gc_tuning in gc.h); no arguments restores defaults."""
    lib = load()
    if not knobs:
        _check(lib.gc_set_tuning(None), "gc_set_tuning")
        return
    t = _Tuning()
    _check(lib.gc_get_tuning(ctypes.byref(t)), "gc_get_tuning")
    for k, v in knobs.items():
        setattr(t, k, int(v))
    _check(lib.gc_set_tuning(ctypes.byref(t)), "gc_set_tuning")


def gc_get_tuning():
    lib = load()
    t = _Tuning()
    _check(lib.gc_get_tuning(ctypes.byref(t)), "gc_get_tuning")
    return {k: getattr(t, k) for k, _ in _Tuning._fields_}


def gc_profile_enable(on: bool = True):
    """Per-kernel CUDA-event timing inside the library (resets the totals)."""
    load().gc_profile_enable(1 if on else 0)


def gc_profile_read():
    """{kernel name: (launches, total ms)} since gc_profile_enable."""
    lib = load()
    cnt = lib.gc_profile_read(None, 0)
    arr = (_KernelTime * max(cnt, 1))()
    cnt = lib.gc_profile_read(arr, cnt)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].ms)) for i in range(cnt)}


PRESETS = {"speed": 0, "quality": 1, "quality10": 2}


def gc_preset_params(preset):
    """The parameter sets of Sec. 4.3 / Sec. 5 ("speed", "quality", "quality10")
    as keyword arguments of gc_color_recolor."""
    lib = load()
    s, x, p, it = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    code = PRESETS[preset] if isinstance(preset, str) else int(preset)
    _check(lib.gc_preset_params(code, ctypes.byref(s), ctypes.byref(x), ctypes.byref(p), ctypes.byref(it)),
           "gc_preset_params")
    return {"strategy": "FF" if s.value == FIRST_FIT else "RXF", "X": x.value,
            "perm": {v: k for k, v in PERM.items()}.get(p.value, p.value), "iterations": it.value}


def gc_inject_alloc_failure(after: int):
    """Testing aid: the library's scratch allocation after the next `after`
    ones fails once (GC_ERR_OOM); a negative value disables."""
    load().gc_inject_alloc_failure(int(after))


def gc_kernel_launches() -> int:
    return int(load().gc_kernel_launches())


def gc_status_string(code: int) -> str:
    return load().gc_status_string(int(code)).decode()


def gc_version() -> int:
    return int(load().gc_version())
