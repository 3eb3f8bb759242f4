"""Autotuning of the scheduling knobs, cached by the shape of the graph.

`autotune(offsets, idx, ...)` asks the library (gc_autotune, coordinate
descent over the knobs, timing the real pipeline on the device) for the
fastest knobs and stores them in a JSON cache keyed by the graph's size and
log2-degree histogram, the strategy and the recoloring settings;
`apply(...)` looks the key up (tuning if missing) and sets the knobs
process-wide; `plan(...)` returns them in a plan instead, which applies them
to its own calls only.  The knobs never change results, only speed.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import threading

import torch

from . import (_Tuning, _check, _graph, _perm, _stream, _strategy, gc_plan_create,
                gc_set_tuning, load)

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("GC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_1407_6745_gb300",
                                       "autotune.json"))


def shape_key(offsets: torch.Tensor, strategy, X: int, perm, iterations: int) -> str:
    deg = (offsets[1:] - offsets[:-1]).to(torch.float64)
    hist = torch.bincount(torch.floor(torch.log2(deg + 1)).to(torch.int64), minlength=32)[:32]
    frac = (hist.to(torch.float64) / max(1, deg.numel())).cpu().tolist()
    sig = {"n_log2": round(float(torch.log2(torch.tensor(float(max(deg.numel(), 1))))), 1),
           "hist": [round(f, 2) for f in frac], "strategy": str(strategy), "X": int(X),
           "perm": str(perm), "iterations": int(iterations)}
    return hashlib.sha1(json.dumps(sig, sort_keys=True).encode()).hexdigest()[:20]


def _load_cache():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(cache):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(offsets, idx, strategy="FF", X: int = 1, seed: int = 0, perm="RV",
             iterations: int = 0, repeats: int = 2, stream=None):
    """Fastest knobs for this graph and these settings: (dict, ms per call)."""
    lib = load()
    g, keep = _graph(offsets, idx)
    best = _Tuning()
    ms = ctypes.c_float(0.0)
    _check(lib.gc_autotune(ctypes.byref(g), _strategy(strategy), int(X), int(seed) & (2**64 - 1),
                           _perm(perm), int(iterations), int(repeats), ctypes.byref(best),
                           ctypes.byref(ms), _stream(keep[0].device, stream)), "gc_autotune")
    return {k: getattr(best, k) for k, _ in _Tuning._fields_}, float(ms.value)


def _cached(offsets, idx, strategy, X, seed, perm, iterations, retune):
    key = shape_key(offsets, strategy, X, perm, iterations)
    with _lock:
        cache = _load_cache()
        entry = None if retune else cache.get(key)
        if entry is None:
            knobs, ms = autotune(offsets, idx, strategy, X, seed, perm, iterations)
            entry = {"knobs": knobs, "ms": ms}
            cache[key] = entry
            _store_cache(cache)
    return entry["knobs"]


def apply(offsets, idx, strategy="FF", X: int = 1, seed: int = 0, perm="RV", iterations: int = 0,
          retune: bool = False):
    """Sets the cached knobs for this graph shape process-wide (tuning and
    caching them on a miss); returns them."""
    knobs = _cached(offsets, idx, strategy, X, seed, perm, iterations, retune)
    gc_set_tuning(**knobs)
    return knobs


def plan(offsets, idx, strategy="FF", X: int = 1, seed: int = 0, perm="RV", iterations: int = 0,
         retune: bool = False):
    """A plan (gc_plan_create) holding the cached knobs for this graph shape
    and these settings, tuning and caching them on a miss; the process-wide
    knobs are left alone."""
    knobs = _cached(offsets, idx, strategy, X, seed, perm, iterations, retune)
    return gc_plan_create(knobs, strategy, X, perm, iterations)
