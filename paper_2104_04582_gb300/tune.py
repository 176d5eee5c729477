"""Autotuner for the summation kernel's tile shape.

The summation kernel is tunable in three ways that change speed but never results (every sample
is summed by one thread in a fixed order, so all choices are bit-identical):

* samples per thread R (the segment tile: one pass covers threads x R consecutive samples),
* threads per block (128 or 256),
* slots per shared-memory stage (the mode tile: each segment's harmonic slot table streams
  through a ring of stages of this many slots, so it also sets the shared memory per CTA).

`tune()` times every candidate on a representative workload with CUDA events (several runs,
best of), picks the fastest, installs it in the context, and records it in a JSON cache keyed by
(precision, slot-count bucket, samples bucket); `apply_cached()` installs a cached choice and
`ensure()` does either, so that a caller (the batched path, the serving engine, the benchmark)
runs every workload with a tuned tile.
"""
from __future__ import annotations

import json
import math
import os
from typing import Any, Callable, Dict, List, Optional, Sequence, Tuple

from . import fewsum as F

CANDIDATES = {
    F.FEW_FP64: [(r, t, s) for r in (1, 2) for t in (128, 256) for s in (128, 256, 512)],
    F.FEW_MIXED: [(r, t, s) for r in (2, 4, 8) for t in (128, 256) for s in (256, 512, 1024)],
}

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "fewsum_tiles.json")


def bucket(prec: int, n_slots: int, n_samples: int) -> str:
    """Cache key: precision, slots rounded to a power of two, samples to a power of four."""
    sb = 1 << max(0, math.ceil(math.log2(max(1, n_slots))))
    nb = 4 ** max(0, math.ceil(math.log(max(1, n_samples), 4)))
    return f"{'fp64' if prec == F.FEW_FP64 else 'mixed'}:{sb}:{nb}"


def _load(path: str) -> Dict[str, dict]:
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def _save(path: str, data: Dict[str, dict]) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def install(ctx_handle: int, prec: int, choice: Tuple[int, int, int]) -> None:
    R, T, S = choice
    F.few_set_tiles(ctx_handle, prec, R, T, S)


def tune(ctx_handle: int, run, prec: int, n_slots: int, n_samples: int, repeats: int = 3,
         cache_path: Optional[str] = DEFAULT_CACHE,
         candidates: Optional[Sequence[Tuple[int, int, int]]] = None,
         prepare: Optional[Callable[[], Any]] = None,
         cleanup: Optional[Callable[[Any], None]] = None) -> Tuple[Tuple[int, int, int], Dict[str, float]]:
    """Time `run` for every candidate tile and keep the fastest.

    Without `prepare`, `run()` must queue one workload on the current stream.  With it, each
    candidate is installed, `prepare()` builds whatever depends on the tile (a batch plan, say)
    outside the timed region, `run(state)` queues the workload and `cleanup(state)` releases it.
    Returns the best (R, threads, stage_slots) and the per-candidate best time in ms; installs
    the winner in the context and stores it in the cache (unless cache_path is None).
    """
    import torch
    cands = list(candidates or CANDIDATES[prec])
    times: Dict[str, float] = {}
    best, best_ms = None, float("inf")
    for c in cands:
        try:
            install(ctx_handle, prec, c)
            state = prepare() if prepare else None
        except F.FewError:
            continue  # e.g. a stage too large for shared memory
        go = (lambda: run(state)) if prepare else run
        try:
            go()  # warm-up (occupancy cache, first launch)
            torch.cuda.synchronize()
            ms = float("inf")
            for _ in range(repeats):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                go()
                b.record()
                b.synchronize()
                ms = min(ms, a.elapsed_time(b))
        except F.FewError:
            ms = float("inf")
        finally:
            if prepare and cleanup:
                cleanup(state)
        times[f"R={c[0]} T={c[1]} S={c[2]}"] = ms
        if ms < best_ms:
            best, best_ms = c, ms
    if best is None:
        raise RuntimeError("no tile candidate ran")
    install(ctx_handle, prec, best)
    if cache_path:
        data = _load(cache_path)
        data[bucket(prec, n_slots, n_samples)] = {"R": best[0], "threads": best[1],
                                                  "stage_slots": best[2], "ms": best_ms}
        _save(cache_path, data)
    return best, times


def apply_cached(ctx_handle: int, prec: int, n_slots: int, n_samples: int,
                 cache_path: str = DEFAULT_CACHE) -> Optional[Tuple[int, int, int]]:
    """Install the cached choice for this bucket, if any; returns it."""
    e = _load(cache_path).get(bucket(prec, n_slots, n_samples))
    if not e:
        return None
    if "stage_slots" not in e:
        return None
    choice = (int(e["R"]), int(e["threads"]), int(e["stage_slots"]))
    install(ctx_handle, prec, choice)
    return choice


def ensure(ctx_handle: int, run, prec: int, n_slots: int, n_samples: int,
           cache_path: Optional[str] = DEFAULT_CACHE, repeats: int = 2,
           prepare: Optional[Callable[[], Any]] = None,
           cleanup: Optional[Callable[[Any], None]] = None) -> Tuple[Tuple[int, int, int], bool]:
    """Install the cached tile for this workload bucket, tuning with `run` on a miss.

    Returns (choice, tuned_now)."""
    if cache_path:
        c = apply_cached(ctx_handle, prec, n_slots, n_samples, cache_path)
        if c is not None:
            return c, False
    best, _ = tune(ctx_handle, run, prec, n_slots, n_samples, repeats=repeats,
                   cache_path=cache_path, prepare=prepare, cleanup=cleanup)
    return best, True
