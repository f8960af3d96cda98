"""Choice by timing of a batch's schedule (mode, threads per block, chunk)
and of a domain's tile shape (the blocks in which its fluid nodes are
numbered in memory).

Every schedule gives the same results bit for bit, so the schedule trials
are real steps of the run: each candidate takes one untimed step (which
records its CUDA graph) and ``trial_steps`` steps timed with CUDA events on
the batch's stream; the fastest wins. The tile shape is fixed when a
domain's geometry is built, so its trials build one domain (or batch) per
candidate from a caller's factory and time it the same way; per-node
results do not depend on the shape. Winners are cached per shape class in
a JSON file, so a batch or domain of the same class later skips the search.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
from typing import Dict, Optional, Tuple

# (mode, threads, chunk): mode 0 = one launch per pass of all cases,
# mode 1 = one persistent launch per call with chunk blocks per work item
CANDIDATES = ((0, 256, 1), (0, 128, 1), (1, 256, 1), (1, 256, 4),
              (1, 256, 16), (1, 128, 4), (1, 128, 16))


# tile shapes (x, y, z) tried per lattice; the first is the library default
TILE_CANDIDATES = {
    19: ((32, 8, 8), (32, 4, 4), (64, 4, 4), (32, 4, 8), (64, 8, 8),
         (32, 16, 16), (128, 2, 2), (128, 8, 4)),
    9: ((64, 32, 1), (32, 32, 1), (32, 64, 1), (128, 16, 1), (64, 64, 1),
        (256, 8, 1)),
}


def default_cache_path() -> str:
    return os.environ.get(
        "LBMGB_TUNE_CACHE",
        os.path.join(os.path.expanduser("~"), ".cache", "lbmgb",
                     "batch_tune.json"))


def _sig2(v: int) -> int:
    if v <= 0:
        return 0
    e = int(math.floor(math.log10(v))) - 1
    return int(round(v / 10 ** e)) * 10 ** e if e > 0 else int(v)


def shape_class(q: int, storage: str, counts) -> str:
    """Key of a batch: counts is a list of (n_fluid, n_solid_boundary)."""
    nf = sum(int(c[0]) for c in counts)
    ns = sum(int(c[1]) for c in counts)
    return f"Q{q}-{storage}-n{len(counts)}-F{_sig2(nf)}-S{_sig2(ns)}"


def load_cache(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path: str, key: str, entry: dict) -> None:
    d = load_cache(path)
    d[key] = entry
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".")
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def fastest(timings: Dict[Tuple[int, int, int], float]) -> Tuple[int, int, int]:
    """Candidate with the least time per step (ties: the earlier one in
    CANDIDATES order)."""
    order = {c: i for i, c in enumerate(CANDIDATES)}
    return min(timings, key=lambda c: (timings[c], order.get(c, len(order))))


def tune(batch, trial_steps: int = 8, cache_path: Optional[str] = None,
         use_cache: bool = True) -> dict:
    """Pick and apply the fastest schedule for `batch` (a lbm.Batch).
    Returns {"config", "key", "cached", "steps_used", "ms_per_step"}; the
    batch has advanced by steps_used steps."""
    torch = batch.torch
    path = cache_path or default_cache_path()
    sess = batch.sessions
    key = shape_class(sess[0].q, sess[0].storage,
                      [(s.counts[1], s.counts[2]) for s in sess])
    if use_cache:
        hit = load_cache(path).get(key)
        if hit and tuple(hit.get("config", ())) in CANDIDATES:
            batch.set_config(*hit["config"])
            return {"config": tuple(hit["config"]), "key": key,
                    "cached": True, "steps_used": 0,
                    "ms_per_step": hit.get("ms_per_step")}
    stream = torch.cuda.current_stream()
    timings = {}
    used = 0
    for cand in CANDIDATES:
        batch.set_config(*cand)
        batch.step(1)  # records the graph of this candidate
        used += 1
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.step(trial_steps)
        e1.record(stream)
        e1.synchronize()
        used += trial_steps
        timings[cand] = e0.elapsed_time(e1) / trial_steps
    if batch.status() != 0:
        raise RuntimeError("a persistent-kernel wait ran out during tuning")
    best = fastest(timings)
    batch.set_config(*best)
    entry = {"config": list(best), "ms_per_step": timings[best],
             "trials": {f"{m}/{t}/{c}": v for (m, t, c), v in timings.items()}}
    if use_cache:
        store_cache(path, key, entry)
    return {"config": best, "key": key, "cached": False, "steps_used": used,
            "ms_per_step": timings[best], "trials": entry["trials"]}


def _time_steps(obj, torch, trial_steps: int) -> float:
    stream = torch.cuda.current_stream()
    obj.step(1)  # records the graph
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    obj.step(trial_steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / trial_steps


def tile_class(q: int, storage: str, shape, counts) -> str:
    """Key of a domain for the tile choice: lattice, storage, box shape
    (nz, ny, nx) and (n_fluid, n_solid_boundary) to two significant digits
    (summed over the cases of a batch)."""
    nf = sum(int(c[0]) for c in counts)
    ns = sum(int(c[1]) for c in counts)
    dims = "x".join(str(int(v)) for v in shape)
    return f"tile-Q{q}-{storage}-{dims}-n{len(counts)}-F{_sig2(nf)}-S{_sig2(ns)}"


def tune_tile(make, q: int, key: Optional[str] = None,
              candidates=None, trial_steps: int = 8,
              cache_path: Optional[str] = None,
              use_cache: bool = True) -> dict:
    """Pick the fastest tile shape. make(tile) builds a ready-to-step
    object (a lbm.Session with parameters and state set, or a lbm.Batch of
    such sessions) whose fluid nodes are numbered in tiles of that shape;
    each candidate's object takes one untimed and ``trial_steps`` timed
    steps and is then dropped. Returns {"tile", "key", "cached",
    "ms_per_step", "trials"}; build the run's own object with the returned
    tile. With a key and use_cache, the winner is read from and stored in
    the cache."""
    cands = tuple(candidates or TILE_CANDIDATES[q])
    path = cache_path or default_cache_path()
    if use_cache and key:
        hit = load_cache(path).get(key)
        if hit and tuple(hit.get("tile", ())) in cands:
            return {"tile": tuple(hit["tile"]), "key": key, "cached": True,
                    "ms_per_step": hit.get("ms_per_step"),
                    "trials": hit.get("trials")}
    timings = {}
    torch = None
    for tile in cands:
        obj = make(tile)
        torch = obj.torch
        timings[tuple(tile)] = _time_steps(obj, torch, trial_steps)
        del obj
    order = {tuple(c): i for i, c in enumerate(cands)}
    best = min(timings, key=lambda t: (timings[t], order[t]))
    trials = {"x".join(map(str, t)): v for t, v in timings.items()}
    if use_cache and key:
        store_cache(path, key, {"tile": list(best),
                                "ms_per_step": timings[best],
                                "trials": trials})
    return {"tile": best, "key": key, "cached": False,
            "ms_per_step": timings[best], "trials": trials}
