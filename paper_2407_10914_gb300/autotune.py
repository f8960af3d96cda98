"""Choice of a batch's schedule (mode, threads per block, chunk) by timing.

Every schedule gives the same results bit for bit, so the trials are real
steps of the run: each candidate takes one untimed step (which records its
CUDA graph) and ``trial_steps`` steps timed with CUDA events on the
batch's stream; the fastest wins. The winner is cached per shape class, the
lattice, storage, case count and the total fluid and solid-boundary node
counts to two significant digits, in a JSON file, so a batch of the same
class later skips the search.
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
