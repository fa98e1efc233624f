"""Autotuner of the batched solve's launch parameters.

The batched kernel runs one tensor per CTA; the best CTA size and the number
of faces (T[o][:][:]) staged and folded per group depend on the mix of
tensor sizes (face size, number of outer indices).  `best_config` times
every candidate pair on the caller's batch (the solve itself, not a model;
the median of a few runs after a warm-up) and caches the winner in a JSON
file keyed by device name and a coarse signature of the batch (counts and
size buckets per order)."""
from __future__ import annotations

import json
import math
import os
import statistics
import time

import torch

from .api import hoscf_solve_batched

CANDIDATES = (256, 512, 1024)          # threads per CTA
FACE_CANDIDATES = (8, 16, 32)          # faces per staged group (at most)
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def signature(tensors) -> str:
    buckets = {}
    for T in tensors:
        b = (T.dim(), int(math.log2(max(1, T.numel()))))
        buckets[b] = buckets.get(b, 0) + 1
    return ";".join(f"d{d}s{s}:{c}" for (d, s), c in sorted(buckets.items()))


def _load():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE)


def _time(tensors, u0s, tol, max_iter, th, fc, reps=3):
    hoscf_solve_batched(tensors, u0s, tol=tol, max_iter=max_iter, batch_threads=th,
                        batch_faces=fc)   # warm (graph capture)
    out = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hoscf_solve_batched(tensors, u0s, tol=tol, max_iter=max_iter, batch_threads=th,
                            batch_faces=fc)
        torch.cuda.synchronize()
        out.append(time.perf_counter() - t0)
    return statistics.median(out)


def best_config(tensors, u0s, tol=1e-6, max_iter=200, force=False):
    """(threads per CTA, faces per group) for this batch (measured once,
    then cached) and the cache record."""
    dev = torch.cuda.get_device_name(tensors[0].device)
    key = f"{dev}|{signature(tensors)}|tol{tol:g}|v2"
    db = _load()
    if key in db and not force:
        return (int(db[key]["threads"]), int(db[key]["faces"])), db[key]
    times = {}
    for th in CANDIDATES:
        for fc in FACE_CANDIDATES:
            times[(th, fc)] = _time(tensors, u0s, tol, max_iter, th, fc)
    best = min(times, key=times.get)
    db[key] = {"threads": best[0], "faces": best[1],
               "seconds": {f"{k[0]}x{k[1]}": v for k, v in times.items()}}
    _store(db)
    return best, db[key]


def best_threads(tensors, u0s, tol=1e-6, max_iter=200, force=False):
    """Threads per CTA of the best configuration (see best_config)."""
    (th, _), rec = best_config(tensors, u0s, tol=tol, max_iter=max_iter, force=force)
    return th, rec
