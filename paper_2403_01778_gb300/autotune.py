"""Autotuner of the batched solve's launch shape (threads per CTA).

The batched kernel runs one tensor per CTA; the best CTA size depends on the
mix of tensor sizes (face size, number of outer indices).  `best_threads`
times each candidate once on the caller's batch (the solve itself, not a
model) and caches the winner in a JSON file keyed by device name and a
coarse signature of the batch (counts and size buckets per order)."""
from __future__ import annotations

import json
import math
import os
import time

import torch

from .api import hoscf_solve_batched

CANDIDATES = (256, 512, 1024)
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


def best_threads(tensors, u0s, tol=1e-6, max_iter=200, force=False):
    """Threads per CTA for this batch (measured once, then cached)."""
    dev = torch.cuda.get_device_name(tensors[0].device)
    key = f"{dev}|{signature(tensors)}|tol{tol:g}"
    db = _load()
    if key in db and not force:
        return int(db[key]["threads"]), db[key]
    times = {}
    for th in CANDIDATES:
        hoscf_solve_batched(tensors, u0s, tol=tol, max_iter=max_iter, batch_threads=th)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hoscf_solve_batched(tensors, u0s, tol=tol, max_iter=max_iter, batch_threads=th)
        torch.cuda.synchronize()
        times[th] = time.perf_counter() - t0
    best = min(times, key=times.get)
    db[key] = {"threads": best, "seconds": {str(k): v for k, v in times.items()}}
    _store(db)
    return best, db[key]
