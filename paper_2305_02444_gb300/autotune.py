"""Autotuner for the batched FT-DGEMM schedule.

The persistent batched kernel takes (problem, tile) work items from a global
counter; the schedule fixes their order (problem order, longest-K first, or
round robin over problems) and how many items a CTA takes per counter access
(1, 2, 4, 8).  For a batch signature (the multiset of shapes and layouts)
this module times every candidate schedule on synthetic problems of the same
shapes through CUDA-graph launches, keeps the fastest, and caches the choice
in a JSON file keyed by the signature and the device.
"""
from __future__ import annotations

import hashlib
import json
import os

CANDIDATES = [order | (c << 4) for order in (0, 1, 2) for c in (0, 1, 2)]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "batched_schedules.json")


def signature(shapes) -> str:
    """shapes: iterable of (ta, tb, M, N, K)."""
    key = ";".join(sorted(f"{ta}{tb}{m}x{n}x{k}" for ta, tb, m, n, k in shapes))
    return hashlib.sha256(key.encode()).hexdigest()[:20]


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(0) if torch.cuda.is_available() else "cpu"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_batched(shapes, reps: int = 5, seed: int = 1, cache_path: str = DEFAULT_CACHE, force: bool = False):
    """Return (best schedule, {schedule: ms}) for `shapes` [(ta, tb, M, N, K)]."""
    import torch
    from . import ftgemm, inputs
    sig = f"{_device_name()}:{signature(shapes)}"
    cache = load_cache(cache_path)
    if not force and sig in cache:
        return cache[sig]["schedule"], cache[sig]["ms"]
    probs, keep = [], []
    for q, (ta, tb, m, n, k) in enumerate(shapes):
        ar, ac = (m, k) if ta == "N" else (k, m)
        br, bc = (k, n) if tb == "N" else (n, k)
        lda, ldb, ldc = ar + (ar & 1), br + (br & 1), m + (m & 1)
        A = inputs.matrix(ar, ac, seed + 3 * q, ld=lda, device="cuda", fill_pad=0.0)
        B = inputs.matrix(br, bc, seed + 3 * q + 1, ld=ldb, device="cuda", fill_pad=0.0)
        C = torch.zeros((n, ldc), dtype=torch.float64, device="cuda")
        keep += [A, B, C]
        probs.append((ta, tb, m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc))
    s = torch.cuda.current_stream()
    times = {}
    for sched in CANDIDATES:
        plan = ftgemm.BatchedPlan(probs, ft=True, schedule=sched)
        for _ in range(2):
            plan.launch()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            plan.launch()
        e1.record(s)
        torch.cuda.synchronize()
        times[sched] = e0.elapsed_time(e1) / reps
        plan.destroy()
    best = min(times, key=times.get)
    cache[sig] = {"schedule": best, "ms": {str(k): v for k, v in times.items()}, "n": len(shapes)}
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:   # closed (flushed) before it replaces the cache
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)
    return best, times
