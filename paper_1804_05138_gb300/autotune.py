"""Autotuner for the batched factorization: block size b per shape bucket.

Shapes are grouped into coarse buckets of (m, n, k).  For each bucket, up to a few
representative matrices are factored with every candidate b (b <= k) through the batched
entry point itself, timed with CUDA events (best of `reps`), and the fastest b is kept.
Tables are cached per GPU name and oversampling in paper_1804_05138_gb300/_build/.
"""
from __future__ import annotations

import json
import os

from . import binding

CANDIDATES = (16, 32, 64)
_HERE = os.path.dirname(os.path.abspath(__file__))


def bucket(m: int, n: int, k: int) -> str:
    return f"{min(m // 1024, 3)}_{min(n // 512, 3)}_{min(k // 64, 3)}"


def default_b(m: int, n: int, k: int) -> int:
    return max(1, min(64, k))


def choose(table: dict, m: int, n: int, k: int) -> int:
    return max(1, min(int(table.get(bucket(m, n, k), default_b(m, n, k))), k, 64))


def _time_batch(mats, ks, bs, p, reps):
    import torch
    orig = [A.clone() for A in mats]
    batch = binding.Batch(mats, ks, bs, p=p)
    best = float("inf")
    for _ in range(reps + 1):
        for A, O in zip(batch.mats, orig):
            A.copy_(O)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        code = batch.run()
        e1.record()
        if code != 0:
            raise binding.RQRCPError(code, "rqrcp_factor_batched (tuning)")
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(shapes, p: int = 8, candidates=CANDIDATES, reps: int = 2, per_bucket: int = 3, seed: int = 0):
    """Return {bucket: b} for the given (m, n, k) shapes, measured on the current GPU."""
    import numpy as np
    import torch
    groups = {}
    for (m, n, k) in shapes:
        groups.setdefault(bucket(m, n, k), []).append((m, n, k))
    rng = np.random.default_rng(seed)
    table = {}
    for key, items in sorted(groups.items()):
        pick = [items[i] for i in rng.choice(len(items), size=min(per_bucket, len(items)), replace=False)]
        kmin = min(k for _, _, k in pick)
        cands = [b for b in candidates if b <= kmin] or [default_b(0, 0, kmin)]
        mats = [torch.randn((n, m), device="cuda").t() for (m, n, _) in pick]
        ks = [k for _, _, k in pick]
        timings = {b: _time_batch(mats, ks, [b] * len(ks), p, reps) for b in cands}
        table[key] = int(min(timings, key=timings.get))
    return table


def cache_path(p: int) -> str:
    import torch
    name = torch.cuda.get_device_name().replace(" ", "_")
    return os.path.join(_HERE, "_build", f"autotune_batched_{name}_p{p}.json")


def load_or_tune(shapes, p: int = 8) -> dict:
    path = cache_path(p)
    table = {}
    if os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
    missing = [s for s in shapes if bucket(*s) not in table]
    if missing:
        table.update(tune(missing, p=p))
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return table
