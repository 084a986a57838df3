"""Autotuner for the batched factorization: block size b and contraction tile shapes per shape bucket.

Shapes are grouped into coarse buckets of (m, n, k).  For each bucket, up to a few representative
matrices are factored through the batched entry point itself, timed with CUDA events (best of
`reps`):
  1. every candidate b (b <= k) with the default tile rules;
  2. with the fastest b, every tile variant (RQRCP_TILES_*): the trailing update on 64 x 128 SIMT
     tiles or on 128 x 64 tcgen05 tiles, the sketch on SIMT tiles, the Gram V^T [V C] on 64 x 128
     tiles; a variant replaces the default only if it is faster by more than `margin`.
Tables map a bucket to {"b": b, "tiles": t}; they are cached per GPU name, precision (the batched
form is FP32) and oversampling p in paper_1804_05138_gb300/_build/.
"""
from __future__ import annotations

import json
import os

from . import binding

CANDIDATES = (16, 32, 64)
TILE_VARIANTS = (binding.RQRCP_TILES_UPDATE_SIMT, binding.RQRCP_TILES_UPDATE_TC, binding.RQRCP_TILES_SKETCH_SIMT,
                 binding.RQRCP_TILES_GRAM_RT64)
_HERE = os.path.dirname(os.path.abspath(__file__))
TABLE_VERSION = 2


def bucket(m: int, n: int, k: int) -> str:
    return f"{min(m // 1024, 3)}_{min(n // 512, 3)}_{min(k // 64, 3)}"


def default_b(m: int, n: int, k: int) -> int:
    return max(1, min(64, k))


def _entry(table: dict, m: int, n: int, k: int) -> dict:
    e = table.get(bucket(m, n, k))
    if e is None:
        return {"b": default_b(m, n, k), "tiles": 0}
    if isinstance(e, dict):
        return {"b": int(e.get("b", default_b(m, n, k))), "tiles": int(e.get("tiles", 0))}
    return {"b": int(e), "tiles": 0}


def choose(table: dict, m: int, n: int, k: int) -> int:
    """Block size b for an m x n matrix with target rank k."""
    return max(1, min(_entry(table, m, n, k)["b"], k, 64))


def choose_tiles(table: dict, m: int, n: int, k: int) -> int:
    """Tile-shape choice (an OR of RQRCP_TILES_*) for an m x n matrix with target rank k."""
    return _entry(table, m, n, k)["tiles"]


def _time_batch(mats, ks, bs, p, reps, tiles=None):
    import torch
    orig = [A.clone() for A in mats]
    batch = binding.Batch(mats, ks, bs, p=p, tiles=tiles)
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


def tune(shapes, p: int = 8, candidates=CANDIDATES, reps: int = 2, per_bucket: int = 3, seed: int = 0,
         variants=TILE_VARIANTS, margin: float = 0.02):
    """Return {bucket: {"b": b, "tiles": t, "ms": {...}}} for the given (m, n, k) shapes, measured on the
    current GPU."""
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
        b_best = int(min(timings, key=timings.get))
        t_best, ms_best = 0, timings[b_best]
        tile_ms = {"0": round(ms_best, 4)}
        for t in variants:
            ms = _time_batch(mats, ks, [b_best] * len(ks), p, reps, tiles=[t] * len(ks))
            tile_ms[str(t)] = round(ms, 4)
            if ms < ms_best * (1.0 - margin):
                t_best, ms_best = t, ms
        table[key] = {"b": b_best, "tiles": t_best, "ms_b": {str(b): round(v, 4) for b, v in timings.items()},
                      "ms_tiles": tile_ms}
    return table


def cache_path(p: int) -> str:
    import torch
    name = torch.cuda.get_device_name().replace(" ", "_")
    return os.path.join(_HERE, "_build", f"autotune_batched_v{TABLE_VERSION}_{name}_fp32_p{p}.json")


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
