"""Measured choice of the object-gradient accumulation tile per problem shape.

The owner-computes accumulation (the one-GPU form of the image-gradient
tessellation, Sec. III) is bandwidth-bound; its tile shape trades the number
of blocks against the positions each block scans.  ``tune_tile`` times a few
shapes on the real inputs with the library's own kernel timers and keeps the
fastest in a JSON cache keyed by the problem shape.  The cache lives in
``$PTYCHO_GB300_CACHE`` (a directory) or ``~/.cache/ptycho_gb300``.
"""
from __future__ import annotations

import json
import os

import torch

from .api import Geometry, Plan

CANDIDATES = ((16, 16), (32, 32), (32, 64), (64, 32), (64, 64), (16, 64))


def cache_path() -> str:
    base = os.environ.get("PTYCHO_GB300_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "ptycho_gb300")
    return os.path.join(base, "autotune.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def key_for(geom: Geometry, precision: str, ckpt_every: int = 0) -> str:
    return f"M{geom.M}_S{geom.S}_H{geom.H}_W{geom.W}_N{geom.N}_{precision}" + (f"_rc{ckpt_every}" if ckpt_every else "")


def tune_tile(geom: Geometry, pos, probe, obj, meas, device, precision: str = "fp32",
              candidates=CANDIDATES, reps: int = 2, use_cache: bool = True, ckpt_every: int = 0) -> tuple[int, int]:
    """Fastest accumulation tile (rows, cols) for this shape, measured on these inputs
    (recompute mode reads finished patches instead of two wave arrays: tuned separately)."""
    key = key_for(geom, precision, ckpt_every)
    cache = _load() if use_cache else {}
    if key in cache:
        return tuple(cache[key]["tile"])
    results = {}
    for tile in candidates:
        plan = Plan(geom, device, tile=tile, timing=True, async_check=True, precision=precision,
                    ckpt_every=ckpt_every)
        plan.loss_grad(pos, probe, obj, meas)  # warm-up
        plan.timing(reset=True)
        for _ in range(reps):
            plan.loss_grad(pos, probe, obj, meas)
        t = plan.timing(reset=True)
        results[tile] = t["accum_ms"] / max(t["accum_launches"], 1)
        plan.close()
    best = min(results, key=results.get)
    if use_cache:
        cache = _load()
        cache[key] = {"tile": list(best), "accum_ms": {f"{a}x{b}": v for (a, b), v in results.items()}}
        _save(cache)
    torch.cuda.synchronize(device)
    return best
