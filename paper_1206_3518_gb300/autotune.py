"""Autotuned pair-kernel tile shapes with a JSON cache keyed by device and problem shape.

The choice for a shape (device name, real-space grid, band counts, sphere sizes) is measured
once by bse_autotune_pair on a range of q points and stored in a JSON file; later plans of the
same shape reuse it without timing.  Marshalling and bookkeeping only: the timing and the
selection run in the CUDA library.
"""
from __future__ import annotations

import json
import os

from . import bse

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune_cache.json")
_FIELDS = ("index", "threads", "rows", "max_products", "max_bands", "points_per_thread", "merged")


def shape_key(plan, s, device_name: str) -> str:
    inf = plan.info(s)
    variants, _ = bse.bse_pair_variants(plan, s)
    ids = ",".join(str(v["index"]) for v in variants)
    return (f"{device_name}|nb{inf['nb']}|dim{inf['dim']}|ng{inf['ng_max']}|npw{inf['npw_max']}|"
            f"nq{inf['nq']}|cand[{ids}]")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(plan, s, forward, q_begin=0, q_end=None, reps=3, cache_path=DEFAULT_CACHE, force=False):
    """Select the pair-kernel variant of system s: from the cache, else by timing.

    forward: a pipeline.Forward of this system (its pair workspace and rho_dir buffer are used;
    rho_dir's contents are overwritten).  Returns a dict with the chosen variant, the per-variant
    times (empty when taken from the cache) and whether the cache was used.
    """
    import torch
    variants, _ = bse.bse_pair_variants(plan, s)
    key = shape_key(plan, s, torch.cuda.get_device_name())
    cache = _load(cache_path)
    hit = cache.get(key)
    if hit is not None and not force:
        for v in variants:
            if all(v[f] == hit["variant"].get(f) for f in _FIELDS):
                bse.bse_set_pair_variant(plan, s, v["index"])
                return {"variant": v, "ms": {}, "cached": True}
    if q_end is None:
        q_end = min(plan.info(s)["nq"], q_begin + forward.qchunk)
    ms, chosen = bse.bse_autotune_pair(plan, s, forward.ws_pair, forward.rho_dir, q_begin, q_end, reps)
    best = next(v for v in variants if v["index"] == chosen)
    times = {str(v["index"]): t for v, t in zip(variants, ms)}
    cache[key] = {"variant": {f: best[f] for f in _FIELDS}, "ms": times}
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return {"variant": best, "ms": times, "cached": False}
