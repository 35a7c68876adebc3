"""Autotuned pair-kernel tile shapes with a JSON cache keyed by device and problem shape.

The choice for a shape (device name, real-space grid, band counts, sphere sizes) is measured
once by bse_autotune_pair on a range of q points and stored in a JSON file; later plans of the
same shape reuse it without timing.  For a mixed-precision build the tensor-core route of the
direct densities (BSE_PD_TENSOR) can be a further candidate: it is timed on the same q range,
through the same C ABI call the build makes, against the fastest variant.  Marshalling and
bookkeeping only: every kernel runs in the CUDA library.
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


def _time_tensor(plan, s, forward, q_begin, q_end, reps):
    """Milliseconds per call of the tensor-core direct densities on [q_begin, q_end) (CUDA events)."""
    import torch
    flags = bse.BSE_PD_DIRECT | bse.BSE_PD_TENSOR
    call = lambda: bse.bse_pair_densities(plan, s, flags, None, None, None, None, forward.rho_dir,  # noqa: E731
                                          q_begin, q_end, forward.ws_pair)
    call()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        call()
    b.record()
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    return a.elapsed_time(b) / reps


def tune(plan, s, forward, q_begin=0, q_end=None, reps=3, cache_path=DEFAULT_CACHE, force=False,
         with_tensor=False):
    """Select the pair-kernel variant of system s: from the cache, else by timing.

    forward: a pipeline.Forward of this system (its pair workspace and rho_dir buffer are used;
    rho_dir's contents are overwritten; the real-space and coefficient images must be in the pair
    workspace).  with_tensor (mixed-precision builds): also time the tensor-core route where the
    system has it and record the faster of the two in forward.tensor_choice, which Forward.build
    then follows.  Returns a dict with the chosen variant, the per-variant times (empty when taken
    from the cache), whether the cache was used and, with with_tensor, "tensor" (the route chosen).
    """
    import torch
    variants, _ = bse.bse_pair_variants(plan, s)
    key = shape_key(plan, s, torch.cuda.get_device_name())
    tensor_ok = with_tensor and bool(plan.info(s)["tensor_pair"])
    if tensor_ok:
        key += f"|tensor|qc{forward.qchunk}"
    cache = _load(cache_path)
    hit = cache.get(key)
    if hit is not None and not force:
        for v in variants:
            if all(v[f] == hit["variant"].get(f) for f in _FIELDS):
                bse.bse_set_pair_variant(plan, s, v["index"])
                out = {"variant": v, "ms": {}, "cached": True}
                if with_tensor:
                    forward.tensor_choice = bool(hit.get("tensor", False))
                    out["tensor"] = forward.tensor_choice
                return out
    if q_end is None:
        q_end = min(plan.info(s)["nq"], q_begin + forward.qchunk)
    ms, chosen = bse.bse_autotune_pair(plan, s, forward.ws_pair, forward.rho_dir, q_begin, q_end, reps)
    best = next(v for v in variants if v["index"] == chosen)
    times = {str(v["index"]): t for v, t in zip(variants, ms)}
    entry = {"variant": {f: best[f] for f in _FIELDS}, "ms": times}
    tensor = False
    if tensor_ok:
        t_tensor = _time_tensor(plan, s, forward, q_begin, q_end, reps)
        times["tensor"] = t_tensor
        tensor = t_tensor < times[str(chosen)]
        entry["tensor"] = tensor
    if with_tensor:
        forward.tensor_choice = tensor
    cache[key] = entry
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    out = {"variant": best, "ms": times, "cached": False}
    if with_tensor:
        out["tensor"] = tensor
    return out
