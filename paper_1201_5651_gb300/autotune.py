"""Autotuner for the wavefront sweep's tile shape.

For a given grid (size, precision, sources) every tile shape the device can
run is timed on one eager substep (per-launch CUDA events through
oots_profile_substep) and the fastest sweep is kept.  Results are cached as
JSON keyed by device name, precision, grid shape and source count, so a
workload is tuned once per machine.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional

from . import oots

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")


def _key(ctx: "oots.Context", device_name: str, nsrc: int) -> str:
    nz, ny, nx = ctx.shape
    prec = "fp64" if ctx.precision == oots.OOTS_FP64 else "mixed"
    return f"{device_name}|{prec}|{nx}x{ny}x{nz}|S{nsrc}"


def _load_cache() -> Dict[str, dict]:
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def tune(ctx: "oots.Context", device_name: str, nsrc: int, repeats: int = 2, use_cache: bool = True,
         verbose: bool = False) -> Optional[int]:
    """Time every tile shape on ctx (which it advances by a few substeps) and
    select the fastest for the sweep; returns the chosen shape."""
    key = _key(ctx, device_name, nsrc)
    cache = _load_cache()
    if use_cache and key in cache:
        ctx.set_tile_shape(cache[key]["shape"])
        return cache[key]["shape"]
    nshape, _ = oots.oots_tile_shape_info(0)
    times = {}
    for sh in range(nshape):
        try:
            ctx.set_tile_shape(sh)
            ctx.profile_substep()                     # build + warm up this shape
            best = None
            for _ in range(repeats):
                prof = dict()
                for k, ms in ctx.profile_substep():
                    prof[k] = prof.get(k, 0.0) + ms
                t = sum(v for k, v in prof.items() if k.startswith("sweep"))
                best = t if best is None else min(best, t)
            times[sh] = best
        except oots.OotsError:
            continue                                  # shape does not fit at this precision
    if not times:
        return None
    choice = min(times, key=times.get)
    ctx.set_tile_shape(choice)
    if verbose:
        print({oots.oots_tile_shape_info(k)[1]: round(v, 4) for k, v in times.items()})
    cache[key] = {"shape": choice, "dims": oots.oots_tile_shape_info(choice)[1], "sweep_ms": times}
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        json.dump(cache, open(CACHE, "w"), indent=1)
    except OSError:
        pass
    return choice
