"""Autotuner for the wavefront sweep: tile shape and sweep kernel.

The sweep has two kernels (the pipelined one, whose tiles hand their faces on
plane chunk by chunk, and the throughput one, which traces whole 8^3 tiles)
and several tile shapes.  Which is fastest depends on how many tiles the
wavefront keeps in flight per diagonal plane: a single source on a 128^3 grid
leaves most of the machine idle, so the pipelined kernel's early hand-off
wins; sixteen sources on 512^3 give thousands of tiles per plane, and the
lean throughput tiles win.  The tuner therefore keys its choice on a
plane-size class of the launch -- the largest grid side (rounded up to a
power of two), the number of sources per grid and the number of grids, each
bucketed -- rather than on the exact grid, times every shape the device can
run on one substep (per-launch CUDA events through oots_profile_substep, or
whole batched substeps), and caches the fastest as JSON keyed by device name,
precision and class.
"""
from __future__ import annotations

import json
import os
import time
from typing import Dict, Optional, Sequence

from . import oots

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")


def _bucket(v: int, edges: Sequence[int]) -> int:
    """Smallest edge >= v (the last edge for anything larger)."""
    for e in edges:
        if v <= e:
            return e
    return edges[-1]


def plane_class(nx: int, ny: int, nz: int, nsrc: int, ngrids: int = 1) -> str:
    """The class of a launch for tuning: side (next power of two of the largest
    side, at least 16), sources per grid and grids, bucketed.  Together they set
    the number of tiles in flight on a wavefront plane."""
    side = 16
    while side < max(nx, ny, nz):
        side *= 2
    return f"side{side}|S{_bucket(nsrc, (1, 4, 16, 64))}|G{_bucket(ngrids, (1, 8, 64, 1024))}"


def cache_key(device_name: str, precision: int, klass: str) -> str:
    prec = "fp64" if precision == oots.OOTS_FP64 else "mixed"
    return f"{device_name}|{prec}|{klass}"


def _load_cache(path: str = CACHE) -> Dict[str, dict]:
    try:
        return json.load(open(path))
    except Exception:
        return {}


def _store(key: str, entry: dict, path: str = CACHE) -> None:
    cache = _load_cache(path)
    cache[key] = entry
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        json.dump(cache, open(path, "w"), indent=1)
    except OSError:
        pass


def lookup(device_name: str, precision: int, klass: str, path: str = CACHE) -> Optional[int]:
    e = _load_cache(path).get(cache_key(device_name, precision, klass))
    return None if e is None else int(e["shape"])


def _shapes():
    n, _ = oots.oots_tile_shape_info(0)
    return range(n)


def tune(ctx: "oots.Context", device_name: str, nsrc: int, repeats: int = 2, use_cache: bool = True,
         verbose: bool = False, path: str = CACHE) -> Optional[int]:
    """Time every tile shape on ctx (which it advances by a few substeps) and
    select the fastest for the sweep; returns the chosen shape."""
    nz, ny, nx = ctx.shape
    klass = plane_class(nx, ny, nz, nsrc)
    key = cache_key(device_name, ctx.precision, klass)
    if use_cache:
        hit = lookup(device_name, ctx.precision, klass, path)
        if hit is not None:
            ctx.set_tile_shape(hit)
            return hit
    times = {}
    for sh in _shapes():
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
        print({sh: round(v, 4) for sh, v in times.items()})
    _store(key, {"shape": choice, "dims": oots.oots_tile_shape_info(choice)[1], "class": klass,
                 "sweep_ms": {str(k): v for k, v in times.items()}}, path)
    return choice


def tune_batch(ctxs: Sequence["oots.Context"], workloads, device_name: str, repeats: int = 2,
               use_cache: bool = True, path: str = CACHE) -> Optional[int]:
    """Time whole batched substeps of the contexts for every tile shape and keep
    the fastest.  The contexts' states and times are restored afterwards."""
    nside = max(max(w.nx, w.ny, w.nz) for w in workloads)
    nsrc = max(len(w.sources) for w in workloads)
    klass = plane_class(nside, nside, nside, nsrc, len(ctxs))
    prec = ctxs[0].precision
    key = cache_key(device_name, prec, klass)
    if use_cache:
        hit = lookup(device_name, prec, klass, path)
        if hit is not None:
            return hit
    t_end = [10.0 * w.t_rec for w in workloads]
    times = {}
    for sh in _shapes():
        try:
            for c in ctxs:
                c.set_tile_shape(sh)
            b = oots.Batch(ctxs)
        except oots.OotsError:
            continue
        try:
            b.run_substeps(1, t_end)
            ctxs[0].synchronize()
            best = None
            for _ in range(repeats):
                t0 = time.perf_counter()
                b.run_substeps(1, t_end)
                ctxs[0].synchronize()
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            times[sh] = best * 1e3
        except oots.OotsError:
            pass
        finally:
            b.close()
    for c, w in zip(ctxs, workloads):
        c.set_neutral_fraction(w.x0)
        c.set_time(0.0)
        c.reset_budget()
    if not times:
        return None
    choice = min(times, key=times.get)
    _store(key, {"shape": choice, "dims": oots.oots_tile_shape_info(choice)[1], "class": klass,
                 "substep_ms": {str(k): v for k, v in times.items()}}, path)
    return choice
