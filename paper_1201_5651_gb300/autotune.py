"""Autotuner for a substep's launch shapes: the sweep's tile shape and kernel,
and the block size of the closed-form per-cell passes.

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
precision and class.  On the chosen shape it then times the closed-form
per-cell passes (the dt criterion, the half and the full step) with 128- and
256-thread blocks: small blocks hold up fewer cells behind a slow one at their
barriers, large ones set up fewer blocks, and which wins depends on how
uneven the per-cell work is (many sources, fronts).
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


def lookup_cell_block(device_name: str, precision: int, klass: str, path: str = CACHE) -> int:
    """The tuned block size of the closed-form passes (0: none tuned, the library's default)."""
    e = _load_cache(path).get(cache_key(device_name, precision, klass))
    return 0 if e is None else int(e.get("cell_block", 0))


CELL_KINDS = ("ratedt", "ratedt_verify", "half", "full")
CELL_BLOCKS = (128, 256)


def _tune_cell_block(ctx: "oots.Context", repeats: int) -> Dict[int, float]:
    """Closed-form pass time of one substep per block size (ms)."""
    times = {}
    for bs in CELL_BLOCKS:
        try:
            ctx.set_cell_block(bs)
            ctx.profile_substep()
            best = None
            for _ in range(repeats):
                t = sum(ms for k, ms in ctx.profile_substep() if k in CELL_KINDS)
                best = t if best is None else min(best, t)
            times[bs] = best
        except oots.OotsError:
            continue
    return times


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
            cb = lookup_cell_block(device_name, ctx.precision, klass, path)
            if cb:
                ctx.set_cell_block(cb)
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
    ctimes = _tune_cell_block(ctx, repeats)
    cb = min(ctimes, key=ctimes.get) if ctimes else 0
    ctx.set_cell_block(cb)
    if verbose:
        print({sh: round(v, 4) for sh, v in times.items()}, {b: round(v, 4) for b, v in ctimes.items()})
    _store(key, {"shape": choice, "dims": oots.oots_tile_shape_info(choice)[1], "class": klass,
                 "sweep_ms": {str(k): v for k, v in times.items()}, "cell_block": cb,
                 "cell_ms": {str(k): v for k, v in ctimes.items()}}, path)
    return choice


def tune_batch(ctxs: Sequence["oots.Context"], workloads, device_name: str, repeats: int = 2,
               use_cache: bool = True, path: str = CACHE) -> Optional[int]:
    """Time whole batched substeps of the contexts for every tile shape, then
    for each block size of the closed-form passes on the fastest shape; keep
    the fastest of each (the block size is set on the contexts, the shape
    returned).  The contexts' states and times are restored afterwards."""
    nside = max(max(w.nx, w.ny, w.nz) for w in workloads)
    nsrc = max(len(w.sources) for w in workloads)
    klass = plane_class(nside, nside, nside, nsrc, len(ctxs))
    prec = ctxs[0].precision
    key = cache_key(device_name, prec, klass)
    if use_cache:
        hit = lookup(device_name, prec, klass, path)
        if hit is not None:
            cb = lookup_cell_block(device_name, prec, klass, path)
            if cb:
                for c in ctxs:
                    c.set_cell_block(cb)
            return hit
    t_end = [10.0 * w.t_rec for w in workloads]

    def timed(sh, cb):
        for c in ctxs:
            c.set_tile_shape(sh)
            c.set_cell_block(cb)
        b = oots.Batch(ctxs)
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
            return best * 1e3
        finally:
            b.close()

    times, ctimes = {}, {}
    for sh in _shapes():
        try:
            times[sh] = timed(sh, 0)
        except oots.OotsError:
            continue
    choice = min(times, key=times.get) if times else None
    if choice is not None:
        for cb in CELL_BLOCKS:
            try:
                ctimes[cb] = timed(choice, cb)
            except oots.OotsError:
                continue
    cb = min(ctimes, key=ctimes.get) if ctimes else 0
    for c, w in zip(ctxs, workloads):
        c.set_cell_block(cb)
        c.set_neutral_fraction(w.x0)
        c.set_time(0.0)
        c.reset_budget()
    if choice is None:
        return None
    _store(key, {"shape": choice, "dims": oots.oots_tile_shape_info(choice)[1], "class": klass,
                 "substep_ms": {str(k): v for k, v in times.items()}, "cell_block": cb,
                 "cell_substep_ms": {str(k): v for k, v in ctimes.items()}}, path)
    return choice
