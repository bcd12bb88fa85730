#!/usr/bin/env python
"""Benchmark of the OTS photoionisation hot path (one A3 substep = one step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload multisource512_bb|clumpy256_mono|lognormal128_bb|stromgren32|batch64]
                    [--no-extra-configs]

A step is one substep of the second-order explicit scheme A3 (Mackey 2012,
Sect. 2.2) with criterion dt02 (K4 = 1/4, Eq. 4): trace every source, the
Eq. 4 timestep, half step, trace of the half-step state, full step with the
photon budget, on the whole grid.  Throughput is cell-substeps/s.

The default workload is 512^3 cells of lognormal hydrogen (mean 100 cm^-3,
sigma_ln = 1, Gaussian random field with P(k) ~ k^-3, seed 1205) lit by 16
blackbody sources (T uniform in 3e4-5e4 K, Q log-uniform in 1e47-1e49 s^-1,
positions uniform, seed 1205), box 2 Stromgren radii of the summed rate.  The
run is first advanced (untimed) to t0 so that the fronts exist; the timed
window starts there.  The mixed-precision path is timed (the product), the
plain FP64 path beside it on the same state, and the two are compared after
advancing both from that state to a common time.  The same line carries, in
"other_configs", the 256^3 clumpy workload and the batch of 64 uneven grids
advanced in one persistent launch per pass.

Under torchrun each rank runs its own replica of the workload on its own GPU
(independent problems, no data-path collective): weak scaling; the step time
is the maximum over ranks.  --impl reference times the CPU oracle on the host
cores instead (bounded samples of the same workload per step, one process per
core).
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-substeps/s mixed vs FP64 at ≤0.5% I-front error; % of HBM roofline"
UNIT = "cell-substeps/s"
T_END_RUN = 10.0          # end of the advance the timed substeps belong to, in t_rec (Sect. 5.1 runs 10 t_rec)

WORKLOADS = {
    "multisource512_bb": dict(
        t0=0.005, n_oct=8, k64=1,
        describe="512^3 lognormal n_H (mean 100, sigma_ln 1, P(k)~k^-3, seed 1205), 16 blackbody sources "
                 "(T 3e4-5e4 K, Q log-uniform 1e47-1e49 s^-1, random vertices, seed 1205), box 2 R_S(sum Q), "
                 "A3-dt02 (K4=1/4), t0 = 0.005 t_rec"),
    "clumpy256_mono": dict(
        t0=0.05, n_oct=8, k64=2,
        describe="256^3 lognormal (sigma_ln 1.5, seed 1203) x 200 clumps (radius 2-8 cells, overdensity 10-100, "
                 "seed 1303), monochromatic Q=1e48 at the centre vertex, box 2.5 R_S, A3-dt02, t0 = 0.05 t_rec"),
    "lognormal128_bb": dict(
        t0=0.05, n_oct=8, k64=3,
        describe="128^3 lognormal n_H (mean 100, sigma_ln 1, P(k)~k^-3, seed 1202), 4e4 K blackbody Q=1e48 "
                 "at the centre vertex, box 2.5 R_S, A3-dt02 (K4=1/4), t0 = 0.05 t_rec"),
    "stromgren32": dict(
        t0=0.05, n_oct=1, k64=3,
        describe="32^3 uniform n=100, monochromatic Q=1e48 at the corner, box 1.5 R_S, A3-dt02, t0 = 0.05 t_rec"),
    "batch64": dict(
        t0=0.02, n_oct=8, k64=2,
        describe="64 independent uniform grids, sides from {32,48,64,96,128}, n log-uniform 10-1000, Q log-uniform "
                 "1e47-1e50, monochromatic source at a random vertex, box 2 R_S each (seed 1204), A3-dt02 with a "
                 "per-grid dt, one persistent launch per pass for all grids, t0 = 0.02 t_rec of each grid"),
}


_CACHE = {}


def _workload(name):
    if name not in _CACHE:
        _CACHE[name] = _make_workload(name)
    return _CACHE[name]


def _make_workload(name):
    from paper_1201_5651_gb300 import inputs
    if name == "multisource512_bb":
        return inputs.multisource(512)
    if name == "clumpy256_mono":
        return inputs.clumpy(256, 1.5, 1203, 1303, 200, Q=1e48, box_rs=2.5, spectrum="mono")
    if name == "lognormal128_bb":
        return inputs.lognormal_bb(128, 1.0, 1202, Q=1e48, T=4e4, box_rs=2.5)
    if name == "stromgren32":
        return inputs.stromgren_corner(32)
    if name == "batch64":
        return inputs.batch(count=64, seed=1204)
    raise SystemExit(f"unknown workload {name}")


def _reff(x, dx, n_oct):
    """Radius of the sphere holding the ionised volume (the cube root of the ions, Sect. 3.2)."""
    return (3.0 * float((1.0 - x).sum()) * dx ** 3 * (8.0 / n_oct) / (4.0 * math.pi)) ** (1.0 / 3.0)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.skip = 0
        self.index = index
        self.out = os.environ.get("OOTS_CLOCKS_LOG") or os.path.join(tempfile.gettempdir(), f"oots_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.out), exist_ok=True)
            self.fh = open(self.out, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            t0 = time.time()
            self.skip = 0
            while time.time() - t0 < 5.0:
                self.fh.flush()
                n = sum(1 for _ in open(self.out))
                if n > 0:
                    self.skip = n
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for i, line in enumerate(open(self.out)):
            if i < self.skip:
                continue
            p = [q.strip() for q in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def rank_max(v, world, device):
    """Maximum of one float over all ranks (the slowest rank sets the job time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as tdist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, t_ms):
    """Whole-job throughput: the units all ranks processed over the max-over-ranks time."""
    return world * units_per_rank / (t_ms / 1e3)


KERNEL_SOURCES = ("common.cuh", "integrator.cuh", "kernels.h", "oots_internal.h", "sweep_impl.cuh", "sweep_tp.cuh",
                  "sweep_f.cu", "sweep_d.cu", "cell.cu")


def kernel_source_hash():
    """sha1 over the device sources, to tell whether ncu counters still describe the kernels."""
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1201_5651_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic(workload, kinds, tile_shape):
    """DRAM bytes (read + write) per launch, summed over the launch kinds of the
    dominant kernel, from the committed ncu summary of this workload; None
    when it is absent, was taken on other kernel sources or another tile shape."""
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    rows, sha, shape = {}, None, None
    for line in text.splitlines():
        if line.startswith("kernel sources sha1:"):
            sha = line.split(":", 1)[1].strip().strip("`")
        if line.startswith("tile shape:"):
            try:
                shape = int(line.split(":", 1)[1].strip().strip("`").split()[0])
            except ValueError:
                shape = None
        cells = [c.strip().strip("`") for c in line.strip().strip("|").split("|")]
        if len(cells) >= 3 and cells[0] in ("pack", "sweep1", "ratedt", "ratedt_verify", "half", "half_general",
                                            "sweep2", "full", "full_general"):
            try:
                rows[cells[0]] = float(cells[1]) + float(cells[2])
            except ValueError:
                pass
    if sha != kernel_source_hash() or shape != tile_shape or not all(k in rows for k in kinds):
        return None
    return sum(rows[k] for k in kinds)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def kernel_bytes_per_cell(kind, rsz, nsrc, n_array):
    """Algorithmic HBM bytes per cell of one launch of each kernel: state x (or
    the half-step state xh), density n (absent when uniform), per-source entry
    columns N.  A trace reads x and n and writes N once per source."""
    n_b = rsz if n_array else 0
    return {
        "sweep1": nsrc * (rsz + n_b + rsz),            # read x (+n), write N1, per source
        "sweep2": nsrc * (rsz + n_b + rsz),            # read xh (+n), write N2, per source
        "ratedt": rsz + n_b + nsrc * rsz,              # read x, n, N1
        "half": rsz + n_b + nsrc * rsz + rsz,          # read x, n, N1, write xh
        "full": rsz + n_b + nsrc * rsz + rsz,          # read x, n, N2, write x
    }.get(kind, 0)


def step_bytes_per_cell(nsrc, n_array):
    """Algorithmic HBM bytes per cell of a whole A3 mixed substep in its fused form
    (the dt criterion folded into the first trace, both integrations into the
    second): 28 B for one source and a density array, 20 B with uniform
    density, 28 S + 32 B for S sources."""
    if nsrc <= 1:
        return 28 if n_array else 20
    return 28 * nsrc + 32


def _describe_tile(shape, cell_block=None, nsrc=1):
    """The sweep's tile shape and kernel, and (when given) the threads per block of
    the closed-form per-cell passes (0 = the library's default for the source count)."""
    from paper_1201_5651_gb300 import oots
    if shape is None:
        return None
    dims = oots.oots_tile_shape_info(shape)[1]
    d = {"id": shape, "dims": list(dims), "kernel": "throughput" if shape in (7, 8) else "pipelined"}
    if cell_block is not None:
        d["cell_block"] = cell_block if cell_block else (128 if nsrc > 1 else 256)
    return d


def _roofline(prof_avg, ms_per_step, ncell, nsrc, n_array, workload, tile_shape):
    peak, peak_src = _peaks()
    # each pass with its helper launches: a trace with the packing of its input
    # (throughput tiles), the Eq. 4 pass with its verifying re-run, an
    # integration with its general pass
    parts = {"half": ["half", "half_general"], "full": ["full", "full_general"],
             "ratedt": ["ratedt", "ratedt_verify"], "sweep1": ["sweep1", "pack"], "sweep2": ["sweep2", "pack"]}
    label = {"half": " (closed-form + general pass)", "full": " (closed-form + general pass)",
             "ratedt": " (pass + verifying pass)", "sweep1": " (n x packing + sweep)", "sweep2": " (n x packing + sweep)"}
    kern = {k: sum(prof_avg.get(q, 0.0) for q in v) for k, v in parts.items() if v[0] in prof_avg}
    dom = max(kern, key=lambda k: kern[k])
    bpc = kernel_bytes_per_cell(dom, 4, nsrc, n_array)
    achieved = bpc * ncell / (kern[dom] / 1e3) / 1e9
    sbytes = step_bytes_per_cell(nsrc, n_array)
    kinds = [q for q in parts[dom] if q in prof_avg]
    return {"bound": "hbm", "kernel": dom + (label[dom] if len(kinds) > 1 else ""),
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": _traffic(workload, kinds, tile_shape),
            "traffic_unit": "bytes per launch (ncu dram read + write, profiles/)", "peak_source": peak_src,
            "bytes_per_cell": bpc, "kernel_ms": kern[dom],
            "step_bytes_per_cell": sbytes,
            "step_frac": sbytes * ncell / (ms_per_step / 1e3) / 1e9 / peak,
            "impl_step_bytes_per_cell": sum(kernel_bytes_per_cell(k, 4, nsrc, n_array)
                                            for k in ("sweep1", "ratedt", "half", "sweep2", "full"))}


def _cpu_info():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
        else:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


# ------------------------------------------------------------------------------------------ the CUDA path
def _timed_substeps(run_one, sync, stream, flush, steps, warmup):
    import torch
    for _ in range(warmup):
        run_one()
    sync()
    evs = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()                        # evict L2 between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        run_one()
        with torch.cuda.stream(stream):
            e1.record(stream)
        evs.append((e0, e1))
    sync()
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in evs)


def _tuned_context(w, precision, dev, stream, args, devname):
    """A context on `stream`, its tile shape chosen by the autotuner at t = 0 (the
    tuning substeps are then undone: state, time and budget reset)."""
    from paper_1201_5651_gb300 import autotune, oots
    c = oots.Context.from_workload(w, precision, device=dev, scheme=oots.OOTS_A3, K4=0.25)
    c.set_stream(stream.cuda_stream)
    shape = None
    if args.shape >= 0:
        try:
            c.set_tile_shape(args.shape)
            c.compute_dt()                          # builds the launch set: refuses a shape that does not fit
            shape = args.shape
        except oots.OotsError:
            shape = None
    cb = 0
    if shape is None:
        shape = autotune.tune(c, devname, len(w.sources), use_cache=not args.retune)
        cb = autotune.lookup_cell_block(devname, c.precision, autotune.plane_class(w.nx, w.ny, w.nz, len(w.sources)))
    c.set_neutral_fraction(w.x0)
    c.set_time(0.0)
    c.reset_budget()
    return c, shape, cb


def bench_single(args, name, steps, warmup, rank, world, dev, flush, devname, with_fp64=True):
    import torch
    from paper_1201_5651_gb300 import oots
    spec = WORKLOADS[name]
    w = _workload(name)
    trec = w.t_rec
    t_end = T_END_RUN * trec
    s = torch.cuda.Stream(device=dev)
    cm, shape, cblock = _tuned_context(w, "mixed", dev, s, args, devname)
    t_dev0 = time.perf_counter()
    _, ndev = cm.advance(spec["t0"] * trec)            # untimed: develop the fronts
    t_dev = time.perf_counter() - t_dev0
    t0 = cm.get_time()[0]
    x_t0 = cm.get_neutral_fraction()
    ms = _timed_substeps(lambda: cm.run_substeps(1, t_end), cm.synchronize, s, flush, steps, warmup)
    ms = rank_max(ms, world, f"cuda:{dev}")
    value = job_rate(w.ncell * steps, world, ms)
    prof = {}
    for _ in range(3):
        for k, v in cm.profile_substep():
            prof.setdefault(k, []).append(v)
    prof_avg = {k: sum(v) / len(v) for k, v in prof.items()}
    launches = sum(len(v) for v in prof.values()) // 3
    nsrc = len(w.sources)
    out = {"workload": name, "describe": spec["describe"], "ncell": w.ncell, "nsrc": nsrc,
           "value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
           "t0_over_trec": t0 / trec, "develop_substeps": ndev, "develop_s": t_dev,
           "tile_shape": _describe_tile(shape, cblock, len(w.sources)),
           "roofline": _roofline(prof_avg, ms / steps, w.ncell, nsrc, w.uniform_n is None, name, shape),
           "kernel_ms": prof_avg, "launches_per_substep": launches,
           "cell_sweeps_per_s": 2.0 * value}
    if with_fp64:
        # the plain FP64 path on the same state, then both paths from that state to a common time
        cf = oots.Context.from_workload(w, "fp64", device=dev, scheme=oots.OOTS_A3, K4=0.25)
        sf = torch.cuda.Stream(device=dev)
        cf.set_stream(sf.cuda_stream)
        if shape is not None:
            try:
                cf.set_tile_shape(shape)
                cf.compute_dt()
            except oots.OotsError:
                cf.set_tile_shape(0)
        cf.set_neutral_fraction(x_t0)
        cf.set_time(t0)
        # the entry columns of the same state on both paths (float-float against double)
        col_src = sorted({0, nsrc - 1})
        cf.compute_dt()
        col64 = {s_: cf.get_column_density(s_) for s_ in col_src}
        k64 = spec["k64"]
        ms64 = _timed_substeps(lambda: cf.run_substeps(1, t_end), cf.synchronize, sf, flush, k64, 1)
        ms64 = rank_max(ms64, world, f"cuda:{dev}")
        tf = cf.get_time()[0]
        xf = cf.get_neutral_fraction()
        del cf
        torch.cuda.empty_cache()
        cm.set_neutral_fraction(x_t0)
        cm.set_time(t0)
        cm.compute_dt()
        col_err, col_p999 = 0.0, 0.0
        for s_ in col_src:
            nm = cm.get_column_density(s_)
            rel = np.abs(nm - col64[s_]) / np.maximum(col64[s_], 1e10)
            col_err = max(col_err, float(rel.max()))
            col_p999 = max(col_p999, float(np.percentile(rel, 99.9)))
            del nm, rel
        del col64
        cm.advance(tf)
        xm = cm.get_neutral_fraction()
        rm, rf = _reff(xm, w.dx, spec["n_oct"]), _reff(xf, w.dx, spec["n_oct"])
        out["fp64"] = {"value": job_rate(w.ncell * k64, world, ms64), "ms_per_step": ms64 / k64, "steps": k64,
                       "warmup": 1, "tile_shape": _describe_tile(shape)}
        out["mixed_over_fp64"] = value / out["fp64"]["value"]
        out["accuracy_vs_fp64"] = {
            "from_t_over_trec": t0 / trec, "t_over_trec": tf / trec, "fp64_substeps": k64 + 1,
            "reff_rel_err": abs(rm / rf - 1.0),
            "ionised_volume_rel_err": abs(float((1 - xm).sum()) / float((1 - xf).sum()) - 1.0),
            "max_abs_dx": float(np.max(np.abs(xm - xf))),
            "column_rel_err": col_err,
            "column_rel_err_p999": col_p999,
            "column_rel_err_sources": col_src}
    # end to end through the C ABI with host buffers: each step uploads the state
    # (oots_set_neutral_fraction), runs one substep and reads the state back
    # (oots_get_neutral_fraction), from and into pinned host memory
    h_in = torch.from_numpy(np.ascontiguousarray(x_t0.ravel())).pin_memory().numpy()
    h_out = torch.empty(w.ncell, dtype=torch.float64).pin_memory().numpy()
    ke = max(3, min(steps, 5))
    cm.set_time(t0)
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(ke):
        cm.set_neutral_fraction(h_in)
        cm.run_substeps(1, t_end)
        cm.get_neutral_fraction_into(h_out)
    t_e2e = rank_max(time.perf_counter() - te0, world, f"cuda:{dev}")
    out["e2e"] = {"value": job_rate(w.ncell * ke, world, t_e2e * 1e3), "unit": UNIT, "steps": ke,
                  "h2d_bytes_per_step": 8 * w.ncell, "d2h_bytes_per_step": 8 * w.ncell,
                  "path": "oots_set_neutral_fraction + oots_run_substeps + oots_get_neutral_fraction, float64 host "
                          "buffers (pinned)"}
    del cm
    torch.cuda.empty_cache()
    return out


def bench_batch(args, steps, warmup, rank, world, dev, flush, devname):
    import torch
    from paper_1201_5651_gb300 import autotune, oots
    spec = WORKLOADS["batch64"]
    ws = _workload("batch64")
    s = torch.cuda.Stream(device=dev)
    ctxs = []
    for w in ws:
        c = oots.Context.from_workload(w, "mixed", device=dev, scheme=oots.OOTS_A3, K4=0.25)
        c.set_stream(s.cuda_stream)
        ctxs.append(c)
    shape = args.shape if args.shape >= 0 else autotune.tune_batch(ctxs, ws, devname, use_cache=not args.retune)
    nside = max(max(w.nx, w.ny, w.nz) for w in ws)
    cblock = 0 if args.shape >= 0 else autotune.lookup_cell_block(
        devname, oots.OOTS_MIXED, autotune.plane_class(nside, nside, nside, max(len(w.sources) for w in ws), len(ws)))
    for c, w in zip(ctxs, ws):
        if shape is not None:
            c.set_tile_shape(shape)
    b = oots.Batch(ctxs)
    t_dev0 = time.perf_counter()
    nsub = b.advance([spec["t0"] * w.t_rec for w in ws])
    t_dev = time.perf_counter() - t_dev0
    t_end = [T_END_RUN * w.t_rec for w in ws]
    ncell = sum(w.ncell for w in ws)
    ms = _timed_substeps(lambda: b.run_substeps(1, t_end), ctxs[0].synchronize, s, flush, steps, warmup)
    ms = rank_max(ms, world, f"cuda:{dev}")
    value = job_rate(ncell * steps, world, ms)
    peak, peak_src = _peaks()
    sbytes = step_bytes_per_cell(1, False)
    out = {"workload": "batch64", "describe": spec["describe"], "ngrids": len(ws), "ncell": ncell,
           "value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
           "develop_substeps": {"min": int(min(nsub)), "max": int(max(nsub))}, "develop_s": t_dev,
           "tile_shape": _describe_tile(shape, cblock, max(len(w.sources) for w in ws)),
           "roofline": {"bound": "hbm", "kernel": "whole substep (all kernels, one launch each for the 64 grids)",
                        "achieved": sbytes * ncell / (ms / steps / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": sbytes * ncell / (ms / steps / 1e3) / 1e9 / peak, "traffic": None,
                        "peak_source": peak_src, "step_bytes_per_cell": sbytes}}
    b.close()
    del b, ctxs
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dev = local_rank
    devname = torch.cuda.get_device_name(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{dev}")   # 256 MB > L2

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()

    cidx = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(dev)).split(",")[0]) if "CUDA_VISIBLE_DEVICES" in os.environ else dev
    clocks = Clocks(cidx)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    if args.workload == "batch64":
        main = bench_batch(args, args.steps, args.warmup, rank, world, dev, flush, devname)
    else:
        main = bench_single(args, args.workload, args.steps, args.warmup, rank, world, dev, flush, devname)
    clk = clocks.stop()
    barrier()
    extra = {}
    if not args.no_extra_configs and args.workload == "multisource512_bb":
        k = max(3, min(args.steps, 20))
        extra["clumpy256_mono"] = bench_single(args, "clumpy256_mono", k, args.warmup, rank, world, dev, flush, devname)
        extra["batch64"] = bench_batch(args, k, args.warmup, rank, world, dev, flush, devname)
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 state and rates; float-float (~48-bit) columns; f64 photon budget",
        "data": "synthetic (seeded generators)",
        "config": {"workload": main["workload"], "describe": main["describe"], "ncell": main["ncell"],
                   "nsrc": main.get("nsrc", 1), "scheme": "A3", "criterion": "dt02 (K4=1/4)", "precision": "mixed",
                   "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}",
                   "tile_shape": main["tile_shape"], "t0_over_trec": main.get("t0_over_trec")},
    }
    for k in ("fp64", "mixed_over_fp64", "cell_sweeps_per_s", "accuracy_vs_fp64", "roofline", "kernel_ms", "e2e",
              "develop_substeps", "develop_s"):
        if k in main:
            line[k] = main[k]
    line["gpu_launches"] = main.get("launches_per_substep", 0) * args.steps
    line["clocks"] = clk
    if extra:
        line["other_configs"] = extra
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    return line


# ------------------------------------------------------------------------------------------ the CPU oracle
def _oracle_crops(workload, m, count):
    """`count` m^3 crops of the workload with their sources, for the oracle.
    Single-source workloads: crops around the source vertex (shifted per
    crop).  The 16-source workload: crops spread over the box, each with all
    16 sources moved by the box-to-crop scale, so every cell sees 16 sources."""
    w = _workload(workload)
    if isinstance(w, list):
        out = []
        for g in range(count):
            wg = w[g % len(w)]
            n = min(m, wg.nx)
            s = wg.sources[0]
            v = [min(max(int(round(p)), 0), wg.nx) for p in s.pos]
            lo = [min(max(q - n // 2, 0), wg.nx - n) for q in v]
            sub = wg.nH[lo[2]:lo[2] + n, lo[1]:lo[1] + n, lo[0]:lo[0] + n].copy()
            pos = tuple(float(v[q] - lo[q]) for q in range(3))
            out.append((n, wg.dx, sub, [(pos, s.Q, s.spectrum, s.T)], wg.alpha, wg.sigma0, wg.tau0, wg.t_rec))
        return out
    rng = np.random.default_rng(7)
    out = []
    for c in range(count):
        if len(w.sources) > 1:
            lo = [int(q) for q in rng.integers(0, w.nx - m, 3)]
            scale = m / w.nx
            srcs = [(tuple(p * scale for p in s.pos), s.Q, s.spectrum, s.T) for s in w.sources]
        elif workload == "stromgren32":
            lo = [0, 0, 0]
            srcs = [((0.0, 0.0, 0.0), w.sources[0].Q, w.sources[0].spectrum, w.sources[0].T)]
        else:
            shift = (c % 3) - 1
            lo = [w.nx // 2 - m // 2 + shift] * 3
            s = w.sources[0]
            srcs = [(tuple(float(s.pos[q] - lo[q]) for q in range(3)), s.Q, s.spectrum, s.T)]
        sub = w.nH[lo[2]:lo[2] + m, lo[1]:lo[1] + m, lo[0]:lo[0] + m].copy()
        out.append((m, w.dx, sub, srcs, w.alpha, w.sigma0, w.tau0, w.t_rec))
    return out


def _oracle_job(job):
    """One process: the oracle's A3-dt02 substeps on one crop; returns (cells x substeps, seconds)."""
    import oracle
    (m, dx, sub, srcs, alpha, sigma0, tau0, trec), nsteps = job
    P = oracle.Problem(m, m, m, dx, sub, srcs, alpha=alpha, sigma0=sigma0, tau0=tau0)
    x = np.full((m, m, m), 1 - 1e-6)
    t = 0.0
    t0 = time.perf_counter()
    for _ in range(nsteps):
        t, *_ = P.substep(x, t, 1e30, scheme=3, K4=0.25)
    return m ** 3 * nsteps, time.perf_counter() - t0


def _oracle_sample_spec(workload):
    # crop side and substeps per crop: about 5-15 s of work per process
    return {"multisource512_bb": (16, 1), "clumpy256_mono": (24, 2), "lognormal128_bb": (24, 2),
            "stromgren32": (16, 2), "batch64": (16, 2)}.get(workload, (16, 2))


def _run_oracle_pool(workload, nproc):
    m, nsteps = _oracle_sample_spec(workload)
    jobs = [(c, nsteps) for c in _oracle_crops(workload, m, nproc)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(nproc) as pool:
        res = pool.map(_oracle_job, jobs)
    wall = time.perf_counter() - t0
    units = sum(r[0] for r in res)
    return units, wall, m, nsteps


def cpu_baseline(args):
    import oracle
    oracle.build()
    nproc = os.cpu_count() or 1
    units, wall, m, nsteps = _run_oracle_pool(args.workload, nproc)
    info = _cpu_info()
    return {"value": units / wall, "unit": UNIT, "cores": nproc, "kind": "oracle", **info,
            "sample": f"{nproc} processes (one per host core), each {nsteps} A3-dt02 substep(s) of the FP64 oracle "
                      f"from the neutral start on an {m}^3 crop of the {args.workload} workload"
                      + (" with all 16 sources moved into the crop by the box-to-crop scale"
                         if args.workload == "multisource512_bb" else "")
                      + f"; {wall:.1f} s wall"}


def run_reference(args):
    """The CPU oracle on the host cores: each step one pool of A3 substeps on crops
    of the workload, one process per core."""
    import oracle
    oracle.build()
    nproc = os.cpu_count() or 1
    for _ in range(args.warmup):
        _run_oracle_pool(args.workload, nproc)
    units = 0
    wall = 0.0
    for _ in range(args.steps):
        u, wl, m, nsteps = _run_oracle_pool(args.workload, nproc)
        units += u
        wall += wl
    v = units / wall
    info = _cpu_info()
    sample = (f"each step: {nproc} processes (one per host core), each {nsteps} A3-dt02 substep(s) of the FP64 "
              f"oracle on an {m}^3 crop of the {args.workload} workload")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generators)",
            "config": {"workload": args.workload, "describe": WORKLOADS[args.workload]["describe"],
                       "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": sample, **info},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="multisource512_bb", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-configs", action="store_true", help="skip the 256^3 and 64-grid lines")
    ap.add_argument("--shape", type=int, default=-1, help="tile shape id (-1: autotuned)")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
