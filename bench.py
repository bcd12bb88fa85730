#!/usr/bin/env python
"""Benchmark of the OTS photoionisation hot path (one A3 substep = one step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload lognormal128_bb|clumpy256_mono|stromgren32]

A step is one substep of the second-order explicit scheme A3 (Mackey 2012,
Sect. 2.2): trace, Eq. 4 timestep, half step, trace of the half-step state,
full step with the photon budget, on the whole grid.  Throughput is
cell-substeps/s.  The default workload is a 128^3 lognormal hydrogen field
(mean 100 cm^-3, sigma_ln = 1, Gaussian random field with P(k) ~ k^-3,
seed 1202) lit by a 4e4 K blackbody (Q = 1e48 s^-1) at the centre vertex,
box 2.5 Stromgren radii, criterion dt02 (K4 = 1/4).  Before timing, the run
is advanced (untimed) to t0 = 0.05 t_rec so the ionisation front is developed.
The mixed-precision path is timed (the product), the plain FP64 path beside
it, and the two are compared on the front radius at a common time.

Under torchrun each rank runs its own replica of the workload on its own GPU
(independent problems, no data-path collective): weak scaling; the step time
is the maximum over ranks.  --impl reference times the CPU oracle on the
host cores instead (a bounded crop of the same workload per step).
"""
import argparse
import json
import math
import os
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


def _workload(name):
    from paper_1201_5651_gb300 import inputs
    if name == "lognormal128_bb":
        return inputs.lognormal_bb(128, 1.0, 1202, Q=1e48, T=4e4, box_rs=2.5)
    if name == "clumpy256_mono":
        return inputs.clumpy(256, 1.5, 1203, 1303, 200, Q=1e48, box_rs=2.5, spectrum="mono")
    if name == "stromgren32":
        return inputs.stromgren_corner(32)
    raise SystemExit(f"unknown workload {name}")


def _describe(name):
    return {
        "lognormal128_bb": "128^3 lognormal n_H (mean 100, sigma_ln 1, P(k)~k^-3, seed 1202), 4e4 K blackbody Q=1e48 "
                           "at the centre vertex, box 2.5 R_S, A3-dt02 (K4=1/4), t0 = 0.05 t_rec",
        "clumpy256_mono": "256^3 lognormal (sigma_ln 1.5, seed 1203) x 200 clumps, monochromatic Q=1e48 at the centre, "
                          "A3-dt02, t0 = 0.05 t_rec",
        "stromgren32": "32^3 uniform n=100, monochromatic Q=1e48 at the corner, box 1.5 R_S, A3-dt02, t0 = 0.05 t_rec",
    }[name]


def _reff(x, dx, n_oct):
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
            # wait for the sampler's first line, then count only the lines that
            # arrive from here on (the timed region starts right after this)
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


KERNEL_SOURCES = ("common.cuh", "integrator.cuh", "kernels.h", "oots_internal.h", "sweep_impl.cuh", "sweep_f.cu", "sweep_d.cu", "cell.cu")
TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "dram_traffic_lognormal128_mixed.md")


def kernel_source_hash():
    """sha1 over the device sources, to tell whether ncu counters still describe the kernels."""
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1201_5651_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic(kinds):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch summed over the launch kinds of
    the dominant kernel, from the committed ncu summary; None when that summary is absent or was
    taken on other kernel sources."""
    try:
        text = open(TRAFFIC_SUMMARY).read()
    except OSError:
        return None
    rows, sha = {}, None
    for line in text.splitlines():
        if line.startswith("kernel sources sha1:"):
            sha = line.split(":", 1)[1].strip().strip("`")
        cells = [c.strip().strip("`") for c in line.strip().strip("|").split("|")]
        if len(cells) >= 3 and cells[0] in ("sweep1", "ratedt", "half", "half_general", "sweep2", "full",
                                            "full_general"):
            try:
                rows[cells[0]] = float(cells[1]) + float(cells[2])
            except ValueError:
                pass
    if sha != kernel_source_hash() or not all(k in rows for k in kinds):
        return None
    return sum(rows[k] for k in kinds)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def _bytes_per_cell(kind, rsz, nsrc, n_array):
    """Algorithmic bytes per cell of one launch of each kernel (state x, density
    n, per-source entry columns N, half-step state xh)."""
    n_b = rsz if n_array else 0
    return {
        "sweep1": nsrc * (rsz + n_b + rsz),            # read x (+n), write N1, per source sweep
        "sweep2": nsrc * (rsz + n_b + rsz),            # read xh (+n), write N2
        "ratedt": rsz + n_b + nsrc * rsz,              # read x, n, N1
        "half": rsz + n_b + nsrc * rsz + rsz,          # read x, n, N1, write xh
        "full": rsz + n_b + nsrc * rsz + rsz,          # read x, n, N2, write x
        "final0": 0, "final1": 0,
    }.get(kind, 0)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1201_5651_gb300 import oots

    torch.cuda.set_device(local_rank)
    dev = local_rank
    w = _workload(args.workload)
    n_oct = 1 if args.workload == "stromgren32" else 8
    big = 1e30

    from paper_1201_5651_gb300 import autotune
    devname = torch.cuda.get_device_name(dev)
    tuned = {}

    def make(precision):
        c = oots.Context.from_workload(w, precision, device=dev, scheme=oots.OOTS_A3, K4=0.25)
        s = torch.cuda.Stream(device=dev)
        c.set_stream(s.cuda_stream)
        c.advance(args.t0 * w.t_rec)          # untimed: develop the front
        shape = None
        if args.shape >= 0:
            try:
                c.set_tile_shape(args.shape)
                c.profile_substep()           # builds the launch set: refuses a shape that does not fit
                shape = args.shape
            except oots.OotsError:
                shape = None                  # not at this precision: tune instead
        tuned[precision] = shape if shape is not None else autotune.tune(c, devname, len(w.sources),
                                                                          use_cache=not args.retune)
        return c, s

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{dev}")   # 256 MB > L2

    def timed(c, s, steps, warmup):
        for _ in range(warmup):
            c.run_substeps(1, big)
        c.synchronize()
        tot = 0.0
        evs = []
        for _ in range(steps):
            with torch.cuda.stream(s):
                flush.zero_()                  # evict L2 between timed steps (not timed)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
            c.run_substeps(1, big)
            with torch.cuda.stream(s):
                e1.record(s)
            evs.append((e0, e1))
        c.synchronize()
        torch.cuda.synchronize()
        for e0, e1 in evs:
            tot += e0.elapsed_time(e1)
        return tot

    def dist_max(v):
        return rank_max(v, world, f"cuda:{dev}")

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()

    # ---------------- mixed precision (the product) ----------------
    cm, sm_ = make("mixed")
    clocks = Clocks(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(dev)).split(",")[0]) if "CUDA_VISIBLE_DEVICES" in os.environ else dev)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_mixed = timed(cm, sm_, args.steps, args.warmup)
    clk = clocks.stop()
    barrier()
    t_mixed = dist_max(t_mixed)
    value = job_rate(w.ncell * args.steps, world, t_mixed)

    # per-kernel durations of one substep (eager, events around every launch)
    prof = {}
    for _ in range(3):
        for k, ms in cm.profile_substep():
            prof.setdefault(k, []).append(ms)
    prof_avg = {k: sum(v) / len(v) for k, v in prof.items()}
    launches_per_substep = sum(len(v) for v in prof.values()) // 3
    # an integration is its closed-form pass plus its general pass over the queued cells
    kern = {k: prof_avg.get(k, 0.0) + prof_avg.get(k + "_general", 0.0) for k in ("half", "full")}
    kern.update({k: prof_avg[k] for k in ("sweep1", "sweep2", "ratedt") if k in prof_avg})
    dom = max(kern, key=lambda k: kern[k])
    peak, peak_src = _peaks()
    nsrc = len(w.sources)
    bpc = _bytes_per_cell(dom, 4, nsrc, w.uniform_n is None)
    achieved = bpc * w.ncell / (kern[dom] / 1e3) / 1e9
    step_bytes = sum(_bytes_per_cell(k, 4, nsrc, w.uniform_n is None) for k in ("sweep1", "ratedt", "half", "sweep2", "full"))

    # ---------------- plain FP64 beside it ----------------
    cf, sf_ = make("fp64")
    k64 = max(3, min(args.steps, 10))
    t_fp64 = dist_max(timed(cf, sf_, k64, 1))
    value_fp64 = job_rate(w.ncell * k64, world, t_fp64)

    # ---------------- accuracy of mixed vs FP64 at a common time ----------------
    tm, _ = cm.get_time()
    tf, _ = cf.get_time()
    tc = max(tm, tf) * 1.02
    cm.advance(tc)
    cf.advance(tc)
    xm, xf = cm.get_neutral_fraction(), cf.get_neutral_fraction()
    rm, rf = _reff(xm, w.dx, n_oct), _reff(xf, w.dx, n_oct)
    acc = {"t_over_trec": tc / w.t_rec, "reff_rel_err": abs(rm / rf - 1.0),
           "ionised_volume_rel_err": abs(float((1 - xm).sum()) / float((1 - xf).sum()) - 1.0),
           "max_abs_dx": float(np.max(np.abs(xm - xf)))}

    # ---------------- end to end through the API with pinned host buffers ----------------
    host_in = torch.from_numpy(np.ascontiguousarray(xm.ravel().astype(np.float32))).pin_memory()
    host_out = torch.empty(w.ncell, dtype=torch.float32).pin_memory()
    dbuf = torch.empty(w.ncell, dtype=torch.float32, device=f"cuda:{dev}")
    ke = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        with torch.cuda.stream(sm_):
            dbuf.copy_(host_in, non_blocking=True)
        cm.set_neutral_fraction_device(dbuf.data_ptr(), True)
        cm.run_substeps(1, big)
        cm.get_neutral_fraction_device(dbuf.data_ptr(), True)
        with torch.cuda.stream(sm_):
            host_out.copy_(dbuf, non_blocking=True)
        sm_.synchronize()
    t_e2e = dist_max(time.perf_counter() - t0)
    e2e = {"value": job_rate(w.ncell * ke, world, t_e2e * 1e3), "unit": UNIT, "h2d_bytes_per_step": 4 * w.ncell,
           "d2h_bytes_per_step": 4 * w.ncell}

    if rank != 0:
        return None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_mixed / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (state, rates; float-float columns)", "data": "synthetic (seeded generators)",
        "config": {"workload": args.workload, "describe": _describe(args.workload), "ncell": w.ncell,
                   "nsrc": nsrc, "scheme": "A3", "criterion": "dt02 (K4=1/4)", "precision": "mixed",
                   "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}",
                   "tile_shape": {k: oots.oots_tile_shape_info(v)[1] if v is not None else None for k, v in tuned.items()}},
        "fp64": {"value": value_fp64, "ms_per_step": t_fp64 / k64, "steps": k64},
        "mixed_over_fp64": value / value_fp64,
        # an A3 substep traces every cell twice: cell-sweeps/s compares A3 with A2 (one trace per substep)
        "cell_sweeps_per_s": 2.0 * value,
        "accuracy_vs_fp64": acc,
        "roofline": {"bound": "hbm", "kernel": dom + (" (closed-form + general pass)" if dom in ("half", "full") else ""),
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": _traffic([dom, dom + "_general"] if dom in ("half", "full") else [dom]),
                     "traffic_unit": "bytes per launch (ncu dram read + write, profiles/)", "peak_source": peak_src,
                     "bytes_per_cell": bpc, "step_bytes_per_cell": step_bytes,
                     "step_frac": step_bytes * w.ncell / (t_mixed / args.steps / 1e3) / 1e9 / peak},
        "kernel_ms": prof_avg,
        "e2e": e2e,
        "gpu_launches": launches_per_substep * args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    return out


def _oracle_sample(args, m):
    """The oracle on the central m^3 crop of the workload (source at its centre vertex)."""
    import oracle
    w = _workload(args.workload)
    if args.workload == "stromgren32":
        sub = w.nH[:m, :m, :m].copy()
        srcs = [((0.0, 0.0, 0.0), w.sources[0].Q, w.sources[0].spectrum, w.sources[0].T)]
    else:
        lo = w.nx // 2 - m // 2
        sub = w.nH[lo:lo + m, lo:lo + m, lo:lo + m].copy()
        s = w.sources[0]
        srcs = [((m / 2, m / 2, m / 2), s.Q, s.spectrum, s.T)]
    P = oracle.Problem(m, m, m, w.dx, sub, srcs, alpha=w.alpha, sigma0=w.sigma0, tau0=w.tau0)
    return P, np.full((m, m, m), 1 - 1e-6)


def cpu_baseline(args, m=48, nsteps=3):
    P, x = _oracle_sample(args, m)
    t = 0.0
    t0 = time.perf_counter()
    for _ in range(nsteps):
        t, dt, _, _ = P.substep(x, t, 1e30, scheme=3, K4=0.25)
    el = time.perf_counter() - t0
    return {"value": m ** 3 * nsteps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{nsteps} A3-dt02 substeps of the FP64 oracle from the initial state on the central {m}^3 crop "
                      f"of the {args.workload} field (source at the crop's centre vertex); {el:.1f} s single-threaded"}


def run_reference(args):
    """The CPU oracle on the host cores: each step one A3 substep on a 32^3 crop."""
    m = 32
    P, x = _oracle_sample(args, m)
    t = 0.0
    for _ in range(args.warmup):
        t, *_ = P.substep(x, t, 1e30, scheme=3, K4=0.25)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t, *_ = P.substep(x, t, 1e30, scheme=3, K4=0.25)
    el = time.perf_counter() - t0
    v = m ** 3 * args.steps / el
    sample = f"each step: one A3-dt02 substep of the FP64 oracle on the central {m}^3 crop of the {args.workload} field"
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generators)",
            "config": {"workload": args.workload, "describe": _describe(args.workload), "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lognormal128_bb")
    ap.add_argument("--t0", type=float, default=0.05)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
