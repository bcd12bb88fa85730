"""Accuracy and cost of the three schemes against the cell optical depth, for
a multi-frequency Stromgren sphere in 3D (Mackey 2012, Sect. 4.1 and 4.2).

For each cell optical depth dtau0 the grid resolves the same problem
(inputs.stromgren_bb: uniform gas, blackbody source at the corner vertex,
Stromgren radius tau_s optical depths).  Every (scheme, criterion) run is
advanced to t_rec and compared with the A3-dt12 run on the same grid, the
reference of Sect. 4.1:
  - front: R_eff = (3 V_ion 8 / 4 pi)^(1/3) (one octant around the source) at
    0.1, 0.3 and 1 t_rec, relative to the reference;
  - L1 error (Eq. 6): mean over cells of |x - x_ref| at t_rec;
  - cost: substeps and wall time of the run (substeps are enqueued in
    batches of 32 and synchronised between batches).
The output times cap the step, as outputs do in the paper's runs.
Runs go through the public C ABI on the mixed path.

    python -m paper_1201_5651_gb300.accuracy_study --dtau 1 3 10 30 --schemes 1 3 --criteria 0 1 2 3 4 \
        --out study.json
    python -m paper_1201_5651_gb300.accuracy_study --density 100 1000 --dtau 3 10 30 --schemes 1 2 3 \
        --criteria 0 1 2 3 4 5 6 7 8 9 10 11 12 --budget 20 --out map.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs, oots

TIMES = (0.1, 0.3, 1.0)      # output times in units of t_rec


def r_eff(x: np.ndarray, dx: float) -> float:
    return (3.0 * float((1.0 - x).sum()) * dx ** 3 * 8.0 / (4.0 * math.pi)) ** (1.0 / 3.0)


def run(w, scheme: int, crit: int, precision: str = "mixed", budget_s: float = 120.0):
    """Advance one run to t_rec.  Returns R_eff at TIMES, x at t_rec, the
    substeps and seconds, or a partial record if budget_s ran out."""
    c = oots.Context.from_workload(w, precision)
    c.set_scheme(scheme, preset=crit)
    out = {"scheme": scheme, "crit": crit, "reff": [], "nsub": 0, "seconds": 0.0, "complete": True}
    t0 = time.perf_counter()
    for f in TIMES:
        # the output times cap the step (as outputs do in any run); between
        # them the substeps go in batches so that a run over budget stops
        target = f * w.t_rec
        while True:
            t, nsub = c.get_time()
            if t >= target * (1 - 1e-12):
                break
            c.run_substeps(32, target)
            c.synchronize()
            if time.perf_counter() - t0 > budget_s:
                out["complete"] = False
                break
        if not out["complete"]:
            break
        out["reff"].append(r_eff(c.get_neutral_fraction(), w.dx))
    out["seconds"] = time.perf_counter() - t0
    out["nsub"] = c.get_time()[1]
    x = c.get_neutral_fraction() if out["complete"] else None
    return out, x


def study(dtau0: float, schemes, criteria, tau_s: float, precision: str, budget_s: float, n_H: float = 10.0):
    w = inputs.stromgren_bb(dtau0, tau_s=tau_s, n_H=n_H)
    ref, xref = run(w, 3, 12, precision, budget_s=10 * budget_s)
    rows = []
    for s in schemes:
        for k in criteria:
            if s == 3 and k == 12:
                r, x = ref, xref
            else:
                r, x = run(w, s, k, precision, budget_s)
            if r["complete"] and ref["complete"]:
                r["front_err"] = [a / b - 1.0 for a, b in zip(r["reff"], ref["reff"])]
                r["l1"] = float(np.abs(x - xref).mean())
            rows.append(r)
    return {"dtau0": dtau0, "n_H": n_H, "n": w.nx, "tau_s": tau_s, "t_rec": w.t_rec, "reference": ref, "runs": rows}


def cheapest(res, scheme: int, l1_max: float, cost: str = "seconds"):
    """The cheapest complete run of `scheme` whose L1 error (Eq. 6) is at most
    l1_max: (cost, criterion), or None.  cost "traces" counts the traces a run
    did (A3 two per substep, A2 and A1 one), a cost that does not depend on the
    machine's load."""
    best = None
    for q in res["runs"]:
        if q["scheme"] != scheme or "l1" not in q or q["l1"] > l1_max:
            continue
        v = q["seconds"] if cost == "seconds" else q["nsub"] * (2 if scheme == 3 else 1)
        if best is None or v < best[0]:
            best = (v, q["crit"])
    return best


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtau", type=float, nargs="+", default=[1.0, 3.0, 10.0, 30.0])
    ap.add_argument("--schemes", type=int, nargs="+", default=[1, 3])
    ap.add_argument("--criteria", type=int, nargs="+", default=[0, 1, 2, 3, 4])
    ap.add_argument("--tau-s", type=float, default=240.0)
    ap.add_argument("--density", type=float, nargs="+", default=[10.0], help="hydrogen densities n_H [cm^-3]")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--budget", type=float, default=60.0, help="wall seconds per run before it is cut short")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    res = []
    for nh in args.density:
        for d in args.dtau:
            r = study(d, args.schemes, args.criteria, args.tau_s, args.precision, args.budget, n_H=nh)
            res.append(r)
            print(f"n_H {nh:g}, dtau0 {d:g}: {r['n']}^3 cells, reference A3-dt12 {r['reference']['nsub']} substeps "
                  f"{r['reference']['seconds']:.1f} s", flush=True)
            for q in r["runs"]:
                fe = " ".join(f"{v:+.4f}" for v in q.get("front_err", [])) or "incomplete"
                l1 = f"{q['l1']:.2e}" if "l1" in q else "-"
                print(f"  A{q['scheme']}-dt{q['crit']:02d}  front err at {TIMES} t_rec: {fe}  L1 {l1}  "
                      f"{q['nsub']} substeps {q['seconds']:.2f} s", flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
