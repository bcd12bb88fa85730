"""Run one A3 substep of a named workload inside a CUDA profiler range.

For profilers started with their capture off (``ncu --profile-from-start
off``): the workload is built, advanced to t0 (untimed, outside the range),
and one eager substep runs between cudaProfilerStart and cudaProfilerStop, so
a capture sees exactly the launches of that substep.  Prints the per-launch
durations that the library's own events measured for the same substep.

    python -m paper_1201_5651_gb300.profile_substep --workload lognormal128_bb --precision mixed --shape 2
    python -m paper_1201_5651_gb300.profile_substep --workload multisource512_bb --shape 7 --t0 0.005 --substeps 3
"""
from __future__ import annotations

import argparse

from . import inputs, oots

WORKLOADS = {
    # 16 blackbody sources in lognormal gas (the many-source workload at full size and at 1/8 of its cells)
    "multisource512_bb": lambda: inputs.multisource(512),
    "multisource256_bb": lambda: inputs.multisource(256),
    "clumpy256_mono": lambda: inputs.clumpy(256, 1.5, 1203, 1303, 200, Q=1e48, box_rs=2.5, spectrum="mono"),
    "lognormal128_bb": lambda: inputs.lognormal_bb(128, 1.0, 1202, Q=1e48, T=4e4, box_rs=2.5),
    "lognormal64_bb": lambda: inputs.lognormal_bb(64, 1.0, 1202, Q=1e48, T=4e4, box_rs=2.5),
    "stromgren32": lambda: inputs.stromgren_corner(32),
    # plane-parallel blackbody source along each axis (rows along x: one warp
    # per row; along y or z: one thread per row)
    "plane256_x": lambda: inputs.plane_random(n=256, seed=31, axis=0, spectrum="bb", F=1e10, x_lo=0.9),
    "plane256_y": lambda: inputs.plane_random(n=256, seed=31, axis=1, spectrum="bb", F=1e10, x_lo=0.9),
    "plane256_z": lambda: inputs.plane_random(n=256, seed=31, axis=2, spectrum="bb", F=1e10, x_lo=0.9),
}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lognormal128_bb", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--shape", type=int, default=-1, help="tile shape id (-1: library default)")
    ap.add_argument("--t0", type=float, default=0.05, help="start time in units of t_rec (0: start at once)")
    ap.add_argument("--substeps", type=int, default=1, help="substeps inside the profiler range")
    args = ap.parse_args(argv)

    import torch
    w = WORKLOADS[args.workload]()
    c = oots.Context.from_workload(w, args.precision, scheme=oots.OOTS_A3, K4=0.25)
    if args.shape >= 0:
        c.set_tile_shape(args.shape)
    if args.t0 > 0:
        c.advance(args.t0 * w.t_rec)
    c.profile_substep()                       # build and warm up every launch
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    profs = [c.profile_substep() for _ in range(args.substeps)]
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    for i, prof in enumerate(profs):
        for k, ms in prof:
            print(f"{i:3d} {k:14s} {ms * 1e3:10.1f} us")


if __name__ == "__main__":
    main()
