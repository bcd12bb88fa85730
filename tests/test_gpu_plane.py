"""Parity of the plane-parallel source path (Sect. 3.1) with the FP64 oracle,
through the C ABI.

FP64: columns within 1e-12 relative, dt within 1e-10, per-cell x within 1e-9,
the photon budget within 1e-8 of the absorbed total.  Mixed: photon
conservation of A1 on the slab and the front against the FP64 path.
"""
import numpy as np
import pytest

import oracle
from paper_1201_5651_gb300 import inputs, oots

pytestmark = pytest.mark.gpu

XTOL = 1e-9
DIRS = [(a, b) for a in range(3) for b in range(2)]


def _rel(a, b, floor=1.0):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


@pytest.mark.parametrize("axis,back", DIRS)
def test_plane_columns_every_direction(axis, back):
    """Rows shorter than a warp (axis 0: 19 cells), longer than two warp
    chunks (70 cells along the axis) and ragged transverse sizes."""
    for dims in [(19, 13, 11), (70, 5, 3), (3, 70, 2), (4, 3, 70)]:
        nx, ny, nz = dims
        w = inputs.plane_random(n=nx, ny=ny, nz=nz, seed=7 + axis + 3 * back, axis=axis, back=back)
        c = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A3, K4=0.25)
        dt = c.compute_dt()
        P = oracle.Problem.from_workload(w)
        assert abs(dt / P.compute_dt(w.x0, K4=0.25) - 1) <= 1e-10
        assert _rel(c.get_column_density(0), P.trace(0, w.x0), floor=1e10) <= 1e-12, dims


@pytest.mark.parametrize("scheme", [3, 2, 1])
@pytest.mark.parametrize("spectrum", ["mono", "bb"])
def test_plane_substeps_fp64(scheme, spectrum):
    w = inputs.plane_random(n=13, ny=9, nz=10, seed=40 + scheme, axis=scheme % 3, back=scheme & 1,
                            spectrum=spectrum, F=3e10)
    dt = 0.01 * w.t_rec
    c = oots.Context.from_workload(w, "fp64", scheme=scheme, dt_fixed=dt)
    P = oracle.Problem.from_workload(w)
    x = w.x0.copy()
    t = 0.0
    tot = np.zeros(4)
    for k in range(3):
        c.step(dt)
        t, _, bud, _ = P.substep(x, t, t + dt, scheme=scheme, dt_fixed=dt)
        tot += bud
        assert np.max(np.abs(c.get_neutral_fraction() - x)) <= XTOL, (scheme, k)
    b = c.get_budget()
    assert abs(b[0] / tot[0] - 1) <= 1e-12
    for q in (1, 2, 3):
        assert abs(b[q] - tot[q]) <= 1e-8 * abs(tot[1]), (q, b, tot)


def test_plane_and_point_sources_adaptive_fp64():
    """A plane source along -y plus a blackbody point source, A3-dt02, three
    adaptive substeps: same dt each substep, x within 1e-9."""
    w = inputs.plane_random(n=12, ny=11, nz=9, seed=5, axis=1, back=1, point_Q=1e48, spectrum="bb", F=1e10)
    c = oots.Context.from_workload(w, "fp64", scheme=3, K4=0.25)
    P = oracle.Problem.from_workload(w)
    x = w.x0.copy()
    t = 0.0
    for k in range(3):
        dt = c.compute_dt()
        t_new, dtr, _, _ = P.substep(x, t, 1e30, scheme=3, K4=0.25)
        assert abs(dt / dtr - 1) <= 1e-10
        c.step(dtr)
        t = t_new
        assert np.max(np.abs(c.get_neutral_fraction() - x)) <= XTOL, k


def test_slab_photon_conservation():
    """Sect. 3.1: with no recombinations the ions per unit area are F t; A1
    conserves photons whatever the step.  FP64 to 1e-9, mixed to 1e-5; and
    the A3-dt02 front error equals the oracle's."""
    w = inputs.planar_slab(n=100, ny=3, nz=2)
    F, n = w.sources[0].Q, 100.0
    tc = n * w.dx / F
    area_cells = w.ny * w.nz
    ions = lambda y: float(((1.0 - np.ravel(y)) * w.nH.ravel() * w.dx).sum()) / area_cells
    i0 = ions(w.x0.ravel())
    for prec, tol in [("fp64", 1e-9), ("mixed", 1e-5)]:
        c = oots.Context.from_workload(w, prec, scheme=oots.OOTS_A1, dt_fixed=0.7 * tc)
        t, nsub = c.advance(40 * tc)
        err = (ions(c.get_neutral_fraction()) - i0) / (F * t) - 1
        assert abs(err) <= tol, (prec, err)
    # A3-dt02 through the graph path, one substep at a time: each substep
    # equals the oracle's from the same state.  (Whole runs are not compared
    # cell by cell: with alpha = 0 the adaptive dt feeds state differences
    # back, and the oracle alone turns a 1e-15 change of one cell into 1e-4
    # after these 127 substeps.  The front error is stable to 1e-5.)
    P = oracle.Problem.from_workload(w)
    c = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A3, K4=0.25)
    T = 40 * tc
    for k in range(400):
        xp = c.get_neutral_fraction().reshape(w.nz, w.ny, w.nx).copy()
        t0, _ = c.get_time()
        c.run_substeps(1, T)
        c.synchronize()
        t1, _ = c.get_time()
        t, dt, _, _ = P.substep(xp, t0, T, scheme=3, K4=0.25)
        assert abs((t1 - t0) / dt - 1) <= 1e-9, k
        assert np.max(np.abs(c.get_neutral_fraction().ravel() - xp.ravel())) <= XTOL, k
        if t1 >= T:
            break
    x = w.x0.copy()
    tr, nr, _ = P.run(x, 0.0, T, scheme=3, K4=0.25)
    assert k + 1 == nr
    err_g = (ions(c.get_neutral_fraction()) - i0) / (F * T) - 1
    err_o = (ions(x) - i0) / (F * T) - 1
    assert 0.005 < err_o < 0.03 and abs(err_g - err_o) <= 1e-4, (err_g, err_o)


def test_plane_mixed_against_fp64():
    """Mixed path on a 48^3 grid lit along +z, A3-dt02 to a front about 20
    cells deep: ionised volume within 1e-3, max |dx| within 1e-3."""
    w = inputs.plane_random(n=48, seed=9, axis=2, back=0, x_lo=1.0 - 1e-6, F=1e10, dtau=1.0)
    tc = 100.0 * w.dx / 1e10
    cm = oots.Context.from_workload(w, "mixed", scheme=oots.OOTS_A3, K4=0.25)
    cf = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A3, K4=0.25)
    cm.advance(20 * tc)
    cf.advance(20 * tc)
    xm, xf = cm.get_neutral_fraction(), cf.get_neutral_fraction()
    assert float((1 - xf).sum()) > 100
    assert abs(float((1 - xm).sum()) / float((1 - xf).sum()) - 1) <= 1e-3
    assert float(np.abs(xm - xf).max()) <= 1e-3
    Nm, Nf = cm.get_column_density(0), cf.get_column_density(0)
    assert _rel(Nm, Nf, floor=1e14) <= 1e-3
