"""Oracle pins for plane-parallel sources (a source at infinity whose rays run
along a grid axis: the slab test of Sect. 3.1).

What fixes the oracle here, independently of its own code:
- the paper's slab (Sect. 3.1): 100 cells over about 0.51 pc with cell optical
  depth about 10 at n_H = 100, front speed F/n = 100 km/s;
- photon conservation with no recombinations: the ions per unit area are F t
  exactly for a photon-conserving integration, which A1 is by construction
  (Sect. 2.1); the absorbed-photon tally equals the photons that entered;
- the closed form x(t) = ln(1 + (e^{b x0} - 1) e^{-A b t}) / b of a cell with
  no recombinations (Eq. 2 with alpha = 0), for the first two cells of a row;
- the paper's convergence findings for the explicit schemes on this test
  (Sect. 3.1, Fig. 2): A2 first order, about a factor 2 per halving of K4 and
  above 1% error for dt00-dt04; A3 much faster;
- symmetry: a mirrored or axis-permuted grid gives the mirrored or permuted
  result exactly; rates of several sources add.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1201_5651_gb300 import inputs

SIG = inputs.SIGMA0
PC = 3.0857e18


def _golden():
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


def _front_error(w, scheme, t_end, **crit):
    """N_i(t) / (F t) - 1 of a slab run (ions per unit area of the face)."""
    P = oracle.Problem.from_workload(w)
    x = w.x0.copy()
    area_cells = x.size // {0: w.nx, 1: w.ny, 2: w.nz}[w.sources[0].plane // 2]
    ions = lambda y: float(((1.0 - y) * w.nH * w.dx).sum()) / area_cells
    i0 = ions(x)
    t, nsub, bud = P.run(x, 0.0, t_end, scheme=scheme, **crit)
    return (ions(x) - i0) / (w.sources[0].Q * t) - 1.0, nsub, bud, x


def test_slab_matches_paper_setup():
    g = _golden()
    w = inputs.planar_slab(n=int(g["plane_cells"]), F=g["plane_flux"], n_H=g["plane_n"], dtau=g["plane_dtau"])
    assert w.nx == 100 and w.alpha == 0.0
    assert abs(w.nx * w.dx / PC / g["plane_length_pc"] - 1) < 0.01
    assert abs(SIG * g["plane_n"] * w.dx - g["plane_dtau"]) < 1e-12
    # the front speed of a photon-conserving run is F/n = 100 km/s
    t_end = 40 * g["plane_n"] * w.dx / g["plane_flux"]
    err, _, _, x = _front_error(w, 1, t_end, dt_fixed=t_end / 57)
    v = (1 + err) * g["plane_flux"] / g["plane_n"] / 1e5
    assert abs(v / g["v_IF_kms"] - 1) < 1e-9
    # the front sits where F t / n puts it: 40 cells ionised, the rest neutral
    assert np.all(x.ravel()[:39] < 1e-3) and np.all(x.ravel()[42:] > 0.999)


@pytest.mark.parametrize("crossings", [0.3, 1.0, 7.0])
def test_a1_conserves_photons(crossings):
    """A1 hands each cell the time-averaged transmission of the cells before it
    (Eq. 3), so with no recombinations every photon that enters makes one ion,
    whatever the step: ions = F t and absorbed = emitted."""
    w = inputs.planar_slab(n=60, dtau=3.0)
    tc = 100.0 * w.dx / w.sources[0].Q          # time for the front to cross one cell
    t_end = 30 * tc
    err, nsub, bud, _ = _front_error(w, 1, t_end, dt_fixed=crossings * tc)
    assert abs(err) < 1e-10, err
    assert abs(bud[1] / bud[0] - 1) < 1e-10 and abs(bud[2] / bud[1] - 1) < 1e-10
    assert bud[3] == 0.0


def test_first_cells_closed_form():
    """Eq. 2 with alpha = 0 and the column frozen over the step has the closed
    form x(h) = ln(1 + (e^{b x0} - 1) e^{-A b h}) / b with A = F e^{-sigma N_in}
    / (n dx) and b = sigma n dx: the first cell (N_in = 0) and the second
    (N_in = n x0 dx of the first) of an A2 step, in each direction."""
    for axis, back in [(0, 0), (0, 1), (2, 1)]:
        w = inputs.planar_slab(n=3, dtau=2.5, axis=axis, back=back)
        w.x0[...] = 0.7
        P = oracle.Problem.from_workload(w)
        x = w.x0.copy()
        F, n = w.sources[0].Q, 100.0
        h = 0.4 * n * w.dx / F
        P.substep(x, 0.0, h, scheme=2, dt_fixed=h)
        b = SIG * n * w.dx
        row = np.moveaxis(x, 2 - axis, 0).ravel()
        if back:
            row = row[::-1]
        for m, Nin in [(0, 0.0), (1, n * 0.7 * w.dx)]:
            A = F * np.exp(-SIG * Nin) / (n * w.dx)
            xe = np.log1p(np.expm1(b * 0.7) * np.exp(-A * b * h)) / b
            assert abs(row[m] - xe) < 1e-12, (axis, back, m, row[m], xe)


def test_explicit_schemes_converge_as_the_paper_finds():
    """Sect. 3.1 / Fig. 2: A2 errors fall by about 2 per halving of K4 and stay
    above 1% for dt00-dt04; A3 converges much faster.  (The paper puts A3-dt02
    below 1%; this reading gives 1.4%, so only the ordering is pinned.)"""
    w = inputs.planar_slab(n=80)
    t_end = 50 * 100.0 * w.dx / w.sources[0].Q
    k4s = [0.5, 0.25, 0.125, 0.0625]
    e2 = [abs(_front_error(w, 2, t_end, K4=k)[0]) for k in k4s]
    e3 = [abs(_front_error(w, 3, t_end, K4=k)[0]) for k in k4s]
    assert all(e > 0.01 for e in e2), e2
    for a, b in zip(e2[1:], e2[2:]):
        assert 1.5 < a / b < 2.6, e2
    assert e3[2] < 0.003 and e3[3] < e3[2] / 4, e3
    assert all(c < a / 5 for a, c in zip(e2[1:], e3[1:])), (e2, e3)


def test_plane_trace_mirror_and_axis_permutation():
    """A source shining along -x on a grid is the source along +x on the grid
    mirrored in x; a source along y is the source along x on the grid with x
    and y exchanged.  Columns, rates and whole A3 substeps agree exactly."""
    w = inputs.plane_random(n=7, ny=5, nz=4, seed=3, axis=0, back=1)
    P = oracle.Problem.from_workload(w)
    x = w.x0.copy()
    N = P.trace(0, x)
    wm = inputs.plane_random(n=7, ny=5, nz=4, seed=3, axis=0, back=0)
    wm.nH = w.nH[:, :, ::-1].copy()
    Pm = oracle.Problem.from_workload(wm)
    Nm = Pm.trace(0, x[:, :, ::-1].copy())
    assert np.array_equal(N, Nm[:, :, ::-1])
    # axis permutation: y-directed source on the grid transposed in (x, y)
    wy = inputs.plane_random(n=5, ny=7, nz=4, seed=3, axis=1, back=1)
    wy.nH = np.ascontiguousarray(w.nH.transpose(0, 2, 1))
    Py = oracle.Problem.from_workload(wy)
    xt = np.ascontiguousarray(x.transpose(0, 2, 1))
    assert np.array_equal(Py.trace(0, xt), np.ascontiguousarray(N.transpose(0, 2, 1)))
    # whole A3 substep
    a = x.copy(); P.substep(a, 0.0, 1e30, scheme=3, K4=0.25)
    b = xt.copy(); Py.substep(b, 0.0, 1e30, scheme=3, K4=0.25)
    assert np.max(np.abs(a - b.transpose(0, 2, 1))) <= 1e-15


def test_rates_of_plane_and_point_sources_add():
    w = inputs.plane_random(n=6, ny=5, nz=7, seed=4, axis=2, back=0, point_Q=1e48, spectrum="bb")
    P = oracle.Problem.from_workload(w)
    x = w.x0.copy()
    N = np.stack([P.trace(0, x), P.trace(1, x)])
    F, _ = P.rates(x, N)
    parts = []
    for s in range(2):
        ws = inputs.plane_random(n=6, ny=5, nz=7, seed=4, axis=2, back=0, point_Q=1e48, spectrum="bb")
        ws.sources = [ws.sources[s]]
        Ps = oracle.Problem.from_workload(ws)
        parts.append(Ps.rates(x, N[s:s + 1])[0])
    assert np.max(np.abs(F - parts[0] - parts[1]) / np.maximum(F, 1e-300)) < 1e-13
    assert np.all(parts[0] > 0) and np.all(parts[1] > 0)


def test_tabulated_plane_source_with_delta_spectrum_equals_monochromatic():
    """A plane source with a tabulated delta spectrum (all photons at nu0) gives
    the same columns and the same A3 substeps as the monochromatic plane source:
    pins the tabulated rate of a plane source against the exponential one."""
    w = inputs.plane_random(n=7, ny=6, nz=5, seed=8, axis=1, back=0, F=3e10)
    Pm = oracle.Problem.from_workload(w)
    srcs = [(s.pos, s.Q, "tab", 0.0, s.plane) for s in w.sources]
    Pt = oracle.Problem(w.nx, w.ny, w.nz, w.dx, w.nH, srcs, alpha=w.alpha, sigma0=w.sigma0, tau0=w.tau0,
                        tables=[oracle.table_build("delta")])
    a = w.x0.copy()
    b = w.x0.copy()
    dt = 0.02 * w.t_rec
    for _ in range(2):
        Pm.substep(a, 0.0, dt, scheme=3, dt_fixed=dt)
        Pt.substep(b, 0.0, dt, scheme=3, dt_fixed=dt)
    assert np.max(np.abs(a - b)) <= 1e-9
    assert np.max(np.abs(a - w.x0)) > 1e-3


def test_a1_and_a3_converge_together_with_recombinations():
    """With recombinations on, the implicit row sweep (A1, fixed small steps)
    and the explicit scheme (A3, tight K4) are different algorithms for the same
    equations; at small steps both converge to one solution.  A front in an
    optically thick slab (cell dtau 5), six crossing times."""
    w = inputs.plane_random(n=16, ny=3, nz=2, seed=12, axis=0, back=0, F=1e9, x_lo=1 - 1e-6, dtau=5.0,
                            sigma_ln=0.3)
    P = oracle.Problem.from_workload(w)
    T = 6 * 100.0 * w.dx / 1e9
    a1 = w.x0.copy()
    P.run(a1, 0.0, T, scheme=1, dt_fixed=T / 400)
    a3 = w.x0.copy()
    P.run(a3, 0.0, T, scheme=3, K4=1 / 64)
    coarse = w.x0.copy()
    P.run(coarse, 0.0, T, scheme=3, K4=1 / 4)
    assert float((1 - a3).sum()) > 20                      # the front has moved several cells in
    assert np.max(np.abs(a1 - a3)) <= 5e-4
    assert abs(float((1 - a1).sum()) / float((1 - a3).sum()) - 1) <= 1e-4
    assert np.max(np.abs(coarse - a3)) > 10 * np.max(np.abs(a1 - a3))   # the agreement is not trivial
