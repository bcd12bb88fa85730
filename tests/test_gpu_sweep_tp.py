"""The throughput form of the sweep (tile shape 7: 8^3 tiles traced whole,
layer by layer along the dominant axis off the octants' diagonal planes,
plane by plane on them) against the CPU oracle.

The grids are large enough that every octant holds tiles of each kind: tiles
where x, y or z dominates every cell, and tiles crossed by the diagonal
planes i = j, j = k, i = k where tied cells average two or three
interpolations (Sect. 2, short characteristics; Sect. 5, octants)."""
import numpy as np
import pytest

import oracle
from paper_1201_5651_gb300 import inputs, oots

pytestmark = pytest.mark.gpu
TP = 7          # 8 x 8 x 8 tiles
TP16 = 8        # 16 x 8 x 8 tiles
XTOL = 1e-9


def _rel(a, b, floor=1e10):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def _three_sources(seed=5, n=41, ny=33, nz=29, spectrum="mono"):
    w = inputs.small_random(n=n, ny=ny, nz=nz, seed=seed, nsrc=3, spectrum=spectrum)
    w.sources[0].pos = (0.0, 0.0, 0.0)          # corner: one octant spans the grid
    w.sources[1].pos = (17.0, 9.0, 22.0)        # interior: eight uneven octants
    w.sources[2].pos = (41.0, 16.0, 3.0)        # on a face
    return w


@pytest.mark.parametrize("tp", [TP, TP16])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_tp_columns_match_the_oracle(precision, tol, tp):
    """FP64: the oracle's columns to 1e-12.  Mixed (float density, state and
    weights, float-float columns): within 1e-5 over paths of ~60 cells, and no
    further from the oracle than the pipelined kernel's columns (plus 1e-7)."""
    w = _three_sources()
    P = oracle.Problem.from_workload(w)
    ref = [P.trace(s, w.x0) for s in range(3)]
    err = {}
    for shape in (0, tp):
        c = oots.Context.from_workload(w, precision, scheme=oots.OOTS_A3, K4=0.25)
        c.set_tile_shape(shape)
        c.compute_dt()
        err[shape] = [_rel(c.get_column_density(s), ref[s]) for s in range(3)]
    for s in range(3):
        assert err[tp][s] <= tol, (precision, s, err)
        assert err[tp][s] <= 2.0 * err[0][s] + 1e-7, (precision, s, err)


def test_tp_columns_partially_ionised_state_fp64():
    """A state with ionised holes (x from 0 to 1): the optical-depth weights vary
    strongly from cell to cell, and the weighted differences of neighbouring
    columns lose a few more digits than on neutral gas (both kernels)."""
    w = _three_sources(seed=9)
    rng = np.random.default_rng(3)
    w.x0 = np.where(rng.uniform(size=w.x0.shape) < 0.3, 1e-4, w.x0)
    P = oracle.Problem.from_workload(w)
    ref = [P.trace(s, w.x0) for s in range(3)]
    err = {}
    for shape in (0, TP, TP16):
        c = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A3, K4=0.25)
        c.set_tile_shape(shape)
        c.compute_dt()
        err[shape] = [_rel(c.get_column_density(s), ref[s]) for s in range(3)]
    for s in range(3):
        for tp in (TP, TP16):
            assert err[tp][s] <= 1e-10, (s, tp, err)
            assert err[tp][s] <= 4.0 * err[0][s] + 1e-13, (s, tp, err)


@pytest.mark.parametrize("tp", [TP, TP16])
@pytest.mark.parametrize("scheme", [2, 3])
def test_tp_adaptive_substeps_fp64(scheme, tp):
    """A2 and A3 with Eq. 4 (K4 = 1/4) on the throughput sweep: the step and every
    cell's neutral fraction follow the oracle for three substeps (both traces of A3)."""
    w = _three_sources(seed=21, spectrum="bb")
    c = oots.Context.from_workload(w, "fp64", scheme=scheme, K4=0.25)
    c.set_tile_shape(tp)
    P = oracle.Problem.from_workload(w)
    x = np.ascontiguousarray(w.x0.astype(np.float64))
    t = 0.0
    for k in range(3):
        dt_g = c.compute_dt()
        t_new, dt, _, _ = P.substep(x, t, 1e300, scheme=scheme, K4=0.25)
        assert abs(dt_g / dt - 1.0) <= 1e-10, (k, dt_g, dt)
        c.step(dt_g)
        t = t_new
        assert float(np.max(np.abs(c.get_neutral_fraction() - x))) <= XTOL, (scheme, k)


@pytest.mark.parametrize("tp", [TP, TP16])
def test_tp_shape_runs_A1_on_the_pipelined_kernel(tp):
    """The implicit sweep (A1) integrates on the chain; with shape 7 it runs the
    pipelined kernel on the same 8^3 tiles and still follows the oracle."""
    w = inputs.small_random(n=19, ny=17, nz=15, seed=4, nsrc=1)
    dt = 0.05 * w.t_rec
    c = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A1, dt_fixed=dt)
    c.set_tile_shape(tp)
    c.step(dt)
    P = oracle.Problem.from_workload(w)
    x = np.ascontiguousarray(w.x0.astype(np.float64))
    P.substep(x, 0.0, dt, scheme=1, dt_fixed=dt)
    assert float(np.max(np.abs(c.get_neutral_fraction() - x))) <= XTOL


def test_tp_many_sources_advance_mixed_matches_pipelined():
    """Sixteen blackbody sources, adaptive A3 on the mixed path to 0.02 t_rec: the
    throughput and pipelined sweeps agree on the front (ionised volume) and per cell."""
    w = inputs.multisource(40, 1.0, 1205, nsrc=16, box_rs=2.0)
    out = []
    for shape in (0, TP, TP16):
        c = oots.Context.from_workload(w, "mixed", scheme=3, K4=0.25)
        c.set_tile_shape(shape)
        c.advance(0.02 * w.t_rec)
        out.append(c.get_neutral_fraction())
    v0 = float((1 - out[0]).sum())
    for o in out[1:]:
        assert abs(float((1 - o).sum()) / v0 - 1.0) <= 1e-4
        assert float(np.abs(out[0] - o).max()) <= 1e-3


@pytest.mark.parametrize("shape", [0, 4, TP, TP16])
def test_octant_aligned_tiles_match_the_oracle(shape):
    """Tiles started at each octant's origin (tuning key 4) instead of at global
    multiples of the tile size: the same columns, to 1e-12 (FP64)."""
    w = _three_sources(seed=13)
    c = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A3, K4=0.25)
    c.set_tile_shape(shape)
    c.debug_set(4, 1)
    c.compute_dt()
    P = oracle.Problem.from_workload(w)
    for s in range(3):
        assert _rel(c.get_column_density(s), P.trace(s, w.x0)) <= 1e-12, (shape, s)


def test_mixed_columns_near_source_vertices():
    """Mixed (float-float) against FP64 entry columns of one developed state of the
    16-source lognormal workload at 64^3: every cell within 2e-3, 99.9% within
    1e-6.  Near a vertex an entry column can be a weighted average of
    neighbours that differ by orders of magnitude; tied cells take their
    reference on a neighbour that carries weight, so no result is a difference
    of far larger columns."""
    w = inputs.multisource(64)
    cm = oots.Context.from_workload(w, "mixed", scheme=3, K4=0.25)
    cm.set_tile_shape(TP)
    cm.advance(0.005 * w.t_rec)
    x = cm.get_neutral_fraction()
    cf = oots.Context.from_workload(w, "fp64", scheme=3, K4=0.25)
    cf.set_tile_shape(TP)
    cf.set_neutral_fraction(x)
    cf.compute_dt()
    cm.compute_dt()
    for s in range(len(w.sources)):
        nf, nm = cf.get_column_density(s), cm.get_column_density(s)
        rel = np.abs(nm - nf) / np.maximum(nf, 1e10)
        assert float(rel.max()) <= 2e-3, (s, float(rel.max()))
        assert float(np.percentile(rel, 99.9)) <= 1e-6, s


@pytest.mark.parametrize("shape", [TP, TP16])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_on_throughput_tiles_matches_solo_runs(shape, precision):
    """Grids of different sizes and source counts in one batch on the throughput
    tiles (one packing launch for all grids, tile items carrying their grid, the
    per-tile end-time check of launches with several grids): each grid ends where
    its own run ends, bit for bit, although the grids reach their end times at
    different substeps."""
    ws = [inputs.small_random(n=n, ny=n - 2, nz=n - 3, seed=70 + n, nsrc=k, spectrum="bb")
          for n, k in ((14, 1), (20, 3), (17, 2))]
    ends = [f * w.t_rec for f, w in zip((0.01, 0.03, 0.02), ws)]
    solo = []
    for w, te in zip(ws, ends):
        c = oots.Context.from_workload(w, precision, scheme=3, K4=0.25)
        c.set_tile_shape(shape)
        _, nsub = c.advance(te)
        solo.append((nsub, c.get_neutral_fraction()))
    ctxs = []
    for w in ws:
        c = oots.Context.from_workload(w, precision, scheme=3, K4=0.25)
        c.set_tile_shape(shape)
        ctxs.append(c)
    b = oots.Batch(ctxs)
    nsub = b.advance(ends)
    b.close()
    for g, (c, (ns, xs)) in enumerate(zip(ctxs, solo)):
        assert nsub[g] == ns, (g, nsub[g], ns)
        assert np.array_equal(c.get_neutral_fraction(), xs), g
