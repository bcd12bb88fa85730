"""The partitioned substep through the C ABI (oots_set_partition,
oots_run_phase, oots_array_device) on one GPU: two contexts, each tracing
half of the sources and integrating half of the z-slabs, driven by two
threads that exchange columns and states (shard.run_threads).  They must
reproduce the whole-grid run of one context (Sect. 5: sources and octants
traced independently; the decomposition changes no arithmetic)."""
import numpy as np
import pytest

import oracle
from paper_1201_5651_gb300 import inputs, oots, shard

pytestmark = pytest.mark.gpu


def _w():
    return inputs.small_random(n=26, ny=21, nz=23, seed=5, nsrc=4, spectrum="bb")


@pytest.mark.parametrize("shape", [None, 7])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_two_partitions_equal_the_whole_grid(precision, tol, shape):
    """On the default tiles and on the 8^3 throughput tiles (packed input).  The
    FP64 bound allows for the source selection: a part whose own cells ask for a
    longer step than the dt hint re-runs its dt pass without the hint, keeping
    sources that the whole run's pass left out (each below a thousandth of the
    rounding), and adaptive steps carry such rounding-level differences on."""
    w = _w()
    t_end = 0.01 * w.t_rec

    def ctx():
        c = oots.Context.from_workload(w, precision, scheme=oots.OOTS_A3, K4=0.25)
        if shape is not None:
            c.set_tile_shape(shape)
        return c
    whole = ctx()
    t_w, n_w = whole.advance(t_end)
    parts = [ctx() for _ in range(2)]
    n = shard.run_threads(parts, len(w.sources), t_end, scheme=oots.OOTS_A3)
    assert n[0] == n[1] == n_w
    xw = whole.get_neutral_fraction()
    for c in parts:
        assert abs(c.get_time()[0] / t_w - 1.0) <= 1e-14
        assert float(np.max(np.abs(c.get_neutral_fraction() - xw))) <= tol


def test_two_partitions_follow_the_oracle_fp64():
    """A3 and A2, Eq. 4 steps (K4 = 1/4, K3 = 1/8): per-cell x within 1e-9 of the oracle."""
    w = _w()
    for scheme, crit in ((oots.OOTS_A3, dict(K4=0.25)), (oots.OOTS_A2, dict(K3=0.125))):
        parts = [oots.Context.from_workload(w, "fp64", scheme=scheme, **crit) for _ in range(2)]
        shard.run_threads(parts, len(w.sources), 1e300, scheme=scheme, max_steps=2)
        P = oracle.Problem.from_workload(w)
        x = np.ascontiguousarray(w.x0.astype(np.float64))
        t = 0.0
        for _ in range(2):
            t, *_ = P.substep(x, t, 1e300, scheme=scheme, **crit)
        for c in parts:
            assert abs(c.get_time()[0] / t - 1.0) <= 1e-10
            assert float(np.max(np.abs(c.get_neutral_fraction() - x))) <= 1e-9, scheme


def test_phases_refuse_what_they_do_not_cover():
    w = _w()
    c = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A1, K1=0.1)
    with pytest.raises(oots.OotsError) as e:
        c.run_phase(oots.OOTS_PH_TRACE1)
    assert e.value.code == oots.OOTS_E_UNSUPPORTED
    c.set_scheme(oots.OOTS_A2, K4=0.25)
    with pytest.raises(oots.OotsError) as e:
        c.run_phase(oots.OOTS_PH_TRACE2)
    assert e.value.code == oots.OOTS_E_INVAL
    with pytest.raises(oots.OotsError) as e:
        c.set_partition((1 << 64) - 1, 5, 2)
    assert e.value.code == oots.OOTS_E_INVAL
    p = inputs.plane_random(n=8, seed=2)
    cp = oots.Context.from_workload(p, "fp64", scheme=oots.OOTS_A3, K4=0.25)
    with pytest.raises(oots.OotsError) as e:
        cp.run_phase(oots.OOTS_PH_TRACE1)
    assert e.value.code == oots.OOTS_E_UNSUPPORTED
