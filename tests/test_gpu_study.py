"""The paper's multi-frequency accuracy findings (Sect. 4.1), reproduced in 3D
through the C ABI (paper_1201_5651_gb300.accuracy_study): a blackbody
Stromgren sphere at cell optical depths 3 and 10, every run compared with
A3-dt12 on the same grid.

- A1 leads: its front runs ahead of the reference under the recombination-time
  criteria dt00 and dt02, and by more in the optically thicker cells;
- A3 lags (it over-attenuates), and by less in the optically thicker cells;
- A3-dt02 is within 0.5% at t_rec at both resolutions.
"""
import pytest

from paper_1201_5651_gb300 import accuracy_study

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def results():
    return {d: accuracy_study.study(d, [1, 3], [0, 2], tau_s=240.0, precision="mixed", budget_s=60.0)
            for d in (3.0, 10.0)}


def _err(res, scheme, crit, i):
    r = next(q for q in res["runs"] if q["scheme"] == scheme and q["crit"] == crit)
    assert r["complete"]
    return r["front_err"][i]


def test_a1_leads_and_worsens_with_cell_optical_depth(results):
    for crit in (0, 2):
        e3, e10 = _err(results[3.0], 1, crit, 1), _err(results[10.0], 1, crit, 1)
        assert e3 > 0.005 and e10 > e3, (crit, e3, e10)


def test_a3_lags_and_improves_with_cell_optical_depth(results):
    for crit in (0, 2):
        e3, e10 = _err(results[3.0], 3, crit, 2), _err(results[10.0], 3, crit, 2)
        assert e3 < 0 and abs(e10) < abs(e3), (crit, e3, e10)
    for d in (3.0, 10.0):
        assert abs(_err(results[d], 3, 2, 2)) < 0.005


# ------------------------------------------------------------------ cost against L1 error (Sect. 4.2, Eq. 6)
@pytest.fixture(scope="module")
def panels():
    """Delta tau0 = 10 (27^3 cells) at n_H = 10, 100 and 1000 cm^-3 (the paper's three densities), A2
    and A3 under the absolute-change criteria dt01-dt04 and the relative-change criteria dt10-dt12."""
    crit = [1, 2, 3, 4, 10, 11, 12]
    return {nh: accuracy_study.study(10.0, [2, 3], crit, tau_s=240.0, precision="mixed", budget_s=30.0, n_H=nh)
            for nh in (10.0, 100.0, 1000.0)}


def test_a3_reaches_each_error_level_cheapest_and_a2_costs_most(panels):
    """Per L1 level (Eq. 6 against A3-dt12), the cheapest A3 run costs fewer traces
    than the cheapest A2 run (A3 traces twice per substep, A2 once), at every density."""
    for nh, res in panels.items():
        compared = 0
        for l1 in (3e-3, 1e-3, 3e-4):
            a3 = accuracy_study.cheapest(res, 3, l1, cost="traces")
            a2 = accuracy_study.cheapest(res, 2, l1, cost="traces")
            assert a3 is not None, (nh, l1)
            if a2 is not None:
                assert a3[0] < a2[0], (nh, l1, a3, a2)
                compared += 1
        assert compared >= 1, nh


def test_front_error_does_not_depend_on_density(panels):
    """At fixed cell optical depth the scheme's error is almost independent of the
    density (Sect. 3.2 and 4): A3-dt02's front error at t_rec agrees across n_H = 10,
    100, 1000 to 0.1% (absolute)."""
    errs = []
    for res in panels.values():
        r = next(q for q in res["runs"] if q["scheme"] == 3 and q["crit"] == 2)
        assert r["complete"]
        errs.append(r["front_err"][2])
    assert max(errs) - min(errs) <= 1e-3, errs
