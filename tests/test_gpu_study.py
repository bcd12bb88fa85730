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
