"""CPU checks of the seeded workload generators added for plane-parallel
sources and the cell-optical-depth study, and of the study's front radius."""
import math

import numpy as np

from paper_1201_5651_gb300 import accuracy_study, inputs


def test_planar_slab_layout():
    for axis in range(3):
        for back in range(2):
            w = inputs.planar_slab(n=10, ny=3, nz=2, axis=axis, back=back, dtau=4.0)
            dims = (w.nx, w.ny, w.nz)
            assert dims[axis] == 10 and sorted(dims) == [2, 3, 10]
            assert w.nH.shape == (w.nz, w.ny, w.nx) and w.x0.shape == w.nH.shape
            assert w.sources[0].plane == 2 * axis + back and w.alpha == 0.0
            assert abs(inputs.SIGMA0 * 100.0 * w.dx - 4.0) < 1e-12


def test_plane_random_is_seeded():
    a = inputs.plane_random(n=6, ny=5, nz=4, seed=3, axis=1, back=1, point_Q=1e48)
    b = inputs.plane_random(n=6, ny=5, nz=4, seed=3, axis=1, back=1, point_Q=1e48)
    assert np.array_equal(a.nH, b.nH) and np.array_equal(a.x0, b.x0)
    assert a.sources[0].plane == 3 and a.sources[1].plane == -1 and a.sources[1].pos == b.sources[1].pos


def test_stromgren_bb_scales_with_cell_optical_depth():
    ws = [inputs.stromgren_bb(d) for d in (1.0, 3.0, 10.0, 30.0)]
    assert [w.nx for w in ws] == [264, 88, 27, 9]
    for w, d in zip(ws, (1.0, 3.0, 10.0, 30.0)):
        assert abs(inputs.SIGMA0 * 10.0 * w.dx / d - 1) < 1e-12
        # the Stromgren radius of the source is 240 optical depths at nu0
        R = inputs.stromgren_radius(w.sources[0].Q, 10.0)
        assert abs(inputs.SIGMA0 * 10.0 * R / 240.0 - 1) < 1e-9
        assert w.sources[0].spectrum == "bb" and w.sources[0].T == 37500.0


def test_study_front_radius():
    # an ionised octant of radius R around the corner: (3 V 8 / 4 pi)^(1/3) = R
    n, dx, R = 40, 1.0, 25.0
    c = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    x = np.where(X ** 2 + Y ** 2 + Z ** 2 < R ** 2, 0.0, 1.0)
    assert abs(accuracy_study.r_eff(x, dx) / R - 1) < 0.01
    assert accuracy_study.r_eff(np.ones((3, 3, 3)), 1.0) == 0.0
    assert math.isclose(accuracy_study.r_eff(np.zeros((2, 2, 2)), 1.0), (3 * 8 * 8 / (4 * math.pi)) ** (1 / 3))
