"""Extended-precision pin of the oracle's table difference ln P(Na + dN) - ln P(Na).

The multi-frequency rate of a cell (Sect. 2, the frequency-integrated rate
tables; Sect. 4) is the photon rate lost between the column at the cell's
entry, Na, and its exit, Na + dN.  The oracle evaluates it from its table by
integrating the interpolant piecewise over node intervals.  Here the same
quantity comes straight from the spectrum, with no table: for a blackbody
photon spectrum phi(u) = u^2/(e^{theta u} - 1) on u = nu/nu0 in [1, 40] and
sigma(u) = sigma0 u^-3,

    1 - P(Na + dN)/P(Na) = int phi e^{-sigma Na} (1 - e^{-sigma dN}) du / int phi e^{-sigma Na} du,

integrated with mpmath at 40 digits (1 - e^{-z} is formed without
cancellation).  The thin steps (dN/Na down to 1e-9) are where a cancelling
difference of two table values would lose every digit.
"""
import math

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")

SIG = 6.3e-18
THETA_OVER_T = 13.6 / 8.617333262e-5     # h nu0 / k in kelvin (h nu0 = 13.6 eV)


def _dlnp_direct(T, Na, dN):
    mp.mp.dps = 40
    theta = mp.mpf(THETA_OVER_T) / T
    sig = mp.mpf(SIG)
    Na, dN = mp.mpf(Na), mp.mpf(dN)

    def phi(u):
        return u * u / mp.expm1(theta * u)

    pts = [1, 1.5, 2, 3, 4, 6, 9, 14, 20, 28, 40]
    den = mp.quad(lambda u: phi(u) * mp.exp(-sig * Na / u ** 3), pts)
    num = mp.quad(lambda u: phi(u) * mp.exp(-sig * Na / u ** 3) * (-mp.expm1(-sig * dN / u ** 3)), pts)
    return float(mp.log1p(-num / den))


def _problem(T):
    tab = oracle.table_build("bb", T, SIG)
    return oracle.Problem(2, 2, 2, 1e16, 100.0, [((0, 0, 0), 1e48, "tab", 0.0)], tables=[tab], sigma0=SIG)


@pytest.mark.parametrize("T", [3e4, 5e4])
@pytest.mark.parametrize("Na,rel", [
    (0.0, None), (3e9, None),              # below the first node (linear piece), then into the table
    (1e12, 1e-9), (1e12, 1e-3),
    (4e16, 1e-9), (4e16, 1e-4), (4e16, 3.0),
    (2e18, 1e-6), (2e18, 0.5),
    (6e19, 1e-9), (6e19, 0.2),
])
def test_table_difference_matches_the_spectrum(T, Na, rel):
    P = _problem(T)
    dN = 5e9 if rel is None else Na * rel
    ref = _dlnp_direct(T, Na, dN)
    got = P.dlnp(0, Na, dN)
    assert got < 0.0
    # inside the table (quintic Hermite in ln N with exact first and second
    # derivatives at 512 nodes) the difference is good to ~1e-12 relative, and a
    # thin difference keeps that accuracy instead of dropping to
    # eps |ln P| / |difference|; below the first node (1e10 cm^-2) P is the
    # straight line Q - N S(0), which departs from the spectrum by ~1e-8
    tol = 3e-8 if Na + dN <= 1e10 else 1e-10
    assert abs(got / ref - 1.0) <= tol, (Na, dN, got, ref)
