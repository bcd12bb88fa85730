"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This module holds no arithmetic of the photoionisation method: it only draws
density fields, source positions, rates and spectra from fixed seeds and
packages them with the physical constants of each workload.  Both the CUDA
path and the CPU oracle are fed from here; neither is imported by it.

Workloads (sizes, distributions and seeds):
  * ``stromgren_corner``: uniform hydrogen, monochromatic source at the corner
    vertex, box side 1.5 Stromgren radii (the 3D analogue of the spherical
    Stromgren test of Sect. 3.2 of Mackey 2012);
  * ``lognormal_bb``: lognormal density from a Gaussian random field with
    P(k) ~ k^-3, blackbody source at the centre vertex;
  * ``clumpy``: lognormal density times spherical clumps;
  * ``batch``: many uniform grids of uneven sizes, densities and rates;
  * ``multisource``: lognormal density with many blackbody sources;
  * ``planar_slab``: the plane-parallel slab of Sect. 3.1 (source at infinity,
    uniform hydrogen, no recombinations);
  * ``plane_random``: small random grid lit by a plane-parallel source;
  * ``stromgren_bb``: uniform gas and a blackbody source at the corner vertex,
    at a chosen cell optical depth (the multi-frequency test of Sect. 4).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Physical constants of the workloads (CGS).
ALPHA_B = 2.59e-13      # case-B recombination coefficient at 1e4 K [cm^3/s]
SIGMA0 = 6.3e-18        # threshold photoionisation cross-section [cm^2]
TAU0 = 0.6              # optical-depth floor of the short-characteristics weights
X_NEUTRAL = 1.0 - 1e-6  # initial neutral fraction of neutral gas


@dataclasses.dataclass
class Source:
    pos: tuple            # position in cell units (vertex coordinates), snapped by the consumer
    Q: float              # ionising photons per second
    spectrum: str = "mono"  # "mono" or "bb"
    T: float = 0.0        # blackbody temperature [K] for "bb"
    plane: int = -1       # -1: point source; else 2*axis + back, a plane-parallel source whose
                          # rays run along +axis (back 0) or -axis (back 1); Q is then a flux [cm^-2 s^-1]


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float                     # cell side [cm]
    nH: np.ndarray                # (nz, ny, nx) float64 hydrogen density [cm^-3]
    x0: np.ndarray                # (nz, ny, nx) float64 initial neutral fraction
    sources: List[Source]
    alpha: float = ALPHA_B
    sigma0: float = SIGMA0
    tau0: float = TAU0
    uniform_n: Optional[float] = None   # set when nH is uniform
    t_rec: float = 0.0            # 1/(alpha <n>) [s]

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz


def stromgren_radius(Q: float, n: float, alpha: float = ALPHA_B) -> float:
    """R_S = (3 Q / (4 pi n^2 alpha))^(1/3)  [cm]."""
    return (3.0 * Q / (4.0 * math.pi * n * n * alpha)) ** (1.0 / 3.0)


def gaussian_random_field(n: int, seed: int, slope: float = -3.0) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian random field on an n^3 grid
    with power spectrum P(k) ~ k^slope (k = 0 removed), float64, shape (n,n,n)."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    fk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kz = np.fft.rfftfreq(n)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)          # sqrt(P) = k^(slope/2)
    amp[0, 0, 0] = 0.0
    g = np.fft.irfftn(fk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_density(n: int, sigma_ln: float, seed: int, mean: float = 100.0) -> np.ndarray:
    """n_H = mean * exp(sigma g - sigma^2/2), rescaled to a sample mean of exactly `mean`."""
    g = gaussian_random_field(n, seed)
    rho = np.exp(sigma_ln * g - 0.5 * sigma_ln * sigma_ln)
    rho *= mean / rho.mean()
    return rho


def add_clumps(rho: np.ndarray, count: int, seed: int, rmin: float = 2.0, rmax: float = 8.0,
               od_min: float = 10.0, od_max: float = 100.0) -> np.ndarray:
    """Multiply `count` spheres (centres uniform, radius uniform in [rmin,rmax]
    cells, overdensity log-uniform in [od_min, od_max]) into rho (in place)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = rho.shape
    for _ in range(count):
        c = rng.uniform(0.0, 1.0, 3) * np.array([nx, ny, nz])
        r = rng.uniform(rmin, rmax)
        od = math.exp(rng.uniform(math.log(od_min), math.log(od_max)))
        lo = np.maximum(np.floor(c - r).astype(int), 0)
        hi = np.minimum(np.ceil(c + r).astype(int) + 1, [nx, ny, nz])
        zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2]) + 0.5, np.arange(lo[1], hi[1]) + 0.5,
                                 np.arange(lo[0], hi[0]) + 0.5, indexing="ij")
        inside = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r
        sub = rho[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[inside] *= od
    return rho


def _uniform(n: int, value: float) -> np.ndarray:
    return np.full((n, n, n), value, dtype=np.float64)


def stromgren_corner(n: int = 32, n_H: float = 100.0, Q: float = 1e48, box_rs: float = 1.5) -> Workload:
    """Uniform static hydrogen, monochromatic source at the corner vertex,
    box side box_rs * R_S (R_S from alpha_B)."""
    L = box_rs * stromgren_radius(Q, n_H)
    w = Workload("stromgren_corner", n, n, n, L / n, _uniform(n, n_H), _uniform(n, X_NEUTRAL),
                 [Source((0.0, 0.0, 0.0), Q, "mono")], uniform_n=n_H)
    w.t_rec = 1.0 / (ALPHA_B * n_H)
    return w


def lognormal_bb(n: int = 128, sigma_ln: float = 1.0, seed: int = 1202, Q: float = 1e48,
                 T: float = 4e4, box_rs: float = 2.5, spectrum: str = "bb") -> Workload:
    """Lognormal density (mean 100), source at the centre vertex."""
    nH = lognormal_density(n, sigma_ln, seed)
    L = box_rs * stromgren_radius(Q, 100.0)
    w = Workload("lognormal_" + spectrum, n, n, n, L / n, nH, _uniform(n, X_NEUTRAL),
                 [Source((n / 2, n / 2, n / 2), Q, spectrum, T if spectrum == "bb" else 0.0)])
    w.t_rec = 1.0 / (ALPHA_B * 100.0)
    return w


def clumpy(n: int = 256, sigma_ln: float = 1.5, seed: int = 1203, clump_seed: int = 1303,
           n_clumps: int = 200, Q: float = 1e48, T: float = 4e4, box_rs: float = 2.5,
           spectrum: str = "mono") -> Workload:
    """Lognormal density (sigma_ln 1.5) times clumps, source at the centre vertex."""
    nH = add_clumps(lognormal_density(n, sigma_ln, seed), n_clumps, clump_seed)
    L = box_rs * stromgren_radius(Q, 100.0)
    w = Workload("clumpy_" + spectrum, n, n, n, L / n, nH, _uniform(n, X_NEUTRAL),
                 [Source((n / 2, n / 2, n / 2), Q, spectrum, T if spectrum == "bb" else 0.0)])
    w.t_rec = 1.0 / (ALPHA_B * 100.0)
    return w


def batch(count: int = 64, seed: int = 1204, sides=(32, 48, 64, 96, 128), box_rs: float = 2.0) -> List[Workload]:
    """Independent uniform grids: side uniform in `sides`, n log-uniform in
    [10, 1000], Q log-uniform in [1e47, 1e50], source at a random interior
    vertex, box side box_rs * R_S of that grid."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(count):
        n = int(rng.choice(sides))
        nH = math.exp(rng.uniform(math.log(10.0), math.log(1000.0)))
        Q = math.exp(rng.uniform(math.log(1e47), math.log(1e50)))
        v = rng.integers(1, n, size=3)
        L = box_rs * stromgren_radius(Q, nH)
        w = Workload(f"batch{g}", n, n, n, L / n, _uniform(n, nH), _uniform(n, X_NEUTRAL),
                     [Source((float(v[0]), float(v[1]), float(v[2])), Q, "mono")], uniform_n=nH)
        w.t_rec = 1.0 / (ALPHA_B * nH)
        out.append(w)
    return out


def multisource(n: int = 512, sigma_ln: float = 1.0, seed: int = 1205, nsrc: int = 16,
                box_rs: float = 2.0) -> Workload:
    """Lognormal density (mean 100) with nsrc blackbody sources: T uniform in
    [3e4, 5e4] K, Q log-uniform in [1e47, 1e49], positions uniform in the box."""
    nH = lognormal_density(n, sigma_ln, seed)
    rng = np.random.default_rng(seed + 10000)
    srcs = []
    Qtot = 0.0
    for _ in range(nsrc):
        T = rng.uniform(3e4, 5e4)
        Q = math.exp(rng.uniform(math.log(1e47), math.log(1e49)))
        pos = tuple(float(p) for p in rng.uniform(0.0, n, 3))
        srcs.append(Source(pos, Q, "bb", T))
        Qtot += Q
    L = box_rs * stromgren_radius(Qtot, 100.0)
    w = Workload("multisource", n, n, n, L / n, nH, _uniform(n, X_NEUTRAL), srcs)
    w.t_rec = 1.0 / (ALPHA_B * 100.0)
    return w


def small_random(n: int = 12, seed: int = 7, nsrc: int = 1, spectrum: str = "mono",
                 sigma_ln: float = 1.0, x_lo: float = 0.0, Q: float = 1e48,
                 box_rs: float = 1.0, ny: Optional[int] = None, nz: Optional[int] = None) -> Workload:
    """Small non-cubic grid with a lognormal-like random density, random
    neutral fractions in [x_lo, 1] and random source vertices; for parity tests."""
    rng = np.random.default_rng(seed)
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    nH = 100.0 * np.exp(sigma_ln * rng.standard_normal((nz, ny, n)) - 0.5 * sigma_ln ** 2)
    x0 = rng.uniform(x_lo, 1.0, (nz, ny, n))
    srcs = []
    for _ in range(nsrc):
        pos = (float(rng.integers(0, n + 1)), float(rng.integers(0, ny + 1)), float(rng.integers(0, nz + 1)))
        T = float(rng.uniform(3e4, 5e4))
        srcs.append(Source(pos, Q * float(rng.uniform(0.5, 2.0)), spectrum, T if spectrum == "bb" else 0.0))
    L = box_rs * stromgren_radius(Q, 100.0)
    w = Workload("small_random", n, ny, nz, L / n, nH, x0, srcs)
    w.t_rec = 1.0 / (ALPHA_B * 100.0)
    return w


def planar_slab(n: int = 100, F: float = 1e9, n_H: float = 100.0, dtau: float = 10.0, ny: int = 1, nz: int = 1,
                axis: int = 0, back: int = 0) -> Workload:
    """Sect. 3.1: a slab of n cells of uniform hydrogen lit from one face by a
    monochromatic plane-parallel flux F [cm^-2 s^-1], cell optical depth dtau
    at x = 1, recombinations off (alpha = 0).  The cell count n lies along
    `axis`; the grid is n x ny x nz cells in that axis order."""
    dx = dtau / (SIGMA0 * n_H)
    dims = [ny, nz]
    shape_xyz = [0, 0, 0]
    shape_xyz[axis] = n
    shape_xyz[(axis + 1) % 3] = dims[0]
    shape_xyz[(axis + 2) % 3] = dims[1]
    nx_, ny_, nz_ = shape_xyz
    full = np.full((nz_, ny_, nx_), n_H, dtype=np.float64)
    w = Workload("planar_slab", nx_, ny_, nz_, dx, full, np.full((nz_, ny_, nx_), X_NEUTRAL),
                 [Source((0.0, 0.0, 0.0), F, "mono", 0.0, 2 * axis + back)], alpha=0.0, uniform_n=n_H)
    return w


def plane_random(n: int = 12, seed: int = 11, axis: int = 0, back: int = 0, F: float = 1e9,
                 spectrum: str = "mono", T: float = 4e4, sigma_ln: float = 1.0, x_lo: float = 0.0,
                 dtau: float = 2.0, ny: Optional[int] = None, nz: Optional[int] = None,
                 point_Q: float = 0.0) -> Workload:
    """Small non-cubic grid with a lognormal-like random density and random
    neutral fractions in [x_lo, 1], lit by one plane-parallel source (flux F)
    and, if point_Q > 0, also by a point source at a random vertex.  The cell
    optical depth at the mean density and x = 1 is dtau."""
    rng = np.random.default_rng(seed)
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    nH = 100.0 * np.exp(sigma_ln * rng.standard_normal((nz, ny, n)) - 0.5 * sigma_ln ** 2)
    x0 = rng.uniform(x_lo, 1.0, (nz, ny, n))
    srcs = [Source((0.0, 0.0, 0.0), F, spectrum, T if spectrum == "bb" else 0.0, 2 * axis + back)]
    if point_Q > 0:
        pos = (float(rng.integers(0, n + 1)), float(rng.integers(0, ny + 1)), float(rng.integers(0, nz + 1)))
        srcs.append(Source(pos, point_Q, spectrum, T if spectrum == "bb" else 0.0))
    w = Workload("plane_random", n, ny, nz, dtau / (SIGMA0 * 100.0), nH, x0, srcs)
    w.t_rec = 1.0 / (ALPHA_B * 100.0)
    return w


def stromgren_bb(dtau0: float, tau_s: float = 240.0, n_H: float = 10.0, T: float = 37500.0,
                 box: float = 1.1) -> Workload:
    """Multi-frequency Stromgren test (Sect. 4) in 3D: uniform hydrogen n_H, a
    blackbody source at the corner vertex, cell optical depth dtau0 at nu0 and
    x = 1.  The source rate is set so that the Stromgren radius is tau_s
    optical depths at nu0 (R_S = tau_s / (sigma0 n_H)); the box side is box R_S,
    so the grid has ceil(box tau_s / dtau0) cells per side."""
    R_S = tau_s / (SIGMA0 * n_H)
    Q = 4.0 * math.pi / 3.0 * ALPHA_B * n_H ** 2 * R_S ** 3
    dx = dtau0 / (SIGMA0 * n_H)
    n = int(math.ceil(box * tau_s / dtau0))
    w = Workload(f"stromgren_bb_dtau{dtau0:g}", n, n, n, dx, _uniform(n, n_H), _uniform(n, X_NEUTRAL),
                 [Source((0.0, 0.0, 0.0), Q, "bb", T)], uniform_n=n_H)
    w.t_rec = 1.0 / (ALPHA_B * n_H)
    return w
