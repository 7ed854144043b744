"""Seeded synthetic inputs for the spherical-polar Poisson solve.

This module is shared by the CPU oracle, the tests, the smoke check and the
benchmark.  It only builds grids and source densities; it holds none of the
solver's arithmetic (no Laplacian, no transform, no eigenproblem).

Grids follow the discretisation of Sect. 3.1 of Mueller & Chan (2018):
cell interfaces in r and theta, a uniform periodic phi grid, and cell
centres taken as the midpoints of their interfaces (the paper's point-source
zone (j,k)=(32,128) at theta=0.246 pi, phi=0.996 pi in Sect. 5.1 matches
midpoint centres with 1-based indices).

Workload recipes (all densities sampled at cell centres, G = 1):

* ``sphere_blob``  32x16x32, uniform r in (0,1]: a homogeneous sphere rho=1
  for r<0.5 plus a Gaussian blob (sigma 0.05, amplitude 10) centred at r=0.3
  in a seeded direction.
* ``stellar_noise`` 128x64x128 on the log grid: the profile
  (1+(r/0.1)^2)^-1.5 times (1 + 0.05 N(0,1) per zone) plus one off-centre
  zone near r=0.3 holding 1% of the profile's mass.
* ``stellar_sh``   550x128x256 on the log grid: the same profile times
  (1 + 0.1 P/max|P|), P a seeded sum of real spherical harmonics with
  1 <= l <= 20 and N(0,1) coefficients.
* ``ragged_batch`` 64 instances, Nr uniform in [64,512], Ntheta in
  {32,64,96,128}, Nphi = 2 Ntheta, profile core radius uniform in
  [0.05,0.2] and one point-mass zone (1% of the mass) at a random position.
* ``served_stream`` Poisson arrivals (mean 200/s); 90% of the requests solve one of
  the 64 ragged-batch instances, 10% the 550x128x256 stellar workload.

The log-stretched radial grid has an origin cell: r_{1/2} = 0 and
r_{i+1/2} = 10^(-3 + 3 (i-1)/(Nr-1)) for i = 1..Nr, so it spans [1e-3, 1]
after the first cell.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

OUTER_MULTIPOLE = 0
OUTER_DIRICHLET = 1


@dataclass
class Problem:
    """One Poisson problem: grid interfaces, phi resolution and rho[i][j][k]."""

    name: str
    r_if: np.ndarray          # (Nr+1,) radial interfaces, strictly increasing, r_if[0] >= 0
    th_if: np.ndarray         # (Ntheta+1,) polar interfaces from 0 to pi
    nphi: int                 # number of uniform phi zones
    rho: np.ndarray           # (Nr, Ntheta, Nphi) float64, phi fastest
    outer_bc: int = OUTER_MULTIPOLE
    G: float = 1.0
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (len(self.r_if) - 1, len(self.th_if) - 1, self.nphi)

    @property
    def zones(self) -> int:
        nr, nt, npf = self.shape
        return nr * nt * npf


# --------------------------------------------------------------------- grids

def uniform_r_interfaces(nr: int, r_in: float = 0.0, r_out: float = 1.0) -> np.ndarray:
    return np.linspace(r_in, r_out, nr + 1)


def log_r_interfaces(nr: int, r_min: float = 1e-3, r_max: float = 1.0,
                     origin_cell: bool = True) -> np.ndarray:
    """Log-spaced interfaces; with ``origin_cell`` the first cell reaches r=0."""
    if origin_cell:
        out = np.empty(nr + 1)
        out[0] = 0.0
        out[1:] = np.logspace(math.log10(r_min), math.log10(r_max), nr)
        return out
    return np.logspace(math.log10(r_min), math.log10(r_max), nr + 1)


def uniform_theta_interfaces(nth: int) -> np.ndarray:
    return np.linspace(0.0, math.pi, nth + 1)


def centres(interfaces: np.ndarray) -> np.ndarray:
    return 0.5 * (interfaces[:-1] + interfaces[1:])


def phi_centres(nphi: int) -> np.ndarray:
    return (np.arange(nphi) + 0.5) * (2.0 * math.pi / nphi)


def cell_volumes(r_if, th_if, nphi) -> np.ndarray:
    """Exact volume of every spherical-polar cell, shape (Nr, Ntheta)."""
    dv_r = (r_if[1:] ** 3 - r_if[:-1] ** 3) / 3.0
    dv_t = np.cos(th_if[:-1]) - np.cos(th_if[1:])
    return dv_r[:, None] * dv_t[None, :] * (2.0 * math.pi / nphi)


# ----------------------------------------------------------------- densities

def _cartesian(r_if, th_if, nphi):
    r = centres(r_if)[:, None, None]
    t = centres(th_if)[None, :, None]
    p = phi_centres(nphi)[None, None, :]
    return (r * np.sin(t) * np.cos(p), r * np.sin(t) * np.sin(p),
            r * np.cos(t) * np.ones_like(p))


def _random_direction(rng):
    mu = rng.uniform(-1.0, 1.0)
    ph = rng.uniform(0.0, 2.0 * math.pi)
    return math.acos(mu), ph


def _profile(r_if, core=0.1):
    r = centres(r_if)
    return (1.0 + (r / core) ** 2) ** -1.5


def _add_point_mass(rho, r_if, th_if, nphi, rng, r_target=0.3, frac=0.01, i=None):
    vol = cell_volumes(r_if, th_if, nphi)
    mass = float(np.sum(rho * vol[:, :, None]))
    if i is None:
        i = int(np.argmin(np.abs(centres(r_if) - r_target)))
    j = int(rng.integers(0, len(th_if) - 1))
    k = int(rng.integers(0, nphi))
    rho[i, j, k] += frac * mass / vol[i, j]
    return (i, j, k)


def _legendre_assoc(l, m, x):
    """Associated Legendre P_l^m(x) (no Condon-Shortley phase), by recurrence."""
    pmm = np.ones_like(x)
    if m > 0:
        somx2 = np.sqrt(np.maximum(0.0, 1.0 - x * x))
        fact = 1.0
        for _ in range(m):
            pmm = pmm * fact * somx2
            fact += 2.0
    if l == m:
        return pmm
    pmmp1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pmmp1
    pll = pmmp1
    for ll in range(m + 2, l + 1):
        pll = ((2 * ll - 1) * x * pmmp1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pmmp1 = pmmp1, pll
    return pll


def _real_sh_field(th_c, ph_c, lmax, rng):
    """sum_{l=1..lmax} sum_{m=-l..l} a_lm Y^real_lm(theta, phi), a ~ N(0,1)."""
    x = np.cos(th_c)
    out = np.zeros((len(th_c), len(ph_c)))
    for l in range(1, lmax + 1):
        for m in range(0, l + 1):
            norm = math.sqrt((2 * l + 1) / (4 * math.pi)
                             * math.exp(math.lgamma(l - m + 1) - math.lgamma(l + m + 1)))
            plm = norm * _legendre_assoc(l, m, x)
            if m == 0:
                out += rng.standard_normal() * plm[:, None]
            else:
                a, b = rng.standard_normal(2)
                out += math.sqrt(2.0) * plm[:, None] * (a * np.cos(m * ph_c)[None, :]
                                                        + b * np.sin(m * ph_c)[None, :])
    return out


def sphere_blob(seed: int = 1, nr=32, nth=16, nphi=32) -> Problem:
    rng = np.random.default_rng(seed)
    r_if = uniform_r_interfaces(nr)
    th_if = uniform_theta_interfaces(nth)
    x, y, z = _cartesian(r_if, th_if, nphi)
    r = np.sqrt(x * x + y * y + z * z)
    t0, p0 = _random_direction(rng)
    x0 = 0.3 * np.array([math.sin(t0) * math.cos(p0), math.sin(t0) * math.sin(p0), math.cos(t0)])
    d2 = (x - x0[0]) ** 2 + (y - x0[1]) ** 2 + (z - x0[2]) ** 2
    rho = (r < 0.5).astype(np.float64) + 10.0 * np.exp(-d2 / (2 * 0.05 ** 2))
    return Problem("sphere_blob", r_if, th_if, nphi, np.ascontiguousarray(rho), seed=seed,
                   meta={"blob_centre": x0.tolist()})


def stellar_noise(seed: int = 2, nr=128, nth=64, nphi=128) -> Problem:
    rng = np.random.default_rng(seed)
    r_if = log_r_interfaces(nr)
    th_if = uniform_theta_interfaces(nth)
    prof = _profile(r_if)[:, None, None]
    rho = prof * (1.0 + 0.05 * rng.standard_normal((nr, nth, nphi)))
    pm = _add_point_mass(rho, r_if, th_if, nphi, rng)
    return Problem("stellar_noise", r_if, th_if, nphi, np.ascontiguousarray(rho), seed=seed,
                   meta={"point_mass_zone": pm})


def stellar_sh(seed: int = 3, nr=550, nth=128, nphi=256, lmax=20) -> Problem:
    rng = np.random.default_rng(seed)
    r_if = log_r_interfaces(nr)
    th_if = uniform_theta_interfaces(nth)
    p = _real_sh_field(centres(th_if), phi_centres(nphi), lmax, rng)
    ang = 1.0 + 0.1 * p / np.max(np.abs(p))
    rho = _profile(r_if)[:, None, None] * ang[None, :, :]
    return Problem("stellar_sh", r_if, th_if, nphi, np.ascontiguousarray(rho), seed=seed)


RAGGED_NTHETA = (32, 64, 96, 128)


def ragged_instance(idx: int, base_seed: int = 4) -> Problem:
    rng = np.random.default_rng(base_seed + idx)
    nr = int(rng.integers(64, 513))
    nth = int(RAGGED_NTHETA[int(rng.integers(0, len(RAGGED_NTHETA)))])
    nphi = 2 * nth
    core = float(rng.uniform(0.05, 0.2))
    r_if = log_r_interfaces(nr)
    th_if = uniform_theta_interfaces(nth)
    rho = np.repeat(np.repeat(_profile(r_if, core)[:, None, None], nth, 1), nphi, 2)
    i = int(rng.integers(0, nr))
    pm = _add_point_mass(rho, r_if, th_if, nphi, rng, i=i)
    return Problem(f"ragged_{idx}", r_if, th_if, nphi, np.ascontiguousarray(rho),
                   seed=base_seed + idx, meta={"core": core, "point_mass_zone": pm})


def ragged_batch(n: int = 64, base_seed: int = 4):
    return [ragged_instance(i, base_seed) for i in range(n)]


def served_stream(n_requests: int, rate_hz: float = 200.0, seed: int = 5,
                  big_fraction: float = 0.1, n_grids: int = 64):
    """Arrival times (s) and problems of the served workload: Poisson arrivals; 90% of
    the requests solve one of the ``n_grids`` ragged-batch instances (their grids and
    densities), 10% the 550x128x256 stellar workload.

    Returns a list of dicts with keys ``t`` (arrival time) and ``problem`` (an index
    into the ragged batch, or -1 for the 550x128x256 workload)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for q in range(n_requests):
        big = rng.uniform() < big_fraction
        out.append({"t": float(t[q]), "problem": -1 if big else int(rng.integers(0, n_grids))})
    return out


def stellar_request(shape, seed: int) -> Problem:
    """Density for one served request of the given shape (log grid, stellar profile)."""
    nr, nth, nphi = shape
    rng = np.random.default_rng(seed)
    core = float(rng.uniform(0.05, 0.2))
    r_if = log_r_interfaces(nr)
    th_if = uniform_theta_interfaces(nth)
    rho = np.repeat(np.repeat(_profile(r_if, core)[:, None, None], nth, 1), nphi, 2)
    pm = _add_point_mass(rho, r_if, th_if, nphi, rng, i=int(rng.integers(0, nr)))
    return Problem(f"served_{nr}x{nth}x{nphi}", r_if, th_if, nphi, np.ascontiguousarray(rho),
                   seed=seed, meta={"core": core, "point_mass_zone": pm})


def random_small(nr, nth, nphi, seed=0, grid="log", r_inner=0.0,
                 outer_bc=OUTER_MULTIPOLE) -> Problem:
    """Small random problem for parity tests: rho ~ U(0,1) plus a smooth part."""
    rng = np.random.default_rng(seed)
    if grid == "log":
        if r_inner > 0:
            r_if = np.logspace(math.log10(r_inner), 0.0, nr + 1)
        else:
            r_if = log_r_interfaces(nr, r_min=1e-2)
    elif grid == "uniform":
        r_if = uniform_r_interfaces(nr, r_in=r_inner)
    else:  # random strictly increasing spacing
        d = rng.uniform(0.5, 1.5, nr)
        r_if = np.concatenate([[r_inner], r_inner + np.cumsum(d) / d.sum() * (1.0 - r_inner)])
    th_if = uniform_theta_interfaces(nth)
    rho = rng.uniform(0.0, 1.0, (nr, nth, nphi)) + _profile(r_if, 0.3)[:, None, None]
    return Problem(f"small_{nr}x{nth}x{nphi}", r_if, th_if, nphi, np.ascontiguousarray(rho),
                   outer_bc=outer_bc, seed=seed)


def random_theta_interfaces(nth, seed=0) -> np.ndarray:
    """Non-uniform, strictly increasing polar interfaces from 0 to pi."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.6, 1.4, nth)
    return np.concatenate([[0.0], np.cumsum(d) / d.sum() * math.pi])


def symmetric_theta_interfaces(nth, seed=0) -> np.ndarray:
    """Non-uniform polar interfaces from 0 to pi, mirror-symmetric about the equator
    (theta_j + theta_{nth-j} = pi exactly); nth must be even."""
    if nth % 2:
        raise ValueError("a mirror-symmetric grid needs an even number of zones")
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.6, 1.4, nth // 2)
    half = np.cumsum(d) / d.sum() * (0.5 * math.pi)
    lower = np.concatenate([[0.0], half[:-1]])
    th = np.concatenate([lower, [0.5 * math.pi], (math.pi - lower[::-1])])
    th[-1] = math.pi
    return th


# ------------------------------------------- ellipsoid of Sect. 5.2 (a, b, c) = (1, 1.5, 2)
def ellipsoid_r_interfaces(kind: str, nr: int = 512) -> np.ndarray:
    """The three radial grids of Sect. 5.2 at Nr zones: "uniform" in (0, 5]; "stretched",
    the same uniform zones up to r = 1.5 and beyond a constant ratio r_{i+1}/r_i = 1 + dr
    (dr = 5/Nr: r_out = 48.7 at Nr = 512); "jump", the uniform spacing up to r = 1.5 and
    1.5 dr beyond."""
    dr = 5.0 / nr
    if kind == "uniform":
        return np.arange(nr + 1) * dr
    n_in = int(math.ceil(1.5 / dr - 1e-9))          # first interface at or beyond 1.5
    inner = np.arange(n_in + 1) * dr
    m = nr - n_in
    if kind == "stretched":
        outer = inner[-1] * (1.0 + dr) ** np.arange(1, m + 1)
    elif kind == "jump":
        outer = inner[-1] + 1.5 * dr * np.arange(1, m + 1)
    else:
        raise ValueError(kind)
    return np.concatenate([inner, outer])


def ellipsoid_density(r_if, th_if, nphi, a=1.0, b=1.5, c=2.0, q=8) -> np.ndarray:
    """Cell-averaged density of the homogeneous (rho = 1) ellipsoid centred on the origin
    with semi-axes a, b, c along x, y, z: the fraction of each cell's volume inside.
    The ellipsoid is star-shaped about the origin, so along a direction n the inside
    part of a cell is r < r_s(n) = 1/sqrt(n_x^2/a^2 + n_y^2/b^2 + n_z^2/c^2): the radial
    integral of r^2 dr is exact, and the solid angle is integrated with a q x q
    Gauss-Legendre rule in (cos theta, phi) per angular cell (a finer sub-volume
    integration than the recursive octant splitting of Sect. 5.2)."""
    r_if = np.asarray(r_if, dtype=np.float64)
    th_if = np.asarray(th_if, dtype=np.float64)
    nr, nth = len(r_if) - 1, len(th_if) - 1
    gx, gw = np.polynomial.legendre.leggauss(q)
    mu_if = np.cos(th_if)
    dphi = 2.0 * math.pi / nphi
    r3 = r_if ** 3
    dv3 = r3[1:] - r3[:-1]
    rho = np.zeros((nr, nth, nphi))
    rmax = max(a, b, c)
    imax = min(nr, int(np.searchsorted(r_if, rmax, side="right")))
    for j in range(nth):
        # q x q directions of every phi cell of row j: mu in [cos th_{j+1}, cos th_j]
        mu = 0.5 * (mu_if[j] + mu_if[j + 1]) + 0.5 * (mu_if[j] - mu_if[j + 1]) * gx           # (q,)
        ph = (np.arange(nphi)[:, None] + 0.5 + 0.5 * gx[None, :]) * dphi                        # (nphi, q)
        st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
        nx = st[None, :, None] * np.cos(ph)[:, None, :]
        ny = st[None, :, None] * np.sin(ph)[:, None, :]
        nz = np.broadcast_to(mu[None, :, None], nx.shape)
        rs = 1.0 / np.sqrt(nx * nx / a ** 2 + ny * ny / b ** 2 + nz * nz / c ** 2)           # (nphi, q, q)
        w = (gw[:, None] * gw[None, :]) / 4.0                                                   # sums to 1
        rs3 = rs ** 3
        for i in range(imax):
            frac = np.clip((rs3 - r3[i]) / dv3[i], 0.0, 1.0)
            rho[i, j, :] = np.einsum("kab,ab->k", frac, w)
    return rho


def ellipsoid(kind: str = "uniform", nr: int = 512, nth: int = 128, nphi: int = 256) -> Problem:
    """Sect. 5.2's convergence test: the (1, 1.5, 2) ellipsoid on one of its radial grids."""
    r_if = ellipsoid_r_interfaces(kind, nr)
    th_if = uniform_theta_interfaces(nth)
    return Problem(f"ellipsoid_{kind}", r_if, th_if, nphi, ellipsoid_density(r_if, th_if, nphi))


CONFIGS = {
    "sphere_blob": sphere_blob,
    "stellar_noise": stellar_noise,
    "stellar_sh": stellar_sh,
}
