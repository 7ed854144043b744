"""The paper's verification workloads (Sect. 5) through the GPU solver.

Sect. 5.1: a point source in one zone of a 550 x 128 x 256 logarithmic grid; the paper
finds the relative error against the analytic point-mass potential at about 10% even in
the zones adjacent to the source.  Both the float64 and the mixed-precision solve are
checked against that bound and against the oracle's exact discrete solution."""
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
