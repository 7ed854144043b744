"""Pins for the CPU oracle: each test checks it against something other than itself
(brute-force linear algebra, closed forms, continuum limits, invariants, and the
paper's own worked example)."""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import sph_poisson as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def geo_of(p):
    return O.Geometry(p.r_if, p.th_if, p.nphi)


# ------------------------------------------------------------------ O1 vs O2
TINY = [
    # nr, nth, nphi, grid, r_inner, outer_bc
    (5, 4, 6, "log", 0.0, O.OUTER_MULTIPOLE),
    (6, 5, 8, "uniform", 0.0, O.OUTER_MULTIPOLE),
    (4, 3, 5, "rand", 0.2, O.OUTER_MULTIPOLE),
    (5, 4, 6, "log", 0.0, O.OUTER_DIRICHLET),
    (4, 6, 9, "uniform", 0.3, O.OUTER_DIRICHLET),
    (3, 1, 4, "uniform", 0.0, O.OUTER_MULTIPOLE),     # one theta zone
    (4, 4, 1, "uniform", 0.0, O.OUTER_MULTIPOLE),     # axisymmetric, Nphi = 1
    (1, 3, 4, "uniform", 0.5, O.OUTER_MULTIPOLE),     # one radial shell
    (7, 8, 12, "rand", 0.0, O.OUTER_MULTIPOLE),
]


@pytest.mark.parametrize("nr,nth,nphi,grid,rin,bc", TINY)
def test_separated_equals_dense_lu(nr, nth, nphi, grid, rin, bc):
    p = W.random_small(nr, nth, nphi, seed=nr * 7 + nth, grid=grid, r_inner=rin)
    g = geo_of(p)
    a = O.solve_separated(g, p.rho, outer_bc=bc)
    b = O.solve_dense(g, p.rho, outer_bc=bc)
    assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= 1e-13


def test_separated_equals_dense_lu_nonuniform_theta():
    p = W.random_small(5, 6, 8, seed=11, grid="log")
    th = W.random_theta_interfaces(6, seed=3)
    g = O.Geometry(p.r_if, th, p.nphi)
    a = O.solve_separated(g, p.rho)
    b = O.solve_dense(g, p.rho)
    assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= 1e-13


@pytest.mark.parametrize("nr,nth,nphi,grid,rin,bc", TINY[:5])
def test_exact_solve_equals_dense_lu(nr, nth, nphi, grid, rin, bc):
    p = W.random_small(nr, nth, nphi, seed=nr * 7 + nth, grid=grid, r_inner=rin)
    g = geo_of(p)
    a = O.solve_exact(g, p.rho, outer_bc=bc)
    b = O.solve_dense(g, p.rho, outer_bc=bc)
    assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= 2e-14


def test_exact_solve_converges_and_is_a_fixed_point():
    p = W.stellar_noise()
    g = geo_of(p)
    phi, hist = O.solve_exact(g, p.rho, return_history=True)
    assert hist[-1] <= 1e-15 and len(hist) <= 3
    plain = O.solve_separated(g, p.rho)
    # the plain separated solve is within the float64 forward-error level of the exact one
    assert np.max(np.abs(plain - phi)) / np.max(np.abs(phi)) <= 2e-12
    eta, _ = O.residuals(g, phi, p.rho)
    assert eta <= 1e-15


def test_backward_error_moderate_grid():
    p = W.stellar_noise()
    g = geo_of(p)
    phi = O.solve_separated(g, p.rho)
    eta, _ = O.residuals(g, phi, p.rho)
    assert eta <= 1e-14


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("bc", [O.OUTER_MULTIPOLE, O.OUTER_DIRICHLET])
def test_gauss_law_spherical_source(bc):
    """A spherically symmetric source excites only l=0; the conservative form then
    fixes Phi by the enclosed mass (flux through r_{i+1/2} = G M_enc)."""
    p = W.sphere_blob()
    g = geo_of(p)
    rho_r = (g.rc < 0.5).astype(float) + 0.3 * np.exp(-g.rc)
    rho = np.broadcast_to(rho_r[:, None, None], (g.nr, g.nth, g.nphi))
    phi = O.solve_separated(g, rho, outer_bc=bc)
    ex = O.gauss_law_potential(g, rho_r, outer_bc=bc)
    assert np.max(np.abs(phi - ex[:, None, None])) / np.max(np.abs(ex)) <= 1e-13
    # log grid with an inner zero-flux boundary
    r_if = np.logspace(-2, 0, 41)
    g2 = O.Geometry(r_if, W.uniform_theta_interfaces(8), 8)
    rho_r2 = 1.0 / (1.0 + (g2.rc / 0.1) ** 2)
    phi2 = O.solve_separated(g2, np.broadcast_to(rho_r2[:, None, None], (40, 8, 8)), outer_bc=bc)
    ex2 = O.gauss_law_potential(g2, rho_r2, outer_bc=bc)
    assert np.max(np.abs(phi2 - ex2[:, None, None])) / np.max(np.abs(ex2)) <= 1e-13


def test_homogeneous_sphere_second_order():
    """Discrete Phi of a homogeneous sphere converges to the continuum potential at O(dr^2)."""
    errs = []
    for nr in (32, 64, 128):
        g = O.Geometry(W.uniform_r_interfaces(nr), W.uniform_theta_interfaces(4), 4)
        rho_r = (g.rc < 0.5).astype(float)
        phi = O.solve_separated(g, np.broadcast_to(rho_r[:, None, None], (nr, 4, 4)))
        ex = O.homogeneous_sphere_potential(g.rc, 0.5)
        errs.append(np.max(np.abs(phi[:, 0, 0] - ex)) / np.max(np.abs(ex)))
    assert errs[0] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_radial_stencil_exact_on_r_squared():
    """On a uniform radial grid the finite-volume Delta_r of r^2 is exactly 6 away from
    the outer boundary (the flux form integrates r^2 d(r^2)/dr exactly)."""
    g = O.Geometry(W.uniform_r_interfaces(12), W.uniform_theta_interfaces(5), 6)
    phi = np.broadcast_to((g.rc ** 2)[:, None, None], (12, 5, 6)).copy()
    lap = O.apply_laplacian(g, phi, O.OUTER_DIRICHLET)
    assert np.max(np.abs(lap[:-1] - 6.0)) <= 1e-12


@pytest.mark.parametrize("func,eig", [
    (lambda t, p: np.cos(t), -2.0),
    (lambda t, p: np.sin(t) * np.cos(p), -2.0),
    (lambda t, p: np.sin(t) ** 2 * np.sin(2 * p), -6.0),
    (lambda t, p: (3 * np.cos(t) ** 2 - 1) * np.ones_like(p), -6.0),
])
def test_angular_operator_converges_to_spherical_laplacian(func, eig):
    """Delta_hat_theta + S_j Delta_hat_phi applied to a spherical harmonic Y_l tends to
    -l(l+1) Y_l at second order in the angular spacing (solid-angle weighted L2 norm;
    the m=1 pole cells converge at first order in the max norm)."""
    errs = []
    for nth in (16, 32, 64):
        g = O.Geometry(W.uniform_r_interfaces(2), W.uniform_theta_interfaces(nth), 2 * nth)
        t = g.thc[:, None]
        ph = W.phi_centres(2 * nth)[None, :]
        u = np.broadcast_to(func(t, ph), (nth, 2 * nth)).copy()
        e2 = (O.angular_apply(g, u) - eig * u) ** 2
        errs.append(math.sqrt(np.sum(g.w[:, None] * e2) / (2.0 * 2 * nth)) / np.max(np.abs(eig * u)))
    assert errs[0] < 0.02
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_harmonic_function_second_order():
    """x = r sin(theta) cos(phi) is harmonic: the full stencil gives O(h^2) away from
    the radial boundaries (volume-weighted L2 norm; the pole cells are first order)."""
    errs = []
    for n in (8, 16, 32):
        g = O.Geometry(W.uniform_r_interfaces(n, 0.5, 1.5), W.uniform_theta_interfaces(n), 2 * n)
        x = (g.rc[:, None, None] * np.sin(g.thc)[None, :, None]
             * np.cos(W.phi_centres(2 * n))[None, None, :])
        inner = O.apply_laplacian(g, x, O.OUTER_DIRICHLET)[1:-1]
        vol = np.broadcast_to(g.cell_volume()[1:-1, :, None], inner.shape)
        errs.append(math.sqrt(np.sum(vol * inner ** 2) / np.sum(vol)))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


# ------------------------------------------------- |L||Phi| of the backward error
def _assembled_abs(g, phi, bc, kmat):
    """|A| |phi| with A assembled column by column from O3, plus the magnitude of the
    multipole boundary term (A then holds only the local stencil: the outer face is
    given a zero kappa matrix)."""
    n = g.nr * g.nth * g.nphi
    local_k = np.zeros((g.nth * g.nphi, g.nth * g.nphi)) if bc == O.OUTER_MULTIPOLE else None
    a = np.zeros((n, n))
    e = np.zeros(n)
    for c in range(n):
        e[:] = 0.0
        e[c] = 1.0
        a[:, c] = O.apply_laplacian(g, e.reshape(g.nr, g.nth, g.nphi), bc, local_k).reshape(n)
    out = (np.abs(a) @ np.abs(phi).reshape(n)).reshape(phi.shape)
    if bc == O.OUTER_MULTIPOLE:
        # the boundary term alone: full operator minus the local stencil
        term = O.apply_laplacian(g, phi, bc, kmat) - O.apply_laplacian(g, phi, bc, local_k)
        out[-1] += np.abs(term[-1])
    return out


ABS_GRIDS = [
    # nr, nth, nphi, grid, r_inner
    (5, 4, 6, "log", 0.0),
    (4, 6, 9, "rand", 0.3),
    (3, 1, 4, "uniform", 0.0),
    (4, 4, 1, "uniform", 0.0),
    (3, 5, 2, "rand", 0.1),
]


@pytest.mark.parametrize("bc", [O.OUTER_MULTIPOLE, O.OUTER_DIRICHLET])
@pytest.mark.parametrize("nr,nth,nphi,grid,rin", ABS_GRIDS)
def test_abs_apply_equals_assembled_abs_operator(nr, nth, nphi, grid, rin, bc):
    """abs_apply (the |L||Phi| denominator of the backward error eta, R13) equals the
    elementwise absolute value of the assembled finite-volume operator of Eq. fin_vol0-3
    times |Phi|, term for term (the diagonal counted as one coefficient), plus |outer
    term| for the multipole condition.  A dropped R_i, 1/w_j or S_j, or a scaled
    radial/theta/phi coefficient in abs_apply changes some entry and fails this."""
    p = W.random_small(nr, nth, nphi, seed=31 * nr + nth, grid=grid, r_inner=rin)
    g = geo_of(p)
    phi = np.random.default_rng(nr + nth + nphi).standard_normal((nr, nth, nphi))
    kmat = O.outer_operator_dense(g) if bc == O.OUTER_MULTIPOLE else None
    ref = _assembled_abs(g, phi, bc, kmat)
    got = O.abs_apply(g, phi, bc, kmat)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(ref)
    if bc == O.OUTER_MULTIPOLE:
        # the per-m eigenbasis form of the boundary term (used on large grids) agrees
        got_sep = O.abs_apply(g, phi, bc, None)
        assert np.max(np.abs(got_sep - ref)) <= 1e-12 * np.max(ref)


# --------------------------------------------------------- conservation form
@pytest.mark.parametrize("bc", [O.OUTER_MULTIPOLE, O.OUTER_DIRICHLET])
def test_discrete_divergence_theorem(bc):
    """sum_cells dV (L Phi) equals the flux through the outer surface only: every interior
    r, theta and phi flux cancels between neighbours."""
    p = W.random_small(5, 6, 8, seed=2, grid="rand", r_inner=0.1)
    g = geo_of(p)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((5, 6, 8))
    lap = O.apply_laplacian(g, phi, bc)
    vol = g.cell_volume()[:, :, None]
    grad = O.outer_gradient(g, phi[-1], bc)
    outer = g.r_out ** 2 * g.dphi * np.sum(g.w[:, None] * grad)
    total = np.sum(vol * lap)
    assert abs(total - outer) <= 1e-12 * np.sum(np.abs(vol * lap))


@pytest.mark.parametrize("bc", [O.OUTER_MULTIPOLE, O.OUTER_DIRICHLET])
def test_volume_weighted_operator_is_symmetric(bc):
    p = W.random_small(4, 5, 6, seed=5, grid="rand", r_inner=0.0)
    g = geo_of(p)
    mat = O.assemble_dense(g, bc)
    vol = np.repeat(g.cell_volume().reshape(-1), g.nphi)
    a = vol[:, None] * mat
    assert np.max(np.abs(a - a.T)) <= 1e-12 * np.max(np.abs(a))


def test_outer_operator_separated_equals_dense():
    p = W.random_small(3, 6, 10, seed=9)
    g = geo_of(p)
    k = O.outer_operator_dense(g)
    u = np.random.default_rng(1).standard_normal((6, 10))
    a = (k @ u.reshape(-1)).reshape(6, 10)
    b = O.outer_kappa_separated(g, u)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_multipole_boundary_mimics_unbounded_domain():
    """With sources inside r<0.5, the multipole outer boundary at r=1 reproduces the
    solution of a grid extended far outwards (identical zones up to r=1); a Dirichlet
    boundary at r=1 does not."""
    nth, nphi = 8, 8
    n_in = 32
    r_in = W.uniform_r_interfaces(n_in)
    ext = np.concatenate([r_in, 1.0 * np.exp(np.cumsum(np.full(160, 1.0 / 32)))])
    th = W.uniform_theta_interfaces(nth)
    g_in = O.Geometry(r_in, th, nphi)
    g_ext = O.Geometry(ext, th, nphi)
    rng = np.random.default_rng(4)
    rho = np.zeros((len(ext) - 1, nth, nphi))
    mask = g_ext.rc < 0.5
    rho[mask] = rng.uniform(0, 1, (int(mask.sum()), nth, nphi))
    far = O.solve_separated(g_ext, rho, outer_bc=O.OUTER_DIRICHLET)[:n_in]
    mp = O.solve_separated(g_in, rho[:n_in], outer_bc=O.OUTER_MULTIPOLE)
    di = O.solve_separated(g_in, rho[:n_in], outer_bc=O.OUTER_DIRICHLET)
    scale = np.max(np.abs(far))
    err_mp = np.max(np.abs(mp - far)) / scale
    err_di = np.max(np.abs(di - far)) / scale
    assert err_mp < 5e-3 and err_di > 20 * err_mp


# ------------------------------------------------------------- theta basis
def test_theta_eigenvectors_are_w_orthonormal_and_exact():
    g = O.Geometry(W.log_r_interfaces(4), W.uniform_theta_interfaces(128), 256)
    for m in (0, 1, 17, 64, 128):
        lam, h = O.theta_eigen(g, m)
        assert np.max(np.abs(h.T @ (g.w[:, None] * h) - np.eye(128))) <= 1e-13
        d, e = O.theta_matrix(g, m)
        b = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        # residual of the symmetric form T Q = Q Lambda, Q = W^(1/2) H, against ||T|| = max|lambda|
        res = (b @ h - g.w[:, None] * h * lam[None, :]) / np.sqrt(g.w)[:, None]
        assert np.max(np.abs(res)) <= 1e-13 * np.max(np.abs(lam))
        assert np.all(lam <= 1e-9) and np.all(np.diff(lam) <= 0)
        lam2 = scipy.linalg.eigh(b, np.diag(g.w), eigvals_only=True)
        assert np.max(np.abs(np.sort(lam2)[::-1] - lam)) <= 1e-12 * np.max(np.abs(lam))


def test_theta_matrix_matches_angular_stencil():
    """W (Delta_hat_theta + S_j lambda_phi,m) from the tridiagonal builder equals the
    full angular stencil acting on e_j cos(m phi)."""
    g = O.Geometry(W.uniform_r_interfaces(2), W.random_theta_interfaces(7, seed=1), 12)
    phc = W.phi_centres(12)
    for m in (0, 1, 4, 6):
        d, e = O.theta_matrix(g, m)
        b = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        cos = np.cos(m * phc + 0.3)
        for j in range(7):
            u = np.zeros((7, 12))
            u[j] = cos
            a = O.angular_apply(g, u) * g.w[:, None]
            assert np.allclose(a, b[:, j][:, None] * cos[None, :], rtol=0, atol=1e-12 * np.abs(b).max())


def test_theta_eigenvalues_approach_continuum():
    """Low eigenvalues approach -(m+n)(m+n+1), the spherical-harmonic values."""
    g = O.Geometry(W.log_r_interfaces(4), W.uniform_theta_interfaces(128), 256)
    for m in (0, 1, 2, 5):
        lam, h = O.theta_eigen(g, m)
        ell = m + np.arange(4)
        ref = -ell * (ell + 1.0)
        if m == 0:
            assert abs(lam[0]) <= 1e-10
            assert np.allclose(h[:, 0] * np.sign(h[0, 0]), 1.0 / math.sqrt(2.0), atol=1e-13)
            assert np.allclose(lam[1:4], ref[1:], rtol=1e-3)
        else:
            assert np.allclose(lam[:4], ref, rtol=3e-3)


def test_phi_eigenvalues_are_circulant_spectrum():
    for nphi in (6, 8, 12, 32):
        g = O.Geometry(W.uniform_r_interfaces(2), W.uniform_theta_interfaces(2), nphi)
        c = np.zeros((nphi, nphi))
        for k in range(nphi):
            c[k, k] = -2.0
            c[k, (k + 1) % nphi] += 1.0
            c[k, (k - 1) % nphi] += 1.0
        ev = np.sort(np.linalg.eigvalsh(c / g.dphi ** 2))
        ours = np.sort(g.lambda_phi(np.arange(nphi)))
        assert np.max(np.abs(ev - ours)) <= 1e-10 * np.max(np.abs(ev))


def test_kappa_continuum_exponent():
    """For lambda = -l(l+1) the exponent p is l+1: kappa = -(l+1)/r_out (r_out/r_N)^-(l+1)."""
    for ell in range(6):
        k = O.kappa(-ell * (ell + 1.0), 2.0, 1.5)
        assert abs(k - (-(ell + 1) / 2.0 * (2.0 / 1.5) ** (-(ell + 1)))) <= 1e-14


# --------------------------------------------------------- single eigenmode
def test_single_eigenmode_reduces_to_one_radial_solve():
    p = W.random_small(9, 6, 8, seed=3, grid="log")
    g = geo_of(p)
    m, ell = 3, 2
    lam, h = O.theta_eigen(g, m)
    phc = W.phi_centres(8)
    q = np.random.default_rng(2).standard_normal(9)
    ang = h[:, ell][:, None] * np.cos(m * phc)[None, :]
    rho = q[:, None, None] * ang[None] / (4 * math.pi)
    phi = O.solve_separated(g, rho)
    # radial matrix read off the full operator applied to e_i (x) H_l cos(m phi)
    kmat = O.outer_operator_dense(g)
    j0, k0 = int(np.argmax(np.abs(h[:, ell]))), 0
    mr = np.zeros((9, 9))
    for i in range(9):
        u = np.zeros((9, 6, 8))
        u[i] = ang
        mr[:, i] = O.apply_laplacian(g, u, O.OUTER_MULTIPOLE, kmat)[:, j0, k0] / ang[j0, k0]
    assert np.max(np.abs(np.triu(mr, 2))) == 0 and np.max(np.abs(np.tril(mr, -2))) == 0
    ab = np.zeros((3, 9))
    ab[0, 1:] = np.diag(mr, 1)
    ab[1] = np.diag(mr)
    ab[2, :-1] = np.diag(mr, -1)
    f = scipy.linalg.solve_banded((1, 1), ab, q)
    ref = f[:, None, None] * ang[None]
    assert np.max(np.abs(phi - ref)) <= 1e-13 * np.max(np.abs(ref))


# ---------------------------------------------------------------- symmetries
def test_symmetries_shift_reflection_linearity():
    p = W.random_small(6, 8, 12, seed=21, grid="log")
    g = geo_of(p)
    phi = O.solve_separated(g, p.rho)
    sc = np.max(np.abs(phi))
    shifted = O.solve_separated(g, np.roll(p.rho, 1, axis=2))
    assert np.max(np.abs(shifted - np.roll(phi, 1, axis=2))) <= 1e-13 * sc
    refl = O.solve_separated(g, p.rho[:, ::-1, :])
    assert np.max(np.abs(refl - phi[:, ::-1, :])) <= 1e-13 * sc
    rho2 = np.random.default_rng(5).uniform(size=p.rho.shape)
    phi2 = O.solve_separated(g, rho2)
    lin = O.solve_separated(g, 2.0 * p.rho - 3.0 * rho2)
    assert np.max(np.abs(lin - (2.0 * phi - 3.0 * phi2))) <= 1e-13 * np.max(np.abs(lin))


# ------------------------------------------------------- paper's worked example
def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, *v = line.split()
                vals[k] = [float(x) for x in v]
    return vals


@pytest.mark.slow
def test_displaced_point_source_matches_paper():
    """Sect. 5.1: a point source in one zone of a 550x128x256 log grid; the paper finds
    max relative errors of about 10% next to the source."""
    gv = _golden("point_source_sect5_1.txt")
    nr, nth, nphi = int(gv["nr"][0]), int(gv["ntheta"][0]), int(gv["nphi"][0])
    r_if = np.logspace(math.log10(gv["r_in"][0]), math.log10(gv["r_out"][0]), nr + 1)
    g = O.Geometry(r_if, W.uniform_theta_interfaces(nth), nphi)
    i, j, k = (int(x) - 1 for x in gv["zone_1based"])
    rho = np.zeros((nr, nth, nphi))
    rho[i, j, k] = gv["rho"][0]
    phi = O.solve_separated(g, rho)
    mass = g.cell_volume()[i, j] * gv["rho"][0]
    ph = W.phi_centres(nphi)
    st, ct = np.sin(g.thc), np.cos(g.thc)
    x = g.rc[:, None, None] * st[None, :, None] * np.cos(ph)[None, None, :]
    y = g.rc[:, None, None] * st[None, :, None] * np.sin(ph)[None, None, :]
    z = g.rc[:, None, None] * ct[None, :, None] * np.ones(nphi)[None, None, :]
    d = np.sqrt((x - x[i, j, k]) ** 2 + (y - y[i, j, k]) ** 2 + (z - z[i, j, k]) ** 2)
    d[i, j, k] = 1.0
    rel = np.abs(phi + mass / d) / (mass / d)
    rel[i, j, k] = 0.0
    d[i, j, k] = 0.0
    bound = gv["max_rel_err_adjacent"][0]
    adj = [rel[i + 1, j, k], rel[i - 1, j, k], rel[i, j + 1, k], rel[i, j - 1, k],
           rel[i, j, k + 1], rel[i, j, k - 1]]
    assert max(adj) <= bound
    assert 0.5 * bound <= rel.max() <= 1.5 * bound
    assert rel[d > 20 * d[i + 1, j, k]].max() < 1e-2


# ------------------------------------------------ face gradients (acceleration)
@pytest.mark.parametrize("bc", [O.OUTER_MULTIPOLE, O.OUTER_DIRICHLET])
@pytest.mark.parametrize("nr,nth,nphi,grid,rin", [(5, 6, 8, "rand", 0.1), (4, 4, 1, "uniform", 0.0),
                                                   (3, 1, 4, "log", 0.0), (6, 5, 2, "rand", 0.0)])
def test_face_gradient_divergence_is_the_operator(nr, nth, nphi, grid, rin, bc):
    """The face gradients are the ones the finite-volume fluxes of Eq. fin_vol3 use: their
    discrete divergence (outward area x gradient over the cell volume, Sect. 3.1) is the
    operator O3 itself, so accelerations taken from them are exactly consistent with the
    potential (the conservative form the paper's introduction asks of an exact solver)."""
    p = W.random_small(nr, nth, nphi, seed=nr + nth, grid=grid, r_inner=rin)
    g = geo_of(p)
    phi = np.random.default_rng(2).standard_normal((nr, nth, nphi))
    k = O.outer_operator_dense(g) if bc == O.OUTER_MULTIPOLE else None
    div = O.face_divergence(g, *O.face_gradients(g, phi, bc, k))
    lap = O.apply_laplacian(g, phi, bc, k)
    assert np.max(np.abs(div - lap)) <= 1e-13 * np.max(O.abs_apply(g, phi, bc, k))


def test_face_gradient_of_spherical_source_is_enclosed_mass():
    """For a spherically symmetric source the radial face gradient of the discrete
    solution is G M_enc(r_{i+1/2}) / r_{i+1/2}^2 at every interface (inner face 0, outer
    face G M / r_out^2), and the angular gradients vanish."""
    r_if = np.logspace(-2, 0, 41)
    g = O.Geometry(r_if, W.uniform_theta_interfaces(6), 8)
    rho_r = 1.0 / (1.0 + (g.rc / 0.1) ** 2)
    rho = np.broadcast_to(rho_r[:, None, None], (40, 6, 8))
    phi = O.solve_separated(g, rho)
    gr, gt, gp = O.face_gradients(g, phi)
    m_enc = np.concatenate([[0.0], np.cumsum(4.0 * math.pi * rho_r * g.dv3 / 3.0)])
    ex = np.zeros(41)
    ex[1:] = m_enc[1:] / r_if[1:] ** 2
    assert np.max(np.abs(gr[:, 0, 0] - ex)) <= 1e-12 * np.max(ex)
    assert np.max(np.abs(gr - gr[:, :1, :1])) <= 1e-12 * np.max(ex)
    assert np.max(np.abs(gt)) <= 1e-12 * np.max(ex) and np.max(np.abs(gp)) <= 1e-12 * np.max(ex)


def test_face_gradient_closed_forms():
    """r^2 on a uniform radial grid: the radial face gradient is exactly 2 r_{i+1/2};
    cos(theta): the theta face gradient tends to -sin(theta_face)/r at second order."""
    g = O.Geometry(W.uniform_r_interfaces(10), W.uniform_theta_interfaces(4), 4)
    phi = np.broadcast_to((g.rc ** 2)[:, None, None], (10, 4, 4)).copy()
    gr, _, _ = O.face_gradients(g, phi, O.OUTER_DIRICHLET)
    assert np.max(np.abs(gr[1:-1, 0, 0] - 2.0 * g.r_if[1:-1])) <= 1e-14
    errs = []
    for nth in (16, 32, 64):
        g = O.Geometry(W.uniform_r_interfaces(2, 1.0, 2.0), W.uniform_theta_interfaces(nth), 2)
        phi = np.broadcast_to(np.cos(g.thc)[None, :, None], (2, nth, 2)).copy()
        _, gt, _ = O.face_gradients(g, phi, O.OUTER_DIRICHLET)
        ex = -np.sin(g.th_if[1:-1])[None, :] / g.rc[:, None]
        errs.append(np.max(np.abs(gt[:, 1:-1, 0] - ex)))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


# ------------------------------------------------- ellipsoid of Sect. 5.2
def test_ellipsoid_potential_closed_form():
    """The analytic ellipsoid potential (Sect. 5.2, Carlson forms): the homogeneous
    sphere for a = b = c; Laplacian 4 pi G rho inside and 0 outside (finite differences);
    continuous across the surface; -G M / r far away."""
    r = np.linspace(0.01, 3.0, 40)
    n = np.array([0.3, 0.4, math.sqrt(0.75)])
    sph = O.ellipsoid_potential(r * n[0], r * n[1], r * n[2], 0.7, 0.7, 0.7)
    assert np.max(np.abs(sph - O.homogeneous_sphere_potential(r, 0.7))) <= 1e-14 * np.max(np.abs(sph))

    def f(q):
        return O.ellipsoid_potential(np.array([q[0]]), np.array([q[1]]), np.array([q[2]]), 1.0, 1.5, 2.0)[0]

    def lap(p, h=1e-3):
        p = np.asarray(p, dtype=float)
        tot = 0.0
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            tot += (f(p + e) + f(p - e) - 2.0 * f(p)) / h ** 2
        return tot

    assert abs(lap((0.2, 0.3, -0.4)) / (4.0 * math.pi) - 1.0) <= 1e-6
    assert abs(lap((1.2, 1.0, 1.5))) <= 1e-5 and abs(lap((0.0, 0.0, 3.0))) <= 1e-5
    # continuity at a surface point (1/sqrt 3)(a, b, c)
    s = np.array([1.0, 1.5, 2.0]) / math.sqrt(3.0)
    assert abs(f(s * (1 - 1e-9)) - f(s * (1 + 1e-9))) <= 1e-8 * abs(f(s))
    mass = 4.0 * math.pi / 3.0 * 1.0 * 1.5 * 2.0
    assert abs(f((0.0, 0.0, 1e4)) * 1e4 / -mass - 1.0) <= 1e-7


def test_ellipsoid_density_integrates_exactly():
    """The sub-volume integrated source holds the ellipsoid's mass 4/3 pi a b c, every
    cell fraction lies in [0, 1], and cells far inside / outside are 1 / 0."""
    p = W.ellipsoid("uniform", 64, 16, 32)
    vol = W.cell_volumes(p.r_if, p.th_if, p.nphi)[:, :, None]
    assert abs(np.sum(p.rho * vol) / (4.0 * math.pi) - 1.0) <= 1e-12
    assert p.rho.min() >= 0.0 and p.rho.max() <= 1.0
    rc = 0.5 * (p.r_if[1:] + p.r_if[:-1])
    assert np.all(p.rho[rc < 0.9] == 1.0) and np.all(p.rho[rc > 2.1] == 0.0)
    r = W.ellipsoid_r_interfaces("stretched", 512)
    assert abs(r[-1] - 48.7) < 0.1 and np.all(np.diff(r) > 0)


# ------------------------------------ explicit centres, regular-interior inner face
def _centred_geo(nr, nth, nphi, seed, inner_bc=O.INNER_ZERO_FLUX, r_inner=0.2, centres=True):
    p = W.random_small(nr, nth, nphi, seed=seed, grid="rand", r_inner=r_inner)
    rng = np.random.default_rng(seed)
    rc = th = None
    if centres:
        rc = p.r_if[:-1] + rng.uniform(0.2, 0.8, nr) * np.diff(p.r_if)
        th = p.th_if[:-1] + rng.uniform(0.2, 0.8, nth) * np.diff(p.th_if)
    return p, O.Geometry(p.r_if, p.th_if, p.nphi, r_centres=rc, th_centres=th, inner_bc=inner_bc)


@pytest.mark.parametrize("bc", [O.OUTER_MULTIPOLE, O.OUTER_DIRICHLET])
@pytest.mark.parametrize("centres,inner", [(True, O.INNER_ZERO_FLUX), (False, O.INNER_REGULAR),
                                           (True, O.INNER_REGULAR)])
def test_separated_equals_dense_lu_centres_and_inner_face(centres, inner, bc):
    """Explicit cell centres (R8') and the regular-interior inner face (R9) enter the
    separated solve (per-mode inner row) and the assembled operator (dense inner term)
    by independent routes; they agree to rounding."""
    p, g = _centred_geo(5, 6, 8, seed=3, inner_bc=inner, centres=centres)
    a = O.solve_separated(g, p.rho, outer_bc=bc)
    b = O.solve_dense(g, p.rho, outer_bc=bc)
    assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= 1e-13


def test_midpoints_given_explicitly_change_nothing():
    p = W.random_small(6, 5, 8, seed=4, grid="rand")
    g0 = O.Geometry(p.r_if, p.th_if, p.nphi)
    g1 = O.Geometry(p.r_if, p.th_if, p.nphi, r_centres=0.5 * (p.r_if[1:] + p.r_if[:-1]),
                    th_centres=0.5 * (p.th_if[1:] + p.th_if[:-1]))
    assert np.array_equal(O.solve_separated(g0, p.rho), O.solve_separated(g1, p.rho))


def test_regular_interior_mimics_empty_core():
    """With no mass inside r = 0.5, the regular-interior inner face at r_{1/2} = 0.5
    reproduces the solution of the grid that also covers the empty core (same zones
    beyond 0.5), to discretisation accuracy; zero flux there does not (it holds only for
    the l = 0 part)."""
    nth, nphi = 8, 8
    r_full = W.uniform_r_interfaces(64)
    th = W.uniform_theta_interfaces(nth)
    g_full = O.Geometry(r_full, th, nphi)
    rng = np.random.default_rng(6)
    rho = np.zeros((64, nth, nphi))
    rho[40:56] = rng.uniform(0.0, 1.0, (16, nth, nphi))
    ref = O.solve_separated(g_full, rho)[32:]
    g_reg = O.Geometry(r_full[32:], th, nphi, inner_bc=O.INNER_REGULAR)
    g_zf = O.Geometry(r_full[32:], th, nphi)
    reg = O.solve_separated(g_reg, rho[32:])
    zf = O.solve_separated(g_zf, rho[32:])
    scale = np.max(np.abs(ref))
    err_reg = np.max(np.abs(reg - ref)) / scale
    err_zf = np.max(np.abs(zf - ref)) / scale
    assert err_reg < 2e-3 and err_zf > 10 * err_reg


def test_kappa_inner_continuum_exponent():
    """At the continuum eigenvalue -l(l+1) the regular exponent is q = l."""
    for l in range(6):
        k = O.kappa_inner(-l * (l + 1.0), 2.0, 2.0)
        assert abs(k * 2.0 - l) <= 1e-13
