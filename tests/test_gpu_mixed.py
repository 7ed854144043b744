"""Mixed-precision solve (split-bf16 tcgen05 projections, float32 FFT and radial solves,
float64 residual refinement) against the oracle's exact float64 solution.

Gate: max|dPhi|/max|Phi| <= 1e-10 (the requested tolerance), with the solver's own
error estimate also <= 1e-10 and the float64 backward error eta <= 1e-12."""
import numpy as np
import pytest

import workloads as W
from oracle import sph_poisson as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1806_06623_gb300 as S
    S.lib()
    return S


def mixed_solve(S, p, tol=TOL, max_iter=8, precision=None):
    precision = S.SP_MIXED_BF16X3 if precision is None else precision
    plan = S.Plan(p.r_if, p.th_if, p.nphi, outer_bc=p.outer_bc, G=p.G, precision=precision,
                  tol=tol, max_iter=max_iter)
    rho = torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()
    phi, info = plan.solve(rho)
    torch.cuda.synchronize()
    return plan, phi.cpu().numpy(), info


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


CASES = [
    (5, 4, 6, "log", 0.0, 0),
    (7, 8, 12, "rand", 0.0, 0),
    (5, 3, 6, "rand", 0.2, 0),
    (6, 5, 9, "uniform", 0.0, 1),
    (3, 1, 4, "uniform", 0.0, 0),
    (1, 3, 4, "uniform", 0.5, 0),
    (33, 17, 48, "log", 0.0, 0),
    (65, 31, 96, "rand", 0.1, 0),
    (130, 128, 24, "log", 0.0, 0),     # full M tile, ragged N tile
    (300, 96, 192, "log", 0.0, 0),     # radix-3 phi, partial second K block
    (70, 16, 324, "rand", 0.0, 0),     # 163 m x 2 column tiles over one CTA per SM: table reloads mid-range
    (70, 32, 324, "rand", 0.0, 0),     # even/odd mode order of a symmetric grid, table reloads mid-range
    (90, 96, 12, "log", 0.3, 1),       # inner zero-flux face, Dirichlet, partial second K block
    (257, 64, 8, "uniform", 0.0, 1),
    (1600, 6, 4, "log", 0.0, 0),       # radial column beyond the shared-memory scan: ring-staged sweeps
    (4, 4, 1, "uniform", 0.0, 0),      # axisymmetric: one phi zone
    (3, 2, 2, "log", 0.0, 0),          # smallest even phi count
    (20, 16, 80, "log", 0.0, 0),       # radix 4 x 4 x 5
    (33, 12, 360, "rand", 0.1, 1),     # radix 4 x 2 x 3 x 3 x 5 (floor still below 1e-10)
    (7, 5, 25, "uniform", 0.0, 0),     # odd Nphi, radix 5 x 5
    # Nphi = 256 with even Ntheta: the residual fused with its forward FFT
    (40, 34, 256, "rand", 0.1, 0),     # partial 32-line theta block, inner zero-flux face
    (24, 6, 256, "log", 0.0, 1),       # Dirichlet (no shell chain), one short block per row
    (2, 64, 256, "uniform", 0.0, 0),   # two shells: the interior rows and the last shell
    (21, 5, 256, "uniform", 0.0, 0),   # odd Ntheta: the separate residual and FFT
]


@pytest.mark.parametrize("mode", ["x3", "x6"])
@pytest.mark.parametrize("nr,nth,nphi,grid,bc", [(4, 8, 4096, "log", 0), (3, 5, 3072, "rand", 1), (6, 12, 1024, "log", 0),
                                                 (5, 8, 480, "rand", 0)])
def test_mixed_long_phi_lines(S, nr, nth, nphi, grid, bc, mode):
    """Nphi up to 4096 (six radix-4 stages; a long radix-3 line).  The float-float
    iterate's precision floor 8 x 2^-48 x (Nphi/2pi)^2 passes 1e-10 near Nphi = 372, so
    beyond it the plan refines with a float64 iterate and the float64 residual stencil
    (SP_RESIDUAL_AUTO), which meets 1e-10; forced to float-float the same request stops
    with SP_ERR_NOT_CONVERGED instead of claiming it, and a looser request succeeds with
    the estimate bounding the true error."""
    p = W.random_small(nr, nth, nphi, seed=nr + 3 * nth + nphi, grid=grid, outer_bc=bc)
    prec = S.SP_MIXED_BF16X3 if mode == "x3" else S.SP_MIXED_BF16X6
    ref = O.solve_exact(O.Geometry(p.r_if, p.th_if, p.nphi), p.rho, outer_bc=bc)
    rho = torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()
    auto = S.Plan(p.r_if, p.th_if, p.nphi, outer_bc=bc, precision=prec, tol=TOL)
    for _ in range(3):                       # direct, then graph capture and replay
        phi, info = auto.solve(rho)
        err = rel_err(phi.cpu().numpy(), ref)
        assert info.status == S.SP_OK and err <= info.est_rel_error <= TOL
    strict = S.Plan(p.r_if, p.th_if, p.nphi, outer_bc=bc, precision=prec, tol=TOL)
    strict.set_residual(S.SP_RESIDUAL_FLOAT_FLOAT)
    with pytest.raises(S.SpError) as ei:
        strict.solve(rho)
    assert ei.value.status == S.SP_ERR_NOT_CONVERGED
    _, phi, info = mixed_solve(S, p, tol=1e-7, precision=prec)
    err = rel_err(phi, ref)
    assert info.status == S.SP_OK
    assert err <= info.est_rel_error <= 1e-7
    # below the float64 residual's floor (2^-40) the request is refused as well
    tight = S.Plan(p.r_if, p.th_if, p.nphi, outer_bc=bc, precision=prec, tol=1e-13)
    with pytest.raises(S.SpError) as ei:
        tight.solve(rho)
    assert ei.value.status == S.SP_ERR_NOT_CONVERGED


@pytest.mark.parametrize("mode", ["x3", "x6"])
@pytest.mark.parametrize("nr,nth,nphi,grid,rin,bc", [CASES[1], CASES[6], CASES[8], CASES[11]])
def test_mixed_float64_residual(S, nr, nth, nphi, grid, rin, bc, mode):
    """The float64 refinement residual chosen explicitly on grids where float-float would
    do: the same solution within the tolerance, the estimate bounding the error."""
    p = W.random_small(nr, nth, nphi, seed=nr + 3 * nth + nphi, grid=grid, r_inner=rin, outer_bc=bc)
    prec = S.SP_MIXED_BF16X3 if mode == "x3" else S.SP_MIXED_BF16X6
    plan = S.Plan(p.r_if, p.th_if, p.nphi, outer_bc=bc, precision=prec, tol=TOL)
    plan.set_residual(S.SP_RESIDUAL_FLOAT64)
    ref = O.solve_exact(O.Geometry(p.r_if, p.th_if, p.nphi), p.rho, outer_bc=bc)
    rho = torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()
    outs = []
    for _ in range(3):
        phi, info = plan.solve(rho)
        outs.append(phi.cpu().numpy())
        assert info.status == S.SP_OK
        assert rel_err(outs[-1], ref) <= max(info.est_rel_error, 1e-13) and info.est_rel_error <= TOL
    assert np.array_equal(outs[1], outs[2])    # graph replay = direct launches


@pytest.mark.parametrize("mode", ["x3", "x6"])
@pytest.mark.parametrize("nr,nth,nphi,grid,rin,bc", CASES)
def test_mixed_matches_exact_small(S, nr, nth, nphi, grid, rin, bc, mode):
    p = W.random_small(nr, nth, nphi, seed=nr + 3 * nth + nphi, grid=grid, r_inner=rin, outer_bc=bc)
    prec = S.SP_MIXED_BF16X3 if mode == "x3" else S.SP_MIXED_BF16X6
    _, phi, info = mixed_solve(S, p, precision=prec)
    ref = O.solve_exact(O.Geometry(p.r_if, p.th_if, p.nphi), p.rho, outer_bc=bc)
    assert info.status == S.SP_OK
    assert rel_err(phi, ref) <= TOL
    assert info.est_rel_error <= TOL and info.iterations >= 2
    # the estimate (distance to the refinement's fixed point) bounds the actual error down
    # to the rounding floor of the float-float residual on this grid: at least 46 of 53
    # bits, so at most 2^7 x the float64 separated solve's error (measured ratio about 6
    # at 1600 log-spaced radial cells)
    plan64 = S.Plan(p.r_if, p.th_if, p.nphi, outer_bc=p.outer_bc, G=p.G)
    phi64, _ = plan64.solve(torch.from_numpy(np.ascontiguousarray(p.rho)).cuda())
    floor = max(128 * rel_err(phi64.cpu().numpy(), ref), 1e-12)
    assert rel_err(phi, ref) <= max(info.est_rel_error, floor)


@pytest.mark.parametrize("mode", ["x3", "x6"])
@pytest.mark.parametrize("nr,nth,nphi,sym", [(40, 64, 48, True), (24, 10, 16, True), (30, 12, 32, False),
                                              (50, 128, 16, True)])
def test_mixed_nonuniform_theta(S, nr, nth, nphi, sym, mode):
    """Non-uniform theta grids (Sect. 3.1 does not require uniform theta) through the
    mixed path, mirror-symmetric ones (eigenbasis from the parity-split eigensolve, modes
    in even/odd order) and asymmetric ones."""
    p = W.random_small(nr, nth, nphi, seed=nr + nth + nphi, grid="log")
    p.th_if = W.symmetric_theta_interfaces(nth, seed=nth) if sym else W.random_theta_interfaces(nth, seed=nth)
    prec = S.SP_MIXED_BF16X3 if mode == "x3" else S.SP_MIXED_BF16X6
    _, phi, info = mixed_solve(S, p, precision=prec)
    geo = O.Geometry(p.r_if, p.th_if, p.nphi)
    ref = O.solve_exact(geo, p.rho)
    assert info.status == S.SP_OK
    assert rel_err(phi, ref) <= TOL
    eta, _ = O.residuals(geo, phi, p.rho)
    assert eta <= 1e-12


@pytest.mark.parametrize("mode", ["x3", "x6"])
@pytest.mark.parametrize("make", [W.sphere_blob, W.stellar_noise, lambda: W.ragged_instance(0),
                                  lambda: W.ragged_instance(5)])
def test_mixed_matches_exact_workloads(S, make, mode):
    p = make()
    prec = S.SP_MIXED_BF16X3 if mode == "x3" else S.SP_MIXED_BF16X6
    _, phi, info = mixed_solve(S, p, precision=prec)
    geo = O.Geometry(p.r_if, p.th_if, p.nphi)
    ref = O.solve_exact(geo, p.rho)
    assert rel_err(phi, ref) <= TOL
    eta, _ = O.residuals(geo, phi, p.rho)
    assert eta <= 1e-12


@pytest.mark.parametrize("mode", ["x3", "x6"])
def test_mixed_full_size_stellar_sh(S, mode):
    """The 550x128x256 headline workload."""
    p = W.stellar_sh()
    prec = S.SP_MIXED_BF16X3 if mode == "x3" else S.SP_MIXED_BF16X6
    _, phi, info = mixed_solve(S, p, precision=prec)
    geo = O.Geometry(p.r_if, p.th_if, p.nphi)
    ref = O.solve_exact(geo, p.rho)
    err = rel_err(phi, ref)
    assert err <= TOL, (err, info.as_dict())
    assert info.est_rel_error <= TOL
    eta, _ = O.residuals(geo, phi, p.rho)
    assert eta <= 1e-12


def test_mixed_reports_non_convergence(S):
    """An unreachable tolerance with one correction allowed fails with a status, not a fault."""
    p = W.stellar_noise()
    _, phi, info = None, None, None
    plan = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_MIXED_BF16X3, tol=1e-30, max_iter=1)
    rho = torch.from_numpy(p.rho).cuda()
    with pytest.raises(S.SpError) as ei:
        plan.solve(rho)
    assert ei.value.status == S.SP_ERR_NOT_CONVERGED
    # the plan stays usable
    plan2 = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_MIXED_BF16X3)
    out, info = plan2.solve(rho)
    assert info.status == S.SP_OK


@pytest.mark.parametrize("mode", ["x3", "x6"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_mixed_nonfinite_source_is_not_converged(S, mode, bad):
    """A NaN or an infinity in rho reaches the stopping decision (the device reductions
    keep a NaN, which a float max would drop, leaving max|Phi| = 0 and a claimed
    convergence) and the solve returns SP_ERR_NOT_CONVERGED; the plan stays usable, and in
    a batch only the instance with the bad source fails."""
    prec = S.SP_MIXED_BF16X3 if mode == "x3" else S.SP_MIXED_BF16X6
    for nphi in (32, 256):   # the separate and the fused residual
        p = W.random_small(12, 8, nphi, seed=5, grid="log")
        bad_rho = np.ascontiguousarray(p.rho).copy()
        bad_rho[3, 2, 5] = bad
        plan = S.Plan(p.r_if, p.th_if, p.nphi, precision=prec, tol=TOL)
        with pytest.raises(S.SpError) as ei:
            plan.solve(torch.from_numpy(bad_rho).cuda())
        assert ei.value.status == S.SP_ERR_NOT_CONVERGED
        _, info = plan.solve(torch.from_numpy(np.ascontiguousarray(p.rho)).cuda())
        assert info.status == S.SP_OK
        plans = [S.Plan(p.r_if, p.th_if, p.nphi, precision=prec, tol=TOL) for _ in range(2)]
        rhos = [torch.from_numpy(bad_rho).cuda(), torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()]
        infos = S.sp_solve_batched(plans, rhos, [torch.empty_like(r) for r in rhos], check=False)
        torch.cuda.synchronize()
        assert infos[0].status == S.SP_ERR_NOT_CONVERGED and not np.isfinite(infos[0].est_rel_error)
        assert infos[1].status == S.SP_OK


def test_mixed_zero_source(S):
    p = W.random_small(6, 8, 8, seed=1)
    p.rho[:] = 0.0
    _, phi, info = mixed_solve(S, p)
    assert info.status == S.SP_OK and np.all(phi == 0.0)


def test_mixed_equals_fp64_plan_within_tolerance(S):
    p = W.stellar_noise()
    _, phi_m, _ = mixed_solve(S, p)
    plan = S.Plan(p.r_if, p.th_if, p.nphi)
    phi_d, _ = plan.solve(torch.from_numpy(p.rho).cuda())
    assert rel_err(phi_m, phi_d.cpu().numpy()) <= 2 * TOL


def test_mixed_x6_second_correction_rebuilds_iterate(S):
    """With 6 products the first correction stores the iterate in float64 only; a tighter
    tolerance that needs a second correction rebuilds its float-float words from there.
    Checked against the exact solution, and bitwise between launch-by-launch solves and
    graph-replayed ones (the replay restores the iterate's state on the host)."""
    p = W.random_small(24, 12, 16, seed=21, grid="log")
    ref = O.solve_exact(O.Geometry(p.r_if, p.th_if, p.nphi), p.rho)
    rho = torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()
    direct = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_MIXED_BF16X6, tol=1e-12, max_iter=8)
    direct.set_graphs(False)
    phi_d, info_d = direct.solve(rho)
    torch.cuda.synchronize()
    assert info_d.status == S.SP_OK and info_d.iterations >= 3, info_d.as_dict()
    assert rel_err(phi_d.cpu().numpy(), ref) <= 1e-12
    plan = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_MIXED_BF16X6, tol=1e-12, max_iter=8)
    out = torch.empty_like(rho)
    for k in range(4):                 # direct, capture + replay, replay, replay
        _, info = plan.solve(rho, out)
        torch.cuda.synchronize()
        assert torch.equal(out, phi_d), k
        assert info.iterations == info_d.iterations


def test_mixed_rho_on_an_8_byte_boundary(S):
    """Even Nphi with rho 16-byte aligned takes the two-column residual; rho on an 8-byte
    boundary the one-column form. Both meet the tolerance, and agree to rounding."""
    p = W.random_small(40, 24, 32, seed=17, grid="log")
    ref = O.solve_exact(O.Geometry(p.r_if, p.th_if, p.nphi), p.rho)
    plan = S.Plan(p.r_if, p.th_if, p.nphi, precision=S.SP_MIXED_BF16X6)
    plan.set_graphs(False)
    n = p.rho.size
    buf = torch.empty(n + 1, dtype=torch.float64, device="cuda")
    aligned = torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()
    shifted = buf[1:].view(p.rho.shape)              # 8 bytes past a 256-byte boundary
    shifted.copy_(aligned)
    assert shifted.data_ptr() % 16 == 8
    phi_a, info_a = plan.solve(aligned)
    phi_b, info_b = plan.solve(shifted)
    torch.cuda.synchronize()
    a, b = phi_a.cpu().numpy(), phi_b.cpu().numpy()
    assert info_a.status == S.SP_OK and info_b.status == S.SP_OK
    assert rel_err(a, ref) <= TOL and rel_err(b, ref) <= TOL
    assert rel_err(b, a) <= 1e-12


@pytest.mark.parametrize("bc", [0, 1])
def test_timing_spans_of_a_mixed_solve(S, bc):
    """Per-kernel CUDA-event timers: every group of the 6-product solve is timed, the
    residual's interior-row kernel has a span of its own inside the residual's (nested
    spans, one per residual), and the launch counter does not count the nested span."""
    p = W.random_small(12, 8, 256, seed=3, grid="log", outer_bc=bc)
    plan = S.Plan(p.r_if, p.th_if, p.nphi, outer_bc=bc, precision=S.SP_MIXED_BF16X6, tol=TOL)
    rho = torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()
    c0 = S.sp_plan_launch_count(plan.handle)
    plan.solve(rho)   # (launched directly: graphs are captured from the second solve on)
    n0 = S.sp_plan_launch_count(plan.handle)
    plan.set_timing(True)
    _, info = plan.solve(rho)
    torch.cuda.synchronize()
    plan.collect_timing()
    t = plan.timing()
    n1 = S.sp_plan_launch_count(plan.handle)
    plan.set_timing(False)
    for name in ("fft_forward", "project_forward", "radial_solve", "project_inverse", "fft_inverse", "residual"):
        assert name in t and t[name][0] > 0.0
    assert t["residual_rows"][1] == t["residual"][1] == info.iterations - 1
    assert 0.0 < t["residual_rows"][0] <= t["residual"][0]
    assert n1 - n0 == n0 - c0   # the same launches with and without timers (both direct)
