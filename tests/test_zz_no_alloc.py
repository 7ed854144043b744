"""sp_apply_laplacian_noalloc: the operator for callers that cannot allocate device memory
(code that must not synchronise the device, or that runs inside a host framework owning
a fixed memory pool).  It must give bitwise the result of sp_apply_laplacian, call after
call, while drawing its scratch from the library's fixed 4 MiB device array.

This file is collected last on purpose, so a run that stops at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1806_06623_gb300 as S
    S.lib()
    return S


def _call_noalloc(S, plan, phi, out):
    """Through the C ABI directly: (plan, phi, out, stream) -> status."""
    stream = torch.cuda.current_stream().cuda_stream
    return S.lib().sp_apply_laplacian_noalloc(plan.handle, C.c_void_p(phi.data_ptr()),
                                              C.c_void_p(out.data_ptr()), C.c_void_p(stream))


@pytest.mark.parametrize("shape,bc,precision", [((33, 17, 48), 0, 0), ((128, 64, 128), 0, 0), ((20, 16, 32), 1, 0),
                                              ((24, 16, 32), 0, 2)])
def test_noalloc_matches_apply_laplacian_twice(S, shape, bc, precision):
    nr, nth, nphi = shape
    p = W.random_small(nr, nth, nphi, seed=7, grid="log", outer_bc=bc)
    kw = dict(precision=precision, tol=1e-10) if precision else {}
    plan = S.Plan(p.r_if, p.th_if, p.nphi, outer_bc=bc, **kw)
    rng = np.random.default_rng(11)
    for call in range(2):
        phi = torch.from_numpy(rng.standard_normal(shape)).cuda()
        ref = plan.apply_laplacian(phi)
        out = torch.full_like(phi, float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        launches = plan.launch_count()
        assert _call_noalloc(S, plan, phi, out) == S.SP_OK
        torch.cuda.synchronize()
        if call == 1:   # after the first call's one-time set-up nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free_before
        # the same launches as sp_apply_laplacian, counted on the plan
        assert plan.launch_count() - launches == (1 if bc == 1 else 4)
        assert torch.equal(out, ref)


def test_noalloc_full_size_workload(S):
    p = W.stellar_sh()
    plan = S.Plan(p.r_if, p.th_if, p.nphi)
    phi = torch.from_numpy(p.rho).cuda()
    ref = plan.apply_laplacian(phi)
    for _ in range(2):
        out = torch.empty_like(phi)
        assert _call_noalloc(S, plan, phi, out) == S.SP_OK
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_near_its_scratch_limit(S):
    # (2048/2+1) x 2 x 127 doubles, 256-byte aligned, twice: 4,165,632 of the 4,194,304 bytes
    p = W.random_small(3, 127, 2048, seed=2, grid="log")
    plan = S.Plan(p.r_if, p.th_if, p.nphi)
    rng = np.random.default_rng(5)
    for _ in range(2):
        phi = torch.from_numpy(rng.standard_normal(p.rho.shape)).cuda()
        ref = plan.apply_laplacian(phi)
        out = torch.full_like(phi, float("nan"))
        assert _call_noalloc(S, plan, phi, out) == S.SP_OK
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    # one more theta zone: (1025 x 2 x 128 doubles) x 2 = 4,198,400 bytes, over the limit
    q = W.random_small(3, 128, 2048, seed=2, grid="log")
    plan2 = S.Plan(q.r_if, q.th_if, q.nphi)
    x = torch.zeros(q.rho.shape, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _call_noalloc(S, plan2, x, y) == S.SP_ERR_UNSUPPORTED


def test_noalloc_rejects_plans_beyond_its_scratch(S):
    # (4096/2+1) x 2 x 160 doubles, twice, exceeds the fixed 4 MiB array
    p = W.random_small(2, 160, 4096, seed=1)
    plan = S.Plan(p.r_if, p.th_if, p.nphi)
    x = torch.zeros(p.rho.shape, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _call_noalloc(S, plan, x, y) == S.SP_ERR_UNSUPPORTED
    with pytest.raises(S.SpError):
        S.sp_apply_laplacian_noalloc(plan.handle, x, y, p.rho.shape)


def test_noalloc_regular_interior_plan(S):
    """A plan with a regular-interior inner face adds the first shell's term, through the
    same scratch: still bitwise sp_apply_laplacian."""
    p = W.random_small(20, 12, 24, seed=3, grid="log", r_inner=0.2)
    plan = S.Plan(p.r_if, p.th_if, p.nphi, inner_bc=S.SP_INNER_REGULAR)
    rng = np.random.default_rng(2)
    for _ in range(2):
        phi = torch.from_numpy(rng.standard_normal(p.rho.shape)).cuda()
        ref = plan.apply_laplacian(phi)
        out = torch.full_like(phi, float("nan"))
        launches = plan.launch_count()
        assert _call_noalloc(S, plan, phi, out) == S.SP_OK
        torch.cuda.synchronize()
        assert plan.launch_count() - launches == 7
        assert torch.equal(out, ref)
