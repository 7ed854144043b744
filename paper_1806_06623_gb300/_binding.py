"""ctypes binding of libsphpoisson.so (include/sphpoisson.h).

Argument marshalling only: every step of the solve runs in the CUDA library.  The
binding refuses to run without the compiled library; there is no CPU fallback.
Device arrays are torch CUDA tensors (float64, contiguous); streams default to
torch's current stream on the tensor's device."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SP_OK = 0
SP_ERR_INVALID_ARG = 1
SP_ERR_GRID = 2
SP_ERR_CUDA = 3
SP_ERR_OOM = 4
SP_ERR_NOT_CONVERGED = 5
SP_ERR_TIMEOUT = 6
SP_ERR_DEVICE_CHECK = 7
SP_ERR_UNSUPPORTED = 8

SP_OUTER_MULTIPOLE = 0
SP_OUTER_DIRICHLET = 1
SP_INNER_ZERO_FLUX = 0
SP_INNER_REGULAR = 1
SP_RESIDUAL_AUTO = 0
SP_RESIDUAL_FLOAT_FLOAT = 1
SP_RESIDUAL_FLOAT64 = 2
SP_FP64 = 0
SP_MIXED_BF16X3 = 1
SP_MIXED_BF16X6 = 2


class SpError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("precision_used", C.c_int), ("last_update", C.c_double),
                ("est_rel_error", C.c_double), ("status", C.c_int), ("update_history", C.c_double * 8)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "update_history"}
        d["update_history"] = list(self.update_history)[:max(0, min(8, self.iterations))]
        return d


class PlanDesc(C.Structure):
    _fields_ = [("r_interfaces", C.c_void_p), ("Nr", C.c_int), ("theta_interfaces", C.c_void_p), ("Ntheta", C.c_int),
                ("Nphi", C.c_int), ("r_centres", C.c_void_p), ("theta_centres", C.c_void_p), ("inner_bc", C.c_int),
                ("outer_bc", C.c_int), ("G", C.c_double), ("precision", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_longlong), ("failed", C.c_longlong), ("queued", C.c_longlong),
                ("running_peak", C.c_int), ("resident_plans", C.c_int), ("evictions", C.c_longlong),
                ("mem_peak_bytes", C.c_double), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("max_ms", C.c_double), ("zones_per_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None

# name -> (restype, argtypes)
_SIGS = {
    "sp_plan_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double,
                                 C.c_int, C.c_double, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "sp_plan_create_ex": (C.c_int, [C.POINTER(PlanDesc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "sp_plan_clone": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "sp_solve_batched": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "sp_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]),
    "sp_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                   C.c_double, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_longlong)]),
    "sp_server_wait": (C.c_int, [C.c_void_p, C.c_longlong, C.c_double, C.POINTER(SolveInfo)]),
    "sp_server_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "sp_server_destroy": (C.c_int, [C.c_void_p]),
    "sp_server_reset_stats": (C.c_int, [C.c_void_p]),
    "sp_plan_workspace_bytes": (C.c_size_t, [C.c_void_p]),
    "sp_plan_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sp_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveInfo)]),
    "sp_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveInfo)]),
    "sp_solve_host_pipelined": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sp_apply_laplacian": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sp_apply_laplacian_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sp_plan_get_eigen": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sp_face_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sp_plan_last_status": (C.c_int, [C.c_void_p]),
    "sp_plan_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "sp_plan_collect_timing": (C.c_int, [C.c_void_p]),
    "sp_plan_get_timing": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "sp_plan_set_graphs": (C.c_int, [C.c_void_p, C.c_int]),
    "sp_plan_set_residual": (C.c_int, [C.c_void_p, C.c_int]),
    "sp_batched_set_ragged": (C.c_int, [C.c_int]),
    "sp_batched_last_ragged": (C.c_int, []),
    "sp_plan_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_char_p, C.c_void_p, C.POINTER(C.c_int)]),
    "sp_plan_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "sp_plan_launch_count": (C.c_longlong, [C.c_void_p]),
    "sp_plan_destroy": (C.c_int, [C.c_void_p]),
    "sp_status_string": (C.c_char_p, [C.c_int]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libsphpoisson.so (building it with nvcc if it is absent)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"{path} is missing: build it with paper_1806_06623_gb300.build.build()")
        _build.build()
    L = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def declared_symbols():
    return list(_SIGS)


def status_string(status: int) -> str:
    try:
        return lib().sp_status_string(int(status)).decode()
    except Exception:  # library not loadable: still describe the code
        return f"status {status}"


def _check(status: int, what: str):
    if status != SP_OK:
        raise SpError(status, what)


def _stream_ptr(stream, device=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dev_ptr(t, n, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be a contiguous float64 tensor with {n} elements")
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------- C-named calls
def sp_plan_create(r_interfaces, theta_interfaces, nphi, outer_bc=SP_OUTER_MULTIPOLE, G=1.0,
                   precision=SP_FP64, tol=1e-10, max_iter=8, stream=None):
    r = np.ascontiguousarray(r_interfaces, dtype=np.float64)
    th = None if theta_interfaces is None else np.ascontiguousarray(theta_interfaces, dtype=np.float64)
    nth = (len(th) - 1) if th is not None else None
    if nth is None:
        raise ValueError("theta_interfaces is required by the binding (pass uniform interfaces)")
    out = C.c_void_p()
    st = lib().sp_plan_create(r.ctypes.data_as(C.c_void_p), len(r) - 1, th.ctypes.data_as(C.c_void_p), nth,
                              int(nphi), int(outer_bc), float(G), int(precision), float(tol), int(max_iter),
                              _stream_ptr(stream), C.byref(out))
    _check(st, "sp_plan_create")
    return out


def sp_plan_create_ex(r_interfaces, theta_interfaces, nphi, r_centres=None, theta_centres=None,
                      inner_bc=SP_INNER_ZERO_FLUX, outer_bc=SP_OUTER_MULTIPOLE, G=1.0, precision=SP_FP64, tol=1e-10,
                      max_iter=8, stream=None):
    r = np.ascontiguousarray(r_interfaces, dtype=np.float64)
    th = np.ascontiguousarray(theta_interfaces, dtype=np.float64)
    rc = None if r_centres is None else np.ascontiguousarray(r_centres, dtype=np.float64)
    tc = None if theta_centres is None else np.ascontiguousarray(theta_centres, dtype=np.float64)
    if rc is not None and len(rc) != len(r) - 1:
        raise ValueError("r_centres needs one value per radial zone")
    if tc is not None and len(tc) != len(th) - 1:
        raise ValueError("theta_centres needs one value per polar zone")
    d = PlanDesc(r.ctypes.data_as(C.c_void_p), len(r) - 1, th.ctypes.data_as(C.c_void_p), len(th) - 1, int(nphi),
                 None if rc is None else rc.ctypes.data_as(C.c_void_p),
                 None if tc is None else tc.ctypes.data_as(C.c_void_p), int(inner_bc), int(outer_bc), float(G),
                 int(precision), float(tol), int(max_iter))
    out = C.c_void_p()
    _check(lib().sp_plan_create_ex(C.byref(d), _stream_ptr(stream), C.byref(out)), "sp_plan_create_ex")
    return out


def sp_plan_clone(plan):
    out = C.c_void_p()
    _check(lib().sp_plan_clone(plan, C.byref(out)), "sp_plan_clone")
    return out


def sp_solve_batched(plans, rhos, phis, stream=None, check=True):
    """plans: list of Plan; rhos, phis: lists of CUDA float64 tensors (one per plan).
    Returns the per-instance infos; with check=False a failing instance does not raise
    (its info.status says how it failed)."""
    n = len(plans)
    if not (len(rhos) == len(phis) == n):
        raise ValueError("plans, rhos and phis must have the same length")
    hp = (C.c_void_p * n)(*[p.handle.value for p in plans])
    rp = (C.c_void_p * n)(*[_dev_ptr(r, int(np.prod(p.shape)), "rho").value for p, r in zip(plans, rhos)])
    pp = (C.c_void_p * n)(*[_dev_ptr(f, int(np.prod(p.shape)), "phi").value for p, f in zip(plans, phis)])
    infos = (SolveInfo * n)()
    dev = rhos[0].device if n else None
    st = lib().sp_solve_batched(hp, rp, pp, n, _stream_ptr(stream, dev), infos)
    if check:
        _check(st, "sp_solve_batched")
    return list(infos)


def sp_server_create(mem_budget_bytes, slots):
    out = C.c_void_p()
    _check(lib().sp_server_create(int(mem_budget_bytes), int(slots), C.byref(out)), "sp_server_create")
    return out


def sp_server_submit(server, r_interfaces, theta_interfaces, nphi, rho, phi, outer_bc=SP_OUTER_MULTIPOLE, G=1.0,
                     precision=SP_FP64, tol=1e-10, max_iter=8):
    r = np.ascontiguousarray(r_interfaces, dtype=np.float64)
    th = np.ascontiguousarray(theta_interfaces, dtype=np.float64)
    if rho.dtype != np.float64 or not rho.flags.c_contiguous or phi.dtype != np.float64 or not phi.flags.c_contiguous:
        raise ValueError("rho and phi must be contiguous float64 arrays")
    t = C.c_longlong()
    st = lib().sp_server_submit(server, r.ctypes.data_as(C.c_void_p), len(r) - 1, th.ctypes.data_as(C.c_void_p),
                                len(th) - 1, int(nphi), int(outer_bc), float(G), int(precision), float(tol),
                                int(max_iter), rho.ctypes.data_as(C.c_void_p), phi.ctypes.data_as(C.c_void_p),
                                C.byref(t))
    _check(st, "sp_server_submit")
    return t.value, (r, th)


def sp_server_wait(server, ticket, timeout_s=-1.0):
    info = SolveInfo()
    st = lib().sp_server_wait(server, int(ticket), float(timeout_s), C.byref(info))
    return st, info


def sp_server_stats(server):
    s = ServerStats()
    _check(lib().sp_server_stats(server, C.byref(s)), "sp_server_stats")
    return s.as_dict()


def sp_server_reset_stats(server):
    _check(lib().sp_server_reset_stats(server), "sp_server_reset_stats")


def sp_server_destroy(server):
    if server:
        lib().sp_server_destroy(server)


def sp_plan_workspace_bytes(plan) -> int:
    return int(lib().sp_plan_workspace_bytes(plan))


def sp_plan_set_workspace(plan, ws):
    _check(lib().sp_plan_set_workspace(plan, C.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size()),
           "sp_plan_set_workspace")


def sp_solve(plan, rho, phi, shape, stream=None):
    n = int(np.prod(shape))
    info = SolveInfo()
    st = lib().sp_solve(plan, _dev_ptr(rho, n, "rho"), _dev_ptr(phi, n, "phi"),
                        _stream_ptr(stream, rho.device), C.byref(info))
    _check(st, "sp_solve")
    return info


def sp_solve_host(plan, rho, phi, stream=None):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    if phi.dtype != np.float64 or not phi.flags.c_contiguous or phi.size != rho.size:
        raise ValueError("phi must be a contiguous float64 array of rho's size")
    info = SolveInfo()
    st = lib().sp_solve_host(plan, rho.ctypes.data_as(C.c_void_p), phi.ctypes.data_as(C.c_void_p),
                             _stream_ptr(stream), C.byref(info))
    _check(st, "sp_solve_host")
    return info


def sp_solve_host_pipelined(plan, rhos, phis, stream=None):
    """rhos, phis: lists of contiguous float64 host arrays of the plan's size (page-locked
    for overlapped copies); solves q = 0..n-1 in order, returns the n SolveInfo."""
    n = len(rhos)
    if len(phis) != n:
        raise ValueError("rhos and phis must have the same length")
    size = rhos[0].size if n else 0
    for r, f in zip(rhos, phis):
        for a, name in ((r, "rho"), (f, "phi")):
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != size:
                raise ValueError(f"{name} arrays must be contiguous float64 arrays of one size")
    rp = (C.c_void_p * max(n, 1))(*[r.ctypes.data for r in rhos])
    pp = (C.c_void_p * max(n, 1))(*[f.ctypes.data for f in phis])
    infos = (SolveInfo * max(n, 1))()
    st = lib().sp_solve_host_pipelined(plan, n, rp, pp, _stream_ptr(stream), infos)
    _check(st, "sp_solve_host_pipelined")
    return list(infos)[:n]


def sp_apply_laplacian(plan, phi, out, shape, stream=None):
    n = int(np.prod(shape))
    _check(lib().sp_apply_laplacian(plan, _dev_ptr(phi, n, "phi"), _dev_ptr(out, n, "out"),
                                    _stream_ptr(stream, phi.device)), "sp_apply_laplacian")


def sp_face_gradients(plan, phi, g_r, g_theta, g_phi, shape, stream=None):
    nr, nth, nphi = shape
    n = nr * nth * nphi
    _check(lib().sp_face_gradients(plan, _dev_ptr(phi, n, "phi"), _dev_ptr(g_r, n + nth * nphi, "g_r"),
                                   _dev_ptr(g_theta, n + nr * nphi, "g_theta"), _dev_ptr(g_phi, n, "g_phi"),
                                   _stream_ptr(stream, phi.device)), "sp_face_gradients")


def sp_apply_laplacian_noalloc(plan, phi, out, shape, stream=None):
    """sp_apply_laplacian for callers that cannot allocate device memory: its scratch is
    a fixed 4 MiB array in the library (see include/sphpoisson.h)."""
    n = int(np.prod(shape))
    _check(lib().sp_apply_laplacian_noalloc(plan, _dev_ptr(phi, n, "phi"), _dev_ptr(out, n, "out"),
                                            _stream_ptr(stream, phi.device)), "sp_apply_laplacian_noalloc")


def sp_plan_get_eigen(plan, mh, nth):
    lam = np.zeros((mh, nth))
    H = np.zeros((mh, nth, nth))
    kap = np.zeros((mh, nth))
    _check(lib().sp_plan_get_eigen(plan, lam.ctypes.data_as(C.c_void_p), H.ctypes.data_as(C.c_void_p),
                                   kap.ctypes.data_as(C.c_void_p)), "sp_plan_get_eigen")
    return lam, H, kap


def sp_plan_last_status(plan) -> int:
    return int(lib().sp_plan_last_status(plan))


KERNEL_NAMES = ["fft_forward", "project_forward", "radial_solve", "project_inverse", "fft_inverse",
                "stencil", "outer_term", "residual", "split", "update", "eigensolve", "residual_rows"]


def sp_plan_set_timing(plan, enable: bool):
    _check(lib().sp_plan_set_timing(plan, 1 if enable else 0), "sp_plan_set_timing")


def sp_plan_collect_timing(plan):
    _check(lib().sp_plan_collect_timing(plan), "sp_plan_collect_timing")


def sp_plan_get_timing(plan):
    n = len(KERNEL_NAMES)
    ms = (C.c_double * n)()
    cnt = (C.c_longlong * n)()
    _check(lib().sp_plan_get_timing(plan, ms, cnt, n), "sp_plan_get_timing")
    return {KERNEL_NAMES[k]: (ms[k], cnt[k]) for k in range(n) if cnt[k]}


def sp_plan_launch_count(plan) -> int:
    return int(lib().sp_plan_launch_count(plan))


def sp_plan_destroy(plan):
    if plan:
        lib().sp_plan_destroy(plan)


def sp_status_string(status: int) -> str:
    return status_string(status)


# ------------------------------------------------------------ convenience
class Plan:
    """One solver plan: grid, boundary condition, precision and its device tables."""

    def __init__(self, r_interfaces, theta_interfaces, nphi, outer_bc=SP_OUTER_MULTIPOLE, G=1.0,
                 precision=SP_FP64, tol=1e-10, max_iter=8, stream=None, r_centres=None, theta_centres=None,
                 inner_bc=SP_INNER_ZERO_FLUX):
        self.r_if = np.asarray(r_interfaces, dtype=np.float64)
        self.th_if = np.asarray(theta_interfaces, dtype=np.float64)
        self.shape = (len(self.r_if) - 1, len(self.th_if) - 1, int(nphi))
        self.mh = int(nphi) // 2 + 1
        self.precision = precision
        self._h = None
        if r_centres is None and theta_centres is None and inner_bc == SP_INNER_ZERO_FLUX:
            self._h = sp_plan_create(self.r_if, self.th_if, nphi, outer_bc, G, precision, tol, max_iter, stream)
        else:
            self._h = sp_plan_create_ex(self.r_if, self.th_if, nphi, r_centres, theta_centres, inner_bc, outer_bc, G,
                                        precision, tol, max_iter, stream)

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self) -> int:
        return sp_plan_workspace_bytes(self._h)

    def clone(self):
        """A plan sharing this plan's tables with its own workspace."""
        c = Plan.__new__(Plan)
        c.r_if, c.th_if, c.shape, c.mh, c.precision = self.r_if, self.th_if, self.shape, self.mh, self.precision
        c._h = None
        c._h = sp_plan_clone(self._h)
        return c

    def solve(self, rho, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(rho)
        info = sp_solve(self._h, rho, out, self.shape, stream)
        return out, info

    def solve_host(self, rho, out=None, stream=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        info = sp_solve_host(self._h, rho, out, stream)
        return out, info

    def solve_host_pipelined(self, rhos, outs=None, stream=None):
        """n solves from host arrays with the copies of neighbouring solves overlapped;
        returns (outs, infos)."""
        if outs is None:
            outs = [np.empty(self.shape, dtype=np.float64) for _ in rhos]
        infos = sp_solve_host_pipelined(self._h, rhos, outs, stream)
        return outs, infos

    def apply_laplacian(self, phi, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(phi)
        sp_apply_laplacian(self._h, phi, out, self.shape, stream)
        return out

    def face_gradients(self, phi, stream=None):
        """(g_r, g_theta, g_phi) face gradients of phi; the acceleration is minus these."""
        import torch
        nr, nth, nphi = self.shape
        kw = dict(dtype=torch.float64, device=phi.device)
        g_r = torch.empty((nr + 1, nth, nphi), **kw)
        g_t = torch.empty((nr, nth + 1, nphi), **kw)
        g_p = torch.empty((nr, nth, nphi), **kw)
        sp_face_gradients(self._h, phi, g_r, g_t, g_p, self.shape, stream)
        return g_r, g_t, g_p

    def eigen(self):
        return sp_plan_get_eigen(self._h, self.mh, self.shape[1])

    def set_timing(self, enable=True):
        sp_plan_set_timing(self._h, enable)

    def collect_timing(self):
        sp_plan_collect_timing(self._h)

    def timing(self):
        return sp_plan_get_timing(self._h)

    def set_graphs(self, enable=True):
        _check(lib().sp_plan_set_graphs(self._h, int(bool(enable))), "sp_plan_set_graphs")

    def autotune(self, rho, phi=None, cache_path=None, stream=None):
        """Tune the launch configuration on rho (see sp_plan_autotune); returns
        (from_cache, [lines per CTA, radix order, projection CTAs, scan components])."""
        import torch
        n = int(np.prod(self.shape))
        if phi is None:
            phi = torch.empty_like(rho)
        fc = C.c_int(0)
        _check(lib().sp_plan_autotune(self._h, _dev_ptr(rho, n, "rho"), _dev_ptr(phi, n, "phi"),
                                      None if cache_path is None else str(cache_path).encode(),
                                      _stream_ptr(stream, rho.device), C.byref(fc)), "sp_plan_autotune")
        return bool(fc.value), self.tuning()

    def tuning(self):
        v = (C.c_int * 4)()
        _check(lib().sp_plan_get_tuning(self._h, v), "sp_plan_get_tuning")
        return list(v)

    def set_residual(self, mode=SP_RESIDUAL_AUTO):
        """Arithmetic of the mixed modes' refinement residual (SP_RESIDUAL_*)."""
        _check(lib().sp_plan_set_residual(self._h, int(mode)), "sp_plan_set_residual")

    def launch_count(self) -> int:
        return sp_plan_launch_count(self._h)

    def last_status(self) -> int:
        return sp_plan_last_status(self._h)

    def close(self):
        if self._h:
            sp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
