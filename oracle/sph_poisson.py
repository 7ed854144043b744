"""CPU FP64 oracle for the exact discrete Poisson solve on spherical polar grids
(Mueller & Chan 2018, "An FFT-based Solution Method for the Poisson Equation
on 3D Spherical Polar Grids").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this module.  The
GPU library never calls it, and it shares no code with the GPU path.

Three independent pieces, all plain FP64 (NumPy / SciPy):

* O3 ``apply_laplacian`` -- the finite-volume operator of Eq. (fin_vol0)-(fin_vol3)
  with the interface areas and volumes of Sect. 3.1, written out term by term,
  plus the paper's multipole outer boundary condition (Sect. 3.2, last equation).
* O2 ``solve_dense`` -- brute force: assemble the operator by applying O3 to
  unit vectors and solve with dense LU.  Tiny grids only.
* O1 ``solve_separated`` -- the paper's serial algorithm (Sect. 3.2) in its own
  order: FFT in phi, per-m eigenproblem of the theta operator, forward
  projection, one tridiagonal radial solve per (l,m), back projection,
  inverse FFT.

Readings of the paper taken here (the printed formulas are partly garbled):

* R1  the theta operator carries 1/w_j, w_j = cos th_{j-1/2} - cos th_{j+1/2}
      (follows from Eq. fin_vol3 with the printed dA/dV).
* R2  the phi operator is the second difference divided by dphi^2.
* R3  lambda_phi,m = -(sin(m dphi/2)/(dphi/2))^2 (negative; the printed form
      lacks the sign, which the outer-boundary exponent requires).
* R4  the theta/phi face areas carry (r_{i+1/2}^2 - r_{i-1/2}^2)/2.
* R5  the radial equation is  Delta_r f + R_i lambda_Omega f = s_hat.
* R6  outer boundary: the outer-face gradient is replaced by
      -p f_N (r_{N+1/2}/r_N)^(-p) / r_{N+1/2},  p = (1+sqrt(1-4 lambda_Omega))/2.
* R8  cell centres are midpoints of their interfaces.
* R9  inner boundary: zero flux through r_{1/2} (the area vanishes when r_{1/2}=0);
      optionally, for r_{1/2} > 0, a "regular interior": the empty region r < r_{1/2}
      holds the regular Laplace solution, so each mode (l,m) is extrapolated as
      f ~ r^q from the innermost zone, q = (-1 + sqrt(1 - 4 lambda_Omega))/2.
* R8' explicit cell centres may replace the midpoints (any point strictly inside
      the cell); the operator's r_i, theta_j are then those centres.
* R10 forward FFT normalised by 1/Nphi; half spectrum m = 0..Nphi//2.
* R11 eigenvalues sorted descending (l=0 is lambda=0 for m=0); eigenvector
      signs are arbitrary, so only Phi is compared.
* R12 s = 4 pi G rho.
* R13 residual gate: eta = max|s - L Phi| / max(|s| + |L||Phi|).
* R19 the parity reference is the exact float64 solution of L Phi = s, obtained
      from the separated solve by residual correction with the operator itself
      (``solve_exact``); the plain separated solve is ~1e-12 away from it.
A test-only Dirichlet outer boundary Phi(r_{N+1/2}) = 0 is also provided.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

OUTER_MULTIPOLE = 0
OUTER_DIRICHLET = 1
INNER_ZERO_FLUX = 0
INNER_REGULAR = 1


class Geometry:
    """Geometric factors of Sect. 3.1 (areas, volumes, R_i, S_j, w_j)."""

    def __init__(self, r_if, th_if, nphi: int, r_centres=None, th_centres=None, inner_bc=INNER_ZERO_FLUX):
        r_if = np.asarray(r_if, dtype=np.float64)
        th_if = np.asarray(th_if, dtype=np.float64)
        if r_if.ndim != 1 or len(r_if) < 2 or np.any(np.diff(r_if) <= 0) or r_if[0] < 0:
            raise ValueError("r interfaces must be strictly increasing with r[0] >= 0")
        if (th_if.ndim != 1 or len(th_if) < 2 or np.any(np.diff(th_if) <= 0)
                or th_if[0] != 0.0 or abs(th_if[-1] - math.pi) > 1e-15):
            raise ValueError("theta interfaces must increase from 0 to pi")
        if nphi < 1:
            raise ValueError("nphi must be >= 1")
        self.r_if, self.th_if, self.nphi = r_if, th_if, int(nphi)
        self.nr, self.nth = len(r_if) - 1, len(th_if) - 1
        rm, rp = r_if[:-1], r_if[1:]
        self.rc = 0.5 * (rm + rp)                              # R8
        if r_centres is not None:                              # R8'
            self.rc = np.asarray(r_centres, dtype=np.float64).copy()
            if self.rc.shape != rm.shape or np.any(self.rc <= rm) or np.any(self.rc >= rp):
                raise ValueError("radial centres must lie strictly inside their cells")
        self.dv3 = rp ** 3 - rm ** 3                           # 3 dV / (w dphi)
        self.R = 3.0 * (rp ** 2 - rm ** 2) / (2.0 * self.rc * self.dv3)
        self.thc = 0.5 * (th_if[:-1] + th_if[1:])              # R8
        if th_centres is not None:                             # R8'
            self.thc = np.asarray(th_centres, dtype=np.float64).copy()
            if (self.thc.shape != (self.nth,) or np.any(self.thc <= th_if[:-1])
                    or np.any(self.thc >= th_if[1:])):
                raise ValueError("polar centres must lie strictly inside their cells")
        self.w = np.cos(th_if[:-1]) - np.cos(th_if[1:])
        self.dth = th_if[1:] - th_if[:-1]
        self.sin_c = np.sin(self.thc)
        self.S = self.dth / (self.sin_c * self.w)
        sin_if = np.sin(th_if)
        sin_if[0] = 0.0                                        # poles: zero face area
        sin_if[-1] = 0.0
        self.sin_if = sin_if
        self.dphi = 2.0 * math.pi / self.nphi
        self.r_out = r_if[-1]
        self.r_in = r_if[0]
        self.inner_regular = inner_bc == INNER_REGULAR and r_if[0] > 0.0
        self._kin_dense = None

    # ------------------------------------------------------------ volumes
    def cell_volume(self):
        """dV_ijk for one phi cell, shape (Nr, Ntheta)."""
        return (self.dv3 / 3.0)[:, None] * self.w[None, :] * self.dphi

    def lambda_phi(self, m):
        """Eigenvalue of the phi second difference for wavenumber m (R3)."""
        h = 0.5 * self.dphi
        return -(np.sin(np.asarray(m) * h) / h) ** 2


def kappa(lam, r_out, r_last):
    """Outer-face gradient per unit f_N for angular eigenvalue lam (R6)."""
    lam = np.asarray(lam, dtype=np.float64)
    p = 0.5 * (1.0 + np.sqrt(1.0 - 4.0 * lam))
    return -p / r_out * np.exp(-p * math.log(r_out / r_last))


def kappa_inner(lam, r_in, r_first):
    """Inner-face gradient per unit f_1 for angular eigenvalue lam with a regular
    interior (R9): f ~ r^q extrapolated from the innermost zone to r_{1/2},
    q = (-1 + sqrt(1 - 4 lam))/2 >= 0 (q = l for the continuum eigenvalue -l(l+1))."""
    lam = np.asarray(lam, dtype=np.float64)
    q = 0.5 * (-1.0 + np.sqrt(1.0 - 4.0 * lam))
    return q / r_in * np.exp(q * math.log(r_in / r_first))


# =================================================================== O3
def angular_apply(geo: Geometry, u):
    """(Delta_hat_theta + S_j Delta_hat_phi) u on shells; u has shape (..., Ntheta, Nphi)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    # theta fluxes through faces j+1/2 (Eq. fin_vol3, areas of Sect. 3.1, R1/R4)
    if geo.nth > 1:
        t_face = geo.sin_if[1:-1] / (geo.thc[1:] - geo.thc[:-1])       # (Ntheta-1,)
        flux = t_face[:, None] * (u[..., 1:, :] - u[..., :-1, :])
        out[..., :-1, :] += flux
        out[..., 1:, :] -= flux
    out /= geo.w[:, None]
    # phi: periodic second difference (R2)
    if geo.nphi > 1:
        d2 = (np.roll(u, -1, axis=-1) - 2.0 * u + np.roll(u, 1, axis=-1)) / geo.dphi ** 2
        out += geo.S[:, None] * d2
    return out


def outer_operator_dense(geo: Geometry, fn=None):
    """Matrix K of kappa(A_Omega) on the outermost shell (or of another function `fn` of
    the angular eigenvalue), by a dense eigendecomposition of the full 2-D angular
    operator (no FFT, no per-m split).  Tiny grids only."""
    n = geo.nth * geo.nphi
    a = np.zeros((n, n))
    eye = np.eye(n).reshape(n, geo.nth, geo.nphi)
    for c in range(n):
        a[:, c] = angular_apply(geo, eye[c]).reshape(n)
    wf = np.repeat(geo.w, geo.nphi)
    sq = np.sqrt(wf)
    m = (sq[:, None] * a) / sq[None, :]
    m = 0.5 * (m + m.T)
    lam, v = np.linalg.eigh(m)
    kap = kappa(lam, geo.r_out, geo.rc[-1]) if fn is None else fn(lam)
    return ((v * kap[None, :]) @ v.T) / sq[:, None] * sq[None, :]


def inner_gradient(geo: Geometry, phi_first):
    """Inner-face gradient for every (j,k) of the first shell: zero flux, or with a
    regular interior kappa_inner(A_Omega) applied to the first shell (R9)."""
    phi_first = np.asarray(phi_first, dtype=np.float64)
    if not geo.inner_regular:
        return np.zeros_like(phi_first)
    fn = lambda lam: kappa_inner(lam, geo.r_in, geo.rc[0])   # noqa: E731
    if geo.nth * geo.nphi <= 1200:
        if geo._kin_dense is None:
            geo._kin_dense = outer_operator_dense(geo, fn)
        return (geo._kin_dense @ phi_first.reshape(-1)).reshape(phi_first.shape)
    return outer_kappa_separated(geo, phi_first, fn)


def outer_gradient(geo: Geometry, phi_last, outer_bc, kmat=None):
    """Outer-face gradient for every (j,k) of the last shell."""
    if outer_bc == OUTER_DIRICHLET:
        return -phi_last / (geo.r_out - geo.rc[-1])
    if kmat is None:
        return outer_kappa_separated(geo, phi_last)
    return (kmat @ phi_last.reshape(-1)).reshape(phi_last.shape)


def apply_laplacian(geo: Geometry, phi, outer_bc=OUTER_MULTIPOLE, kmat=None):
    """O3: (Delta Phi)_{ijk} of Eq. (fin_vol0)-(fin_vol3) with the boundary conditions."""
    phi = np.asarray(phi, dtype=np.float64)
    out = np.zeros_like(phi)
    # radial fluxes r_{i+1/2}^2 (Phi_{i+1}-Phi_i)/(r_{i+1}-r_i) through interior faces
    if geo.nr > 1:
        k_face = geo.r_if[1:-1] ** 2 / (geo.rc[1:] - geo.rc[:-1])
        flux = k_face[:, None, None] * (phi[1:] - phi[:-1])
        out[:-1] += flux
        out[1:] -= flux
    # inner face r_{1/2}: zero flux or regular interior (R9).  Outer face: boundary
    # condition (R6).
    out[0] -= geo.r_in ** 2 * inner_gradient(geo, phi[0])
    out[-1] += geo.r_out ** 2 * outer_gradient(geo, phi[-1], outer_bc, kmat)
    out *= (3.0 / geo.dv3)[:, None, None]
    # angular part, scaled by R_i
    out += geo.R[:, None, None] * angular_apply(geo, phi)
    return out


def abs_apply(geo: Geometry, phi, outer_bc=OUTER_MULTIPOLE, kmat=None):
    """|L| |Phi| for the backward error of R13: the local stencil with absolute
    coefficients (the diagonal taken as one coefficient), plus the magnitude of the
    outer boundary term (and of its diagonal part for the Dirichlet case)."""
    a = np.abs(np.asarray(phi, dtype=np.float64))
    nr, nth, nphi = geo.nr, geo.nth, geo.nphi
    diag = np.zeros((nr, nth, nphi))
    off = np.zeros((nr, nth, nphi))
    if nr > 1:
        k_face = geo.r_if[1:-1] ** 2 / (geo.rc[1:] - geo.rc[:-1])
        c = (3.0 / geo.dv3)
        off[:-1] += (c[:-1] * k_face)[:, None, None] * a[1:]
        off[1:] += (c[1:] * k_face)[:, None, None] * a[:-1]
        diag[:-1] -= (c[:-1] * k_face)[:, None, None]
        diag[1:] -= (c[1:] * k_face)[:, None, None]
    if nth > 1:
        t_face = geo.sin_if[1:-1] / (geo.thc[1:] - geo.thc[:-1])
        up = geo.R[:, None] * (t_face / geo.w[:-1])[None, :]
        dn = geo.R[:, None] * (t_face / geo.w[1:])[None, :]
        off[:, :-1, :] += up[:, :, None] * a[:, 1:, :]
        off[:, 1:, :] += dn[:, :, None] * a[:, :-1, :]
        diag[:, :-1, :] -= up[:, :, None]
        diag[:, 1:, :] -= dn[:, :, None]
    if nphi > 1:
        cphi = geo.R[:, None] * geo.S[None, :] / geo.dphi ** 2
        off += cphi[:, :, None] * (np.roll(a, -1, -1) + np.roll(a, 1, -1))
        diag -= 2.0 * cphi[:, :, None]
    out = off
    if geo.inner_regular:
        out[0] += np.abs(3.0 * geo.r_in ** 2 / geo.dv3[0] * inner_gradient(geo, np.asarray(phi, dtype=np.float64)[0]))
    if outer_bc == OUTER_DIRICHLET:
        diag[-1] -= 3.0 * geo.r_out ** 2 / ((geo.r_out - geo.rc[-1]) * geo.dv3[-1])
        out += np.abs(diag) * a
    else:
        out += np.abs(diag) * a
        g = outer_gradient(geo, np.asarray(phi, dtype=np.float64)[-1], outer_bc, kmat)
        out[-1] += np.abs(3.0 * geo.r_out ** 2 / geo.dv3[-1] * g)
    return out


def residuals(geo: Geometry, phi, rho, G=1.0, outer_bc=OUTER_MULTIPOLE, kmat=None):
    """(eta, max|s-L Phi|/max|s|) of R13 for a candidate Phi."""
    s = 4.0 * math.pi * G * np.asarray(rho, dtype=np.float64)
    r = s - apply_laplacian(geo, phi, outer_bc, kmat)
    den = np.abs(s) + abs_apply(geo, phi, outer_bc, kmat)
    return float(np.max(np.abs(r)) / np.max(den)), float(np.max(np.abs(r)) / np.max(np.abs(s)))


# =================================================================== O2
def assemble_dense(geo: Geometry, outer_bc=OUTER_MULTIPOLE):
    """The full operator as a dense matrix, column by column from O3."""
    n = geo.nr * geo.nth * geo.nphi
    if n > 4096:
        raise ValueError("assemble_dense is for tiny grids only")
    kmat = outer_operator_dense(geo) if outer_bc == OUTER_MULTIPOLE else None
    mat = np.zeros((n, n))
    e = np.zeros(n)
    for c in range(n):
        e[:] = 0.0
        e[c] = 1.0
        mat[:, c] = apply_laplacian(geo, e.reshape(geo.nr, geo.nth, geo.nphi), outer_bc, kmat).reshape(n)
    return mat


def solve_dense(geo: Geometry, rho, G=1.0, outer_bc=OUTER_MULTIPOLE):
    """O2: Phi = L^{-1} (4 pi G rho) by dense LU."""
    mat = assemble_dense(geo, outer_bc)
    s = 4.0 * math.pi * G * np.asarray(rho, dtype=np.float64).reshape(-1)
    return np.linalg.solve(mat, s).reshape(geo.nr, geo.nth, geo.nphi)


# =================================================================== O1
def theta_matrix(geo: Geometry, m):
    """Symmetric tridiagonal B_m = W (Delta_hat_theta + S_j lambda_phi,m): (diag, offdiag)."""
    t_face = geo.sin_if[1:-1] / (geo.thc[1:] - geo.thc[:-1]) if geo.nth > 1 else np.zeros(0)
    diag = np.zeros(geo.nth)
    diag[:-1] -= t_face
    diag[1:] -= t_face
    diag += geo.lambda_phi(m) * geo.dth / geo.sin_c
    return diag, t_face


def theta_eigen(geo: Geometry, m):
    """Eigenpairs of Delta_hat_theta + S_j lambda_phi,m (Sect. 3.2): returns (lam, H) with
    H^T W H = I, columns sorted by descending eigenvalue (R11)."""
    b_d, b_e = theta_matrix(geo, m)
    sq = np.sqrt(geo.w)
    d = b_d / geo.w
    e = b_e / (sq[:-1] * sq[1:])
    if geo.nth == 1:
        lam, q = d.copy(), np.ones((1, 1))
    else:
        lam, q = scipy.linalg.eigh_tridiagonal(d, e)
    order = np.argsort(-lam, kind="stable")
    lam, q = lam[order], q[:, order]
    return lam, q / sq[:, None]


def all_theta_eigen(geo: Geometry):
    mh = geo.nphi // 2 + 1
    lams = np.zeros((mh, geo.nth))
    hs = np.zeros((mh, geo.nth, geo.nth))
    for m in range(mh):
        lams[m], hs[m] = theta_eigen(geo, m)
    return lams, hs


def radial_system(geo: Geometry, lam, outer_bc=OUTER_MULTIPOLE):
    """Tridiagonal rows of Delta_r + R_i lam for every eigenvalue in ``lam`` (R5, R6, R9).

    Returns (sub, diag, sup), each of shape lam.shape + (Nr,)."""
    lam = np.asarray(lam, dtype=np.float64)
    nr = geo.nr
    sub = np.zeros(nr)
    sup = np.zeros(nr)
    if nr > 1:
        k_face = geo.r_if[1:-1] ** 2 / (geo.rc[1:] - geo.rc[:-1])
        sup[:-1] = 3.0 * k_face / geo.dv3[:-1]
        sub[1:] = 3.0 * k_face / geo.dv3[1:]
    base = -(sub + sup)
    diag = base + geo.R * lam[..., None]
    if geo.inner_regular:
        diag[..., 0] += -3.0 * geo.r_in ** 2 * kappa_inner(lam, geo.r_in, geo.rc[0]) / geo.dv3[0]
    if outer_bc == OUTER_DIRICHLET:
        diag[..., -1] += -3.0 * geo.r_out ** 2 / ((geo.r_out - geo.rc[-1]) * geo.dv3[-1])
    else:
        diag[..., -1] += 3.0 * geo.r_out ** 2 * kappa(lam, geo.r_out, geo.rc[-1]) / geo.dv3[-1]
    shp = lam.shape + (nr,)
    return np.broadcast_to(sub, shp), diag, np.broadcast_to(sup, shp)


def thomas(sub, diag, sup, rhs):
    """Tridiagonal solve along the last axis, vectorised over the leading axes.
    rhs may have one more trailing-batch axis than the coefficients (broadcast)."""
    n = diag.shape[-1]
    cp = np.zeros(diag.shape)
    dp = np.zeros(rhs.shape, dtype=rhs.dtype)
    piv = diag[..., 0]
    cp[..., 0] = sup[..., 0] / piv
    dp[..., 0] = rhs[..., 0] / piv
    for i in range(1, n):
        piv = diag[..., i] - sub[..., i] * cp[..., i - 1]
        cp[..., i] = sup[..., i] / piv
        dp[..., i] = (rhs[..., i] - sub[..., i] * dp[..., i - 1]) / piv
    x = np.zeros_like(dp)
    x[..., n - 1] = dp[..., n - 1]
    for i in range(n - 2, -1, -1):
        x[..., i] = dp[..., i] - cp[..., i] * x[..., i + 1]
    return x


def solve_separated(geo: Geometry, rho, G=1.0, outer_bc=OUTER_MULTIPOLE, eig=None,
                    return_stages=False):
    """O1: the serial algorithm of Sect. 3.2, step by step."""
    s = 4.0 * math.pi * G * np.asarray(rho, dtype=np.float64)        # R12
    nphi = geo.nphi
    # (1) FFT along phi: s_tilde[i,j,m] = (1/Nphi) sum_k s e^{-2 pi i m k/Nphi}  (R10)
    s_tilde = np.fft.rfft(s, axis=2) / nphi                            # (Nr, Nth, Mh)
    mh = s_tilde.shape[2]
    # (2) eigenvectors H_{l,m}(j) of Delta_hat_theta + S_j lambda_phi,m, once per m
    lams, hs = eig if eig is not None else all_theta_eigen(geo)
    # (3) forward projection s_hat[i,l,m] = sum_j H_{l,m}(j) w_j s_tilde[i,j,m]
    s_hat = np.empty_like(s_tilde)
    for m in range(mh):
        s_hat[:, :, m] = s_tilde[:, :, m] @ (hs[m] * geo.w[:, None])
    # (4) radial boundary-value problem per (l,m): Delta_r f + R_i lambda f = s_hat
    sub, diag, sup = radial_system(geo, lams, outer_bc)               # (Mh, Nth, Nr)
    rhs = s_hat.transpose(2, 1, 0)                                     # (Mh, Nth, Nr)
    f = thomas(sub, diag, sup, rhs).transpose(2, 1, 0)                 # (Nr, Nth, Mh)
    # (5) back projection g[i,j,m] = sum_l H_{l,m}(j) f[i,l,m]
    g = np.empty_like(f)
    for m in range(mh):
        g[:, :, m] = f[:, :, m] @ hs[m].T
    # (6) inverse FFT Phi_ijk = sum_m g_ijm e^{2 pi i m k/Nphi}
    phi = np.fft.irfft(g * nphi, n=nphi, axis=2)
    if return_stages:
        return phi, {"s_tilde": s_tilde, "s_hat": s_hat, "f": f, "g": g,
                     "lams": lams, "hs": hs}
    return phi


def solve_exact(geo: Geometry, rho, G=1.0, outer_bc=OUTER_MULTIPOLE, max_steps=6, return_history=False):
    """The exact float64 solution of L Phi = 4 pi G rho (R19).

    The separated solve O1 is exact in exact arithmetic, but in float64 its forward
    error reaches ~1e-12 relative on graded theta operators (the eigenbasis of
    T_m has entries spanning ~1e8 at Ntheta=128), whereas its backward error is
    ~1e-16.  Residual correction with the operator itself (O3) removes that error:
    Phi <- Phi + O1(s - L Phi) until the update is below 1e-15 max|Phi|."""
    eig = all_theta_eigen(geo)
    s = 4.0 * math.pi * G * np.asarray(rho, dtype=np.float64)
    kmat = None
    if outer_bc == OUTER_MULTIPOLE and geo.nth * geo.nphi <= 1200:
        kmat = outer_operator_dense(geo)
    phi = solve_separated(geo, rho, G, outer_bc, eig=eig)
    hist = []
    for _ in range(max_steps):
        r = s - apply_laplacian(geo, phi, outer_bc, kmat)
        e = solve_separated(geo, r, 1.0 / (4.0 * math.pi), outer_bc, eig=eig)
        phi = phi + e
        upd = float(np.max(np.abs(e)) / np.max(np.abs(phi)))
        hist.append(upd)
        if upd <= 1e-15:
            break
    return (phi, hist) if return_history else phi


def outer_kappa_separated(geo: Geometry, u, fn=None):
    """kappa(A_Omega) u on the last shell (or `fn` of the angular eigenvalue) through the
    per-m eigenbasis (FFT, projection, scale, back projection, inverse FFT).  Used for
    O3 on grids too large for the dense K."""
    u = np.asarray(u, dtype=np.float64)
    lams, hs = all_theta_eigen(geo)
    ut = np.fft.rfft(u, axis=-1) / geo.nphi                      # (Nth, Mh)
    kap = kappa(lams, geo.r_out, geo.rc[-1]) if fn is None else fn(lams)   # (Mh, Nth)
    out = np.zeros_like(ut)
    for m in range(ut.shape[-1]):
        c = (hs[m] * geo.w[:, None]).T @ ut[:, m]
        out[:, m] = hs[m] @ (kap[m] * c)
    return np.fft.irfft(out * geo.nphi, n=geo.nphi, axis=-1)


# ------------------------------------------- gravitational acceleration (Sect. 1)
def face_gradients(geo: Geometry, phi, outer_bc=OUTER_MULTIPOLE, kmat=None):
    """Gradient of Phi on every cell face, as the finite-volume operator of Eq.
    fin_vol3 uses it in its fluxes (the gravitational acceleration is minus this):

    * radial faces i = 0..Nr (face i between cells i-1 and i): (Phi_i - Phi_{i-1}) /
      (r_i - r_{i-1}); zero at r_{1/2} (R9); the outer face carries the boundary
      condition's gradient (R6).  Shape (Nr+1, Ntheta, Nphi).
    * theta faces j = 0..Ntheta: (Phi_j - Phi_{j-1}) / (r_i (theta_j - theta_{j-1})),
      zero at the poles.  Shape (Nr, Ntheta+1, Nphi).
    * phi faces k+1/2 (between k and k+1, periodic): (Phi_{k+1} - Phi_k) /
      (r_i sin(theta_j) dphi).  Shape (Nr, Ntheta, Nphi).
    Cell centres r_i, theta_j as in R8."""
    phi = np.asarray(phi, dtype=np.float64)
    nr, nth, nphi = phi.shape
    gr = np.zeros((nr + 1, nth, nphi))
    if nr > 1:
        gr[1:-1] = (phi[1:] - phi[:-1]) / (geo.rc[1:] - geo.rc[:-1])[:, None, None]
    gr[0] = inner_gradient(geo, phi[0])
    gr[-1] = outer_gradient(geo, phi[-1], outer_bc, kmat)
    gt = np.zeros((nr, nth + 1, nphi))
    if nth > 1:
        gt[:, 1:-1, :] = ((phi[:, 1:, :] - phi[:, :-1, :])
                          / (geo.rc[:, None, None] * (geo.thc[1:] - geo.thc[:-1])[None, :, None]))
    gp = np.zeros((nr, nth, nphi))
    if nphi > 1:
        gp = (np.roll(phi, -1, axis=2) - phi) / (geo.rc[:, None, None] * geo.sin_c[None, :, None] * geo.dphi)
    return gr, gt, gp


def face_divergence(geo: Geometry, gr, gt, gp):
    """Discrete divergence of face-centred vector components: the sum over a cell's
    faces of (outward area x component), divided by the cell volume (the areas and
    volumes of Sect. 3.1)."""
    nr, nth, nphi = gp.shape
    r2 = geo.r_if ** 2
    area_r = r2[:, None] * geo.w[None, :] * geo.dphi                          # (Nr+1, Nth)
    half_r2 = 0.5 * (geo.r_if[1:] ** 2 - geo.r_if[:-1] ** 2)                  # (Nr,)
    area_t = half_r2[:, None] * geo.sin_if[None, :] * geo.dphi                 # (Nr, Nth+1)
    area_p = half_r2[:, None] * geo.dth[None, :]                               # (Nr, Nth)
    vol = geo.cell_volume()[:, :, None]
    div = (area_r[1:, :, None] * gr[1:] - area_r[:-1, :, None] * gr[:-1])
    div = div + (area_t[:, 1:, None] * gt[:, 1:, :] - area_t[:, :-1, None] * gt[:, :-1, :])
    div = div + area_p[:, :, None] * (gp - np.roll(gp, 1, axis=2))
    return div / vol


# ------------------------------------------------------- closed forms (pins)
def gauss_law_potential(geo: Geometry, rho_r, G=1.0, outer_bc=OUTER_MULTIPOLE):
    """Exact discrete solution for a spherically symmetric source rho(r_i), from the
    conservative flux form: the flux through r_{i+1/2} equals G times the enclosed mass.
    Returns Phi_i (Nr,)."""
    rho_r = np.asarray(rho_r, dtype=np.float64)
    m_enc = np.cumsum(4.0 * math.pi * rho_r * geo.dv3 / 3.0)
    phi = np.zeros(geo.nr)
    grad_out = G * m_enc[-1] / geo.r_out ** 2
    if outer_bc == OUTER_DIRICHLET:
        phi[-1] = -grad_out * (geo.r_out - geo.rc[-1])
    else:   # multipole BC with l=0 (p=1): grad = -Phi_N r_N / r_out^2
        phi[-1] = -grad_out * geo.r_out ** 2 / geo.rc[-1]
    for i in range(geo.nr - 2, -1, -1):
        grad = G * m_enc[i] / geo.r_if[i + 1] ** 2
        phi[i] = phi[i + 1] - grad * (geo.rc[i + 1] - geo.rc[i])
    return phi


def ellipsoid_potential(x, y, z, a, b, c, rho0=1.0, G=1.0):
    """Continuum potential of the homogeneous ellipsoid x^2/a^2 + y^2/b^2 + z^2/c^2 <= 1
    (Sect. 5.2): Phi = pi G rho0 a b c (A x^2 + B y^2 + C z^2 - D) with
    A = int_u^inf dl / sqrt((a^2+l)^3 (b^2+l) (c^2+l)) (B, C likewise) and
    D = int_u^inf dl / sqrt((a^2+l)(b^2+l)(c^2+l)); u = 0 inside, else the positive
    root of x^2/(a^2+u) + y^2/(b^2+u) + z^2/(c^2+u) = 1.  In Carlson's symmetric forms
    (a library primitive here): D = 2 R_F(a^2+u, b^2+u, c^2+u) and
    A = (2/3) R_D(b^2+u, c^2+u, a^2+u), with B, C by permutation."""
    import scipy.special as sps
    x, y, z = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
    a2, b2, c2 = a * a, b * b, c * c
    q = x * x / a2 + y * y / b2 + z * z / c2
    u = np.zeros_like(q)
    out = q > 1.0
    if np.any(out):
        xo, yo, zo = x[out] ** 2, y[out] ** 2, z[out] ** 2
        # f(u) = sum x_i^2/(a_i^2+u) - 1 is convex and decreasing; its root is the largest
        # root of the cubic prod (a_i^2+u) - sum x_i^2 prod_{k!=i} (a_k^2+u), taken in
        # closed form (trigonometric / Cardano), then polished by Newton steps on f
        c2_ = a2 + b2 + c2 - (xo + yo + zo)
        c1_ = a2 * b2 + b2 * c2 + c2 * a2 - xo * (b2 + c2) - yo * (a2 + c2) - zo * (a2 + b2)
        c0_ = a2 * b2 * c2 - xo * b2 * c2 - yo * a2 * c2 - zo * a2 * b2
        # u = t - c2/3: t^3 + p t + q = 0
        pp = c1_ - c2_ * c2_ / 3.0
        qq = 2.0 * c2_ ** 3 / 27.0 - c2_ * c1_ / 3.0 + c0_
        disc = (qq / 2.0) ** 2 + (pp / 3.0) ** 3
        t_one = np.cbrt(-qq / 2.0 + np.sqrt(np.maximum(disc, 0.0))) + np.cbrt(-qq / 2.0 - np.sqrt(np.maximum(disc, 0.0)))
        mm = 2.0 * np.sqrt(np.maximum(-pp / 3.0, 0.0))
        arg = np.where(mm > 0, 3.0 * qq / (pp * np.where(mm > 0, mm, 1.0)), 0.0)
        t_three = mm * np.cos(np.arccos(np.clip(arg, -1.0, 1.0)) / 3.0)
        uu = np.where(disc > 0, t_one, t_three) - c2_ / 3.0
        uu = np.maximum(uu, np.maximum(0.0, xo + yo + zo - max(a2, b2, c2)))
        for _ in range(2):
            f = xo / (a2 + uu) + yo / (b2 + uu) + zo / (c2 + uu) - 1.0
            df = -(xo / (a2 + uu) ** 2 + yo / (b2 + uu) ** 2 + zo / (c2 + uu) ** 2)
            uu = uu - f / df
        u[out] = uu
    A = (2.0 / 3.0) * sps.elliprd(b2 + u, c2 + u, a2 + u)
    B = (2.0 / 3.0) * sps.elliprd(a2 + u, c2 + u, b2 + u)
    C = (2.0 / 3.0) * sps.elliprd(a2 + u, b2 + u, c2 + u)
    D = 2.0 * sps.elliprf(a2 + u, b2 + u, c2 + u)
    return math.pi * G * rho0 * a * b * c * (A * x * x + B * y * y + C * z * z - D)


def homogeneous_sphere_potential(r, radius, rho0=1.0, G=1.0):
    """Continuum potential of a homogeneous sphere."""
    r = np.asarray(r, dtype=np.float64)
    inside = -2.0 * math.pi * G * rho0 * (radius ** 2 - r ** 2 / 3.0)
    outside = -4.0 * math.pi * G * rho0 * radius ** 3 / (3.0 * np.maximum(r, 1e-300))
    return np.where(r < radius, inside, outside)
