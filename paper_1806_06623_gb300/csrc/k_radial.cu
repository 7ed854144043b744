// Radial boundary-value problems of Sect. 3.2 and the float64 finite-volume operator.
//
// thomas: for every (l,m) the tridiagonal system  Delta_r f + R_i lambda_Omega,l,m f = s_hat
// (Eq. tridiag) with zero flux through r_{1/2} and the outer row carrying the
// mode's boundary term (multipole exponent p or Dirichlet).  One thread per (m,l)
// solves the real and imaginary right-hand sides together by forward elimination and
// back substitution; the systems are diagonally dominant, so no pivoting is needed.
// The spectral layout [m][i][c][l] makes every radial step a coalesced row access.
//
// stencil: (Delta Phi)_{ijk} of Eq. (fin_vol0)-(fin_vol3), one thread per cell with phi
// fastest; the multipole outer term is added by outer_term (FFT of the last shell,
// kappa(lambda) in the eigenbasis, inverse FFT).
#include "sp_internal.h"

namespace sp {
namespace {

// Elimination factors of every (m,l) radial system (plan set-up, float64): the forward
// sweep of the Thomas algorithm without a right-hand side, storing 1/pivot_i and
// c'_i = sup_i / pivot_i; the diagonal carries R_i lambda_lm, the multipole outer row and
// the regular-interior inner row.
__global__ void __launch_bounds__(128) k_radial_factors_f64(const RadialRow* __restrict__ rad,
                                                            const double* __restrict__ lam,
                                                            const double* __restrict__ outer,
                                                            const double* __restrict__ inner, double* __restrict__ tinv,
                                                            double* __restrict__ tcp, int nr, int nth, int mh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= mh * nth) return;
  const int m = t / nth;
  const int l = t - m * nth;
  const double L = lam[t];
  const double od = outer[t];
  const double id = inner[t];
  double* INV = tinv + (size_t)m * nr * nth + l;
  double* CP = tcp + (size_t)m * nr * nth + l;
  double cprev = 0.0;
  for (int i = 0; i < nr; ++i) {
    const RadialRow rr = rad[i];
    double b = fma(rr.R, L, rr.base);
    if (i == 0) b += id;
    if (i == nr - 1) b += od;
    const double piv = b - rr.sub * cprev;
    const double inv = 1.0 / piv;
    cprev = rr.sup * inv;
    INV[(size_t)i * nth] = inv;
    CP[(size_t)i * nth] = cprev;
  }
}

// The radial solves of the separated system (Sect. 3.2, Eq. tridiag), float64, one thread
// per (m,l) and both components: forward elimination d_i = (x_i - sub_i d_{i-1}) / pivot_i
// and back substitution f_i = d_i - c'_i f_{i+1} with the plan's factor tables, so no
// division on the (narrow) float64 pipe; the rows are taken kThomasU at a time with all
// their loads issued before the recurrence uses them.
constexpr int kThomasU = 8;
__global__ void __launch_bounds__(64) k_thomas_f64(const RadialRow* __restrict__ rad, const double* __restrict__ tinv,
                                                   const double* __restrict__ tcp, double* __restrict__ x, int nr,
                                                   int nth, int mh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= mh * nth) return;
  const int m = t / nth;
  const int l = t - m * nth;
  double* X = x + (size_t)m * nr * 2 * nth + l;
  const double* INV = tinv + (size_t)m * nr * nth + l;
  const double* CP = tcp + (size_t)m * nr * nth + l;
  const size_t st = 2 * (size_t)nth;
  double dre = 0.0, dim = 0.0;
  for (int i0 = 0; i0 < nr; i0 += kThomasU) {
    double xr[kThomasU], xi[kThomasU], iv[kThomasU], sb[kThomasU];
#pragma unroll
    for (int u = 0; u < kThomasU; ++u) {
      const int i = i0 + u;
      if (i < nr) {
        xr[u] = X[i * st];
        xi[u] = X[i * st + nth];
        iv[u] = INV[(size_t)i * nth];
        sb[u] = rad[i].sub;
      }
    }
#pragma unroll
    for (int u = 0; u < kThomasU; ++u) {
      const int i = i0 + u;
      if (i < nr) {
        dre = (xr[u] - sb[u] * dre) * iv[u];
        dim = (xi[u] - sb[u] * dim) * iv[u];
        X[i * st] = dre;
        X[i * st + nth] = dim;
      }
    }
  }
  for (int i1 = nr - 2; i1 >= 0; i1 -= kThomasU) {
    double xr[kThomasU], xi[kThomasU], c[kThomasU];
#pragma unroll
    for (int u = 0; u < kThomasU; ++u) {
      const int i = i1 - u;
      if (i >= 0) {
        c[u] = CP[(size_t)i * nth];
        xr[u] = X[i * st];
        xi[u] = X[i * st + nth];
      }
    }
#pragma unroll
    for (int u = 0; u < kThomasU; ++u) {
      const int i = i1 - u;
      if (i >= 0) {
        dre = xr[u] - c[u] * dre;
        dim = xi[u] - c[u] * dim;
        X[i * st] = dre;
        X[i * st + nth] = dim;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_stencil_f64(const double* __restrict__ phi, double* __restrict__ out,
                                                     const RadialRow* __restrict__ rad,
                                                     const ThetaRow* __restrict__ th, int nr, int nth, int nphi,
                                                     double dir_coef) {
  const size_t n = (size_t)nr * nth * nphi;
  const size_t shell = (size_t)nth * nphi;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % nphi);
    const size_t ij = idx / nphi;
    const int j = (int)(ij % nth);
    const int i = (int)(ij / nth);
    const double c = phi[idx];
    const RadialRow rr = rad[i];
    const ThetaRow tr = th[j];
    double v = 0.0;
    if (i > 0) v += rr.sub * (phi[idx - shell] - c);
    if (i < nr - 1) v += rr.sup * (phi[idx + shell] - c);
    double a = 0.0;
    if (j > 0) a += tr.tm * (phi[idx - nphi] - c);
    if (j < nth - 1) a += tr.tp * (phi[idx + nphi] - c);
    const size_t kp = (k + 1 == nphi) ? idx - k : idx + 1;
    const size_t km = (k == 0) ? idx + (nphi - 1) : idx - 1;
    a += tr.sphi * ((phi[kp] - c) + (phi[km] - c));
    v += rr.R * a;
    if (i == nr - 1) v += dir_coef * c;
    out[idx] = v;
  }
}

// Outer-shell operator of the multipole condition per m: O_m = H_m diag(outer_m) (H^T W)_m
// (set-up; one CTA per (j, m) row, threads over j').
__global__ void k_outer_operator(const double* __restrict__ HtW, const double* __restrict__ H,
                                 const double* __restrict__ outer, double* __restrict__ O, int nth) {
  const int j = blockIdx.x, m = blockIdx.y;
  const double* Hm = H + ((size_t)m * nth + j) * nth;
  const double* A = HtW + (size_t)m * nth * nth;
  const double* om = outer + (size_t)m * nth;
  for (int jp = threadIdx.x; jp < nth; jp += blockDim.x) {
    double s = 0.0;
    for (int l = 0; l < nth; ++l) s = fma(Hm[l] * om[l], A[(size_t)l * nth + jp], s);
    O[((size_t)m * nth + j) * nth + jp] = s;
  }
}

// z_m = O_m x_m for the two real columns (re, im) of the outer shell's spectrum: one warp
// per row j of O_m, lanes over j' (coalesced), shuffle reduction.
constexpr int kShellRows = 8;
__device__ __forceinline__ void shell_apply_body(const double* __restrict__ O, const double* __restrict__ xin,
                                                 double* __restrict__ zout, int nth, int bx, int m) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = bx * kShellRows + warp;
  if (j >= nth) return;
  const double* row = O + ((size_t)m * nth + j) * nth;
  const double* x = xin + (size_t)m * 2 * nth;
  double s0 = 0.0, s1 = 0.0;
  for (int jp = lane; jp < nth; jp += 32) {
    const double o = row[jp];
    s0 = fma(o, x[jp], s0);
    s1 = fma(o, x[nth + jp], s1);
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, off);
    s1 += __shfl_down_sync(0xffffffffu, s1, off);
  }
  if (lane == 0) {
    zout[(size_t)m * 2 * nth + j] = s0;
    zout[(size_t)m * 2 * nth + nth + j] = s1;
  }
}

__global__ void __launch_bounds__(32 * kShellRows) k_shell_apply(const double* __restrict__ O,
                                                                 const double* __restrict__ xin,
                                                                 double* __restrict__ zout, int nth) {
  shell_apply_body(O, xin, zout, nth, blockIdx.x, blockIdx.y);
}

// ragged form: local CTA b is row block b mod gx of wavenumber b / gx
__global__ void __launch_bounds__(32 * kShellRows) k_shell_apply_rag(const ShellArgs* __restrict__ tab,
                                                                     const int* __restrict__ start, int n) {
  const int q = rag_instance(start, n, blockIdx.x);
  const ShellArgs& a = tab[q];
  const int b = (int)blockIdx.x - start[q];
  shell_apply_body(a.O, a.x, a.z, a.nth, b % a.gx, b / a.gx);
}

// Face gradients (minus the gravitational acceleration) of Eq. fin_vol3's fluxes: a warp
// per (i, j) line, its lanes over the azimuthal cells, writing the gradient on each cell's
// inner radial face i, its lower polar face j (and the pole face j = Ntheta after the last
// row) and its azimuthal face k+1/2.  The line's coefficient products are formed once,
// so a cell costs three float64 differences and three products.  The outer radial face
// (index nr) holds on entry the multipole term O_m Phi_last computed by the shell
// transforms (scaled here by 1/outer_coef), or is set from the Dirichlet condition; the
// inner face (index 0) holds O_in Phi_first for a regular interior (scaled by
// -1/inner_coef), else it is zero (inner_scale = 0).
constexpr int kFaceWarps = 8;
constexpr int kFaceU = 4;   // cells per lane in flight
__global__ void __launch_bounds__(32 * kFaceWarps) k_face_grad(const double* __restrict__ phi, double* __restrict__ gr,
                                                               double* __restrict__ gt, double* __restrict__ gp,
                                                               const FaceCoef* __restrict__ fr,
                                                               const FaceCoef* __restrict__ ft, int nr, int nth,
                                                               int nphi, int dirichlet, double outer_scale,
                                                               double inner_scale) {
  const int lane = threadIdx.x & 31;
  const int lines = nr * nth;
  const size_t shell = (size_t)nth * nphi;
  for (int ln = blockIdx.x * kFaceWarps + (threadIdx.x >> 5); ln < lines; ln += gridDim.x * kFaceWarps) {
    const int i = ln / nth, j = ln - i * nth;
    const FaceCoef r = fr[i];
    const FaceCoef t = ft[j];
    const double ct = r.inv_c * t.inv_d, cp = r.inv_c * t.inv_c;
    const size_t o = (size_t)ln * nphi;
    const double* row = phi + o;
    double* grl = gr + o;
    double* gtl = gt + ((size_t)i * (nth + 1) + j) * nphi;
    double* gpl = gp + o;
    for (int k0 = lane; k0 < nphi; k0 += 32 * kFaceU) {
      double c[kFaceU], cn[kFaceU], ci[kFaceU], cj[kFaceU];
#pragma unroll
      for (int u = 0; u < kFaceU; ++u) {
        const int k = k0 + 32 * u;
        if (k < nphi) {
          c[u] = row[k];
          cn[u] = row[k + 1 == nphi ? 0 : k + 1];
          ci[u] = i > 0 ? row[(ptrdiff_t)k - (ptrdiff_t)shell] : (inner_scale != 0.0 ? grl[k] : 0.0);
          cj[u] = j > 0 ? row[k - nphi] : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < kFaceU; ++u) {
        const int k = k0 + 32 * u;
        if (k >= nphi) continue;
        // inner face: zero flux, or (regular interior) O_in phi_first on entry, scaled
        grl[k] = i > 0 ? (c[u] - ci[u]) * r.inv_d : ci[u] * inner_scale;
        if (i == nr - 1) {
          double* of = grl + shell + k;   // outer face
          *of = dirichlet ? -c[u] * outer_scale : *of * outer_scale;
        }
        gtl[k] = j > 0 ? (c[u] - cj[u]) * ct : 0.0;
        if (j == nth - 1) gtl[nphi + k] = 0.0;
        gpl[k] = (cn[u] - c[u]) * cp;
      }
    }
  }
}

}  // namespace

cudaError_t face_gradients_f64(const Plan& p, const double* phi, double* gr, double* gt, double* gp, cudaStream_t s) {
  const bool dir = p.outer_bc == SP_OUTER_DIRICHLET;
  const size_t off = (size_t)(p.nr - 1) * p.nth * p.nphi;
  const size_t sh = (size_t)p.nth * p.nphi;
  cudaError_t e;
  if (!dir) {
    // O_m phi_last = outer_coef x kappa(A_Omega) phi_last into the outer face
    if ((e = fft_forward_f64(p, phi + off, 1, 1.0 / p.nphi, p.shell, s)) != cudaSuccess) return e;
    if ((e = shell_kappa_f64(p, p.shell, p.shell2, s)) != cudaSuccess) return e;
    if ((e = fft_inverse_f64(p, p.shell2, 1, gr + off + sh, false, s)) != cudaSuccess) return e;
  }
  const bool reg = p.inner_bc == SP_INNER_REGULAR;
  if (reg) {
    // O_in phi_first = -inner_coef x kappa_in(A_Omega) phi_first into the inner face
    if ((e = fft_forward_f64(p, phi, 1, 1.0 / p.nphi, p.shell, s)) != cudaSuccess) return e;
    if ((e = shell_apply_f64(p, p.d_ishell, p.shell, p.shell2, s)) != cudaSuccess) return e;
    if ((e = fft_inverse_f64(p, p.shell2, 1, gr, false, s)) != cudaSuccess) return e;
  }
  const int lines = p.nr * p.nth;
  int blocks = (lines + kFaceWarps - 1) / kFaceWarps;
  if (blocks > p.num_sms * 8) blocks = p.num_sms * 8;   // one resident wave, 8 CTAs per SM
  const double scale = dir ? 1.0 / (p.r_out - p.r_last) : 1.0 / p.outer_coef;
  k_face_grad<<<(unsigned)blocks, 32 * kFaceWarps, 0, s>>>(phi, gr, gt, gp, p.d_face_r, p.d_face_t, p.nr, p.nth, p.nphi,
                                               dir ? 1 : 0, scale, reg ? -1.0 / p.inner_coef : 0.0);
  return cudaGetLastError();
}

cudaError_t thomas_f64(const Plan& p, double* x, cudaStream_t s) {
  const int n = p.mh * p.nth;
  k_thomas_f64<<<(n + 63) / 64, 64, 0, s>>>(p.d_rad, p.d_tinv, p.d_tcp, x, p.nr, p.nth, p.mh);
  return cudaGetLastError();
}

cudaError_t radial_factors_f64(const Plan& p, cudaStream_t s) {
  const int n = p.mh * p.nth;
  k_radial_factors_f64<<<(n + 127) / 128, 128, 0, s>>>(p.d_rad, p.d_lam, p.d_outer, p.d_inner, p.d_tinv, p.d_tcp,
                                                      p.nr, p.nth, p.mh);
  return cudaGetLastError();
}

cudaError_t stencil_f64(const Plan& p, const double* phi, double* out, cudaStream_t s) {
  const size_t n = (size_t)p.nr * p.nth * p.nphi;
  const double dir = (p.outer_bc == SP_OUTER_DIRICHLET) ? -p.outer_coef / (p.r_out - p.r_last) : 0.0;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_stencil_f64<<<(unsigned)blocks, 256, 0, s>>>(phi, out, p.d_rad, p.d_theta, p.nr, p.nth, p.nphi, dir);
  return cudaGetLastError();
}

void shell_apply_desc(const Plan& p, const double* O, const double* in, double* out, ShellArgs& a, int& ctas) {
  const int gx = (p.nth + kShellRows - 1) / kShellRows;
  a = ShellArgs{O, in, out, p.nth, p.mh, gx};
  ctas = gx * p.mh;
}

cudaError_t shell_apply_rag(const ShellArgs* tab, const int* start, int n, int total, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  k_shell_apply_rag<<<total, 32 * kShellRows, 0, s>>>(tab, start, n);
  return cudaGetLastError();
}

cudaError_t shell_apply_f64(const Plan& p, const double* O, const double* in, double* out, cudaStream_t s) {
  k_shell_apply<<<dim3((p.nth + kShellRows - 1) / kShellRows, p.mh), 32 * kShellRows, 0, s>>>(O, in, out, p.nth);
  return cudaGetLastError();
}

cudaError_t shell_kappa_f64(const Plan& p, const double* in, double* out, cudaStream_t s) {
  return shell_apply_f64(p, p.d_oshell, in, out, s);
}

cudaError_t shell_operator_f64(const Plan& p, const double* diag, double* dst, cudaStream_t s) {
  k_outer_operator<<<dim3(p.nth, p.mh), 128, 0, s>>>(p.d_HtW, p.d_H, diag, dst, p.nth);
  return cudaGetLastError();
}

cudaError_t outer_operator_f64(const Plan& p, cudaStream_t s) { return shell_operator_f64(p, p.d_outer, p.d_oshell, s); }

cudaError_t inner_term_f64(const Plan& p, const double* phi, double* out, cudaStream_t s) {
  cudaError_t e = fft_forward_f64(p, phi, 1, 1.0 / p.nphi, p.shell, s);
  if (e != cudaSuccess) return e;
  e = shell_apply_f64(p, p.d_ishell, p.shell, p.shell2, s);
  if (e != cudaSuccess) return e;
  return fft_inverse_f64(p, p.shell2, 1, out, true, s);
}

cudaError_t outer_term_f64(const Plan& p, const double* phi, double* out, cudaStream_t s) {
  const size_t off = (size_t)(p.nr - 1) * p.nth * p.nphi;
  cudaError_t e = fft_forward_f64(p, phi + off, 1, 1.0 / p.nphi, p.shell, s);
  if (e != cudaSuccess) return e;
  e = shell_kappa_f64(p, p.shell, p.shell2, s);
  if (e != cudaSuccess) return e;
  return fft_inverse_f64(p, p.shell2, 1, out + off, true, s);
}

}  // namespace sp
