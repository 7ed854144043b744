// theta eigenbasis of Sect. 3.2, computed once per plan on the GPU in float64.
//
// For every azimuthal wavenumber m the operator Delta_hat_theta + S_j lambda_phi,m equals
// W^-1 B_m with W = diag(w_j) and B_m symmetric tridiagonal, so its eigenvectors are
// H = W^-1/2 Q with Q the orthonormal eigenvectors of T_m = W^-1/2 B_m W^-1/2 (also
// tridiagonal), and H^T W H = I; the inverse of H is H^T W.
//
// Parity split (Sect. 4.2): on a theta grid symmetric about the equator with an even
// number of zones, T_m commutes with the reflection j -> Ntheta-1-j, so its
// eigenvectors are even or odd in mu = cos(theta).  With h = Ntheta/2 the even vectors
// are [u; reverse(u)]/sqrt(2) with u an eigenvector of the leading h x h block whose
// last diagonal gains +e_{h-1}, the odd ones [u; -reverse(u)]/sqrt(2) with -e_{h-1}.
// Besides halving the work, each half block is graded in one direction only (large
// entries at the pole), which the QL iteration resolves to a much smaller error in the
// equatorial (small-|lambda|) modes than the doubly graded full matrix.
//
// Mode order: on a parity-split grid the even modes take l = 0..h-1 and the odd modes
// l = h..Ntheta-1, each half in descending order of lambda (the radial solves only need
// each mode's own lambda, so any order serves), and the half blocks are also written as
// (Ntheta/2)^2 tables (H^T W)_m,p[l][j] and H_m,p[j][l], p = even/odd, j < Ntheta/2:
// the projections then fold the spectrum into s(j) +- s(Ntheta-1-j) and multiply two
// half-size matrices per m instead of one full one (Sect. 4.2).  Otherwise l ranks all
// Ntheta eigenvalues in descending order.
//
// Each block is diagonalised by the implicit QL iteration with Wilkinson-type shifts
// (Bowdler, Martin, Reinsch & Wilkinson 1968; Golub & Van Loan, Sect. 8.3): each sweep
// chases the bulge from the bottom of the active block to its top with Givens
// rotations.  One CTA per m: thread 0 runs the scalar recurrence and records the
// rotations of a sweep in shared memory, then every thread applies them to its own
// row of the eigenvector matrix Z (column-major in shared memory).  Eigenvalues are
// ranked in descending order (l = 0 is lambda = 0 for m = 0), and the epilogue writes
// lambda, H, H^T W and the outer-boundary coefficient
// kappa = -p/r_out (r_out/r_N)^-p, p = (1 + sqrt(1 - 4 lambda))/2 (Sect. 3.2).
#include <cfloat>

#include "sp_internal.h"

namespace sp {
namespace {

constexpr int kMaxSweepsPerValue = 64;

struct QlControl {
  int lo, hi, done, fail;
};

// Diagonalise the n x n symmetric tridiagonal (d, e) in place; Z (n x n, Z[col*n+row])
// must hold the identity on entry and holds the eigenvectors on exit.  All threads of
// the CTA call this; thread 0 drives the iteration.
__device__ void ql_block(double* d, double* e, double* Z, int n, double* rc, double* rs, QlControl* ctl) {
  const int tid = threadIdx.x;
  int l = 0, iter = 0;
  if (tid == 0) ctl->done = 0;
  __syncthreads();
  while (true) {
    if (tid == 0) {
      int lo = -1, hi = -1;
      while (l < n && lo < 0) {
        int mm = l;
        for (; mm < n - 1; ++mm) {
          const double dd = fabs(d[mm]) + fabs(d[mm + 1]);
          if (fabs(e[mm]) <= DBL_EPSILON * dd) break;
        }
        if (mm == l) { ++l; iter = 0; continue; }
        if (++iter > kMaxSweepsPerValue) { ctl->fail = 1; l = n; break; }
        // shift from the leading 2x2 block of the active part
        double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
        double r = hypot(g, 1.0);
        g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
        double s = 1.0, c = 1.0, p = 0.0;
        int i = mm - 1;
        bool early = false;
        for (; i >= l; --i) {
          const double f = s * e[i];
          const double b = c * e[i];
          r = hypot(f, g);
          e[i + 1] = r;
          if (r == 0.0) { d[i + 1] -= p; e[mm] = 0.0; early = true; break; }
          s = f / r;
          c = g / r;
          g = d[i + 1] - p;
          r = (d[i] - g) * s + 2.0 * c * b;
          p = s * r;
          d[i + 1] = g + p;
          g = c * r - b;
          rc[i] = c;
          rs[i] = s;
        }
        if (!early) { d[l] -= p; e[l] = g; e[mm] = 0.0; }
        lo = early ? i + 1 : l;
        hi = mm;
      }
      if (lo < 0) ctl->done = 1;
      else { ctl->lo = lo; ctl->hi = hi; }
    }
    __syncthreads();
    if (ctl->done) break;
    const int lo = ctl->lo, hi = ctl->hi;
    for (int row = tid; row < n; row += blockDim.x) {
      for (int i = hi - 1; i >= lo; --i) {
        const double c = rc[i], s = rs[i];
        const double zi = Z[i * n + row];
        const double zi1 = Z[(i + 1) * n + row];
        Z[(i + 1) * n + row] = s * zi + c * zi1;
        Z[i * n + row] = c * zi - s * zi1;
      }
    }
    __syncthreads();
  }
  __syncthreads();
}

__global__ void k_theta_eigen(const double* __restrict__ tdiag, const double* __restrict__ toff,
                              const double* __restrict__ sqw, int nth, int parity, int outer_bc, double r_out,
                              double r_last, double outer_coef, int inner_regular, double r_in, double r_first,
                              double inner_coef, double* __restrict__ lam_out,
                              double* __restrict__ kappa_out, double* __restrict__ outer_out,
                              double* __restrict__ inner_out,
                              double* __restrict__ H, double* __restrict__ HtW, double* __restrict__ Hp,
                              double* __restrict__ HtWp, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int h = parity ? nth / 2 : nth;       // block size
  const int nblk = parity ? 2 : 1;
  double* Z = reinterpret_cast<double*>(smem_raw);   // nblk blocks of h*h
  double* d = Z + nblk * h * h;                      // [nth]
  double* e = d + nth;                               // [nth]
  double* rc = e + nth;                              // [h]
  double* rs = rc + h;                               // [h]
  int* rank = reinterpret_cast<int*>(rs + h);        // [nth]
  __shared__ QlControl ctl;

  const int m = blockIdx.x;
  const int tid = threadIdx.x;
  for (int t = tid; t < nblk * h * h; t += blockDim.x) {
    const int q = t % (h * h);
    Z[t] = ((q / h) == (q % h)) ? 1.0 : 0.0;
  }
  if (parity) {
    // even block in d[0..h), odd block in d[h..2h); off-diagonals likewise
    for (int t = tid; t < h; t += blockDim.x) {
      const double dv = tdiag[(size_t)m * nth + t];
      const double mid = (t == h - 1) ? toff[h - 1] : 0.0;
      d[t] = dv + mid;
      d[h + t] = dv - mid;
      e[t] = (t < h - 1) ? toff[t] : 0.0;
      e[h + t] = e[t];
    }
  } else {
    for (int t = tid; t < nth; t += blockDim.x) {
      d[t] = tdiag[(size_t)m * nth + t];
      e[t] = (t < nth - 1) ? toff[t] : 0.0;
    }
  }
  if (tid == 0) ctl.fail = 0;
  __syncthreads();
  for (int b = 0; b < nblk; ++b) ql_block(d + b * h, e + b * h, Z + b * h * h, h, rc, rs, &ctl);
  if (tid == 0 && ctl.fail) atomicOr(err, kErrEigenIter);
  if (m == 0) {
    // The constant is an exact eigenvector with lambda = 0 for m = 0 (every theta flux
    // vanishes).  QL returns it with an absolute eigenvalue error ~eps ||T_0||, which the
    // near-singular l=0 radial problem amplifies; deflate it exactly instead.  In Q
    // coordinates the constant is sqrt(w_j)/sqrt(sum w) (times sqrt(2) in the even half
    // block); the other block-0 vectors are W-orthogonalised against it.
    __shared__ int s_a0;
    __shared__ double s_norm;
    double* uc = rc;   // reuse the rotation buffers: uc[h]
    if (tid == 0) {
      int a0 = 0;
      for (int a = 1; a < h; ++a)
        if (d[a] > d[a0]) a0 = a;
      s_a0 = a0;
      double sw = 0.0;
      for (int j = 0; j < nth; ++j) sw += sqw[j] * sqw[j];
      s_norm = (parity ? sqrt(2.0) : 1.0) / sqrt(sw);
      d[a0] = 0.0;
    }
    __syncthreads();
    for (int j = tid; j < h; j += blockDim.x) uc[j] = sqw[j] * s_norm;
    __syncthreads();
    const int a0 = s_a0;
    for (int k = tid; k < h; k += blockDim.x) {
      double* z = Z + k * h;
      if (k == a0) {
        for (int j = 0; j < h; ++j) z[j] = uc[j];
      } else {
        double dot = 0.0;
        for (int j = 0; j < h; ++j) dot += uc[j] * z[j];
        double nn = 0.0;
        for (int j = 0; j < h; ++j) {
          z[j] -= dot * uc[j];
          nn += z[j] * z[j];
        }
        const double inv = 1.0 / sqrt(nn);
        for (int j = 0; j < h; ++j) z[j] *= inv;
      }
    }
    __syncthreads();
  }
  // descending rank, ties broken by index: within the half block of a parity grid
  // (l = block * h + rank), else over all nth eigenvalues
  for (int a = tid; a < nth; a += blockDim.x) {
    const int b0 = parity ? (a / h) * h : 0, b1 = parity ? b0 + h : nth;
    int rnk = b0;
    const double va = d[a];
    for (int b = b0; b < b1; ++b) {
      const double vb = d[b];
      rnk += (vb > va) || (vb == va && b < a);
    }
    rank[a] = rnk;
  }
  __syncthreads();
  for (int a = tid; a < nth; a += blockDim.x) {
    const int lrow = rank[a];
    const double lam = d[a];
    lam_out[(size_t)m * nth + lrow] = lam;
    const double p = 0.5 * (1.0 + sqrt(1.0 - 4.0 * lam));
    const double kap = -p / r_out * exp(-p * log(r_out / r_last));
    kappa_out[(size_t)m * nth + lrow] = kap;
    outer_out[(size_t)m * nth + lrow] =
        (outer_bc == SP_OUTER_DIRICHLET) ? -outer_coef / (r_out - r_last) : outer_coef * kap;
    // regular interior: inner-face gradient q f_1 (r_in/r_1)^q / r_in, q = (-1 + sqrt(1 - 4 lambda))/2,
    // entering row 1 with minus the face area over the volume
    double in_d = 0.0;
    if (inner_regular) {
      const double q = 0.5 * (-1.0 + sqrt(1.0 - 4.0 * lam));
      in_d = -inner_coef * (q / r_in) * exp(q * log(r_in / r_first));
    }
    inner_out[(size_t)m * nth + lrow] = in_d;
  }
  // H[m][j][l] = q_j/sqrt(w_j), HtW[m][l][j] = q_j sqrt(w_j), l = rank[a]
  double* Hm = H + (size_t)m * nth * nth;
  double* Am = HtW + (size_t)m * nth * nth;
  const double rsq2 = 0.70710678118654752440084436210485;
  for (int t = tid; t < nth * nth; t += blockDim.x) {
    const int a = t / nth;   // eigenvector index
    const int j = t - a * nth;
    double z;
    if (parity) {
      const int blk = a / h, col = a - blk * h;
      const bool upper = j < h;
      const int jj = upper ? j : nth - 1 - j;
      const double v = Z[blk * h * h + col * h + jj] * rsq2;
      z = (upper || blk == 0) ? v : -v;
    } else {
      z = Z[a * nth + j];
    }
    const double sw = sqw[j];
    const int lrow = rank[a];
    Am[(size_t)lrow * nth + j] = z * sw;
    Hm[(size_t)j * nth + lrow] = z / sw;
  }
  if (parity) {
    // half tables [m][p][h][h]: (H^T W)_p[l][j] and H_p[j][l] for j < h, the values of
    // the full tables' upper half (the lower half mirrors them, with a sign for p = odd)
    double* Ap = HtWp + (size_t)m * 2 * h * h;
    double* Hq = Hp + (size_t)m * 2 * h * h;
    for (int t = tid; t < nth * h; t += blockDim.x) {
      const int a = t / h, j = t - a * h;
      const int blk = a / h, col = a - blk * h;
      const int lrow = rank[a] - blk * h;
      const double v = Z[blk * h * h + col * h + j] * rsq2;
      const double sw = sqw[j];
      Ap[((size_t)blk * h + lrow) * h + j] = v * sw;
      Hq[((size_t)blk * h + j) * h + lrow] = v / sw;
    }
  }
}

}  // namespace

size_t theta_eigen_smem(int nth, bool parity) {
  const int h = parity ? nth / 2 : nth;
  const int nblk = parity ? 2 : 1;
  return sizeof(double) * ((size_t)nblk * h * h + 2 * (size_t)nth + 2 * (size_t)h) + sizeof(int) * nth;
}

cudaError_t theta_eigen(const Plan& p, cudaStream_t s) {
  const int nth = p.nth;
  const size_t smem = theta_eigen_smem(nth, p.parity);
  cudaError_t e = allow_smem(k_theta_eigen, smem);
  if (e != cudaSuccess) return e;
  int threads = ((nth + 31) / 32) * 32;
  if (threads < 32) threads = 32;
  k_theta_eigen<<<p.mh, threads, smem, s>>>(p.d_tdiag, p.d_toff, p.d_sqw, nth, p.parity ? 1 : 0, p.outer_bc,
                                            p.r_out, p.r_last, p.outer_coef,
                                            p.inner_bc == SP_INNER_REGULAR ? 1 : 0, p.r_in, p.r_first, p.inner_coef,
                                            p.d_lam, p.d_kappa, p.d_outer, p.d_inner,
                                            p.d_H, p.d_HtW, p.d_Hp, p.d_HtWp, p.d_err);
  return cudaGetLastError();
}

}  // namespace sp
