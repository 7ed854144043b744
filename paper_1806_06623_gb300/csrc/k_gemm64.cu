// float64 theta projections (Sect. 3.2): for every m,
//   forward  s_hat[i,c,l] = sum_j (H^T W)_m[l,j] s_tilde[i,c,j]
//   inverse  g[i,c,j]     = sum_l  H_m[j,l]      f[i,c,l]
// Both are the batched NT product C[b][n][r] = sum_k A[b][r][k] B[b][n][k] with the
// panel column n = (i,c) K-contiguous, as the FFT writes it.  GB300 has no fast float64
// tensor path, so this is a register-tiled DFMA kernel: a 64x64 tile per CTA, 16-wide
// K slices staged through shared memory, a 4x4 accumulator block per thread.
#include "sp_internal.h"

namespace sp {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256) k_gemm_nt_f64(const double* __restrict__ A, const double* __restrict__ B,
                                                     double* __restrict__ C, int M, int ncol, int K) {
  __shared__ double As[BK][BM + 2];
  __shared__ double Bs[BK][BN + 2];
  const int b = blockIdx.z;
  const int n0 = blockIdx.x * BN;
  const int m0 = blockIdx.y * BM;
  const double* Ab = A + (size_t)b * M * K;
  const double* Bb = B + (size_t)b * ncol * K;
  double* Cb = C + (size_t)b * ncol * M;
  const int tid = threadIdx.x;
  const int tm = tid & 15;   // row group (4 rows)
  const int tn = tid >> 4;   // column group (4 columns)
  double acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.0;

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / 256; ++q) {
      const int e = tid + q * 256;
      const int r = e / BK, kk = e % BK;
      const int gr = m0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? Ab[(size_t)gr * K + gk] : 0.0;
      const int gc = n0 + r;
      Bs[kk][r] = (gc < ncol && gk < K) ? Bb[(size_t)gc * K + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], bv[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = As[kk][tm * 4 + x];
#pragma unroll
      for (int y = 0; y < 4; ++y) bv[y] = Bs[kk][tn * 4 + y];
#pragma unroll
      for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) acc[y][x] = fma(a[x], bv[y], acc[y][x]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const int gc = n0 + tn * 4 + y;
    if (gc >= ncol) continue;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int gr = m0 + tm * 4 + x;
      if (gr < M) Cb[(size_t)gc * M + gr] = acc[y][x];
    }
  }
}

// Parity-split projections (Sect. 4.2) on a theta grid symmetric about the equator,
// nth = 2h.  A holds the two half blocks of every m, A[b][p][r][k] (p = 0 even, 1 odd).
//  forward: C[b][n][p*h + r] = sum_{k<h} A[b][p][r][k] (B[b][n][k] +- B[b][n][nth-1-k])
//  inverse: g_p[n][r] = sum_{k<h} A[b][p][r][k] B[b][n][p*h + k];
//           C[b][n][r] = g_0 + g_1, C[b][n][nth-1-r] = g_0 - g_1.
// A CTA computes the same 64x64 (r, n) tile of both parities, so the fold (forward)
// reads each panel value once for both products and the unfold (inverse) has both
// results in registers: half the multiply-adds of the full Nth x Nth product for the
// same panel traffic.
__global__ void __launch_bounds__(256) k_gemm_parity_f64(const double* __restrict__ A, const double* __restrict__ B,
                                                         double* __restrict__ C, int h, int ncol, int inverse) {
  __shared__ double As[2][BK][BM + 2];
  __shared__ double Bs[2][BK][BN + 2];
  const int b = blockIdx.z;
  const int n0 = blockIdx.x * BN;
  const int m0 = blockIdx.y * BM;
  const int nth = 2 * h;
  const double* Ab = A + (size_t)b * 2 * h * h;
  const double* Bb = B + (size_t)b * ncol * nth;
  double* Cb = C + (size_t)b * ncol * nth;
  const int tid = threadIdx.x;
  const int tm = tid & 15;
  const int tn = tid >> 4;
  double acc[2][4][4];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[q][x][y] = 0.0;

  for (int k0 = 0; k0 < h; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / 256; ++q) {
      const int e = tid + q * 256;
      const int r = e / BK, kk = e % BK;
      const int gr = m0 + r, gk = k0 + kk;
      const bool ak = gr < h && gk < h;
      As[0][kk][r] = ak ? Ab[(size_t)gr * h + gk] : 0.0;
      As[1][kk][r] = ak ? Ab[(size_t)(h + gr) * h + gk] : 0.0;
      const int gc = n0 + r;
      double b0 = 0.0, b1 = 0.0;
      if (gc < ncol && gk < h) {
        const double* row = Bb + (size_t)gc * nth;
        if (inverse) {
          b0 = row[gk];
          b1 = row[h + gk];
        } else {
          const double u = row[gk], v = row[nth - 1 - gk];
          b0 = u + v;
          b1 = u - v;
        }
      }
      Bs[0][kk][r] = b0;
      Bs[1][kk][r] = b1;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        double a[4], bv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) a[x] = As[q][kk][tm * 4 + x];
#pragma unroll
        for (int y = 0; y < 4; ++y) bv[y] = Bs[q][kk][tn * 4 + y];
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
          for (int x = 0; x < 4; ++x) acc[q][y][x] = fma(a[x], bv[y], acc[q][y][x]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const int gc = n0 + tn * 4 + y;
    if (gc >= ncol) continue;
    double* row = Cb + (size_t)gc * nth;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int gr = m0 + tm * 4 + x;
      if (gr >= h) continue;
      if (inverse) {
        row[gr] = acc[0][y][x] + acc[1][y][x];
        row[nth - 1 - gr] = acc[0][y][x] - acc[1][y][x];
      } else {
        row[gr] = acc[0][y][x];
        row[h + gr] = acc[1][y][x];
      }
    }
  }
}

}  // namespace

cudaError_t gemm_parity_f64(const double* A, const double* B, double* C, int nb, int h, int ncol, bool inverse,
                            cudaStream_t s) {
  dim3 grid((ncol + BN - 1) / BN, (h + BM - 1) / BM, nb);
  k_gemm_parity_f64<<<grid, 256, 0, s>>>(A, B, C, h, ncol, inverse ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t gemm_nt_f64(const double* A, const double* B, double* C, int nb, int M, int ncol, int K,
                        cudaStream_t s) {
  dim3 grid((ncol + BN - 1) / BN, (M + BM - 1) / BM, nb);
  k_gemm_nt_f64<<<grid, 256, 0, s>>>(A, B, C, M, ncol, K);
  return cudaGetLastError();
}

}  // namespace sp
