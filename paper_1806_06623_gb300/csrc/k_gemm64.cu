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

}  // namespace

cudaError_t gemm_nt_f64(const double* A, const double* B, double* C, int nb, int M, int ncol, int K,
                        cudaStream_t s) {
  dim3 grid((ncol + BN - 1) / BN, (M + BM - 1) / BM, nb);
  k_gemm_nt_f64<<<grid, 256, 0, s>>>(A, B, C, M, ncol, K);
  return cudaGetLastError();
}

}  // namespace sp
