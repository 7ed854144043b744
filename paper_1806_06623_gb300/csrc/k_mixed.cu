// Mixed-precision solve (SP_MIXED_BF16X3): the low-precision separated solve and the
// float64 residual of the finite-volume operator used to refine it.
//
//  low-precision solve of L e = r (Sect. 3.2 steps in float32):
//    FFT (float32, bf16 hi/lo panel out) -> tcgen05 projection with (H^T W)_m
//    -> radial solves (float32; float64 for the near-singular |lambda| < 30 modes)
//    -> tcgen05 projection with H_m -> inverse FFT (float32) with Phi += e in float64
//  residual: r = 4 pi G rho - L Phi in float64 (stencil of Eq. fin_vol3 plus the
//    multipole outer-shell term), stored in float32 as the next right-hand side.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fft_dev.cuh"
#include "sp_internal.h"
#include "tc_gemm.cuh"

namespace sp {
namespace {

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// table [b][rows][n] float64 -> bf16 planes [b][rows][kstride] (x0 = RN(x), x1 = RN(x - x0),
// x2 = RN(x - x0 - x1), differences in float64), zero beyond n
__global__ void k_split_table(const double* __restrict__ src, int n, int kstride, size_t total, Planes pl) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % kstride);
    const size_t br = t / kstride;
    double x = 0.0;
    if (k < n) x = src[br * n + k];
    const __nv_bfloat16 h = __double2bfloat16(x);
    pl.p[0][t] = h;
    const double r = x - (double)__bfloat162float(h);
    const __nv_bfloat16 m = __double2bfloat16(r);
    pl.p[1][t] = m;
    if (pl.n == 3) pl.p[2][t] = __double2bfloat16(r - (double)__bfloat162float(m));
  }
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kTR = 16;       // radial rows per staged chunk
constexpr int kStages = 6;    // chunks in flight per warp

// Radial solves of the low-precision solve.  The elimination factors c'_i and 1/pivot_i
// of every (m,l) system depend on the plan only and are precomputed (float64, rounded
// to float32), so the sweeps carry no division: forward d_i = (x_i - sub_i d_{i-1})/piv_i,
// backward f_i = d_i - c'_i f_{i+1}.  One warp per (m, c = re/im, 32 consecutive l);
// rows of the mode array and of the factor tables stream through a kStages-deep ring
// of cp.async copies (each lane copies its own elements) so each sweep reads shared
// memory while later rows are in flight.  Lanes of near-singular modes (|lambda| < thr)
// idle here; the trailing blocks solve those in float64, one mode per warp.
// x holds s_hat[m][i][c][l] on entry and the forward values afterwards; f leaves as bf16
// planes in the panel layout.
__global__ void __launch_bounds__(32) k_thomas_staged(const float* __restrict__ sub_r, const double* __restrict__ lam,
                                                      float* __restrict__ x, const float* __restrict__ fcp,
                                                      const float* __restrict__ finv, float* __restrict__ pl, int nr, int nth,
                                                      int kstride, double thr, int nblk_f32,
                                                      const int* __restrict__ low_idx, int nlow,
                                                      const RadialRow* __restrict__ rad64,
                                                      const double2* __restrict__ low_fac, double* __restrict__ low_ws) {
  __shared__ float sx[kStages][kTR][2][32];
  const int lane = threadIdx.x;
  const size_t st = 2 * (size_t)nth;
  const int nchunk = (nr + kTR - 1) / kTR;
  if ((int)blockIdx.x >= nblk_f32) {
    // ---- float64 near-singular mode, one per warp: the column and its precomputed
    // elimination factors are loaded in parallel, lane 0 runs both sweeps out of shared
    // memory (or low_ws when the column does not fit), all lanes write the result.
    const int q = (int)blockIdx.x - nblk_f32;
    if (q >= nlow) return;
    const int t = low_idx[q];
    const int m = t / nth;
    const int l = t - m * nth;
    const float* X = x + (size_t)m * nr * st + l;
    const double2* F = low_fac + (size_t)q * nr;     // (c'_i, 1/pivot_i)
    double* W = (3 * nr <= (int)(sizeof(sx) / sizeof(double))) ? reinterpret_cast<double*>(&sx[0][0][0][0])
                                                                 : low_ws + (size_t)q * nr * 3;
    for (int i = lane; i < nr; i += 32) {
      W[3 * i] = (double)X[(size_t)i * st];
      W[3 * i + 1] = (double)X[(size_t)i * st + nth];
      W[3 * i + 2] = F[i].x;
    }
    __threadfence_block();
    __syncwarp();
    if (lane == 0) {
      double dre = 0.0, dim = 0.0;
      for (int i = 0; i < nr; ++i) {
        const double sub = rad64[i].sub;
        const double inv = F[i].y;
        dre = (W[3 * i] - sub * dre) * inv;
        dim = (W[3 * i + 1] - sub * dim) * inv;
        W[3 * i] = dre;
        W[3 * i + 1] = dim;
      }
      for (int i = nr - 2; i >= 0; --i) {
        const double c = W[3 * i + 2];
        dre = W[3 * i] - c * dre;
        dim = W[3 * i + 1] - c * dim;
        W[3 * i] = dre;
        W[3 * i + 1] = dim;
      }
    }
    __threadfence_block();
    __syncwarp();
    const size_t prow = (size_t)m * nr * 2;
    for (int i = lane; i < nr; i += 32) {
      pl[(prow + 2 * i) * kstride + l] = (float)W[3 * i];
      pl[(prow + 2 * i + 1) * kstride + l] = (float)W[3 * i + 1];
    }
    return;
  }
  // ---- float32 modes: block = (m, lb, c)
  const int nlb = (nth + 31) / 32;
  const int c = blockIdx.x & 1;
  const int mb = blockIdx.x >> 1;
  const int m = mb / nlb;
  const int l = (mb - m * nlb) * 32 + lane;
  const bool valid = l < nth;
  const bool work = valid && fabs(lam[m * nth + l]) >= thr;
  float* X = x + (size_t)m * nr * st + (size_t)c * nth + (valid ? l : 0);
  const float* FC = fcp + (size_t)m * nr * nth + (valid ? l : 0);
  const float* FI = finv + (size_t)m * nr * nth + (valid ? l : 0);

  auto fetch = [&](int k, bool fwd) {   // k-th chunk in sweep order into ring slot k % kStages
    const int ch = fwd ? k : nchunk - 1 - k;
    if (ch >= 0 && ch < nchunk && work) {
      const int i0 = ch * kTR;
      const int n = min(kTR, nr - i0);
      float(*b)[2][32] = sx[k % kStages];
      for (int r = 0; r < n; ++r) {
        cp_async4(&b[r][0][lane], X + (size_t)(i0 + r) * st);
        cp_async4(&b[r][1][lane], (fwd ? FI : FC) + (size_t)(i0 + r) * nth);
      }
    }
    cp_async_commit();
  };
  // forward sweep
  for (int k = 0; k < kStages - 1; ++k) fetch(k, true);
  float d = 0.f;
  for (int k = 0; k < nchunk; ++k) {
    fetch(k + kStages - 1, true);
    cp_async_wait<kStages - 1>();
    __syncwarp();
    if (work) {
      const int i0 = k * kTR;
      const int n = min(kTR, nr - i0);
      float(*b)[2][32] = sx[k % kStages];
      for (int r = 0; r < n; ++r) {
        const int i = i0 + r;
        d = fmaf(-sub_r[i], d, b[r][0][lane]) * b[r][1][lane];
        X[(size_t)i * st] = d;
      }
    }
    __syncwarp();
  }
  cp_async_wait<0>();
  __threadfence_block();
  __syncwarp();
  // back substitution, chunks in reverse; each lane re-reads only its own elements
  const size_t prow = (size_t)m * nr * 2 + c;
  for (int k = 0; k < kStages - 1; ++k) fetch(k, false);
  float f = 0.f;
  for (int k = 0; k < nchunk; ++k) {
    fetch(k + kStages - 1, false);
    cp_async_wait<kStages - 1>();
    __syncwarp();
    if (work) {
      const int ch = nchunk - 1 - k;
      const int i0 = ch * kTR;
      const int n = min(kTR, nr - i0);
      float(*b)[2][32] = sx[k % kStages];
      for (int r = n - 1; r >= 0; --r) {
        const int i = i0 + r;
        f = (i == nr - 1) ? b[r][0][lane] : fmaf(-b[r][1][lane], f, b[r][0][lane]);
        pl[(prow + 2 * i) * kstride + l] = f;
      }
    }
    __syncwarp();
  }
  cp_async_wait<0>();
}

// Radial solves of the low-precision solve as segmented scans.  With the factors
// precomputed, the forward sweep d_i = b_i + a_i d_{i-1} (b_i = x_i/piv_i,
// a_i = -sub_i/piv_i) and the back substitution f_i = d_i - c'_i f_{i+1} are first-order
// linear recurrences.  One CTA per (m, kScanCols consecutive l) and NC of the two
// components re/im (NC = 2 whenever two such CTAs fit on an SM): the column block's rows
// are first staged in shared memory with cp.async (all rows in flight at once), then
// each of kScanSegs thread groups sweeps one radial segment from a zero start while
// recording the running product of the coefficients, which depends on the matrix only
// and so serves both components; the first group chains the segment carries and every
// group adds carry x product to its rows.  The forward values stay in shared memory for
// the back substitution.  All coefficients
// are contractive (|a_i|, |c'_i| < 1 for these diagonally dominant systems), so the
// reassociation does not amplify rounding.  Lanes of near-singular modes idle; the
// leading CTAs solve those in float64 with the same segmented scan (one warp per mode
// and component, 32 segments, carries by a shuffle scan), concurrently with the rest.
constexpr int kScanCols = 16;
constexpr int kScanThreads = 256;
constexpr int kScanSegs = kScanThreads / kScanCols;

// float32 CTAs: NC arrays D and one Q [nr][kScanCols] + sub [nr] floats; float64 CTAs:
// 8 warps x 2 x nr doubles
size_t scan_smem_bytes(int nr, int nc) {
  const size_t f32 = ((nc + 1) * (size_t)nr * kScanCols + (size_t)nr) * sizeof(float);
  const size_t f64 = (size_t)(kScanThreads / 32) * 2 * nr * sizeof(double);
  return f32 > f64 ? f32 : f64;
}

template <int NC>
__device__ __forceinline__ void thomas_scan_body(
    const float* __restrict__ sub_r, const double* __restrict__ lam, const float* __restrict__ x,
    const float* __restrict__ fcp, const float* __restrict__ finv, float* __restrict__ pl, int nr, int nth, int kstride,
    double thr, int nlowblk, const int* __restrict__ low_idx, int nlow, const RadialRow* __restrict__ rad64,
    const double2* __restrict__ low_fac, int bx) {
  extern __shared__ __align__(16) float sm[];
  // D[c] [nr][kScanCols]: right-hand side, then d, then f of component c
  float* Q = sm + (size_t)NC * nr * kScanCols;   // [nr][kScanCols] 1/pivot or c', then running products
  float* A = Q + (size_t)nr * kScanCols;         // [nr] sub-diagonal
  __shared__ float sE[NC][kScanSegs][kScanCols], sP[kScanSegs][kScanCols], sC[NC][kScanSegs][kScanCols];
  const int tid = threadIdx.x;
  const size_t st = 2 * (size_t)nth;
  pdl_trigger();
  pdl_wait();
  if (bx < nlowblk) {
    // ---- float64 near-singular modes: warp pair (re, im) per mode, same segmented scan
    // over the warp's 32 lanes, carries by a shuffle scan of the affine segment maps
    const int warp = tid >> 5, lane = tid & 31;
    const int q = bx * (kScanThreads / 64) + (warp >> 1);
    const int cc = warp & 1;
    if (q >= nlow) return;
    const int t = low_idx[q];
    const int m = t / nth;
    const int l = t - m * nth;
    const float* X = x + (size_t)m * nr * st + (size_t)cc * nth + l;
    const double2* F = low_fac + (size_t)q * nr;   // (c'_i, 1/pivot_i)
    double* Wd = reinterpret_cast<double*>(sm) + (size_t)warp * 2 * nr;
    double* Wq = Wd + nr;
    for (int i = lane; i < nr; i += 32) {
      Wd[i] = (double)X[(size_t)i * st];
      Wq[i] = F[i].y;
    }
    __syncwarp();
    int Ll = (nr + 31) / 32;
    Ll += (Ll & 1) ^ 1;
    const int j0 = min(nr, lane * Ll), j1 = min(nr, j0 + Ll);
    double v = 0.0, pr = 1.0;
    for (int i = j0; i < j1; ++i) {
      const double a = -rad64[i].sub * Wq[i];
      v = fma(a, v, Wd[i] * Wq[i]);
      pr *= a;
      Wd[i] = v;
      Wq[i] = pr;
    }
    for (int off = 1; off < 32; off <<= 1) {
      const double e2 = __shfl_up_sync(0xffffffffu, v, off), p2 = __shfl_up_sync(0xffffffffu, pr, off);
      if (lane >= off) {
        v = fma(pr, e2, v);
        pr *= p2;
      }
    }
    double carry = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 0) carry = 0.0;
    for (int i = j0; i < j1; ++i) Wd[i] = fma(Wq[i], carry, Wd[i]);
    __syncwarp();
    for (int i = lane; i < nr; i += 32) Wq[i] = F[i].x;
    __syncwarp();
    v = 0.0;
    pr = 1.0;
    for (int i = j1 - 1; i >= j0; --i) {
      const double g = -Wq[i];
      v = fma(g, v, Wd[i]);
      pr *= g;
      Wd[i] = v;
      Wq[i] = pr;
    }
    for (int off = 1; off < 32; off <<= 1) {
      const double e2 = __shfl_down_sync(0xffffffffu, v, off), p2 = __shfl_down_sync(0xffffffffu, pr, off);
      if (lane + off < 32) {
        v = fma(pr, e2, v);
        pr *= p2;
      }
    }
    carry = __shfl_down_sync(0xffffffffu, v, 1);
    if (lane == 31) carry = 0.0;
    const size_t prow = (size_t)m * nr * 2 + cc;
    for (int i = j0; i < j1; ++i) pl[(prow + 2 * i) * kstride + l] = (float)fma(Wq[i], carry, Wd[i]);
    return;
  }
  const int col = tid % kScanCols, seg = tid / kScanCols;
  const int ncb = (nth + kScanCols - 1) / kScanCols;
  const int bid = bx - nlowblk;
  const int c0 = NC == 2 ? 0 : (bid & 1);   // first component of this CTA
  const int mb = NC == 2 ? bid : (bid >> 1);
  const int m = mb / ncb;
  const int l = (mb - m * ncb) * kScanCols + col;
  const bool valid = l < nth;
  const bool work = valid && fabs(lam[m * nth + l]) >= thr;
  // segments of odd length: the two segments a warp holds then sit 16 banks apart
  int L = (nr + kScanSegs - 1) / kScanSegs;
  L += (L & 1) ^ 1;
  const int i0 = min(nr, seg * L), i1 = min(nr, i0 + L);
  // ---- stage the right-hand sides and 1/pivot of the whole column block: 16-byte copies
  // (4 threads per 16-column row) when rows start on 16-byte boundaries, else 4-byte
  const int lb0 = (mb - m * ncb) * kScanCols;
  const bool vec4 = (nth & 3) == 0;
  auto stage = [&](float* dst, const float* src, size_t rstride) {   // src: column lb0 of row 0
    if (vec4) {
      const int c4 = tid & 3, r0 = tid >> 2;
      if (lb0 + 4 * c4 < nth) {
        const float* g = src + 4 * c4 + (size_t)r0 * rstride;
        float* sd = dst + r0 * kScanCols + 4 * c4;
        for (int i = r0; i < nr; i += kScanThreads / 4, g += (kScanThreads / 4) * rstride, sd += (kScanThreads / 4) * kScanCols)
          cp_async16(sd, g);
      }
    } else if (valid) {
      const float* g = src + col + (size_t)seg * rstride;
      float* sd = dst + seg * kScanCols + col;
      for (int i = seg; i < nr; i += kScanSegs, g += kScanSegs * rstride, sd += kScanSegs * kScanCols) cp_async4(sd, g);
    }
  };
#pragma unroll
  for (int c = 0; c < NC; ++c)
    stage(sm + (size_t)c * nr * kScanCols, x + (size_t)m * nr * st + (size_t)(c0 + c) * nth + lb0, st);
  stage(Q, finv + (size_t)m * nr * nth + lb0, nth);
  cp_async_commit();
  for (int i = tid; i < nr; i += kScanThreads) A[i] = sub_r[i];
  cp_async_wait<0>();
  __syncthreads();
  const int nseg = i1 - i0;
  const size_t cst = (size_t)nr * kScanCols;   // distance between the components' arrays
  // ---- forward sweep of this segment from d = 0
  float d[NC], q = 1.f;
#pragma unroll
  for (int c = 0; c < NC; ++c) d[c] = 0.f;
  if (work) {
    float* Dp = sm + i0 * kScanCols + col;
    float* Qp = Q + i0 * kScanCols + col;
    const float* Ap = A + i0;
#pragma unroll 4
    for (int n = 0; n < nseg; ++n) {
      const float iv = Qp[n * kScanCols];
      const float a = -Ap[n] * iv;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        d[c] = fmaf(a, d[c], Dp[c * cst + n * kScanCols] * iv);
        Dp[c * cst + n * kScanCols] = d[c];
      }
      q *= a;
      Qp[n * kScanCols] = q;
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) sE[c][seg][col] = d[c];
  sP[seg][col] = q;
  __syncthreads();
  if (seg < NC) {   // group c chains the carries of component c
    float carry = 0.f;   // d_{-1} = 0
    for (int w = 0; w < kScanSegs; ++w) {
      sC[seg][w][col] = carry;
      carry = fmaf(sP[w][col], carry, sE[seg][w][col]);
    }
  }
  __syncthreads();
  if (work) {
    float cw[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) cw[c] = sC[c][seg][col];
    float* Dp = sm + i0 * kScanCols + col;
    const float* Qp = Q + i0 * kScanCols + col;
#pragma unroll 4
    for (int n = 0; n < nseg; ++n) {
      const float qn = Qp[n * kScanCols];
#pragma unroll
      for (int c = 0; c < NC; ++c) Dp[c * cst + n * kScanCols] = fmaf(qn, cw[c], Dp[c * cst + n * kScanCols]);
    }
  }
  __syncthreads();
  // ---- stage c' over the running products, then back-substitute from f = 0
  stage(Q, fcp + (size_t)m * nr * nth + lb0, nth);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  float f[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) f[c] = 0.f;
  q = 1.f;
  if (work) {
    float* Dp = sm + (i1 - 1) * kScanCols + col;
    float* Qp = Q + (i1 - 1) * kScanCols + col;
#pragma unroll 4
    for (int n = 0; n < nseg; ++n) {
      const float g = -Qp[-n * kScanCols];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        f[c] = fmaf(g, f[c], Dp[c * cst - n * kScanCols]);
        Dp[c * cst - n * kScanCols] = f[c];
      }
      q *= g;
      Qp[-n * kScanCols] = q;
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) sE[c][seg][col] = f[c];   // value at the segment's first row from a zero start above it
  sP[seg][col] = q;
  __syncthreads();
  if (seg < NC) {
    float carry = 0.f;   // f_{nr} is absent
    for (int w = kScanSegs - 1; w >= 0; --w) {
      sC[seg][w][col] = carry;
      carry = fmaf(sP[w][col], carry, sE[seg][w][col]);
    }
  }
  __syncthreads();
  if (work) {
    float cw[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) cw[c] = sC[c][seg][col];
    const float* Dp = sm + i0 * kScanCols + col;
    const float* Qp = Q + i0 * kScanCols + col;
    float* out = pl + ((size_t)m * nr * 2 + c0 + 2 * (size_t)i0) * kstride + l;
    const size_t ostep = 2 * (size_t)kstride;
#pragma unroll 4
    for (int n = 0; n < nseg; ++n) {
      const float qn = Qp[n * kScanCols];
#pragma unroll
      for (int c = 0; c < NC; ++c) out[n * ostep + c * kstride] = fmaf(qn, cw[c], Dp[c * cst + n * kScanCols]);
    }
  }
}

template <int NC>
__global__ void __launch_bounds__(kScanThreads) k_thomas_scan(
    const float* __restrict__ sub_r, const double* __restrict__ lam, const float* __restrict__ x,
    const float* __restrict__ fcp, const float* __restrict__ finv, float* __restrict__ pl, int nr, int nth, int kstride,
    double thr, int nlowblk, const int* __restrict__ low_idx, int nlow, const RadialRow* __restrict__ rad64,
    const double2* __restrict__ low_fac) {
  thomas_scan_body<NC>(sub_r, lam, x, fcp, finv, pl, nr, nth, kstride, thr, nlowblk, low_idx, nlow, rad64, low_fac,
                       blockIdx.x);
}

template <int NC>
__global__ void __launch_bounds__(kScanThreads) k_thomas_scan_rag(const ScanArgs* __restrict__ tab,
                                                                  const int* __restrict__ start, int n) {
  const int q = rag_instance(start, n, blockIdx.x);
  const ScanArgs& a = tab[q];
  thomas_scan_body<NC>(a.sub_r, a.lam, a.x, a.fcp, a.finv, a.pl, a.nr, a.nth, a.kstride, a.thr, a.nlowblk, a.low_idx,
                       a.nlow, a.rad64, a.low_fac, (int)blockIdx.x - start[q]);
}

// float32 elimination factors of every (m,l) radial system, computed in float64.
__global__ void k_radial_factors(const RadialRow* __restrict__ rad, const double* __restrict__ lam,
                                 const double* __restrict__ outer, int nr, int nth, int mh, float* __restrict__ fcp,
                                 float* __restrict__ finv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= mh * nth) return;
  const int m = t / nth;
  const int l = t - m * nth;
  const double L = lam[t];
  double cprev = 0.0;
  for (int i = 0; i < nr; ++i) {
    const RadialRow rr = rad[i];
    double b = fma(rr.R, L, rr.base);
    if (i == nr - 1) b += outer[t];
    const double inv = 1.0 / (b - rr.sub * cprev);
    cprev = rr.sup * inv;
    const size_t o = ((size_t)m * nr + i) * nth + l;
    fcp[o] = (float)cprev;
    finv[o] = (float)inv;
  }
}

// Elimination factors (c'_i, 1/pivot_i) of the float64 near-singular modes (set-up).
__global__ void k_low_factors(const RadialRow* __restrict__ rad, const double* __restrict__ lam,
                              const double* __restrict__ outer, const int* __restrict__ low_idx, int nlow, int nr,
                              double2* __restrict__ fac) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nlow) return;
  const int t = low_idx[q];
  const double L = lam[t];
  double cprev = 0.0;
  for (int i = 0; i < nr; ++i) {
    const RadialRow rr = rad[i];
    double b = fma(rr.R, L, rr.base);
    if (i == nr - 1) b += outer[t];
    const double inv = 1.0 / (b - rr.sub * cprev);
    cprev = rr.sup * inv;
    fac[(size_t)q * nr + i] = make_double2(cprev, inv);
  }
}

// Unnormalised float-float helpers for the residual: a value is (h, l) with |l| small
// against |h| but not necessarily below half an ulp; one renormalisation at the end.
__device__ __forceinline__ void ffd_diff(float bh, float bl, float ch, float cl, float& dh, float& dl) {
  float e;
  two_sum(bh, -ch, dh, e);
  dl = e + (bl - cl);
}
__device__ __forceinline__ void ffd_mul(ff k, float dh, float dl, float& p, float& e) {
  p = __fmul_rn(k.hi, dh);
  e = fmaf(k.hi, dh, -p);
  e = fmaf(k.hi, dl, e);
  e = fmaf(k.lo, dh, e);
}
__device__ __forceinline__ void ffd_acc(float& ah, float& al, float ph, float pe) {
  float s, e;
  two_sum(ah, ph, s, e);
  ah = s;
  al += e + pe;
}

// Neighbour difference b - c of float-float values; with LO = false both low words are
// zero and the difference is the error-free two-sum of the high words.
template <bool LO>
__device__ __forceinline__ void ffd_diff_lo(float bh, float bl, float ch, float cl, float& dh, float& dl) {
  if (LO) ffd_diff(bh, bl, ch, cl, dh, dl);
  else two_sum(bh, -ch, dh, dl);
}

// Float pair of a float64 source value: hi is x rounded toward zero to float (x truncated
// to 24 significant bits; one conversion instruction), lo the remaining 29 fraction bits
// rounded to float and scaled by 2^(E-52), E the exponent of x and hi, as two exact powers
// of two taken from hi's exponent field; so |hi + lo - x| <= 2^-24 |lo| < 2^-47 |x| for
// 2^-100 <= |x| < 2^128.  Smaller magnitudes keep hi alone (lo = 0, an error below one
// unit of hi's last place); larger ones lie outside the float range of the low-precision
// solve.
__device__ __forceinline__ ff d2ff_trunc(double x) {
  const float hi = __double2float_rz(x);
  const unsigned int hb = __float_as_uint(hi);
  const unsigned int wlo = (unsigned int)__double_as_longlong(x);
  const float lo = (float)(wlo & 0x1FFFFFFFu) * __uint_as_float((hb & 0xFF800000u) - (26u << 23)) * 0x1p-26f;
  return ff{hi, (hb & 0x7F800000u) >= (27u << 23) ? lo : 0.f};
}

// r = 4 pi G rho - (L Phi) of one zone for the float-float iterate Phi = hi + lo,
// evaluated in float-float arithmetic in difference form (every neighbour difference
// Phi_nb - Phi_c is formed first, so products carry errors relative to the small
// differences, not to |L||Phi|) and returned as float32.  (mh, ml) = Phi(i-1) - Phi(i)
// on entry (read when i > 0) and Phi(i) - Phi(i+1) on exit (when i < Nr-1); (qh, ql) is
// the phi second difference (Phi_k+1 - Phi_k) + (Phi_k-1 - Phi_k); (oh, ol) the outer
// boundary term of the last shell (multipole or Dirichlet), added when i = Nr-1.
template <bool LO>
__device__ __forceinline__ float residual_zone(float ch, float cl, float& mh, float& ml, bool has_im, bool has_ip,
                                               float nh, float nl, bool has_jm, float jmh, float jml, bool has_jp,
                                               float jph, float jpl, float qh, float ql, float oh, float ol,
                                               const RadialRowFF& rr, const ThetaRowFF& ar, double rv,
                                               const ff& four_pi_g) {
  float dh, dl, p, e;
  float sh = 0.f, sl = 0.f;   // L Phi as one unnormalised float-float sum
  if (has_im) {
    ffd_mul(rr.sub, mh, ml, p, e);
    sh = p;
    sl = e;
  }
  if (has_ip) {
    ffd_diff_lo<LO>(nh, nl, ch, cl, dh, dl);
    ffd_mul(rr.sup, dh, dl, p, e);
    ffd_acc(sh, sl, p, e);
    mh = -dh;
    ml = -dl;
  }
  if (has_jm) {
    ffd_diff_lo<LO>(jmh, jml, ch, cl, dh, dl);
    ffd_mul(ar.tm, dh, dl, p, e);
    ffd_acc(sh, sl, p, e);
  }
  if (has_jp) {
    ffd_diff_lo<LO>(jph, jpl, ch, cl, dh, dl);
    ffd_mul(ar.tp, dh, dl, p, e);
    ffd_acc(sh, sl, p, e);
  }
  ffd_mul(ar.sphi, qh, ql, p, e);
  ffd_acc(sh, sl, p, e);
  if (!has_ip) ffd_acc(sh, sl, oh, ol);
  const ff sv = ff_mul(four_pi_g, d2ff_trunc(rv));
  float th_, tl;
  two_sum(sv.hi, -sh, th_, tl);
  tl += sv.lo - sl;
  return th_ + tl;
}

// Outer boundary term of zone (Nr-1, j, k): Dirichlet coefficient x Phi, or the
// precomputed multipole term (float64, already scaled by 3 r_out^2/dV3_N).
__device__ __forceinline__ void outer_term(int dirichlet, const ff& dir_coef, float ch, float cl,
                                           const double* outer_shell, size_t idx, float& oh, float& ol) {
  if (dirichlet) {
    ffd_mul(dir_coef, ch, cl, oh, ol);
  } else {
    const ff o = d2ff(outer_shell[idx]);
    oh = o.hi;
    ol = o.lo;
  }
}

// The residual (LO = false: the iterate of a first solve, lo = 0 and not read), stored as
// float32.  One CTA per (j, chunk of kResRows radial rows, block of phi columns); each
// thread marches outward along its (j, k) column with the radial window in registers, so
// the difference across face i+1/2 serves as the inner difference of row i+1 (negated,
// exactly), and the phi neighbours come from the row's line staged in shared memory.
constexpr int kResRows = 16;
constexpr int kResThreads = 256;

template <bool LO>
__global__ void __launch_bounds__(kResThreads) k_residual_ff(const double* __restrict__ rho,
                                                             const float* __restrict__ ph,
                                                             const float* __restrict__ pl,
                                                             const double* __restrict__ outer_shell,
                                                             float* __restrict__ r,
                                                             const RadialRowFF* __restrict__ rad,
                                                             const ThetaRowFF* __restrict__ ang, int nr, int nth,
                                                             int nphi, int row_begin, int row_end, int dirichlet,
                                                             ff dir_coef, ff four_pi_g) {
  __shared__ float line[2][2][kResThreads + 2];   // [row parity][hi, lo][k - k0 + 1]
  pdl_trigger();
  pdl_wait();
  const int j = blockIdx.x;
  const int i0 = row_begin + (int)blockIdx.y * kResRows, i1 = min(row_end, i0 + kResRows);
  const int t = threadIdx.x;
  const int k0 = blockIdx.z * blockDim.x;
  const int nk = min((int)blockDim.x, nphi - k0);   // columns of this CTA
  const bool act = t < nk;
  const int k = k0 + (act ? t : nk - 1);
  const int kl = k0 == 0 ? nphi - 1 : k0 - 1;       // periodic halo columns
  const int kr = k0 + nk == nphi ? 0 : k0 + nk;
  const size_t shell = (size_t)nth * nphi;
  const bool has_jm = j > 0, has_jp = j < nth - 1;
  // pointers at (i, j, 0) and (i, j, k), stepped one shell per row
  const size_t c0 = (size_t)i0 * shell + (size_t)j * nphi;
  const float* hrow = ph + c0;
  const float* lrow = pl + c0;
  const float* hp = hrow + k;
  const float* lp = lrow + k;
  const double* rp = rho + c0 + k;
  float* op = r + c0 + k;
  const ThetaRowFF* angp = ang + (size_t)i0 * nth + j;
  float ch = hp[0], cl = LO ? lp[0] : 0.f;
  float mh = 0.f, ml = 0.f;   // Phi(i-1) - Phi(i)
  if (i0 > 0) ffd_diff_lo<LO>(hp[-(ptrdiff_t)shell], LO ? lp[-(ptrdiff_t)shell] : 0.f, ch, cl, mh, ml);
  for (int i = i0; i < i1; ++i) {
    float* bh = line[i & 1][0];
    float* bl = line[i & 1][1];
    if (act) {
      bh[t + 1] = ch;
      if (LO) bl[t + 1] = cl;
    }
    if (t == 0) {
      bh[0] = hrow[kl];
      bh[nk + 1] = hrow[kr];
      if (LO) {
        bl[0] = lrow[kl];
        bl[nk + 1] = lrow[kr];
      }
    }
    const bool has_ip = i < nr - 1;
    float nh = 0.f, nl = 0.f, jmh = 0.f, jml = 0.f, jph = 0.f, jpl = 0.f;
    if (has_ip) {
      nh = hp[shell];
      if (LO) nl = lp[shell];
    }
    if (has_jm) {
      jmh = hp[-nphi];
      if (LO) jml = lp[-nphi];
    }
    if (has_jp) {
      jph = hp[nphi];
      if (LO) jpl = lp[nphi];
    }
    const double rv = *rp;
    const RadialRowFF rr = rad[i];
    const ThetaRowFF ar = *angp;   // R_i x (t_j+1/2, t_j-1/2, S_j lambda-free phi coefficient)
    __syncthreads();
    float qh, ql, dh, dl;
    ffd_diff_lo<LO>(bh[t + 2], LO ? bl[t + 2] : 0.f, ch, cl, qh, ql);
    ffd_diff_lo<LO>(bh[t], LO ? bl[t] : 0.f, ch, cl, dh, dl);
    ffd_acc(qh, ql, dh, dl);
    float oh = 0.f, ol = 0.f;
    if (!has_ip) outer_term(dirichlet, dir_coef, ch, cl, outer_shell, (size_t)j * nphi + k, oh, ol);
    const float res = residual_zone<LO>(ch, cl, mh, ml, i > 0, has_ip, nh, nl, has_jm, jmh, jml, has_jp, jph, jpl, qh,
                                        ql, oh, ol, rr, ar, rv, four_pi_g);
    if (act) *op = res;
    ch = nh;
    cl = nl;
    hrow += shell;
    lrow += shell;
    hp += shell;
    lp += shell;
    rp += shell;
    op += shell;
    angp += nth;
  }
}

// The float-float helpers on column pairs: paired float32 instructions (one instruction
// per operation for both columns, each component rounded to nearest as in the scalar
// forms, the operations in the same order).  No operand of a paired instruction is
// negated: a - b is the fused (-1) b + a (one rounding, the same value), and where an
// algorithm needs -x the helpers carry the negated quantity instead (round to nearest is
// symmetric, so every value is exactly that of the form with the negation).
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.f), a); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// two_sum2(a, -b): s = a - b and its exact error
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2& s, float2& e) {
  s = sub2(a, b);
  const float2 bb = sub2(s, a);
  e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
// Neighbour difference b - c of float-float values (LO = false: the error-free
// difference of the high words).  The result is antisymmetric: the difference c - b is
// exactly its negation.
template <bool LO>
__device__ __forceinline__ void ffd_diff2(float2 bh, float2 bl, float2 ch, float2 cl, float2& dh, float2& dl) {
  if (LO) {
    float2 e;
    two_diff2(bh, ch, dh, e);
    dl = add2(e, sub2(bl, cl));
  } else {
    two_diff2(bh, ch, dh, dl);
  }
}
// A float-float coefficient with its negation, each word broadcast to both columns.
struct ffc2 {
  float2 hi, nhi, nlo;
};
__device__ __forceinline__ ffc2 coef2(const ff& k) { return ffc2{f2s(k.hi), f2s(-k.hi), f2s(-k.lo)}; }
// the coefficient -k
__device__ __forceinline__ ffc2 ncoef2(const ff& k) { return ffc2{f2s(-k.hi), f2s(k.hi), f2s(k.lo)}; }
// k (dh + dl) = p + e, returned as p and ne = -e
__device__ __forceinline__ void ffd_mul2(const ffc2& k, float2 dh, float2 dl, float2& p, float2& ne) {
  p = __fmul2_rn(k.hi, dh);
  ne = __ffma2_rn(k.nhi, dh, p);
  ne = __ffma2_rn(k.nhi, dl, ne);
  ne = __ffma2_rn(k.nlo, dh, ne);
}
// Sum (ah, -nal) += (ph, -npe): the low word is carried negated.
__device__ __forceinline__ void ffd_nacc2(float2& ah, float2& nal, float2 ph, float2 npe) {
  float2 s, e;
  two_sum2(ah, ph, s, e);
  ah = s;
  nal = sub2(nal, sub2(e, npe));
}
// (ah, al) += (ph, pe), both low words as they are
__device__ __forceinline__ void ffd_acc2(float2& ah, float2& al, float2 ph, float2 pe) {
  float2 s, e;
  two_sum2(ah, ph, s, e);
  ah = s;
  al = add2(al, add2(e, pe));
}

// 4 pi G rho - (sh - nsl) of both columns, rounded to float32: the float-float source
// term (ff_mul, then fast two-sum), then the difference.
__device__ __forceinline__ float2 residual_finish2(float2 sh, float2 nsl, double2 rv, const ffc2& fpg) {
  const ff rx = d2ff_trunc(rv.x), ry = d2ff_trunc(rv.y);
  const float2 rh = make_float2(rx.hi, ry.hi), rl = make_float2(rx.lo, ry.lo);
  float2 sp, nse;
  ffd_mul2(fpg, rh, rl, sp, nse);
  const float2 svh = sub2(sp, nse);
  const float2 nsvl = add2(nse, sub2(svh, sp));
  float2 th_, tl;
  two_diff2(svh, sh, th_, tl);
  tl = add2(tl, sub2(nsl, nsvl));
  return add2(th_, tl);
}

// residual_zone for the two columns of a pair at once.  (mh, ml) = Phi(i) - Phi(i-1) on
// entry (read when i > 0) and Phi(i+1) - Phi(i) on exit (when i < Nr-1): the radial
// difference is carried with its sign and the inner face's term takes the coefficient
// -sub.
template <bool LO>
__device__ __forceinline__ float2 residual_zone2(float2 ch, float2 cl, float2& mh, float2& ml, bool has_im,
                                                 bool has_ip, float2 nh, float2 nl, bool has_jm, float2 jmh,
                                                 float2 jml, bool has_jp, float2 jph, float2 jpl, float2 qh, float2 ql,
                                                 float2 oh, float2 ol, const RadialRowFF& rr, const ThetaRowFF& ar,
                                                 double2 rv, const ff& four_pi_g) {
  float2 dh, dl, p, ne;
  float2 sh = f2s(0.f), nsl = f2s(0.f);
  if (has_im) {
    ffd_mul2(ncoef2(rr.sub), mh, ml, p, ne);
    sh = p;
    nsl = ne;
  }
  if (has_ip) {
    ffd_diff2<LO>(nh, nl, ch, cl, dh, dl);
    ffd_mul2(coef2(rr.sup), dh, dl, p, ne);
    ffd_nacc2(sh, nsl, p, ne);
    mh = dh;
    ml = dl;
  }
  if (has_jm) {
    ffd_diff2<LO>(jmh, jml, ch, cl, dh, dl);
    ffd_mul2(coef2(ar.tm), dh, dl, p, ne);
    ffd_nacc2(sh, nsl, p, ne);
  }
  if (has_jp) {
    ffd_diff2<LO>(jph, jpl, ch, cl, dh, dl);
    ffd_mul2(coef2(ar.tp), dh, dl, p, ne);
    ffd_nacc2(sh, nsl, p, ne);
  }
  ffd_mul2(coef2(ar.sphi), qh, ql, p, ne);
  ffd_nacc2(sh, nsl, p, ne);
  if (!has_ip) {
    float2 s, e;
    two_sum2(sh, oh, s, e);
    sh = s;
    nsl = sub2(nsl, add2(e, ol));
  }
  return residual_finish2(sh, nsl, rv, coef2(four_pi_g));
}

// The same for an even number of phi zones, two adjacent columns (k, k+1) per thread:
// 8- and 16-byte accesses, the per-row work done once per pair, and the phi face between
// the pair's columns differenced once for both.  rho must be 16-byte aligned.
template <bool LO>
__device__ __forceinline__ void residual_ff2_body(const double* __restrict__ rho, const float* __restrict__ ph,
                                                  const float* __restrict__ pl, const double* __restrict__ outer_shell,
                                                  float* __restrict__ r, const RadialRowFF* __restrict__ rad,
                                                  const ThetaRowFF* __restrict__ ang, int nr, int nth, int nphi,
                                                  int row_begin, int row_end, int dirichlet, ff dir_coef, ff four_pi_g,
                                                  int bx, int by, int bz) {
  // [row parity][hi, lo][even, odd column of the pair][pair - p0 + 1]
  __shared__ float line[2][2][2][kResThreads + 2];
  pdl_trigger();
  pdl_wait();
  const int j = bx;
  const int i0 = row_begin + by * kResRows, i1 = min(row_end, i0 + kResRows);
  const int t = threadIdx.x;
  const int np2 = nphi >> 1;                          // column pairs per line
  const int p0 = bz * blockDim.x;                     // first pair of this CTA
  const int nk = min((int)blockDim.x, np2 - p0);      // pairs of this CTA
  const bool act = t < nk;
  const int k = 2 * (p0 + (act ? t : nk - 1));        // even column of the pair
  const int kl = p0 == 0 ? nphi - 1 : 2 * p0 - 1;     // periodic halo columns (odd, even)
  const int kr = p0 + nk == np2 ? 0 : 2 * (p0 + nk);
  const size_t shell = (size_t)nth * nphi;
  const size_t sh2 = shell >> 1;                      // strides in pairs
  const ptrdiff_t nph2 = np2;
  const bool has_jm = j > 0, has_jp = j < nth - 1;
  const size_t c0 = (size_t)i0 * shell + (size_t)j * nphi;
  const float* hrow = ph + c0;
  const float* lrow = pl + c0;
  const float2* hp = reinterpret_cast<const float2*>(hrow + k);
  const float2* lp = reinterpret_cast<const float2*>(lrow + k);
  const double2* rp = reinterpret_cast<const double2*>(rho + c0 + k);
  float2* op = reinterpret_cast<float2*>(r + c0 + k);
  const ThetaRowFF* angp = ang + (size_t)i0 * nth + j;
  const float2 z2 = make_float2(0.f, 0.f);
  float2 ch = hp[0], cl = LO ? lp[0] : z2;
  float2 m2h = z2, m2l = z2;   // Phi(i) - Phi(i-1) of both columns
  if (i0 > 0) ffd_diff2<LO>(ch, cl, hp[-(ptrdiff_t)sh2], LO ? lp[-(ptrdiff_t)sh2] : z2, m2h, m2l);
  for (int i = i0; i < i1; ++i) {
    float* ev = line[i & 1][0][0];   // high words of the even and odd columns
    float* od = line[i & 1][0][1];
    float* evl = line[i & 1][1][0];
    float* odl = line[i & 1][1][1];
    if (act) {
      ev[t + 1] = ch.x;
      od[t + 1] = ch.y;
      if (LO) {
        evl[t + 1] = cl.x;
        odl[t + 1] = cl.y;
      }
    }
    if (t == 0) {
      od[0] = hrow[kl];
      ev[nk + 1] = hrow[kr];
      if (LO) {
        odl[0] = lrow[kl];
        evl[nk + 1] = lrow[kr];
      }
    }
    const bool has_ip = i < nr - 1;
    float2 nh = z2, nl = z2, jmh = z2, jml = z2, jph = z2, jpl = z2;
    if (has_ip) {
      nh = hp[sh2];
      if (LO) nl = lp[sh2];
    }
    if (has_jm) {
      jmh = hp[-nph2];
      if (LO) jml = lp[-nph2];
    }
    if (has_jp) {
      jph = hp[nph2];
      if (LO) jpl = lp[nph2];
    }
    const double2 rv = *rp;
    const RadialRowFF rr = rad[i];
    const ThetaRowFF ar = *angp;
    __syncthreads();
    // phi second differences: the face between the pair's columns once for both
    float dmh, dml;
    ffd_diff_lo<LO>(ch.y, cl.y, ch.x, cl.x, dmh, dml);   // Phi(k+1) - Phi(k)
    float2 qh, ql;                                       // Phi(k-1) - Phi(k), Phi(k+2) - Phi(k+1)
    ffd_diff2<LO>(make_float2(od[t], ev[t + 2]), LO ? make_float2(odl[t], evl[t + 2]) : z2, ch, cl, qh, ql);
    ffd_acc2(qh, ql, make_float2(dmh, -dmh), make_float2(dml, -dml));
    float2 oh = z2, ol = z2;
    if (!has_ip) {
      outer_term(dirichlet, dir_coef, ch.x, cl.x, outer_shell, (size_t)j * nphi + k, oh.x, ol.x);
      outer_term(dirichlet, dir_coef, ch.y, cl.y, outer_shell, (size_t)j * nphi + k + 1, oh.y, ol.y);
    }
    const float2 res = residual_zone2<LO>(ch, cl, m2h, m2l, i > 0, has_ip, nh, nl, has_jm, jmh, jml, has_jp, jph, jpl,
                                          qh, ql, oh, ol, rr, ar, rv, four_pi_g);
    if (act) *op = res;
    ch = nh;
    cl = nl;
    hrow += shell;
    lrow += shell;
    hp += sh2;
    lp += sh2;
    rp += sh2;
    op += sh2;
    angp += nth;
  }
}

template <bool LO>
__global__ void __launch_bounds__(kResThreads) k_residual_ff2(const double* __restrict__ rho,
                                                              const float* __restrict__ ph,
                                                              const float* __restrict__ pl,
                                                              const double* __restrict__ outer_shell,
                                                              float* __restrict__ r,
                                                              const RadialRowFF* __restrict__ rad,
                                                              const ThetaRowFF* __restrict__ ang, int nr, int nth,
                                                              int nphi, int row_begin, int row_end, int dirichlet,
                                                              ff dir_coef, ff four_pi_g) {
  residual_ff2_body<LO>(rho, ph, pl, outer_shell, r, rad, ang, nr, nth, nphi, row_begin, row_end, dirichlet, dir_coef,
                        four_pi_g, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Ragged form: local CTA b of an instance is (b mod gx, (b / gx) mod gy, b / (gx gy)) of
// its single-plan grid; the block size is the batch's largest, the unused threads of a
// narrower instance idle as in a partial column block.
template <bool LO>
__global__ void __launch_bounds__(kResThreads) k_residual_ff2_rag(const ResArgs* __restrict__ tab,
                                                                  const int* __restrict__ start, int n) {
  const int q = rag_instance(start, n, blockIdx.x);
  const ResArgs& a = tab[q];
  const int b = (int)blockIdx.x - start[q];
  const int bx = b % a.gx, byz = b / a.gx;
  residual_ff2_body<LO>(a.rho, a.ph, a.pl, a.outer_shell, a.r, a.rad, a.ang, a.nr, a.nth, a.nphi, a.row_begin, a.row_end,
                        a.dirichlet, a.dir_coef, a.four_pi_g, bx, byz % a.gy, byz / a.gy);
}

// ---- The residual fused with its forward phi FFT (Nphi = 256, float-float iterate).
//
// residual_zone2 with the theta window carried instead of the radial one: the difference
// Phi(j) - Phi(j-1) comes in (dmh, dml; the Phi(j+1) - Phi(j) of the previous line) and
// the lower polar face's term takes the coefficient -tm; Phi(i-1) comes as values.  The
// terms are summed in the same order with the same operations, so the residual is
// bitwise that of k_residual_ff2.
template <bool LO>
__device__ __forceinline__ float2 residual_zone2j(float2 ch, float2 cl, bool has_im, float2 imh, float2 iml,
                                                  bool has_ip, float2 nh, float2 nl, bool has_jm, float2& dmh,
                                                  float2& dml, bool has_jp, float2 jph, float2 jpl, float2 qh,
                                                  float2 ql, float2 oh, float2 ol, const ffc2& csub,
                                                  const ffc2& csup, const ThetaRowFF& ar, double2 rv,
                                                  const ffc2& fpg) {
  float2 dh, dl, p, ne;
  float2 sh = f2s(0.f), nsl = f2s(0.f);
  if (has_im) {
    ffd_diff2<LO>(ch, cl, imh, iml, dh, dl);   // Phi(i) - Phi(i-1), the term's coefficient -sub
    ffd_mul2(csub, dh, dl, p, ne);
    sh = p;
    nsl = ne;
  }
  if (has_ip) {
    ffd_diff2<LO>(nh, nl, ch, cl, dh, dl);
    ffd_mul2(csup, dh, dl, p, ne);
    ffd_nacc2(sh, nsl, p, ne);
  }
  if (has_jm) {
    ffd_mul2(ncoef2(ar.tm), dmh, dml, p, ne);
    ffd_nacc2(sh, nsl, p, ne);
  }
  if (has_jp) {
    ffd_diff2<LO>(jph, jpl, ch, cl, dh, dl);
    ffd_mul2(coef2(ar.tp), dh, dl, p, ne);
    ffd_nacc2(sh, nsl, p, ne);
    dmh = dh;
    dml = dl;
  }
  ffd_mul2(coef2(ar.sphi), qh, ql, p, ne);
  ffd_nacc2(sh, nsl, p, ne);
  if (!has_ip) {
    float2 s, e;
    two_sum2(sh, oh, s, e);
    sh = s;
    nsl = sub2(nsl, add2(e, ol));
  }
  return residual_finish2(sh, nsl, rv, fpg);
}

// One CTA per (radial row i, block of lpc consecutive j; even lpc <= 32): each half of the
// 256 threads takes lpc/2 consecutive lines of the block, a thread per phi column pair,
// and marches in j with the theta window in registers (Phi(j+1) loaded, Phi(j) and the
// face difference kept; Phi(i-1), Phi(i+1), rho and the (i, j) coefficients loaded per
// line; the line's phi neighbours from a shared-memory copy of it).  The residual lines
// go planar into the in-place radix-16 buffer, then the block's half spectrum (scaled by
// `scale`) to the panel spec[m][i][c][j] with row stride rs.  This drops the float32
// residual's round trip through HBM (write, then the FFT's read: 8 bytes per zone).
// Ntheta even, so every block starts on an even line and pairs the lines as the
// stand-alone transform does: the spectrum is bitwise that of k_residual_ff2 followed by
// k_fft_fwd<float, float>.
constexpr int kRfN = 256;               // Nphi
constexpr int kRfPairs = kRfN / 2;      // column pairs per line = threads per half
template <bool LO>
__global__ void __launch_bounds__(256, 4) k_residual_fft(
    const double* __restrict__ rho, const float* __restrict__ ph, const float* __restrict__ pl,
    const double* __restrict__ outer_shell, const RadialRowFF* __restrict__ rad, const ThetaRowFF* __restrict__ ang,
    int nr, int nth, int row_begin, int lpc, int dirichlet, ff dir_coef, ff four_pi_g,
    const float* __restrict__ twid, float scale, float* __restrict__ spec, int rs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [step parity][half][hi, lo][even, odd column of the pair][pair + 1, with the wrap]
  __shared__ float line[2][2][2][2][kRfPairs + 2];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* buf = tw + kRfN;
  load_twiddles<float>(tw, twid, kRfN);   // plan-constant: before the dependency wait
  pdl_trigger();
  pdl_wait();
  const int ncb = (nth + lpc - 1) / lpc;
  const int i = row_begin + (int)blockIdx.x / ncb;
  const int j0 = ((int)blockIdx.x % ncb) * lpc;
  const int nl = min(lpc, nth - j0);
  const int half = lpc >> 1;
  const int t = threadIdx.x & (kRfPairs - 1);
  const int h = threadIdx.x >> 7;
  const int l0 = h * half;                        // first line of this half in the block
  const int nlh = max(0, min(half, nl - l0));     // lines of this half
  const size_t shell = (size_t)nth * kRfN;
  const size_t sh2 = shell >> 1;                  // strides in pairs
  const bool has_im = i > 0, has_ip = i < nr - 1;
  const float2 z2 = make_float2(0.f, 0.f);
  const RadialRowFF rr = rad[i];
  const ffc2 csub = ncoef2(rr.sub), csup = coef2(rr.sup), fpg = coef2(four_pi_g);
  const int k = 2 * t;                            // even column of the pair
  // pair pointers of line (i, j) at step 0
  int j = j0 + l0;
  size_t c0 = (size_t)i * shell + (size_t)j * kRfN + k;
  const float2* hp = reinterpret_cast<const float2*>(ph + c0);
  const float2* lp = reinterpret_cast<const float2*>(pl + c0);
  float2 ch = z2, cl = z2, dmh = z2, dml = z2;
  if (nlh > 0) {
    ch = hp[0];
    if (LO) cl = lp[0];
    if (j > 0) {
      const float2 bh = hp[-(ptrdiff_t)(kRfN / 2)], bl = LO ? lp[-(ptrdiff_t)(kRfN / 2)] : z2;
      ffd_diff2<LO>(ch, cl, bh, bl, dmh, dml);   // Phi(j) - Phi(j-1)
    }
  }
  for (int st = 0; st < half; ++st) {
    const bool act = st < nlh;
    float* ev = line[st & 1][h][0][0];
    float* od = line[st & 1][h][0][1];
    float* evl = line[st & 1][h][1][0];
    float* odl = line[st & 1][h][1][1];
    if (act) {
      ev[t + 1] = ch.x;
      od[t + 1] = ch.y;
      if (t == kRfPairs - 1) od[0] = ch.y;   // column Nphi-1, left of column 0
      if (t == 0) ev[kRfPairs + 1] = ch.x;   // column 0, right of column Nphi-1
      if (LO) {
        evl[t + 1] = cl.x;
        odl[t + 1] = cl.y;
        if (t == kRfPairs - 1) odl[0] = cl.y;
        if (t == 0) evl[kRfPairs + 1] = cl.x;
      }
    }
    const bool has_jm = j > 0, has_jp = j < nth - 1;
    float2 nh = z2, nl2 = z2, imh = z2, iml = z2, jph = z2, jpl = z2;
    double2 rv = make_double2(0.0, 0.0);
    ThetaRowFF ar{};
    if (act) {
      if (has_ip) {
        nh = hp[sh2];
        if (LO) nl2 = lp[sh2];
      }
      if (has_im) {
        imh = hp[-(ptrdiff_t)sh2];
        if (LO) iml = lp[-(ptrdiff_t)sh2];
      }
      if (has_jp) {
        jph = hp[kRfN / 2];
        if (LO) jpl = lp[kRfN / 2];
      }
      rv = *reinterpret_cast<const double2*>(rho + c0);
      ar = ang[(size_t)i * nth + j];
    }
    // the halves exchange nothing: each waits for its own 4 warps only (barriers 1, 2)
    asm volatile("bar.sync %0, %1;" ::"r"(1 + h), "r"(kRfPairs) : "memory");
    if (act) {
      float dmh_, dml_;
      ffd_diff_lo<LO>(ch.y, cl.y, ch.x, cl.x, dmh_, dml_);   // Phi(k+1) - Phi(k)
      float2 qh, ql;                                          // Phi(k-1) - Phi(k), Phi(k+2) - Phi(k+1)
      ffd_diff2<LO>(make_float2(od[t], ev[t + 2]), LO ? make_float2(odl[t], evl[t + 2]) : z2, ch, cl, qh, ql);
      ffd_acc2(qh, ql, make_float2(dmh_, -dmh_), make_float2(dml_, -dml_));
      float2 oh = z2, ol = z2;
      if (!has_ip) {
        outer_term(dirichlet, dir_coef, ch.x, cl.x, outer_shell, (size_t)j * kRfN + k, oh.x, ol.x);
        outer_term(dirichlet, dir_coef, ch.y, cl.y, outer_shell, (size_t)j * kRfN + k + 1, oh.y, ol.y);
      }
      const float2 res = residual_zone2j<LO>(ch, cl, has_im, imh, iml, has_ip, nh, nl2, has_jm, dmh, dml, has_jp,
                                             jph, jpl, qh, ql, oh, ol, csub, csup, ar, rv, fpg);
      // planar into the transform buffer: line l = l0 + st of pair l / 2
      const int l = l0 + st;
      *reinterpret_cast<float2*>(reinterpret_cast<float*>(buf + (l >> 1) * kPsInplace) + (l & 1) * kRfN + k) = res;
      ch = jph;
      cl = jpl;
      hp += kRfN / 2;
      lp += kRfN / 2;
      c0 += kRfN;
      ++j;
    }
  }
  __syncthreads();
  const int npairs = (nl + 1) / 2;
  if (nl & 1)   // (not with even Ntheta and lpc; kept for the general form)
    for (int q = threadIdx.x; q < kRfN; q += blockDim.x) reinterpret_cast<float*>(buf + (nl >> 1) * kPsInplace)[kRfN + q] = 0.f;
  __syncthreads();
  float2* Z = warp_fft256_inplace<false, true, float>(buf, tw, npairs);
  __syncthreads();
  store_half_spectrum<float>(Z, kPsInplace, nl, i * nth + j0, nth, nr, kRfN, scale, spec, rs);
}

// float64 Phi = hi + lo (pl null: lo = 0)
__device__ __forceinline__ void finish_body(const float* __restrict__ ph, const float* __restrict__ pl,
                                            double* __restrict__ phi, size_t n, int bx, int gx) {
  for (size_t idx = bx * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gx * blockDim.x)
    phi[idx] = ff2d(ff{ph[idx], pl ? pl[idx] : 0.f});
}

__global__ void __launch_bounds__(256) k_finish(const float* __restrict__ ph, const float* __restrict__ pl,
                                                double* __restrict__ phi, size_t n) {
  finish_body(ph, pl, phi, n, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_finish_rag(const FinishArgs* __restrict__ tab, const int* __restrict__ start,
                                                    int n) {
  const int q = rag_instance(start, n, blockIdx.x);
  const FinishArgs& a = tab[q];
  finish_body(a.ph, a.pl, a.phi, a.n, (int)blockIdx.x - start[q], start[q + 1] - start[q]);
}

// float64 iterate -> float-float (hi, lo): the inverse of k_finish up to 2^-48 relative.
__global__ void __launch_bounds__(256) k_split64(const double* __restrict__ phi, float* __restrict__ ph,
                                                 float* __restrict__ pl, size_t n) {
  pdl_wait();
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const ff v = d2ff(phi[idx]);
    ph[idx] = v.hi;
    pl[idx] = v.lo;
  }
}

// The same for 16-byte aligned arrays (pl null or 16-byte aligned), four values per
// thread and step.
__global__ void __launch_bounds__(256) k_finish4(const float4* __restrict__ ph, const float4* __restrict__ pl,
                                                 double2* __restrict__ phi, size_t n4) {
  pdl_wait();
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n4; q += (size_t)gridDim.x * blockDim.x) {
    const float4 h = __ldg(ph + q), l = pl ? __ldg(pl + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    phi[2 * q] = make_double2(ff2d(ff{h.x, l.x}), ff2d(ff{h.y, l.y}));
    phi[2 * q + 1] = make_double2(ff2d(ff{h.z, l.z}), ff2d(ff{h.w, l.w}));
  }
}

}  // namespace

size_t mixed_workspace_bytes(const Plan& p) {
  const MixedTables& x = *p.mixed;
  const size_t zones = (size_t)p.nr * p.nth * p.nphi;
  const size_t rows = (size_t)p.mh * 2 * p.nr;
  return 3 * al256(zones * 4) + al256(rows * x.kstride * 4) + al256(rows * p.nth * 4) +
         al256((size_t)(x.nlow ? x.nlow : 1) * p.nr * 3 * 8) +
         2 * al256((size_t)p.nth * p.nphi * 8) + 2 * al256((size_t)p.mh * 2 * p.nth * 8) + 256;
}

void mixed_bind_workspace(Plan& p, char* c) {
  MixedTables& x = *p.mixed;
  const size_t zones = (size_t)p.nr * p.nth * p.nphi;
  const size_t rows = (size_t)p.mh * 2 * p.nr;
  x.r32 = reinterpret_cast<float*>(c);
  c += al256(zones * 4);
  x.phi_hi = reinterpret_cast<float*>(c);
  c += al256(zones * 4);
  x.phi_lo = reinterpret_cast<float*>(c);
  c += al256(zones * 4);
  x.panel = reinterpret_cast<float*>(c);
  c += al256(rows * x.kstride * 4);
  x.d32 = reinterpret_cast<float*>(c);
  c += al256(rows * p.nth * 4);
  x.low_ws = reinterpret_cast<double*>(c);
  c += al256((size_t)(x.nlow ? x.nlow : 1) * p.nr * 3 * 8);
  x.outer_shell = reinterpret_cast<double*>(c);
  c += al256((size_t)p.nth * p.nphi * 8);
  x.shell_phi = reinterpret_cast<double*>(c);
  c += al256((size_t)p.nth * p.nphi * 8);
  p.shell = reinterpret_cast<double*>(c);
  c += al256((size_t)p.mh * 2 * p.nth * 8);
  p.shell2 = reinterpret_cast<double*>(c);
  c += al256((size_t)p.mh * 2 * p.nth * 8);
  x.red = reinterpret_cast<unsigned int*>(c);
  p.specA = p.specB = nullptr;
}

int mixed_create_tables(Plan& p, cudaStream_t s) {
  MixedTables* x = new (std::nothrow) MixedTables();
  if (!x) return SP_ERR_OOM;
  p.mixed = x;
  const int nth = p.nth, mh = p.mh;
  x->kstride = (nth + 7) / 8 * 8;
  x->np = (p.precision == SP_MIXED_BF16X6) ? 3 : 2;
  const size_t tab = (size_t)mh * nth * x->kstride;
  for (int q = 0; q < x->np; ++q)
    if (cudaMalloc(&x->HtW[q], tab * 2) != cudaSuccess || cudaMalloc(&x->Hm[q], tab * 2) != cudaSuccess)
      return SP_ERR_OOM;
  if (cudaMalloc(&x->radf, sizeof(RadialRowF) * p.nr) != cudaSuccess) return SP_ERR_OOM;
  const size_t fac = (size_t)mh * p.nr * nth;
  if (cudaMalloc(&x->fcp, sizeof(float) * fac) != cudaSuccess || cudaMalloc(&x->finv, sizeof(float) * fac) != cudaSuccess ||
      cudaMalloc(&x->sub_r, sizeof(float) * p.nr) != cudaSuccess)
    return SP_ERR_OOM;
  k_radial_factors<<<(mh * nth + 127) / 128, 128, 0, s>>>(p.d_rad, p.d_lam, p.d_outer, p.nr, nth, mh, x->fcp, x->finv);
  k_split_table<<<1024, 256, 0, s>>>(p.d_HtW, nth, x->kstride, tab, Planes{{x->HtW[0], x->HtW[1], x->HtW[2]}, x->np});
  k_split_table<<<1024, 256, 0, s>>>(p.d_H, nth, x->kstride, tab, Planes{{x->Hm[0], x->Hm[1], x->Hm[2]}, x->np});
  if (cudaGetLastError() != cudaSuccess) return SP_ERR_CUDA;
  std::vector<RadialRow> rad(p.nr);
  std::vector<double> lam((size_t)mh * nth);
  if (cudaMemcpyAsync(rad.data(), p.d_rad, sizeof(RadialRow) * p.nr, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(lam.data(), p.d_lam, sizeof(double) * lam.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SP_ERR_CUDA;
  std::vector<RadialRowF> rf(p.nr);
  for (int i = 0; i < p.nr; ++i) rf[i] = {(float)rad[i].sub, (float)rad[i].sup, (float)rad[i].R, (float)rad[i].base};
  auto split = [](double v) { const float h = (float)v; return ff{h, (float)(v - (double)h)}; };
  std::vector<RadialRowFF> rff(p.nr);
  for (int i = 0; i < p.nr; ++i) rff[i] = {split(rad[i].sub), split(rad[i].sup), split(rad[i].R), ff{0.f, 0.f}};
  std::vector<ThetaRow> thr(p.nth);
  if (cudaMemcpy(thr.data(), p.d_theta, sizeof(ThetaRow) * p.nth, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SP_ERR_CUDA;
  // R_i x angular coefficients of every (i, j), split from their float64 products
  std::vector<ThetaRowFF> thff((size_t)p.nr * p.nth);
  for (int i = 0; i < p.nr; ++i)
    for (int j = 0; j < p.nth; ++j)
      thff[(size_t)i * p.nth + j] = {split(rad[i].R * thr[j].tp), split(rad[i].R * thr[j].tm),
                                     split(rad[i].R * thr[j].sphi), ff{0.f, 0.f}};
  x->four_pi_g = split(4.0 * 3.14159265358979323846264338327950288 * p.G);
  x->dir_coef = split(-p.outer_coef / (p.r_out - p.r_last));
  if (cudaMalloc(&x->radff, sizeof(RadialRowFF) * p.nr) != cudaSuccess ||
      cudaMalloc(&x->thff, sizeof(ThetaRowFF) * thff.size()) != cudaSuccess)
    return SP_ERR_OOM;
  if (cudaMemcpy(x->radff, rff.data(), sizeof(RadialRowFF) * p.nr, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(x->thff, thff.data(), sizeof(ThetaRowFF) * thff.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return SP_ERR_CUDA;
  std::vector<int> low;
  for (size_t t = 0; t < lam.size(); ++t)
    if (std::fabs(lam[t]) < x->low_threshold) low.push_back((int)t);
  x->nlow = (int)low.size();
  if (cudaMalloc(&x->low_idx, sizeof(int) * (low.empty() ? 1 : low.size())) != cudaSuccess) return SP_ERR_OOM;
  if (cudaMemcpy(x->radf, rf.data(), sizeof(RadialRowF) * p.nr, cudaMemcpyHostToDevice) != cudaSuccess) return SP_ERR_CUDA;
  std::vector<float> subr(p.nr);
  for (int i = 0; i < p.nr; ++i) subr[i] = (float)rad[i].sub;
  if (cudaMemcpy(x->sub_r, subr.data(), sizeof(float) * p.nr, cudaMemcpyHostToDevice) != cudaSuccess) return SP_ERR_CUDA;
  if (!low.empty() &&
      cudaMemcpy(x->low_idx, low.data(), sizeof(int) * low.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return SP_ERR_CUDA;
  if (x->nlow) {
    if (cudaMalloc(&x->low_fac, sizeof(double2) * (size_t)x->nlow * p.nr) != cudaSuccess) return SP_ERR_OOM;
    k_low_factors<<<(x->nlow + 63) / 64, 64, 0, s>>>(p.d_rad, p.d_lam, p.d_outer, x->low_idx, x->nlow, p.nr,
                                                     x->low_fac);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return SP_ERR_CUDA;
  }
  bool ok = true;
  for (int q = 0; q < x->np; ++q)
    ok = ok && tc::make_map(reinterpret_cast<CUtensorMap*>(x->map_Af[q]), x->HtW[q], nth, x->kstride, nth, mh, tc::kM) &&
         tc::make_map(reinterpret_cast<CUtensorMap*>(x->map_Ai[q]), x->Hm[q], nth, x->kstride, nth, mh, tc::kM);
  return ok ? SP_OK : SP_ERR_CUDA;
}

void mixed_free_shared(MixedTables& x) {
  for (int q = 0; q < 3; ++q) {
    cudaFree(x.HtW[q]);
    cudaFree(x.Hm[q]);
  }
  cudaFree(x.radf);
  cudaFree(x.fcp);
  cudaFree(x.finv);
  cudaFree(x.sub_r);
  cudaFree(x.low_idx);
  cudaFree(x.low_fac);
  cudaFree(x.radff);
  cudaFree(x.thff);
}

void mixed_clear_workspace(MixedTables& x) {
  x.r32 = nullptr;
  x.phi_hi = x.phi_lo = nullptr;
  x.panel = nullptr;
  x.d32 = nullptr;
  x.low_ws = nullptr;
  x.outer_shell = x.shell_phi = nullptr;
  x.red = nullptr;
}

template <int NP>
cudaError_t tc_project_np(const Plan& p, bool inverse, cudaStream_t s) {
  const MixedTables& x = *p.mixed;
  tc::Maps maps;
  for (int q = 0; q < NP; ++q) std::memcpy(&maps.a[q], inverse ? x.map_Ai[q] : x.map_Af[q], sizeof(CUtensorMap));
  // one CTA per SM, each with an equal share of the (m, column tile) list
  const int tiles = (2 * p.nr + tc::Cfg<NP>::BN - 1) / tc::Cfg<NP>::BN;
  const long long total = (long long)tiles * p.mh;
  const int grid = (int)std::min<long long>(total, p.tune.tc_ctas > 0 ? p.tune.tc_ctas : p.num_sms);
  tc::Params prm{x.d32, x.panel, p.nth, p.nth, x.kstride, 2 * p.nr, (p.nth + tc::kKBlk - 1) / tc::kKBlk, p.mh, p.d_err};
  constexpr uint32_t smem = tc::smem_bytes<NP>();
  cudaError_t e = allow_smem(tc::k_tc_gemm_split<NP>, smem);
  if (e != cudaSuccess) return e;
  e = launch_pdl(tc::k_tc_gemm_split<NP>, dim3(grid), dim3(tc::kThreads), smem, s, maps, prm);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t tc_project(const Plan& p, bool inverse, cudaStream_t s) {
  return p.mixed->np == 3 ? tc_project_np<3>(p, inverse, s) : tc_project_np<2>(p, inverse, s);
}

cudaError_t thomas_mixed(const Plan& p, cudaStream_t s) {
  const MixedTables& x = *p.mixed;
  // both components per CTA while two such CTAs fit on an SM, else one
  int nc = scan_smem_bytes(p.nr, 2) <= 108 * 1024 ? 2 : 1;
  if (p.tune.scan_nc == 1 || (p.tune.scan_nc == 2 && scan_smem_bytes(p.nr, 2) <= 200 * 1024)) nc = p.tune.scan_nc;
  const size_t smem = scan_smem_bytes(p.nr, nc);
  if (smem <= 200 * 1024) {
    const int nblk = (2 / nc) * p.mh * ((p.nth + kScanCols - 1) / kScanCols);
    const int nlowblk = (x.nlow + kScanThreads / 64 - 1) / (kScanThreads / 64);
    auto kern = nc == 2 ? k_thomas_scan<2> : k_thomas_scan<1>;
    cudaError_t e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(kern, dim3(nlowblk + nblk), dim3(kScanThreads), smem, s, (const float*)x.sub_r,
                   (const double*)p.d_lam, (const float*)x.d32, (const float*)x.fcp, (const float*)x.finv, x.panel,
                   p.nr, p.nth, x.kstride, x.low_threshold, nlowblk, (const int*)x.low_idx, x.nlow,
                   (const RadialRow*)p.d_rad, (const double2*)x.low_fac);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  const int nblk = 2 * p.mh * ((p.nth + 31) / 32);
  const int nlowblk = x.nlow;   // one warp per float64 mode
  k_thomas_staged<<<nblk + nlowblk, 32, 0, s>>>(x.sub_r, p.d_lam, x.d32, x.fcp, x.finv,
                                                 x.panel, p.nr, p.nth,
                                                 x.kstride, x.low_threshold, nblk, x.low_idx, x.nlow, p.d_rad,
                                                 x.low_fac, x.low_ws);
  return cudaGetLastError();
}

int create_side_stream(Plan& p) {
  if (!p.mixed || p.outer_bc != SP_OUTER_MULTIPOLE) return SP_OK;
  int lo = 0, hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&p.side, cudaStreamNonBlocking, hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&p.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p.ev_join, cudaEventDisableTiming) != cudaSuccess)
    return SP_ERR_CUDA;
  return SP_OK;
}

cudaError_t residual_ff(Plan& p, const double* rho, cudaStream_t s) {
  const MixedTables& x = *p.mixed;
  const size_t sh = (size_t)p.nth * p.nphi;
  // column pairs per thread when Nphi is even and rho allows 16-byte loads
  const bool pairs = (p.nphi & 1) == 0 && (reinterpret_cast<uintptr_t>(rho) & 15u) == 0;
  const int ncols = pairs ? p.nphi / 2 : p.nphi;
  const int tpb = ncols >= kResThreads ? kResThreads : ((ncols + 31) / 32) * 32;
  auto rows = [&](int r0, int r1, cudaStream_t st) {   // rows [r0, r1)
    const dim3 grid(p.nth, (r1 - r0 + kResRows - 1) / kResRows, (ncols + tpb - 1) / tpb);
    auto kern = pairs ? (x.lo_zero ? k_residual_ff2<false> : k_residual_ff2<true>)
                      : (x.lo_zero ? k_residual_ff<false> : k_residual_ff<true>);
    const cudaError_t e = launch_pdl(kern, grid, dim3(tpb), 0, st, rho, (const float*)x.phi_hi,
                                     (const float*)x.phi_lo, (const double*)x.outer_shell, x.r32,
                                     (const RadialRowFF*)x.radff, (const ThetaRowFF*)x.thff, p.nr, p.nth, p.nphi, r0,
                                     r1, p.outer_bc == SP_OUTER_DIRICHLET ? 1 : 0, x.dir_coef, x.four_pi_g);
    return e != cudaSuccess ? e : cudaGetLastError();
  };
  if (p.outer_bc != SP_OUTER_MULTIPOLE) return timed_span(p, kKResidualRows, s, [&] { return rows(0, p.nr, s); });
  // The multipole term of the last shell (small: Ntheta x Nphi zones, float64 FFTs and
  // per-m operator) and then the last shell's residual run on the high-priority side
  // stream while the interior rows, which do not need the term, run here; the join
  // follows both.
  cudaError_t e;
  if ((e = cudaEventRecord(p.ev_fork, s)) != cudaSuccess || (e = cudaStreamWaitEvent(p.side, p.ev_fork, 0)) != cudaSuccess)
    return e;
  const size_t off = (size_t)(p.nr - 1) * sh;
  k_finish<<<(unsigned)((sh + 255) / 256), 256, 0, p.side>>>(x.phi_hi + off, x.lo_zero ? nullptr : x.phi_lo + off,
                                                              x.shell_phi, sh);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = fft_forward_f64(p, x.shell_phi, 1, 1.0 / p.nphi, p.shell, p.side)) != cudaSuccess) return e;
  if ((e = shell_kappa_f64(p, p.shell, p.shell2, p.side)) != cudaSuccess) return e;
  if ((e = fft_inverse_f64(p, p.shell2, 1, x.outer_shell, false, p.side)) != cudaSuccess) return e;
  if ((e = rows(p.nr - 1, p.nr, p.side)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(p.ev_join, p.side)) != cudaSuccess) return e;
  if (p.nr > 1 && (e = timed_span(p, kKResidualRows, s, [&] { return rows(0, p.nr - 1, s); })) != cudaSuccess)
    return e;
  return cudaStreamWaitEvent(s, p.ev_join, 0);
}

bool residual_fft_supported(const Plan& p, const double* rho) {
  return p.nphi == kRfN && (p.nth & 1) == 0 && (reinterpret_cast<uintptr_t>(rho) & 15u) == 0 && !p.mixed->resid64;
}

// The float-float residual fused with its forward FFT into the panel (see k_residual_fft),
// with the same side-stream shell term as residual_ff: interior rows in blocks of 32
// lines here while the shell chain and then the last shell (in blocks of 4 lines: more
// CTAs for the one row) run on the side stream; the join follows both.
cudaError_t residual_fft(Plan& p, const double* rho, cudaStream_t s) {
  const MixedTables& x = *p.mixed;
  auto kern = x.lo_zero ? k_residual_fft<false> : k_residual_fft<true>;
  auto rows = [&](int r0, int r1, int lpc, cudaStream_t st) {
    const size_t smem = sizeof(float2) * ((size_t)kRfN + (size_t)(lpc / 2) * kPsInplace);
    cudaError_t e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const int ncb = (p.nth + lpc - 1) / lpc;
    e = launch_pdl(kern, dim3((unsigned)((r1 - r0) * ncb)), dim3(256), smem, st, rho, (const float*)x.phi_hi,
                   (const float*)x.phi_lo, (const double*)x.outer_shell, (const RadialRowFF*)x.radff,
                   (const ThetaRowFF*)x.thff, p.nr, p.nth, r0, lpc, p.outer_bc == SP_OUTER_DIRICHLET ? 1 : 0,
                   x.dir_coef, x.four_pi_g, (const float*)p.d_twid32, (float)(1.0 / p.nphi), x.panel, x.kstride);
    return e != cudaSuccess ? e : cudaGetLastError();
  };
  if (p.outer_bc != SP_OUTER_MULTIPOLE) return timed_span(p, kKResidualRows, s, [&] { return rows(0, p.nr, 32, s); });
  cudaError_t e;
  if ((e = cudaEventRecord(p.ev_fork, s)) != cudaSuccess || (e = cudaStreamWaitEvent(p.side, p.ev_fork, 0)) != cudaSuccess)
    return e;
  const size_t sh = (size_t)p.nth * p.nphi;
  const size_t off = (size_t)(p.nr - 1) * sh;
  k_finish<<<(unsigned)((sh + 255) / 256), 256, 0, p.side>>>(x.phi_hi + off, x.lo_zero ? nullptr : x.phi_lo + off,
                                                              x.shell_phi, sh);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = fft_forward_f64(p, x.shell_phi, 1, 1.0 / p.nphi, p.shell, p.side)) != cudaSuccess) return e;
  if ((e = shell_kappa_f64(p, p.shell, p.shell2, p.side)) != cudaSuccess) return e;
  if ((e = fft_inverse_f64(p, p.shell2, 1, x.outer_shell, false, p.side)) != cudaSuccess) return e;
  if ((e = rows(p.nr - 1, p.nr, 4, p.side)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(p.ev_join, p.side)) != cudaSuccess) return e;
  if (p.nr > 1 && (e = timed_span(p, kKResidualRows, s, [&] { return rows(0, p.nr - 1, 32, s); })) != cudaSuccess)
    return e;
  return cudaStreamWaitEvent(s, p.ev_join, 0);
}

// Refinement residual in float64 for a float64 iterate: r = 4 pi G rho - (Delta Phi) with
// the operator of Eq. fin_vol3 (the float64 stencil's arithmetic), stored in float32 as
// the next low-precision right-hand side; the multipole term of the last shell comes
// from outer_shell.
__global__ void __launch_bounds__(256) k_residual_f64(const double* __restrict__ rho, const double* __restrict__ phi,
                                                      const double* __restrict__ outer_shell, float* __restrict__ r,
                                                      const RadialRow* __restrict__ rad,
                                                      const ThetaRow* __restrict__ th, int nr, int nth, int nphi,
                                                      int dirichlet, double dir_coef, double four_pi_g) {
  pdl_wait();
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
    if (i == nr - 1) v += dirichlet ? dir_coef * c : outer_shell[idx - (size_t)(nr - 1) * shell];
    r[idx] = (float)(four_pi_g * rho[idx] - v);
  }
}

cudaError_t residual_f64(const Plan& p, const double* rho, const double* phi, cudaStream_t s) {
  const MixedTables& x = *p.mixed;
  const size_t sh = (size_t)p.nth * p.nphi;
  const size_t n = (size_t)p.nr * sh;
  const bool dir = p.outer_bc == SP_OUTER_DIRICHLET;
  cudaError_t e;
  if (!dir) {
    // the multipole term of the last shell from the float64 iterate itself
    const size_t off = (size_t)(p.nr - 1) * sh;
    if ((e = fft_forward_f64(p, phi + off, 1, 1.0 / p.nphi, p.shell, s)) != cudaSuccess) return e;
    if ((e = shell_kappa_f64(p, p.shell, p.shell2, s)) != cudaSuccess) return e;
    if ((e = fft_inverse_f64(p, p.shell2, 1, x.outer_shell, false, s)) != cudaSuccess) return e;
  }
  size_t blocks = (n + 255) / 256;
  if (blocks > (size_t)p.num_sms * 32) blocks = (size_t)p.num_sms * 32;
  e = launch_pdl(k_residual_f64, dim3((unsigned)blocks), dim3(256), 0, s, rho, phi, (const double*)x.outer_shell, x.r32,
                 (const RadialRow*)p.d_rad, (const ThetaRow*)p.d_theta, p.nr, p.nth, p.nphi, dir ? 1 : 0,
                 dir ? -p.outer_coef / (p.r_out - p.r_last) : 0.0, 4.0 * 3.14159265358979323846264338327950288 * p.G);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t split_iterate(const Plan& p, const double* phi, cudaStream_t s) {
  const MixedTables& x = *p.mixed;
  const size_t n = (size_t)p.nr * p.nth * p.nphi;
  size_t blocks = (n + 255) / 256;
  if (blocks > (size_t)p.num_sms * 16) blocks = (size_t)p.num_sms * 16;
  const cudaError_t e = launch_pdl(k_split64, dim3((unsigned)blocks), dim3(256), 0, s, phi, x.phi_hi, x.phi_lo, n);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t finish_mixed(const Plan& p, double* phi, cudaStream_t s) {
  const MixedTables& x = *p.mixed;
  const size_t n = (size_t)p.nr * p.nth * p.nphi;
  const float* lo = x.lo_zero ? nullptr : x.phi_lo;   // a first solve's iterate: lo = 0, not stored
  const bool aligned = ((reinterpret_cast<uintptr_t>(phi) | reinterpret_cast<uintptr_t>(x.phi_hi) |
                         reinterpret_cast<uintptr_t>(lo)) & 15u) == 0 && (n & 3) == 0;
  if (aligned) {
    size_t blocks = (n / 4 + 255) / 256;
    if (blocks > (size_t)p.num_sms * 8) blocks = (size_t)p.num_sms * 8;
    const cudaError_t e = launch_pdl(k_finish4, dim3((unsigned)blocks), dim3(256), 0, s,
                                     reinterpret_cast<const float4*>(x.phi_hi), reinterpret_cast<const float4*>(lo),
                                     reinterpret_cast<double2*>(phi), n / 4);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  size_t blocks = (n + 255) / 256;
  if (blocks > (size_t)p.num_sms * 16) blocks = (size_t)p.num_sms * 16;
  k_finish<<<(unsigned)blocks, 256, 0, s>>>(x.phi_hi, lo, phi, n);
  return cudaGetLastError();
}

// ---- ragged batches: per-instance descriptions (the single-plan launchers' choices)

// both components per CTA while two fit on an SM (2), one component (1), or 0 when the
// column needs the ring-staged kernel (no ragged form)
int scan_components(const Plan& p) {
  if (scan_smem_bytes(p.nr, 1) > 200 * 1024) return 0;
  if (p.tune.scan_nc == 1 || (p.tune.scan_nc == 2 && scan_smem_bytes(p.nr, 2) <= 200 * 1024)) return p.tune.scan_nc;
  return scan_smem_bytes(p.nr, 2) <= 108 * 1024 ? 2 : 1;
}

void scan_desc(const Plan& p, int nc, ScanArgs& a, int& ctas, size_t& smem) {
  const MixedTables& x = *p.mixed;
  smem = scan_smem_bytes(p.nr, nc);
  const int nblk = (2 / nc) * p.mh * ((p.nth + kScanCols - 1) / kScanCols);
  const int nlowblk = (x.nlow + kScanThreads / 64 - 1) / (kScanThreads / 64);
  a = ScanArgs{x.sub_r, p.d_lam, x.d32, x.fcp, x.finv, x.panel, x.low_idx, p.d_rad, x.low_fac, x.low_threshold,
               p.nr, p.nth, x.kstride, nlowblk, x.nlow};
  ctas = nlowblk + nblk;
}

cudaError_t scan_rag(int nc, const ScanArgs* tab, const int* start, int n, int total, size_t smem, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  auto kern = nc == 2 ? k_thomas_scan_rag<2> : k_thomas_scan_rag<1>;
  cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  e = launch_pdl(kern, dim3(total), dim3(kScanThreads), smem, s, tab, start, n);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// whether the two-column residual serves this plan and source (even Nphi, 16-byte rho)
bool residual_pairs(const Plan& p, const double* rho) {
  return (p.nphi & 1) == 0 && (reinterpret_cast<uintptr_t>(rho) & 15u) == 0;
}

int residual_threads(const Plan& p) {
  const int ncols = p.nphi / 2;
  return ncols >= kResThreads ? kResThreads : ((ncols + 31) / 32) * 32;
}

// tpb: the block size the launch uses (at least residual_threads(p)); column blocks of it
void residual_desc(const Plan& p, const double* rho, int r0, int r1, int tpb, ResArgs& a, int& ctas) {
  const MixedTables& x = *p.mixed;
  const int ncols = p.nphi / 2;
  const int gy = (r1 - r0 + kResRows - 1) / kResRows, gz = (ncols + tpb - 1) / tpb;
  a = ResArgs{rho, x.phi_hi, x.phi_lo, x.outer_shell, x.r32, x.radff, x.thff, x.dir_coef, x.four_pi_g,
              p.nr, p.nth, p.nphi, r0, r1, p.outer_bc == SP_OUTER_DIRICHLET ? 1 : 0, p.nth, gy};
  ctas = r1 > r0 ? p.nth * gy * gz : 0;
}

cudaError_t residual_rag(bool lo_read, const ResArgs* tab, const int* start, int n, int total, int tpb,
                         cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  auto kern = lo_read ? k_residual_ff2_rag<true> : k_residual_ff2_rag<false>;
  const cudaError_t e = launch_pdl(kern, dim3(total), dim3(tpb), 0, s, tab, start, n);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// float64 value of the float-float iterate's last shell (the multipole term's input)
void shell_finish_desc(const Plan& p, FinishArgs& a, int& ctas) {
  const MixedTables& x = *p.mixed;
  const size_t sh = (size_t)p.nth * p.nphi;
  const size_t off = (size_t)(p.nr - 1) * sh;
  a = FinishArgs{x.phi_hi + off, x.lo_zero ? nullptr : x.phi_lo + off, x.shell_phi, sh};
  ctas = (int)((sh + 255) / 256);
}

cudaError_t finish_rag(const FinishArgs* tab, const int* start, int n, int total, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  k_finish_rag<<<total, 256, 0, s>>>(tab, start, n);
  return cudaGetLastError();
}

namespace {
__global__ void __launch_bounds__(256) k_post_words(const unsigned int* __restrict__ src, unsigned int* dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
__global__ void __launch_bounds__(256) k_post_words2(const unsigned int* __restrict__ a, unsigned int* da, int na,
                                                     const unsigned int* __restrict__ b, unsigned int* db, int nb) {
  for (int i = threadIdx.x; i < na; i += blockDim.x) da[i] = a[i];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) db[i] = b[i];
}
}  // namespace

// A few result words of the device into page-locked host memory by the GPU's own stores:
// no copy-engine transfer, so the host's read of a refinement decision does not queue
// behind bulk host copies that other streams have in flight.
cudaError_t post_words(const unsigned int* src, unsigned int* host_dst, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_post_words<<<1, 256, 0, s>>>(src, host_dst, n);
  return cudaGetLastError();
}

// Two such groups of words in one launch.
cudaError_t post_words2(const unsigned int* a, unsigned int* host_a, int na, const unsigned int* b,
                        unsigned int* host_b, int nb, cudaStream_t s) {
  k_post_words2<<<1, 256, 0, s>>>(a, host_a, na, b, host_b, nb);
  return cudaGetLastError();
}

}  // namespace sp
