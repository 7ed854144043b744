// Real FFTs along phi (Sect. 3.2: expansion in h_m(k) = exp(2 pi i m k / Nphi)).
//
// One CTA transforms a chunk of consecutive phi lines (line g = i*Ntheta + j, each
// Nphi contiguous doubles).  Two real lines are packed into one complex line
// z = x_A + i x_B, transformed by a mixed-radix (4, 2, 3) Stockham FFT staged in
// shared memory, and separated with X_A[m] = (Z[m] + conj Z[N-m])/2,
// X_B[m] = (Z[m] - conj Z[N-m])/(2i).  The half spectrum m = 0..Nphi/2 is written in
// the spectral layout [m][i][c][j] (c = re/im, j fastest) that the theta projection
// reads as a K-contiguous panel.  The inverse kernel rebuilds the Hermitian spectrum
// of two lines, runs the inverse FFT and writes both real lines.
#include "sp_internal.h"

namespace sp {
namespace {

template <typename T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

template <typename CT>
__device__ __forceinline__ CT cmul(CT a, CT b) {
  CT r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename CT>
__device__ __forceinline__ CT cadd(CT a, CT b) { CT r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename CT>
__device__ __forceinline__ CT csub(CT a, CT b) { CT r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename CT>
__device__ __forceinline__ CT mul_mi(CT a) {
  CT r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// One Stockham stage of radix R over `npairs` independent length-n transforms.
// Butterfly b reads src[b + r n/R], applies twiddles exp(-+2 pi i r k/(Ns R)),
// k = b mod Ns, and writes dst[(b/Ns) Ns R + k + r Ns].
template <bool INV, typename T>
__device__ __forceinline__ void stockham_stage(const typename C2<T>::t* __restrict__ src,
                                               typename C2<T>::t* __restrict__ dst,
                                               const typename C2<T>::t* __restrict__ tw,
                                               int n, int R, int Ns, int npairs) {
  using CT = typename C2<T>::t;
  const int nb = n / R;
  const int stride = n / R;
  const int tstep = n / (Ns * R);
  const int total = npairs * nb;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int p = t / nb;
    const int b = t - p * nb;
    const int k = b % Ns;
    const CT* s = src + p * n;
    CT* d = dst + p * n;
    const int base = (b / Ns) * Ns * R + k;
    if (R == 4) {
      CT v0 = s[b], v1 = s[b + stride], v2 = s[b + 2 * stride], v3 = s[b + 3 * stride];
      if (k != 0) {
        CT w1 = tw[k * tstep], w2 = tw[2 * k * tstep], w3 = tw[3 * k * tstep];
        if (INV) { w1.y = -w1.y; w2.y = -w2.y; w3.y = -w3.y; }
        v1 = cmul(v1, w1); v2 = cmul(v2, w2); v3 = cmul(v3, w3);
      }
      CT a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = mul_mi<INV>(csub(v1, v3));
      d[base] = cadd(a0, a2);
      d[base + Ns] = cadd(a1, a3);
      d[base + 2 * Ns] = csub(a0, a2);
      d[base + 3 * Ns] = csub(a1, a3);
    } else if (R == 2) {
      CT v0 = s[b], v1 = s[b + stride];
      if (k != 0) {
        CT w1 = tw[k * tstep];
        if (INV) w1.y = -w1.y;
        v1 = cmul(v1, w1);
      }
      d[base] = cadd(v0, v1);
      d[base + Ns] = csub(v0, v1);
    } else {  // R == 3
      CT v0 = s[b], v1 = s[b + stride], v2 = s[b + 2 * stride];
      if (k != 0) {
        CT w1 = tw[k * tstep], w2 = tw[2 * k * tstep];
        if (INV) { w1.y = -w1.y; w2.y = -w2.y; }
        v1 = cmul(v1, w1); v2 = cmul(v2, w2);
      }
      const T h = T(0.8660254037844386467637231707529362);  // sin(2 pi/3)
      CT t1 = cadd(v1, v2), t2 = csub(v1, v2);
      CT a; a.x = v0.x - T(0.5) * t1.x; a.y = v0.y - T(0.5) * t1.y;
      CT bb; bb.x = h * t2.x; bb.y = h * t2.y;
      CT jb = mul_mi<INV>(bb);  // -i b forward, +i b inverse
      d[base] = cadd(v0, t1);
      d[base + Ns] = cadd(a, jb);
      d[base + 2 * Ns] = csub(a, jb);
    }
  }
}

template <bool INV, typename T>
__device__ typename C2<T>::t* run_fft(typename C2<T>::t* bufA, typename C2<T>::t* bufB,
                                      const typename C2<T>::t* tw, const FftSchedule& sch, int npairs) {
  using CT = typename C2<T>::t;
  CT* src = bufA;
  CT* dst = bufB;
  int Ns = 1;
  for (int s = 0; s < sch.nstages; ++s) {
    const int R = sch.radix[s];
    stockham_stage<INV, T>(src, dst, tw, sch.n, R, Ns, npairs);
    __syncthreads();
    CT* t = src; src = dst; dst = t;
    Ns *= R;
  }
  return src;
}

template <typename T>
__device__ void load_twiddles(typename C2<T>::t* tw, const T* __restrict__ g, int n) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    tw[t].x = g[2 * t];
    tw[t].y = g[2 * t + 1];
  }
}

// Forward: lines [line0, line0+nl) of `in` -> half spectrum (scaled) in spec.
template <typename T, typename Tin>
__global__ void __launch_bounds__(256) k_fft_forward(const Tin* __restrict__ in, int nlines, int nth, int nrs,
                                                     FftSchedule sch, const T* __restrict__ twid, T scale,
                                                     int lpc, T* __restrict__ spec) {
  using CT = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = sch.n;
  const int P = lpc / 2;
  CT* tw = reinterpret_cast<CT*>(smem_raw);
  CT* bufA = tw + n;
  CT* bufB = bufA + P * (n + 2);
  load_twiddles<T>(tw, twid, n);
  const int line0 = blockIdx.x * lpc;
  const int nl = min(lpc, nlines - line0);
  const int npairs = (nl + 1) / 2;
  const Tin* src = in + (size_t)line0 * n;
  const int tot = nl * n;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e / n;
    const int q = e - l * n;
    T v = T(src[e]);
    CT* z = bufA + (l >> 1) * n + q;
    if (l & 1) z->y = v; else z->x = v;
  }
  if (nl & 1) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) bufA[(nl >> 1) * n + q].y = T(0);
  }
  __syncthreads();
  CT* Z = run_fft<false, T>(bufA, bufB, tw, sch, npairs);
  const int mh = n / 2 + 1;
  const size_t cstride = nth;
  for (int t = threadIdx.x; t < mh * nl; t += blockDim.x) {
    const int m = t / nl;
    const int l = t - m * nl;
    const CT* zp = Z + (l >> 1) * n;
    const CT a = zp[m];
    const CT b = zp[(n - m) % n];
    T re, im;
    if (l & 1) {   // (Z - conj Zc)/(2i)
      re = T(0.5) * (a.y + b.y);
      im = T(-0.5) * (a.x - b.x);
    } else {       // (Z + conj Zc)/2
      re = T(0.5) * (a.x + b.x);
      im = T(0.5) * (a.y - b.y);
    }
    const int g = line0 + l;
    const int i = g / nth;
    const int j = g - i * nth;
    T* o = spec + ((size_t)(m * nrs + i) * 2) * cstride + j;
    o[0] = re * scale;
    o[cstride] = im * scale;
  }
}

// Inverse: half spectra of lines [line0, line0+nl) -> real lines (optionally accumulated).
template <typename T, typename Tout>
__global__ void __launch_bounds__(256) k_fft_inverse(const T* __restrict__ spec, int nlines, int nth, int nrs,
                                                     FftSchedule sch, const T* __restrict__ twid, int lpc,
                                                     Tout* __restrict__ out, int accumulate) {
  using CT = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = sch.n;
  const int P = lpc / 2;
  CT* tw = reinterpret_cast<CT*>(smem_raw);
  CT* bufA = tw + n;
  CT* bufB = bufA + P * (n + 2);
  load_twiddles<T>(tw, twid, n);
  const int line0 = blockIdx.x * lpc;
  const int nl = min(lpc, nlines - line0);
  const int npairs = (nl + 1) / 2;
  const int mh = n / 2 + 1;
  const size_t cstride = nth;
  // half spectra into bufB as HS[m][l] (padded to an even number of lines)
  const int nle = npairs * 2;
  for (int t = threadIdx.x; t < mh * nle; t += blockDim.x) {
    const int m = t / nle;
    const int l = t - m * nle;
    CT v;
    v.x = T(0); v.y = T(0);
    if (l < nl) {
      const int g = line0 + l;
      const int i = g / nth;
      const int j = g - i * nth;
      const T* s = spec + ((size_t)(m * nrs + i) * 2) * cstride + j;
      v.x = s[0];
      v.y = (m == 0 || 2 * m == n) ? T(0) : s[cstride];
    }
    bufB[m * nle + l] = v;
  }
  __syncthreads();
  // Z[m] = G_A[m] + i G_B[m], Z[n-m] = conj G_A[m] + i conj G_B[m]
  for (int t = threadIdx.x; t < mh * npairs; t += blockDim.x) {
    const int m = t / npairs;
    const int p = t - m * npairs;
    const CT A = bufB[m * nle + 2 * p];
    const CT B = bufB[m * nle + 2 * p + 1];
    CT* z = bufA + p * n;
    CT zm; zm.x = A.x - B.y; zm.y = A.y + B.x;
    z[m] = zm;
    if (m != 0 && 2 * m != n) {
      CT zn; zn.x = A.x + B.y; zn.y = B.x - A.y;
      z[n - m] = zn;
    }
  }
  __syncthreads();
  CT* Z = run_fft<true, T>(bufA, bufB, tw, sch, npairs);
  Tout* dst = out + (size_t)line0 * n;
  const int tot = nl * n;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e / n;
    const int q = e - l * n;
    const CT z = Z[(l >> 1) * n + q];
    const T v = (l & 1) ? z.y : z.x;
    if (accumulate) dst[e] += Tout(v); else dst[e] = Tout(v);
  }
}

template <typename T>
int lines_per_cta(int n) {
  // keep two ping-pong buffers near 64 KB
  const int budget = 65536 / (2 * 2 * (int)sizeof(T));  // complex elements per buffer pair
  int lpc = budget / (n + 2) * 2;
  if (lpc > 32) lpc = 32;
  if (lpc < 2) lpc = 2;
  return lpc & ~1;
}

template <typename T>
size_t fft_smem(int n, int lpc) {
  return sizeof(typename C2<T>::t) * ((size_t)n + 2 * (size_t)(lpc / 2) * (n + 2));
}

}  // namespace

cudaError_t fft_forward_f64(const Plan& p, const double* in, int nrs, double scale, double* spec,
                            cudaStream_t s) {
  const int nlines = nrs * p.nth;
  const int lpc = lines_per_cta<double>(p.nphi);
  const size_t smem = fft_smem<double>(p.nphi, lpc);
  auto kern = k_fft_forward<double, double>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (nlines + lpc - 1) / lpc;
  kern<<<grid, 256, smem, s>>>(in, nlines, p.nth, nrs, p.sched, p.d_twid, scale, lpc, spec);
  return cudaGetLastError();
}

cudaError_t fft_inverse_f64(const Plan& p, const double* spec, int nrs, double* out, bool accumulate,
                            cudaStream_t s) {
  const int nlines = nrs * p.nth;
  const int lpc = lines_per_cta<double>(p.nphi);
  const size_t smem = fft_smem<double>(p.nphi, lpc);
  auto kern = k_fft_inverse<double, double>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (nlines + lpc - 1) / lpc;
  kern<<<grid, 256, smem, s>>>(spec, nlines, p.nth, nrs, p.sched, p.d_twid, lpc, out, accumulate ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace sp
