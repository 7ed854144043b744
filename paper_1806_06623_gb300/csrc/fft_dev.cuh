// Device building blocks of the phi FFTs (Sect. 3.2: expansion in exp(2 pi i m k / Nphi)),
// shared by the FFT kernels and by the kernels that transform lines they compute
// themselves (the refinement residual).  Two real lines are packed into one complex
// line; each packed line is transformed by one warp (mixed radix 4, 2, 3, 5) or one
// half-warp (Nphi = 256: two radix-16 passes) in shared memory.
#pragma once

#include "sp_internal.h"

namespace sp {
namespace {

constexpr int kWarps = 8;
constexpr int kLoadU = 16;   // input values in flight per thread in the forward load

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

__device__ __forceinline__ int div_ns(int x, const FftSchedule& sch, int s) {
  return sch.shift[s] >= 0 ? (x >> sch.shift[s]) : (int)__umulhi((unsigned int)x, sch.magic[s]);
}

// One radix-R Stockham butterfly b of a stage on one line: reads src[b + r n/R],
// applies twiddles exp(-+2 pi i r k/(Ns R)), k = b mod Ns, writes dst[(b/Ns) Ns R + k + r Ns].
template <bool INV, typename T>
__device__ __forceinline__ void butterfly(const typename C2<T>::t* __restrict__ s, typename C2<T>::t* __restrict__ d,
                                          const typename C2<T>::t* __restrict__ tw, int n, int R, int Ns, int tstep,
                                          int b, int bq) {
  using CT = typename C2<T>::t;
  const int stride = n / R;
  const int k = b - bq * Ns;
  const int base = bq * Ns * R + k;
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
  } else if (R == 5) {
    CT v0 = s[b], v1 = s[b + stride], v2 = s[b + 2 * stride], v3 = s[b + 3 * stride], v4 = s[b + 4 * stride];
    if (k != 0) {
      CT w1 = tw[k * tstep], w2 = tw[2 * k * tstep], w3 = tw[3 * k * tstep], w4 = tw[4 * k * tstep];
      if (INV) { w1.y = -w1.y; w2.y = -w2.y; w3.y = -w3.y; w4.y = -w4.y; }
      v1 = cmul(v1, w1); v2 = cmul(v2, w2); v3 = cmul(v3, w3); v4 = cmul(v4, w4);
    }
    // X_q = sum_r v_r w^(r q), w = exp(-+2 pi i / 5), from the pairs r and 5-r:
    // X_1, X_4 = a1 -+ i b1 and X_2, X_3 = a2 -+ i b2 (forward signs)
    const T c1 = T(0.30901699437494742410229341718281906);    // cos(2 pi/5)
    const T c2 = T(-0.80901699437494742410229341718281906);   // cos(4 pi/5)
    const T s1 = T(0.95105651629515357211643933337938214);    // sin(2 pi/5)
    const T s2 = T(0.58778525229247312916870595463907277);    // sin(4 pi/5)
    CT t1 = cadd(v1, v4), t2 = cadd(v2, v3), t3 = csub(v1, v4), t4 = csub(v2, v3);
    CT a1, a2, b1, b2;
    a1.x = v0.x + c1 * t1.x + c2 * t2.x; a1.y = v0.y + c1 * t1.y + c2 * t2.y;
    a2.x = v0.x + c2 * t1.x + c1 * t2.x; a2.y = v0.y + c2 * t1.y + c1 * t2.y;
    b1.x = s1 * t3.x + s2 * t4.x; b1.y = s1 * t3.y + s2 * t4.y;
    b2.x = s2 * t3.x - s1 * t4.x; b2.y = s2 * t3.y - s1 * t4.y;
    const CT jb1 = mul_mi<INV>(b1), jb2 = mul_mi<INV>(b2);
    d[base] = cadd(v0, cadd(t1, t2));
    d[base + Ns] = cadd(a1, jb1);
    d[base + 2 * Ns] = cadd(a2, jb2);
    d[base + 3 * Ns] = csub(a2, jb2);
    d[base + 4 * Ns] = csub(a1, jb1);
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

// All stages for the line pairs owned by this warp (p = warp, warp+kWarps, ...).
// Returns the buffer holding the result.
template <bool INV, typename T>
__device__ typename C2<T>::t* warp_fft(typename C2<T>::t* bufA, typename C2<T>::t* bufB,
                                       const typename C2<T>::t* tw, const FftSchedule& sch, int npairs, int PS) {
  using CT = typename C2<T>::t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  CT* src = bufA;
  CT* dst = bufB;
  const int n = sch.n;
  for (int st = 0; st < sch.nstages; ++st) {
    const int R = sch.radix[st];
    const int Ns = sch.ns[st];
    const int tstep = sch.tstep[st];
    const int nb = n / R;
    for (int p = warp; p < npairs; p += kWarps) {
      const CT* s = src + p * PS;
      CT* d = dst + p * PS;
      for (int b = lane; b < nb; b += 32) butterfly<INV, T>(s, d, tw, n, R, Ns, tstep, b, div_ns(b, sch, st));
    }
    __syncwarp();
    CT* t = src; src = dst; dst = t;
  }
  return src;
}

// ---- Nphi = 256: two radix-16 Stockham passes, each butterfly a 4 x 4 DFT in registers.
// Pass 1 (Ns = 1) reads z[b + 16 r] and writes the padded intermediate w[17 b + r];
// pass 2 (Ns = 16) reads w[17 r + b], twiddles by exp(-+2 pi i r b / 256) and writes
// the spectrum z[b + 16 q].  Half a warp per line pair (lane = butterfly b), so a warp
// runs two pairs per pass (pairs w and w + kWarps, as in the generic path, so the owner
// of a pair is the same in every phase); the padding keeps both passes free of bank
// conflicts.
constexpr int kPad256 = 272;   // 16 x 17 intermediate stride per line pair

template <bool INV, typename CT>
__device__ __forceinline__ void dft4(CT& a, CT& b, CT& c, CT& d) {
  const CT y0 = cadd(a, c), y1 = csub(a, c), y2 = cadd(b, d), y3 = mul_mi<INV>(csub(b, d));
  a = cadd(y0, y2);
  b = cadd(y1, y3);
  c = csub(y0, y2);
  d = csub(y1, y3);
}

// In-register 16-point DFT of v[r] (r = 0..15); result X[q] in v[q].
template <bool INV, typename T>
__device__ __forceinline__ void dft16(typename C2<T>::t (&v)[16]) {
  using CT = typename C2<T>::t;
  // 4-point DFTs over r1 for each r2 (r = r2 + 4 r1): u[r2][q1] in v[r2 + 4 q1]
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) dft4<INV>(v[r2], v[r2 + 4], v[r2 + 8], v[r2 + 12]);
  // twiddles exp(-+2 pi i r2 q1 / 16)
  const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), h = T(0.70710678118654752440);
  auto tw = [&](CT& x, T c, T sn) {   // x *= c - i sn (forward) or c + i sn (inverse)
    const T sg = INV ? sn : -sn;
    CT r;
    r.x = x.x * c - x.y * sg;
    r.y = x.x * sg + x.y * c;
    x = r;
  };
  tw(v[5], c1, s1);   // r2 = 1, q1 = 1: w^1
  tw(v[9], h, h);     // r2 = 1, q1 = 2: w^2
  tw(v[13], s1, c1);  // r2 = 1, q1 = 3: w^3
  tw(v[6], h, h);     // r2 = 2, q1 = 1: w^2
  v[10] = mul_mi<INV>(v[10]);   // r2 = 2, q1 = 2: w^4 = -+i
  tw(v[14], -h, h);   // r2 = 2, q1 = 3: w^6
  tw(v[7], s1, c1);   // r2 = 3, q1 = 1: w^3
  tw(v[11], -h, h);   // r2 = 3, q1 = 2: w^6
  tw(v[15], -c1, -s1);   // r2 = 3, q1 = 3: w^9
  // 4-point DFTs over r2 for each q1: X[q1 + 4 q2] lands in v[4 q1 + q2]
#pragma unroll
  for (int q1 = 0; q1 < 4; ++q1) dft4<INV>(v[4 * q1], v[4 * q1 + 1], v[4 * q1 + 2], v[4 * q1 + 3]);
}

template <bool INV, typename T>
__device__ typename C2<T>::t* warp_fft256(typename C2<T>::t* bufA, typename C2<T>::t* bufB,
                                          const typename C2<T>::t* tw, int npairs, int PS) {
  using CT = typename C2<T>::t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = lane & 15;
  CT v[16];
  for (int p0 = warp; p0 < npairs; p0 += 2 * kWarps) {
    const int p = p0 + (lane >> 4) * kWarps;   // pair p stays with warp p mod kWarps
    if (p < npairs) {
      const CT* z = bufA + p * PS;
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = z[b + 16 * r];
      dft16<INV, T>(v);
      CT* w = bufB + p * kPad256;
      // X[q] with q = q1 + 4 q2 is in v[4 q1 + q2]; Stockham pass 1 output index 16 b + q
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) w[17 * b + q1 + 4 * q2] = v[4 * q1 + q2];
    }
  }
  __syncwarp();
  for (int p0 = warp; p0 < npairs; p0 += 2 * kWarps) {
    const int p = p0 + (lane >> 4) * kWarps;   // pair p stays with warp p mod kWarps
    if (p < npairs) {
      const CT* w = bufB + p * kPad256;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        CT x = w[17 * r + b];
        if (r != 0 && b != 0) {
          CT t = tw[r * b];
          if (INV) t.y = -t.y;
          x = cmul(x, t);
        }
        v[r] = x;
      }
      dft16<INV, T>(v);
      CT* z = bufA + p * PS;
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) z[b + 16 * (q1 + 4 * q2)] = v[4 * q1 + q2];
    }
  }
  __syncwarp();
  return bufA;
}

// The same two passes in place (float panels): each half-warp reads its line pair into
// registers before it overwrites the pair's region, so one buffer of kPsInplace entries
// per pair holds the line, the padded intermediate and the spectrum in turn.  The stride
// is odd, so a lane pair per line pair in the load and store phases (stride PS between
// lanes) spreads over the banks too.
constexpr int kPsInplace = 273;

// PLANAR: the pair's region holds the two real lines one after the other (line A in the
// first 256 values, line B in the next 256) rather than as complex values; the first
// pass then reads A and B separately (the half-warps' pairs sit kWarps pairs = 16 banks
// apart, so the 32-bit reads do not conflict).
template <bool INV, bool PLANAR, typename T>
__device__ typename C2<T>::t* warp_fft256_inplace(typename C2<T>::t* buf, const typename C2<T>::t* tw, int npairs) {
  using CT = typename C2<T>::t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = lane & 15;
  CT v[16];
  for (int p0 = warp; p0 < npairs; p0 += 2 * kWarps) {
    const int p = p0 + (lane >> 4) * kWarps;   // pair p stays with warp p mod kWarps
    CT* z = buf + p * kPsInplace;
    if (p < npairs) {
      if (PLANAR) {
        const T* za = reinterpret_cast<const T*>(z);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          v[r].x = za[b + 16 * r];
          v[r].y = za[256 + b + 16 * r];
        }
      } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = z[b + 16 * r];
      }
      dft16<INV, T>(v);
    }
    __syncwarp();   // the half-warp has read its whole pair
    if (p < npairs) {
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) z[17 * b + q1 + 4 * q2] = v[4 * q1 + q2];
    }
  }
  __syncwarp();
  for (int p0 = warp; p0 < npairs; p0 += 2 * kWarps) {
    const int p = p0 + (lane >> 4) * kWarps;
    CT* z = buf + p * kPsInplace;
    if (p < npairs) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        CT x = z[17 * r + b];
        if (r != 0 && b != 0) {
          CT t = tw[r * b];
          if (INV) t.y = -t.y;
          x = cmul(x, t);
        }
        v[r] = x;
      }
      dft16<INV, T>(v);
    }
    __syncwarp();
    if (p < npairs) {
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) z[b + 16 * (q1 + 4 * q2)] = v[4 * q1 + q2];
    }
  }
  __syncwarp();
  return buf;
}

// Float panels of Nphi = 256 run the in-place radix-16 passes.
template <typename T>
__host__ __device__ constexpr bool fft_inplace(int n) { return sizeof(T) == 4 && n == 256; }

// Bulk prefetch of the `lines` contiguous lines starting at `line` into L2 (16-byte
// multiples only; a hint, so nothing happens otherwise).
template <typename Tv>
__device__ __forceinline__ void prefetch_lines_l2(const Tv* base, int line, int lines, int n) {
  const size_t bytes = (size_t)lines * n * sizeof(Tv);
  const size_t off = (size_t)line * n * sizeof(Tv);
  if (lines <= 0 || ((bytes | off | reinterpret_cast<uintptr_t>(base)) & 15u) || bytes >= (1u << 31)) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const char*>(base) + off),
               "r"((unsigned int)bytes)
               : "memory");
}

template <typename T>
__device__ void load_twiddles(typename C2<T>::t* tw, const T* __restrict__ g, int n) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    tw[t].x = g[2 * t];
    tw[t].y = g[2 * t + 1];
  }
}

// Half spectrum of the CTA's nl transformed lines (line pairs in Z at stride PS), lines
// line0 + l = i Ntheta + j: X_A[m] = (Z[m] + conj Z[N-m])/2, X_B[m] = (Z[m] - conj
// Z[N-m])/(2i), times `scale`, written to spec[m][i][c][j] with row stride `rs`; lane l
// owns line l (l < 32), so each warp store is a run of consecutive j.
template <typename T>
__device__ __forceinline__ void store_half_spectrum(const typename C2<T>::t* __restrict__ Z, int PS, int nl,
                                                    int line0, int nth, int nrs, int n, T scale,
                                                    T* __restrict__ spec, int rs) {
  using CT = typename C2<T>::t;
  const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int mh = n / 2 + 1;
  if (l < nl) {
    const int g = line0 + l;
    const int i = g / nth;
    const int j = g - i * nth;
    const CT* zp = Z + (l >> 1) * PS;
    for (int m = warp; m < mh; m += (int)(blockDim.x >> 5)) {
      const CT a = zp[m];
      const CT b = zp[m == 0 ? 0 : n - m];
      T re, im;
      if (l & 1) { re = T(0.5) * (a.y + b.y); im = T(-0.5) * (a.x - b.x); }   // (Z - conj Zc)/(2i)
      else { re = T(0.5) * (a.x + b.x); im = T(0.5) * (a.y - b.y); }          // (Z + conj Zc)/2
      re *= scale;
      im *= scale;
      T* o = spec + ((size_t)(m * nrs + i) * 2) * rs + j;
      o[0] = re;
      o[rs] = im;
    }
  }
}

}  // namespace
}  // namespace sp
