// Real FFTs along phi (Sect. 3.2: expansion in h_m(k) = exp(2 pi i m k / Nphi)).
//
// One CTA (8 warps) transforms a chunk of up to 32 consecutive phi lines (line
// g = i*Ntheta + j, Nphi contiguous values each).  Two real lines are packed into one
// complex line z = x_A + i x_B; every packed line is owned by one warp, which runs a
// mixed-radix (4, 2, 3, 5) Stockham FFT on it in shared memory with only warp-level
// synchronisation.  Lines are stored at a padded stride of Nphi+1 complex values so
// that lanes addressing consecutive lines hit different banks.  The forward kernel
// separates X_A[m] = (Z[m] + conj Z[N-m])/2, X_B[m] = (Z[m] - conj Z[N-m])/(2i) and
// writes the half spectrum m = 0..Nphi/2 in the layout [m][i][c][j] that the theta
// projection reads (lane = line, so each warp store is a run of consecutive j).  The
// inverse kernel rebuilds the Hermitian spectrum of each line pair with one lane-pair
// shuffle, runs the inverse FFT and writes (or accumulates, or adds into a
// float-float iterate) both real lines.
#include <algorithm>

#include "fft_dev.cuh"

namespace sp {
namespace {

// float64 input to the transform's type; to float by the rounding conversion, one
// instruction on the float64 pipe, which the transform leaves otherwise idle
template <typename T>
__device__ __forceinline__ T load_in(const double* p) { return (T)*p; }
template <typename T>
__device__ __forceinline__ T load_in(const float* p) { return (T)*p; }
template <typename T>
__device__ __forceinline__ T cvt_in(double x) { return (T)x; }
template <typename T>
__device__ __forceinline__ T cvt_in(float x) { return (T)x; }

// 16-byte vector of the input type: V values of one line
template <typename Tin> struct Vec16;
template <> struct Vec16<double> {
  using t = double2;
  static constexpr int V = 2;
  __device__ static double at(const double2& w, int i) { return i ? w.y : w.x; }
};
template <> struct Vec16<float> {
  using t = float4;
  static constexpr int V = 4;
  __device__ static float at(const float4& w, int i) { return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w)); }
};

// Forward: lines [line0, line0+nl) of `in` -> half spectrum scaled by `scale`,
// spec[m][i][c][j] with row stride `rs` (Ntheta, or the padded panel stride).
template <typename T, typename Tin>
__device__ __forceinline__ void fft_fwd_body(const Tin* __restrict__ in, int nlines, int nth, int nrs,
                                             const FftSchedule& sch, const T* __restrict__ twid, T scale, int lpc,
                                             T* __restrict__ spec, int rs, int ahead, int bx, int gx) {
  using CT = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = sch.n;
  const bool inplace = fft_inplace<T>(n);
  const int PS = inplace ? kPsInplace : n + 1;
  const int P = lpc / 2;
  CT* tw = reinterpret_cast<CT*>(smem_raw);
  CT* bufA = tw + n;
  CT* bufB = inplace ? nullptr : bufA + P * PS;
  load_twiddles<T>(tw, twid, n);   // plan-constant: before the dependency wait
  pdl_trigger();
  pdl_wait();
  const int line0 = bx * lpc;
  const int nl = min(lpc, nlines - line0);
  const int npairs = (nl + 1) / 2;
  // the input of the CTA one resident wave ahead goes on its way into L2 now
  if (threadIdx.x == 0 && ahead > 0 && bx + ahead < gx) {
    const int l2 = (bx + ahead) * lpc;
    prefetch_lines_l2(in, l2, min(lpc, nlines - l2), n);
  }
  // The CTA's lines are contiguous in memory: all threads load them together with
  // kLoadU values per thread in flight, then scatter into the packed complex lines.
  const int tot = nl * n;
  const Tin* src = in + (size_t)line0 * n;
  using VT = typename Vec16<Tin>::t;
  constexpr int V = Vec16<Tin>::V;
  if (n % V == 0 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
    // 16-byte loads (V values of one line each), kLoadU values per thread in flight
    constexpr int U = kLoadU / V;
    const VT* vsrc = reinterpret_cast<const VT*>(src);
    const int totv = tot / V;
    for (int e0 = threadIdx.x; e0 < totv; e0 += blockDim.x * U) {
      VT w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * (int)blockDim.x;
        if (e < totv) w[u] = __ldg(vsrc + e);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * (int)blockDim.x;
        if (e < totv) {
          const int ev = e * V;
          const int line = sch.nshift >= 0 ? (ev >> sch.nshift) : (int)__umulhi((unsigned int)ev, sch.nmagic);
          const int q = ev - line * n;
          if (inplace) {
            // planar: V consecutive values of one line in 8-byte stores (the pair stride
            // is even in values); with V = 4 the upper half of each 16 threads stores its
            // second half first, so that a half-warp's 8-byte stores cover all 32 banks
            T* dst = reinterpret_cast<T*>(bufA + (line >> 1) * PS) + (line & 1) * n + q;
            const int i0 = (V == 4 && (threadIdx.x & 8)) ? 2 : 0;
#pragma unroll
            for (int h = 0; h < V; h += 2) {
              const int i = h ^ i0;
              typename C2<T>::t t2;
              t2.x = cvt_in<T>(Vec16<Tin>::at(w[u], i));
              t2.y = cvt_in<T>(Vec16<Tin>::at(w[u], i + 1));
              *reinterpret_cast<typename C2<T>::t*>(dst + i) = t2;
            }
          } else {
            T* dst = reinterpret_cast<T*>(bufA + (line >> 1) * PS + q) + (line & 1);
#pragma unroll
            for (int i = 0; i < V; ++i) dst[2 * i] = cvt_in<T>(Vec16<Tin>::at(w[u], i));
          }
        }
      }
    }
  } else
  for (int e0 = threadIdx.x; e0 < tot; e0 += blockDim.x * kLoadU) {
    T v[kLoadU];
#pragma unroll
    for (int u = 0; u < kLoadU; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      v[u] = e < tot ? load_in<T>(src + e) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kLoadU; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < tot) {
        const int line = sch.nshift >= 0 ? (e >> sch.nshift) : (int)__umulhi((unsigned int)e, sch.nmagic);
        const int q = e - line * n;
        if (inplace) reinterpret_cast<T*>(bufA + (line >> 1) * PS)[(line & 1) * n + q] = v[u];
        else reinterpret_cast<T*>(bufA + (line >> 1) * PS + q)[line & 1] = v[u];
      }
    }
  }
  if (nl & 1)
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      if (inplace) reinterpret_cast<T*>(bufA + (nl >> 1) * PS)[n + q] = T(0);
      else bufA[(nl >> 1) * PS + q].y = T(0);
    }
  __syncthreads();
  // the two-pass radix-16 form keeps a half-warp per line pair: it pays only with every
  // warp busy; few pairs (one shell) take the radix-4 passes with a whole warp per pair
  CT* Z = inplace ? warp_fft256_inplace<false, true, T>(bufA, tw, npairs)
          : (n == 256 && npairs >= 2 * kWarps) ? warp_fft256<false, T>(bufA, bufB, tw, npairs, PS)
                                               : warp_fft<false, T>(bufA, bufB, tw, sch, npairs, PS);
  __syncthreads();
  store_half_spectrum<T>(Z, PS, nl, line0, nth, nrs, n, scale, spec, rs);
}

// max(m, |x|) for m >= 0 that keeps a NaN: non-negative float bit patterns order as
// unsigned integers, every NaN above +inf (a NaN in a correction then reaches the host's
// stopping decision instead of being dropped as fmaxf drops it)
__device__ __forceinline__ float amax(float m, float x) {
  return __uint_as_float(max(__float_as_uint(m), __float_as_uint(fabsf(x))));
}

enum InvOut { kInvWrite = 0, kInvAccumulate = 1, kInvPairUpdate = 2, kInvF64Update = 3, kInvPairToF64 = 4 };
// spectrum rows a warp has in flight in the inverse transform's load (float: 16; double:
// 8, where 16 would spill)
template <typename T>
constexpr int inv_rows() { return sizeof(T) == 4 ? 16 : 8; }

// Inverse: half spectra spec[m][i][c][j] (row stride Ntheta) of lines [line0, line0+nl)
// -> real lines:
//  MODE kInvWrite / kInvAccumulate: out = / += value
//  MODE kInvPairUpdate: float-float iterate (out, phi_lo) = (e, 0) if first (the zero
//    low word is not stored) else (out, phi_lo) + e, phi_lo read only with lo_read (else
//    the stored iterate's low word is zero), with max|e| and max|hi| reduced into red[0], red[1]
//    (non-negative float bit patterns, so integer max orders them); with phi64 given,
//    the updated iterate is also written as float64 (the solve's output when this
//    correction turns out to be the last), and with hilo = 0 only there (out and phi_lo
//    are then left as they were).
//  MODE kInvF64Update: float64 iterate out = e (first) or out + e, with the same two
//    reductions (max|e|, max|out| as float).
//  MODE kInvPairToF64: kInvPairUpdate of an iterate with a zero low word (not first,
//    lo_read = 0) that writes only phi64 (hilo = 0): phi64 = out + e in one float64
//    addition, the value the float-float sum gives, and max|out + e| from the float sum,
//    its high word.
template <typename T, typename Tout, int MODE>
__device__ __forceinline__ void fft_inv_body(const T* __restrict__ spec, int nlines, int nth, int nrs,
                                             const FftSchedule& sch, const T* __restrict__ twid, int lpc,
                                             Tout* __restrict__ out, float* __restrict__ phi_lo, int first,
                                             int lo_read, int hilo, unsigned int* __restrict__ red, int ahead,
                                             double* __restrict__ phi64, int bx, int gx) {
  using CT = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_me[kWarps], s_mp[kWarps];
  const int n = sch.n;
  const bool inplace = fft_inplace<T>(n);
  const int PS = inplace ? kPsInplace : n + 1;
  const int P = lpc / 2;
  CT* tw = reinterpret_cast<CT*>(smem_raw);
  CT* bufA = tw + n;
  CT* bufB = inplace ? nullptr : bufA + P * PS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  load_twiddles<T>(tw, twid, n);   // plan-constant: before the dependency wait
  pdl_trigger();
  const int line0 = bx * lpc;
  const int nl = min(lpc, nlines - line0);
  const int npairs = (nl + 1) / 2;
  const int mh = n / 2 + 1;
  // this CTA's iterate lines (not written by the preceding kernels) head for L2 while the
  // spectra are read and transformed; a prefetch moves no data into the program
  if ((MODE == kInvPairUpdate || MODE == kInvPairToF64) && !first && threadIdx.x == 0) {
    prefetch_lines_l2(out, line0, nl, n);
    if (lo_read) prefetch_lines_l2(phi_lo, line0, nl, n);
  }
  pdl_wait();
  // the iterate lines of the CTA one resident wave ahead go on their way into L2 now
  if ((MODE == kInvPairUpdate || MODE == kInvPairToF64) && !first && threadIdx.x == 0 && ahead > 0 && bx + ahead < gx) {
    const int l2 = (bx + ahead) * lpc;
    prefetch_lines_l2(out, l2, min(lpc, nlines - l2), n);
    if (lo_read) prefetch_lines_l2(phi_lo, l2, min(lpc, nlines - l2), n);
  }
  {
    const int l = lane;
    int i = 0, j = 0;
    if (l < nl) {
      const int g = line0 + l;
      i = g / nth;
      j = g - i * nth;
    }
    // Z[m] = G_A[m] + i G_B[m] (even lane writes), Z[n-m] = conj G_A[m] + i conj G_B[m] (odd lane);
    // inv_rows m-rows are loaded before any is consumed
    constexpr int kRows = inv_rows<T>();
    for (int m0 = warp; m0 < mh; m0 += kRows * kWarps) {
      CT vv[kRows];
#pragma unroll
      for (int u = 0; u < kRows; ++u) {
        const int m = m0 + u * kWarps;
        vv[u].x = T(0);
        vv[u].y = T(0);
        if (l < nl && m < mh) {
          const T* s = spec + ((size_t)(m * nrs + i) * 2) * nth + j;
          vv[u].x = s[0];
          vv[u].y = (m == 0 || 2 * m == n) ? T(0) : s[nth];
        }
      }
#pragma unroll
      for (int u = 0; u < kRows; ++u) {
        const int m = m0 + u * kWarps;
        const CT v = vv[u];
        CT o;
        o.x = __shfl_xor_sync(0xffffffffu, v.x, 1);
        o.y = __shfl_xor_sync(0xffffffffu, v.y, 1);
        if (m < mh && (l >> 1) < npairs) {
          CT* z = bufA + (l >> 1) * PS;
          if (!(l & 1)) {
            CT zm; zm.x = v.x - o.y; zm.y = v.y + o.x;   // A = v, B = o
            z[m] = zm;
          } else if (m != 0 && 2 * m != n) {
            CT zn; zn.x = o.x + v.y; zn.y = v.x - o.y;   // A = o, B = v
            z[n - m] = zn;
          }
        }
      }
    }
  }
  __syncthreads();
  CT* Z = inplace ? warp_fft256_inplace<true, false, T>(bufA, tw, npairs)
          : (n == 256 && npairs >= 2 * kWarps) ? warp_fft256<true, T>(bufA, bufB, tw, npairs, PS)
                                               : warp_fft<true, T>(bufA, bufB, tw, sch, npairs, PS);
  float me = 0.f, mp = 0.f;
  for (int p = warp; p < npairs; p += kWarps) {
    const CT* z = Z + p * PS;
    const bool hasb = 2 * p + 1 < nl;
    const size_t o0 = (size_t)(line0 + 2 * p) * n;
    if (MODE == kInvF64Update) {
      for (int q = lane; q < n; q += 32) {
        const CT v = z[q];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !hasb) continue;
          const size_t o = o0 + (size_t)h * n + q;
          const float e = (float)(h ? v.y : v.x);
          const double nv = first ? (double)e : (double)out[o] + (double)e;
          out[o] = (Tout)nv;
          me = amax(me, e);
          mp = amax(mp, (float)nv);
        }
      }
    } else if (MODE == kInvPairToF64) {
      // each lane owns 4 consecutive points of two segments of both lines: the iterate's
      // high words in 16-byte loads (all four in flight), Phi in 16-byte stores (the
      // launcher checks n and the alignment)
      for (int qb = 4 * lane; qb < n; qb += 256) {
        float4 w[2][2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int sg = 0; sg < 2; ++sg) {
            const int q = qb + 128 * sg;
            w[h][sg] = q < n && (h == 0 || hasb) ? *reinterpret_cast<const float4*>(out + o0 + (size_t)h * n + q)
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
          const int q = qb + 128 * sg;
          if (q >= n) continue;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (h == 1 && !hasb) continue;
            const float oh4[4] = {w[h][sg].x, w[h][sg].y, w[h][sg].z, w[h][sg].w};
            double* d = phi64 + o0 + (size_t)h * n + q;
#pragma unroll
            for (int i = 0; i < 4; i += 2) {
              const CT v0 = z[q + i], v1 = z[q + i + 1];
              const float e0 = (float)(h ? v0.y : v0.x), e1 = (float)(h ? v1.y : v1.x);
              reinterpret_cast<double2*>(d)[i >> 1] =
                  make_double2(f2d_bits(oh4[i]) + f2d_bits(e0), f2d_bits(oh4[i + 1]) + f2d_bits(e1));
              me = amax(amax(me, e0), e1);
              mp = amax(amax(mp, __fadd_rn(oh4[i], e0)), __fadd_rn(oh4[i + 1], e1));
            }
          }
        }
      }
    } else if (MODE != kInvPairUpdate) {
      for (int q = lane; q < n; q += 32) {
        const CT v = z[q];
        if (MODE == kInvWrite) {
          out[o0 + q] = (Tout)v.x;
          if (hasb) out[o0 + n + q] = (Tout)v.y;
        } else {
          out[o0 + q] += (Tout)v.x;
          if (hasb) out[o0 + n + q] += (Tout)v.y;
        }
      }
    } else {
      if ((n & 3) == 0 && (reinterpret_cast<uintptr_t>(phi64) & 15u) == 0) {
        // 16-byte accesses (a float64 output on an 8-byte boundary takes the scalar
        // path): each lane owns 4 consecutive points; two lines x two
        // segments of the iterate in flight per lane
        for (int qb = 4 * lane; qb < n; qb += 256) {
          float4 oh[2][2], ol[2][2];
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int sg = 0; sg < 2; ++sg) {
              const int q = qb + 128 * sg;
              const size_t o = o0 + (size_t)h * n + q;
              const bool ok = q < n && (h == 0 || hasb) && !first;
              oh[h][sg] = ok ? *reinterpret_cast<const float4*>(out + o) : make_float4(0.f, 0.f, 0.f, 0.f);
              ol[h][sg] = ok && lo_read ? *reinterpret_cast<const float4*>(phi_lo + o) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
          for (int sg = 0; sg < 2; ++sg) {
            const int q = qb + 128 * sg;
            if (q >= n) continue;
            CT v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = z[q + i];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              if (h == 1 && !hasb) continue;
              const size_t o = o0 + (size_t)h * n + q;
              const float oh4[4] = {oh[h][sg].x, oh[h][sg].y, oh[h][sg].z, oh[h][sg].w};
              const float ol4[4] = {ol[h][sg].x, ol[h][sg].y, ol[h][sg].z, ol[h][sg].w};
              float nh[4], nl[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const float e = (float)(h ? v[i].y : v[i].x);
                const ff nv = first ? ff{e, 0.f} : ff_add_f(ff{oh4[i], ol4[i]}, e);
                nh[i] = nv.hi;
                nl[i] = nv.lo;
                me = amax(me, e);
                mp = amax(mp, nv.hi);
              }
              if (hilo) {
                *reinterpret_cast<float4*>(out + o) = make_float4(nh[0], nh[1], nh[2], nh[3]);
                if (!first) *reinterpret_cast<float4*>(phi_lo + o) = make_float4(nl[0], nl[1], nl[2], nl[3]);
              }
              if (phi64) {
                reinterpret_cast<double2*>(phi64 + o)[0] = make_double2(ff2d(ff{nh[0], nl[0]}), ff2d(ff{nh[1], nl[1]}));
                reinterpret_cast<double2*>(phi64 + o)[1] = make_double2(ff2d(ff{nh[2], nl[2]}), ff2d(ff{nh[3], nl[3]}));
              }
            }
          }
        }
      } else
      // two lines x four segments of the iterate in flight per lane
      for (int q0 = lane; q0 < n; q0 += 128) {
        float oh[2][4], ol[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int q = q0 + 32 * u;
            const size_t o = o0 + (size_t)h * n + q;
            const bool ok = q < n && (h == 0 || hasb) && !first;
            oh[h][u] = ok ? (float)out[o] : 0.f;
            ol[h][u] = ok && lo_read ? phi_lo[o] : 0.f;
          }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + 32 * u;
          if (q >= n) continue;
          const CT v = z[q];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (h == 1 && !hasb) continue;
            const size_t o = o0 + (size_t)h * n + q;
            const float e = (float)(h ? v.y : v.x);
            const ff nv = first ? ff{e, 0.f} : ff_add_f(ff{oh[h][u], ol[h][u]}, e);
            if (hilo) {
              out[o] = (Tout)nv.hi;
              if (!first) phi_lo[o] = nv.lo;
            }
            if (phi64) phi64[o] = ff2d(nv);
            me = amax(me, e);
            mp = amax(mp, nv.hi);
          }
        }
      }
    }
  }
  if (MODE == kInvPairUpdate || MODE == kInvF64Update || MODE == kInvPairToF64) {
    for (int o = 16; o > 0; o >>= 1) {
      me = amax(me, __shfl_xor_sync(0xffffffffu, me, o));
      mp = amax(mp, __shfl_xor_sync(0xffffffffu, mp, o));
    }
    if (lane == 0) { s_me[warp] = me; s_mp[warp] = mp; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kWarps; ++w) { me = amax(me, s_me[w]); mp = amax(mp, s_mp[w]); }
      atomicMax(red, __float_as_uint(me));
      atomicMax(red + 1, __float_as_uint(mp));
    }
  }
}

template <typename T, typename Tin>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_fft_fwd(const Tin* __restrict__ in, int nlines, int nth, int nrs,
                                                 FftSchedule sch, const T* __restrict__ twid, T scale, int lpc,
                                                 T* __restrict__ spec, int rs, int ahead) {
  fft_fwd_body<T, Tin>(in, nlines, nth, nrs, sch, twid, scale, lpc, spec, rs, ahead, blockIdx.x, gridDim.x);
}

template <typename T, typename Tout, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_fft_inv(const T* __restrict__ spec, int nlines, int nth, int nrs,
                                                 FftSchedule sch, const T* __restrict__ twid, int lpc,
                                                 Tout* __restrict__ out, float* __restrict__ phi_lo, int first,
                                                 int lo_read, int hilo, unsigned int* __restrict__ red, int ahead,
                                                 double* __restrict__ phi64) {
  fft_inv_body<T, Tout, MODE>(spec, nlines, nth, nrs, sch, twid, lpc, out, phi_lo, first, lo_read, hilo, red, ahead,
                              phi64, blockIdx.x, gridDim.x);
}

// ---- ragged batches: one launch over the CTAs of several instances; CTA b belongs to
// the instance q with start[q] <= b < start[q+1] and runs that instance's transform
// as its CTA b - start[q].
template <typename T, typename Tin>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_fft_fwd_rag(const FwdArgs* __restrict__ tab,
                                                     const int* __restrict__ start, int n) {
  const int q = rag_instance(start, n, blockIdx.x);
  const FwdArgs& a = tab[q];
  fft_fwd_body<T, Tin>(static_cast<const Tin*>(a.in), a.nlines, a.nth, a.nrs, a.sch,
                       static_cast<const T*>(a.twid), (T)a.scale, a.lpc, static_cast<T*>(a.spec), a.rs, a.ahead,
                       (int)blockIdx.x - start[q], start[q + 1] - start[q]);
}

template <typename T, typename Tout, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_fft_inv_rag(const InvArgs* __restrict__ tab,
                                                     const int* __restrict__ start, int n) {
  const int q = rag_instance(start, n, blockIdx.x);
  const InvArgs& a = tab[q];
  fft_inv_body<T, Tout, MODE>(static_cast<const T*>(a.spec), a.nlines, a.nth, a.nrs, a.sch,
                              static_cast<const T*>(a.twid), a.lpc, static_cast<Tout*>(a.out), a.phi_lo, a.first,
                              a.lo_read, a.hilo, a.red, a.ahead, a.phi64, (int)blockIdx.x - start[q],
                              start[q + 1] - start[q]);
}

template <typename T>
int lines_per_cta(int n, int nlines) {
  // two padded line buffers within ~100 KB (float) / ~140 KB (double), at most 32 lines;
  // with few lines (one shell), fewer per CTA so that about two CTAs per SM have work
  const size_t budget = sizeof(T) == 4 ? 100000 : 140000;
  const size_t per_pair = 2 * (size_t)(n + 1) * 2 * sizeof(T);
  size_t pairs = budget / per_pair;
  if (pairs > 16) pairs = 16;
  const size_t few = (size_t)nlines / (2 * 2 * 152);
  if (pairs > few) pairs = few;
  if (pairs < 1) pairs = 1;
  return (int)(2 * pairs);
}

template <typename T>
size_t fft_smem(int n, int lpc);
}  // namespace

int panel_lpc(const Plan& p, int nlines) {
  const int dflt = lines_per_cta<float>(p.nphi, nlines);
  // a tuned value is used when it is even and no larger than the default (which the
  // shared-memory budget allows)
  return (p.tune.lpc >= 2 && p.tune.lpc <= dflt && (p.tune.lpc & 1) == 0) ? p.tune.lpc : dflt;
}

namespace {
template <typename T>
size_t fft_smem(int n, int lpc) {
  const size_t P = (size_t)(lpc / 2);
  if (fft_inplace<T>(n)) return sizeof(typename C2<T>::t) * ((size_t)n + P * kPsInplace);
  const size_t psb = n == 256 ? (size_t)kPad256 : (size_t)n + 1;
  return sizeof(typename C2<T>::t) * ((size_t)n + P * (n + 1) + P * psb);
}

template <typename K>
cudaError_t prep(K kern, size_t smem) {
  return allow_smem(kern, smem);
}

// CTAs of `kern` resident on the device at once (one wave), 0 if unknown.
template <typename K>
int resident_ctas(K kern, size_t smem, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kWarps, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * num_sms;
}

}  // namespace

cudaError_t fft_forward_f64(const Plan& p, const double* in, int nrs, double scale, double* spec, cudaStream_t s) {
  const int nlines = nrs * p.nth;
  const int lpc = lines_per_cta<double>(p.nphi, nlines);
  const size_t smem = fft_smem<double>(p.nphi, lpc);
  auto kern = k_fft_fwd<double, double>;
  cudaError_t e = prep(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<(nlines + lpc - 1) / lpc, 32 * kWarps, smem, s>>>(in, nlines, p.nth, nrs, p.sched, p.d_twid, scale, lpc, spec,
                                                           p.nth, 0);
  return cudaGetLastError();
}

cudaError_t fft_inverse_f64(const Plan& p, const double* spec, int nrs, double* out, bool accumulate, cudaStream_t s) {
  const int nlines = nrs * p.nth;
  const int lpc = lines_per_cta<double>(p.nphi, nlines);
  const size_t smem = fft_smem<double>(p.nphi, lpc);
  const int grid = (nlines + lpc - 1) / lpc;
  cudaError_t e;
  if (accumulate) {
    auto kern = k_fft_inv<double, double, kInvAccumulate>;
    if ((e = prep(kern, smem)) != cudaSuccess) return e;
    kern<<<grid, 32 * kWarps, smem, s>>>(spec, nlines, p.nth, nrs, p.sched, p.d_twid, lpc, out, nullptr, 0, 0, 1, nullptr,
                                         0, nullptr);
  } else {
    auto kern = k_fft_inv<double, double, kInvWrite>;
    if ((e = prep(kern, smem)) != cudaSuccess) return e;
    kern<<<grid, 32 * kWarps, smem, s>>>(spec, nlines, p.nth, nrs, p.sched, p.d_twid, lpc, out, nullptr, 0, 0, 1, nullptr,
                                         0, nullptr);
  }
  return cudaGetLastError();
}

// How many CTAs ahead the forward transform prefetches its input: one resident wave, but
// no more than ~16 MB of input in flight towards L2 (a farther prefetch is evicted again
// before its CTA reads it: the float64 source of 144 MB was read as 190 MB with the
// full wave of 608 CTAs ahead, 174 MB at 32 MB ahead, 149 MB at 16 MB).
static int prefetch_ahead(int resident, size_t bytes_per_cta) {
  const size_t cap = (size_t(16) << 20) / (bytes_per_cta ? bytes_per_cta : 1);
  return (int)std::min<size_t>((size_t)resident, cap);
}

cudaError_t fft_forward_panel(const Plan& p, const void* in, bool in_double, float scale, int kstride, float* out,
                              cudaStream_t s) {
  const int nlines = p.nr * p.nth;
  const int lpc = panel_lpc(p, nlines);
  const size_t smem = fft_smem<float>(p.nphi, lpc);
  const int grid = (nlines + lpc - 1) / lpc;
  const size_t cta_bytes = (size_t)lpc * p.nphi * (in_double ? sizeof(double) : sizeof(float));
  cudaError_t e;
  if (in_double) {
    auto kern = k_fft_fwd<float, double>;
    if ((e = prep(kern, smem)) != cudaSuccess) return e;
    e = launch_pdl(kern, dim3(grid), dim3(32 * kWarps), smem, s, static_cast<const double*>(in), nlines, p.nth, p.nr,
                   p.sched, (const float*)p.d_twid32, scale, lpc, out, kstride,
                   prefetch_ahead(resident_ctas(kern, smem, p.num_sms), cta_bytes));
    if (e != cudaSuccess) return e;
  } else {
    auto kern = k_fft_fwd<float, float>;
    if ((e = prep(kern, smem)) != cudaSuccess) return e;
    e = launch_pdl(kern, dim3(grid), dim3(32 * kWarps), smem, s, static_cast<const float*>(in), nlines, p.nth, p.nr,
                   p.sched, (const float*)p.d_twid32, scale, lpc, out, kstride,
                   prefetch_ahead(resident_ctas(kern, smem, p.num_sms), cta_bytes));
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t fft_inverse_update64(const Plan& p, const float* spec, double* phi, bool first, unsigned int* red,
                                 cudaStream_t s) {
  const int nlines = p.nr * p.nth;
  const int lpc = panel_lpc(p, nlines);
  const size_t smem = fft_smem<float>(p.nphi, lpc);
  auto kern = k_fft_inv<float, double, kInvF64Update>;
  cudaError_t e = prep(kern, smem);
  if (e != cudaSuccess) return e;
  e = launch_pdl(kern, dim3((nlines + lpc - 1) / lpc), dim3(32 * kWarps), smem, s, spec, nlines, p.nth, p.nr, p.sched,
                 (const float*)p.d_twid32, lpc, phi, (float*)nullptr, first ? 1 : 0, 0, 1, red, 0, (double*)nullptr);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t fft_inverse_update(const Plan& p, const float* spec, float* phi_hi, float* phi_lo, bool first, bool lo_read,
                               bool f64_only, unsigned int* red, double* phi64, cudaStream_t s) {
  const int nlines = p.nr * p.nth;
  const int lpc = panel_lpc(p, nlines);
  const size_t smem = fft_smem<float>(p.nphi, lpc);
  const bool hilo = !(f64_only && !first && phi64);
  // an iterate with a zero low word that is written only as float64 Phi: the direct
  // float64 update (16-byte accesses)
  const bool direct = !hilo && !lo_read && (p.nphi & 3) == 0 && (reinterpret_cast<uintptr_t>(phi64) & 15u) == 0 &&
                      (reinterpret_cast<uintptr_t>(phi_hi) & 15u) == 0;
  auto kern = direct ? k_fft_inv<float, float, kInvPairToF64> : k_fft_inv<float, float, kInvPairUpdate>;
  cudaError_t e = prep(kern, smem);
  if (e != cudaSuccess) return e;
  // (prefetching the iterate a wave ahead measured slower here: ahead = 0)
  e = launch_pdl(kern, dim3((nlines + lpc - 1) / lpc), dim3(32 * kWarps), smem, s, spec, nlines, p.nth, p.nr, p.sched,
                 (const float*)p.d_twid32, lpc, phi_hi, phi_lo, first ? 1 : 0, lo_read ? 1 : 0, hilo ? 1 : 0, red, 0,
                 first ? nullptr : phi64);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// ---- ragged batches: per-instance descriptions (the single-plan launchers' choices) and
// one launch over all instances
namespace {
template <typename K, typename A>
cudaError_t rag_launch(K kern, const A* tab, const int* start, int n, int total, size_t smem, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  cudaError_t e = prep(kern, smem);
  if (e != cudaSuccess) return e;
  e = launch_pdl(kern, dim3(total), dim3(32 * kWarps), smem, s, tab, start, n);
  return e != cudaSuccess ? e : cudaGetLastError();
}
}  // namespace

void fft_fwd_panel_desc(const Plan& p, const void* in, float scale, int kstride, float* out, FwdArgs& a, int& ctas,
                        size_t& smem) {
  const int nlines = p.nr * p.nth;
  const int lpc = panel_lpc(p, nlines);
  smem = fft_smem<float>(p.nphi, lpc);
  ctas = (nlines + lpc - 1) / lpc;
  a = FwdArgs{p.sched, in, out, p.d_twid32, (double)scale, nlines, p.nth, p.nr, lpc, kstride, 0};
}

void fft_fwd_shell_desc(const Plan& p, const double* in, double* spec, FwdArgs& a, int& ctas, size_t& smem) {
  const int nlines = p.nth;
  const int lpc = lines_per_cta<double>(p.nphi, nlines);
  smem = fft_smem<double>(p.nphi, lpc);
  ctas = (nlines + lpc - 1) / lpc;
  a = FwdArgs{p.sched, in, spec, p.d_twid, 1.0 / p.nphi, nlines, p.nth, 1, lpc, p.nth, 0};
}

void fft_inv_update_desc(const Plan& p, const float* spec, float* phi_hi, float* phi_lo, bool first, bool lo_read,
                         bool f64_only, unsigned int* red, double* phi64, InvArgs& a, int& ctas, size_t& smem) {
  const int nlines = p.nr * p.nth;
  const int lpc = panel_lpc(p, nlines);
  smem = fft_smem<float>(p.nphi, lpc);
  ctas = (nlines + lpc - 1) / lpc;
  a = InvArgs{p.sched, spec, phi_hi, phi_lo, red, first ? nullptr : phi64, p.d_twid32, nlines, p.nth, p.nr, lpc,
              first ? 1 : 0, lo_read ? 1 : 0, (f64_only && !first && phi64) ? 0 : 1, 0};
}

void fft_inv_shell_desc(const Plan& p, const double* spec, double* out, InvArgs& a, int& ctas, size_t& smem) {
  const int nlines = p.nth;
  const int lpc = lines_per_cta<double>(p.nphi, nlines);
  smem = fft_smem<double>(p.nphi, lpc);
  ctas = (nlines + lpc - 1) / lpc;
  a = InvArgs{p.sched, spec, out, nullptr, nullptr, nullptr, p.d_twid, nlines, p.nth, 1, lpc, 0, 0, 1, 0};
}

cudaError_t fft_fwd_rag(int kind, const FwdArgs* tab, const int* start, int n, int total, size_t smem, cudaStream_t s) {
  if (kind == 0) return rag_launch(k_fft_fwd_rag<float, double>, tab, start, n, total, smem, s);
  if (kind == 1) return rag_launch(k_fft_fwd_rag<float, float>, tab, start, n, total, smem, s);
  return rag_launch(k_fft_fwd_rag<double, double>, tab, start, n, total, smem, s);
}

cudaError_t fft_inv_rag(int kind, const InvArgs* tab, const int* start, int n, int total, size_t smem, cudaStream_t s) {
  if (kind == 0) return rag_launch(k_fft_inv_rag<float, float, kInvPairUpdate>, tab, start, n, total, smem, s);
  return rag_launch(k_fft_inv_rag<double, double, kInvWrite>, tab, start, n, total, smem, s);
}

int fft_resident_ctas(const Plan& p, size_t smem) {
  return resident_ctas(k_fft_fwd_rag<float, float>, smem, p.num_sms);
}

}  // namespace sp
