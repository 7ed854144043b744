// sp_apply_laplacian_noalloc: the finite-volume operator without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// operator: a hydrodynamics step driven by a host framework that owns a fixed memory
// pool and forbids other allocations, or a callback that must not synchronise the
// device (cudaMalloc and cudaFree can).  For them this entry point keeps the only
// scratch the operator needs -- the spectrum of the outermost shell for the multipole
// boundary term -- in a fixed array that is part of the library's device image, so a
// call allocates nothing.
#include <mutex>

#include "sp_internal.h"

namespace {

// Two outer-shell spectra of (Nphi/2+1) x 2 x Ntheta doubles, each 256-byte aligned.
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;   // 4 MiB on every device that loads the library

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (looked up once per device;
// in host code the array's name is only a host-side stand-in, not a device address).
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return SP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SP_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return SP_OK;
}

}  // namespace

extern "C" int sp_apply_laplacian_noalloc(sp_plan* plan, const double* phi, double* out, void* stream) {
  cudaGetLastError();   // an earlier failed call of this thread is not this call's error
  if (!plan || !phi || !out) return SP_ERR_INVALID_ARG;
  sp::Plan& P = *reinterpret_cast<sp::Plan*>(plan);
  const size_t bytes = sizeof(double) * (size_t)P.nr * P.nth * P.nphi;
  const char* a = reinterpret_cast<const char*>(phi);
  const char* b = reinterpret_cast<const char*>(out);
  if (a < b + bytes && b < a + bytes) return SP_ERR_INVALID_ARG;
  const size_t shell = align256(sizeof(double) * (size_t)P.mh * 2 * P.nth);
  if (2 * shell > kNoAllocScratchBytes) return SP_ERR_UNSUPPORTED;

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return SP_ERR_CUDA;
  if (prev != P.device && cudaSetDevice(P.device) != cudaSuccess) return SP_ERR_CUDA;
  void* base = nullptr;
  int st = scratch_address(P.device, &base);
  if (st == SP_OK) {
    double* shell_a = static_cast<double*>(base);
    double* shell_b = reinterpret_cast<double*>(static_cast<char*>(base) + shell);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the same launches as sp_apply_laplacian, counted and timed on the plan
    cudaError_t e = sp::timed_launch(P, sp::kKStencil, s, [&] { return sp::stencil_f64(P, phi, out, s); });
    if (e == cudaSuccess && P.outer_bc == SP_OUTER_MULTIPOLE) {
      // FFT of the last shell, kappa in the eigenbasis, inverse FFT accumulated into out
      const size_t off = (size_t)(P.nr - 1) * P.nth * P.nphi;
      e = sp::timed_launch(P, sp::kKOuter, s, [&] {
        cudaError_t r = sp::fft_forward_f64(P, phi + off, 1, 1.0 / P.nphi, shell_a, s);
        if (r == cudaSuccess) r = sp::shell_kappa_f64(P, shell_a, shell_b, s);
        if (r == cudaSuccess) r = sp::fft_inverse_f64(P, shell_b, 1, out + off, true, s);
        return r;
      });
      P.launches += 2;
    }
    if (e == cudaSuccess && P.inner_bc == SP_INNER_REGULAR) {
      // the regular-interior term of the first shell, through the same scratch (stream order)
      e = sp::timed_launch(P, sp::kKOuter, s, [&] {
        cudaError_t r = sp::fft_forward_f64(P, phi, 1, 1.0 / P.nphi, shell_a, s);
        if (r == cudaSuccess) r = sp::shell_apply_f64(P, P.d_ishell, shell_a, shell_b, s);
        if (r == cudaSuccess) r = sp::fft_inverse_f64(P, shell_b, 1, out, true, s);
        return r;
      });
      P.launches += 2;
    }
    if (e != cudaSuccess) st = SP_ERR_CUDA;
  }
  if (prev != P.device) cudaSetDevice(prev);
  return st;
}
