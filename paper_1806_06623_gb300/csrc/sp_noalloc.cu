// sp_apply_laplacian_noalloc: the finite-volume operator without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// operator: code running inside a captured CUDA graph, a hydrodynamics step driven by
// a host framework that owns a fixed memory pool, or a callback that must not
// synchronise (cudaMalloc/cudaFree can synchronise the device).  For them this entry
// point keeps the only scratch the operator needs -- the spectrum of the outermost
// shell for the multipole boundary term -- in a fixed array that is part of the
// library's device image, so a call allocates nothing.
#include <atomic>
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

// Device address of the scratch array on the current device (set up once per device).
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
  if (!plan || !phi || !out) return SP_ERR_INVALID_ARG;
  const sp::Plan* p = reinterpret_cast<const sp::Plan*>(plan);
  const size_t bytes = sizeof(double) * (size_t)p->nr * p->nth * p->nphi;
  const char* a = reinterpret_cast<const char*>(phi);
  const char* b = reinterpret_cast<const char*>(out);
  if (a < b + bytes && b < a + bytes) return SP_ERR_INVALID_ARG;
  const size_t shell = align256(sizeof(double) * (size_t)p->mh * 2 * p->nth);
  if (2 * shell > kNoAllocScratchBytes) return SP_ERR_UNSUPPORTED;

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return SP_ERR_CUDA;
  if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) return SP_ERR_CUDA;
  void* base = nullptr;
  int st = scratch_address(p->device, &base);
  if (st == SP_OK) {
    // the plan's tables with the outer-shell buffers pointed at the static scratch
    sp::Plan q = *p;
    q.shell = static_cast<double*>(base);
    q.shell2 = reinterpret_cast<double*>(static_cast<char*>(base) + shell);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = sp::stencil_f64(q, phi, out, s);
    if (e == cudaSuccess && q.outer_bc == SP_OUTER_MULTIPOLE) e = sp::outer_term_f64(q, phi, out, s);
    if (e != cudaSuccess) st = SP_ERR_CUDA;
  }
  if (prev != p->device) cudaSetDevice(prev);
  return st;
}
