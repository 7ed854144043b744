// Host side of the C ABI: validation, the geometry of Sect. 3.1, the per-plan tables,
// workspace management and the float64 solve sequence of Sect. 3.2.
#include <algorithm>
#include <cmath>
#include <limits>
#include <cstdio>
#include <mutex>
#include <unordered_map>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "sp_internal.h"

using sp::Plan;

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else if (prev == dev) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

#define SP_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      return e_ == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA; \
    }                                                  \
  } while (0)

bool make_schedule(int n, sp::FftSchedule* s, int order = 0) {
  s->n = n;
  s->nstages = 0;
  int r = n;
  while (r % 4 == 0) { if (s->nstages >= sp::kMaxStages) return false; s->radix[s->nstages++] = 4; r /= 4; }
  while (r % 2 == 0) { if (s->nstages >= sp::kMaxStages) return false; s->radix[s->nstages++] = 2; r /= 2; }
  while (r % 3 == 0) { if (s->nstages >= sp::kMaxStages) return false; s->radix[s->nstages++] = 3; r /= 3; }
  while (r % 5 == 0) { if (s->nstages >= sp::kMaxStages) return false; s->radix[s->nstages++] = 5; r /= 5; }
  if (r != 1) return false;
  if (order == 1) std::reverse(s->radix, s->radix + s->nstages);
  int ns = 1;
  for (int st = 0; st < s->nstages; ++st) {
    s->ns[st] = ns;
    s->tstep[st] = n / (ns * s->radix[st]);
    int sh = -1;
    for (int b = 0; b < 31; ++b)
      if ((1 << b) == ns) sh = b;
    s->shift[st] = sh;
    s->magic[st] = (unsigned int)((1ull << 32) / (unsigned long long)ns + 1ull);
    ns *= s->radix[st];
  }
  s->nshift = -1;
  for (int b = 0; b < 31; ++b)
    if ((1 << b) == n) s->nshift = b;
  s->nmagic = s->nshift >= 0 ? 0u : (unsigned int)(((1ull << 32) + (unsigned long long)n - 1ull) / (unsigned long long)n);
  return true;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

namespace sp {
bool make_fft_schedule(int n, int order, FftSchedule* s) { return make_schedule(n, s, order); }
}  // namespace sp

namespace {

template <typename T>
int upload(T** dst, const T* src, size_t n) {
  SP_CUDA(cudaMalloc(reinterpret_cast<void**>(dst), sizeof(T) * (n ? n : 1)));
  if (n) SP_CUDA(cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice));
  return SP_OK;
}

// Release what the plan owns; the shared tables go with the last plan using them.
void free_pipe(Plan* p) {
  if (!p->pipe) return;
  Plan::HostPipe& q = *p->pipe;
  for (int b = 0; b < 2; ++b) {
    cudaFree(q.rho[b]);
    cudaFree(q.phi[b]);
    if (q.in[b]) cudaEventDestroy(q.in[b]);
    if (q.solved[b]) cudaEventDestroy(q.solved[b]);
    if (q.out[b]) cudaEventDestroy(q.out[b]);
  }
  if (q.join) cudaEventDestroy(q.join);
  if (q.h2d) cudaStreamDestroy(q.h2d);
  if (q.d2h) cudaStreamDestroy(q.d2h);
  delete p->pipe;
  p->pipe = nullptr;
}

void free_tables(Plan* p) {
  const bool last = !p->table_refs || p->table_refs->fetch_sub(1) == 1;
  if (last) {
    cudaFree(p->d_rad);
    cudaFree(p->d_theta);
    cudaFree(p->d_twid);
    cudaFree(p->d_twid32);
    cudaFree(p->d_tdiag);
    cudaFree(p->d_toff);
    cudaFree(p->d_sqw);
    cudaFree(p->d_lam);
    cudaFree(p->d_kappa);
    cudaFree(p->d_outer);
    cudaFree(p->d_inner);
    cudaFree(p->d_tinv);
    cudaFree(p->d_tcp);
    cudaFree(p->d_ishell);
    cudaFree(p->d_HtW);
    cudaFree(p->d_H);
    cudaFree(p->d_HtWp);
    cudaFree(p->d_Hp);
    cudaFree(p->d_oshell);
    cudaFree(p->d_face_r);
    cudaFree(p->d_face_t);
    if (p->mixed) sp::mixed_free_shared(*p->mixed);
    delete p->table_refs;
  }
  delete p->mixed;
  p->mixed = nullptr;
  cudaFree(p->d_err);
  cudaFree(p->d_rho_io);
  cudaFree(p->d_phi_io);
  free_pipe(p);
  if (p->h_red) cudaFreeHost(p->h_red);
  if (p->ws_owned) cudaFree(p->ws);
  for (int i = 0; i < 2 * sp::kMaxTimedLaunches; ++i)
    if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  sp::drop_phase_graph(*p);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->side) cudaStreamDestroy(p->side);
}

bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bytes && y < x + bytes;
}

int ensure_workspace(Plan* p) {
  if (p->ws) return SP_OK;
  const size_t b = sp::workspace_bytes(*p);
  void* w = nullptr;
  SP_CUDA(cudaMalloc(&w, b));
  p->ws = w;
  p->ws_bytes = b;
  p->ws_owned = true;
  sp::bind_workspace(*p, w);
  return SP_OK;
}

int launch_status(cudaError_t e) {
  if (e == cudaSuccess) return SP_OK;
  return e == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA;
}

int solve_fp64(Plan* p, const double* rho, double* phi, cudaStream_t s) {
  const int nth = p->nth, nr = p->nr, mh = p->mh;
  Plan& P = *p;
  int st;
  // (1) s_tilde = FFT_phi(4 pi G rho)/Nphi
  if ((st = launch_status(sp::timed_launch(P, sp::kKFftFwd, s, [&] {
         return sp::fft_forward_f64(P, rho, nr, 4.0 * kPi * P.G / P.nphi, P.specA, s); }))))
    return st;
  // (2) s_hat = (H^T W)_m s_tilde (parity grids: two half-size products on the folded spectrum)
  if ((st = launch_status(sp::timed_launch(P, sp::kKGemmFwd, s, [&] {
         return P.parity ? sp::gemm_parity_f64(P.d_HtWp, P.specA, P.specB, mh, nth / 2, 2 * nr, false, s)
                         : sp::gemm_nt_f64(P.d_HtW, P.specA, P.specB, mh, nth, 2 * nr, nth, s); }))))
    return st;
  // (3) radial solves per (l,m)
  if ((st = launch_status(sp::timed_launch(P, sp::kKThomas, s, [&] { return sp::thomas_f64(P, P.specB, s); }))))
    return st;
  // (4) g = H_m f (parity grids: two half-size products, then g(j), g(Ntheta-1-j) = g_even +- g_odd)
  if ((st = launch_status(sp::timed_launch(P, sp::kKGemmInv, s, [&] {
         return P.parity ? sp::gemm_parity_f64(P.d_Hp, P.specB, P.specA, mh, nth / 2, 2 * nr, true, s)
                         : sp::gemm_nt_f64(P.d_H, P.specB, P.specA, mh, nth, 2 * nr, nth, s); }))))
    return st;
  // (5) Phi = inverse FFT
  return launch_status(sp::timed_launch(P, sp::kKFftInv, s, [&] {
    return sp::fft_inverse_f64(P, P.specA, nr, phi, false, s); }));
}

// One low-precision separated solve of L e = (scale*Nphi) * input: FFT (float32, bf16
// split), tcgen05 projection, float32/float64 radial solves, tcgen05 back projection,
// inverse FFT with Phi (+)= e and the max|e|, max|Phi| reductions.
// in == nullptr: the panel already holds the right-hand side's spectrum.
int lp_solve(Plan* p, const void* in, bool in_double, float scale, double* phi, bool first, cudaStream_t s) {
  Plan& P = *p;
  sp::MixedTables& x = *P.mixed;
  int st;
  if (in && (st = launch_status(sp::timed_launch(P, sp::kKFftFwd, s, [&] {
                return sp::fft_forward_panel(P, in, in_double, scale, x.kstride, x.panel, s); }))))
    return st;
  if ((st = launch_status(sp::timed_launch(P, sp::kKGemmFwd, s, [&] { return sp::tc_project(P, false, s); }))))
    return st;
  if ((st = launch_status(sp::timed_launch(P, sp::kKThomas, s, [&] { return sp::thomas_mixed(P, s); })))) return st;
  if ((st = launch_status(sp::timed_launch(P, sp::kKGemmInv, s, [&] { return sp::tc_project(P, true, s); }))))
    return st;
  if (x.resid64) {
    // float64 iterate in the caller's output: phi = e (first) or phi + e
    st = launch_status(sp::timed_launch(P, sp::kKFftInv, s, [&] {
      return sp::fft_inverse_update64(P, x.d32, phi, first, x.red, s); }));
    x.lo_zero = false;
    x.iter64 = nullptr;
    return st;
  }
  const bool lo_read = !first && !x.lo_zero;
  const bool f64_only = !first && phi && x.lo_zero && sp::first_correction_f64_only(P);
  st = launch_status(sp::timed_launch(P, sp::kKFftInv, s, [&] {
    return sp::fft_inverse_update(P, x.d32, x.phi_hi, x.phi_lo, first, lo_read, f64_only, x.red, phi, s); }));
  x.lo_zero = first;
  x.iter64 = f64_only ? phi : nullptr;
  return st;
}

}  // namespace

namespace sp {

// First low-precision solve of L Phi = 4 pi G rho (asynchronous); with a float64 iterate
// its result goes straight to phi.
int mixed_start(Plan* p, const double* rho, double* phi, cudaStream_t s) {
  p->phi64_written = nullptr;
  SP_CUDA(cudaMemsetAsync(p->mixed->red, 0, 2 * sizeof(unsigned int), s));
  const bool r64 = p->mixed->resid64;
  const int st = lp_solve(p, rho, true, (float)(4.0 * kPi * p->G / p->nphi), r64 ? phi : nullptr, true, s);
  if (st == SP_OK && r64) p->phi64_written = phi;
  return st;
}

// Precision floor of the refinement (see decide_one).  Float-float iterate and residual:
// 8 x 2^-48 x (Nphi / 2 pi)^2.  Float64 iterate and residual: 2^-40, flat (measured fixed
// points 1.2e-14 .. 3.2e-14 for Nphi = 256 .. 4096 at Nr x Ntheta = 4x8, 16x64, 40x32,
// the level of the float64 separated solve itself).
double mixed_floor(const Plan& p, bool resid64) {
  if (resid64) return 9.094947017729282e-13;
  const double kq = p.nphi / (2.0 * kPi);
  return 8.0 * 3.552713678800501e-15 * kq * kq;
}

// Whether the first correction stores the updated iterate only as the float64 output:
// with 6 products it is normally the last one, so the float-float words it would write
// are rebuilt from float64 (split_iterate) only when another correction follows.
bool first_correction_f64_only(const Plan& p) { return p.mixed->np == 3; }

// One correction: float-float residual, then the low-precision solve of L e = r
// (asynchronous); its inverse FFT also writes the updated iterate to phi in float64.
int mixed_correct(Plan* p, const double* rho, double* phi, cudaStream_t s) {
  Plan& P = *p;
  int st;
  if (P.mixed->resid64) {
    // float64 residual of the float64 iterate held in phi (shell term first on this stream)
    if ((st = launch_status(timed_launch(P, kKResidual, s, [&] { return residual_f64(P, rho, phi, s); })))) return st;
    if (P.outer_bc == SP_OUTER_MULTIPOLE) P.launches += 3;   // shell FFT, apply, inverse FFT
    SP_CUDA(cudaMemsetAsync(P.mixed->red, 0, 2 * sizeof(unsigned int), s));
    st = lp_solve(p, P.mixed->r32, false, (float)(1.0 / P.nphi), phi, false, s);
    if (st == SP_OK) P.phi64_written = phi;
    return st;
  }
  if (P.mixed->iter64) {   // the iterate lives in float64 only: rebuild its float-float words
    if ((st = launch_status(timed_launch(P, kKUpdate, s, [&] { return split_iterate(P, P.mixed->iter64, s); }))))
      return st;
    P.mixed->iter64 = nullptr;
  }
  // the residual and its forward FFT in one kernel where supported (the spectrum goes
  // straight to the panel), else the residual to r32 and the transform in lp_solve
  const bool fused = residual_fft_supported(P, rho);
  if ((st = launch_status(timed_launch(P, kKResidual, s, [&] {
         return fused ? residual_fft(P, rho, s) : residual_ff(P, rho, s); }))))
    return st;
  if (P.outer_bc == SP_OUTER_MULTIPOLE) P.launches += 5;   // shell: finish, FFT, apply, inverse FFT; split residual
  SP_CUDA(cudaMemsetAsync(P.mixed->red, 0, 2 * sizeof(unsigned int), s));
  st = lp_solve(p, fused ? nullptr : P.mixed->r32, false, (float)(1.0 / P.nphi), phi, false, s);
  if (st == SP_OK) P.phi64_written = phi;
  return st;
}

// Queue the copy of the reductions of the last low-precision solve to the next of two
// pinned host slots.
int mixed_issue_read(Plan* p, cudaStream_t s, MixedRun& R) {
  SP_CUDA(post_words(p->mixed->red, p->h_red_dev + 2 * R.next_slot, 2, s));
  ++p->launches;
  R.next_slot ^= 1;
  ++R.pending;
  return SP_OK;
}

namespace {

// Phase A ends with the copy of the device status word too (with the correction's
// reductions, one launch), so that a solve which stops after it (the usual case) returns
// without another kernel or synchronisation.  The first solve's reductions are copied on
// the side stream beside the correction's residual when the residual's multipole chain
// joins that stream back before the reductions are cleared (float-float residual); else
// here.
int phase_a_direct(Plan* p, const double* rho, double* phi, cudaStream_t s, MixedRun& R) {
  int st;
  if ((st = mixed_start(p, rho, phi, s))) return st;
  if (p->max_iter >= 1 && p->side && !p->mixed->resid64 && p->outer_bc == SP_OUTER_MULTIPOLE) {
    SP_CUDA(cudaEventRecord(p->ev_fork, s));
    SP_CUDA(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
    if ((st = mixed_issue_read(p, p->side, R))) return st;
  } else if ((st = mixed_issue_read(p, s, R))) {
    return st;
  }
  const unsigned int* err = reinterpret_cast<const unsigned int*>(p->d_err);
  if (p->max_iter >= 1) {
    if ((st = mixed_correct(p, rho, phi, s))) return st;
    SP_CUDA(post_words2(p->mixed->red, p->h_red_dev + 2 * R.next_slot, 2, err, p->h_red_dev + kRedErrWord, 1, s));
    R.next_slot ^= 1;
    ++R.pending;
  } else {
    SP_CUDA(post_words(err, p->h_red_dev + kRedErrWord, 1, s));
  }
  ++p->launches;
  return SP_OK;
}

// Capture phase A on the plan's private stream (thread-local capture mode, so other host
// threads' calls are unaffected) and instantiate it into `g`; false leaves the plan
// without graphs.
bool capture_phase_a(Plan* p, const double* rho, double* phi, Plan::PhaseGraph& g) {
  if (!p->cap_stream && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    p->cap_stream = nullptr;
    return false;
  }
  const long long l0 = p->launches;
  MixedRun Rc;
  if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  const int st = phase_a_direct(p, rho, phi, p->cap_stream, Rc);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
  g.launches = p->launches - l0;
  p->launches = l0;   // nothing ran yet
  bool ok = st == SP_OK && e == cudaSuccess && graph != nullptr;
  if (ok && cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
    g.exec = nullptr;
    ok = false;
  }
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();   // clear a capture error; the plan runs phase A directly from now on
    p->graphs = false;
    drop_phase_graph(*p);
    return false;
  }
  g.rho = rho;
  g.phi = phi;
  g.ws = p->ws;
  g.pending = Rc.pending;
  return true;
}

}  // namespace

void drop_phase_graph(Plan& p) {
  for (auto& g : p.ga) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = Plan::PhaseGraph{};
  }
  p.ga_victim = 0;
}

// The first call runs directly (it sets the kernels' shared-memory attributes and binds the
// workspace); later calls replay a graph captured for the same rho, phi and workspace
// (captured when none of the plan's two graphs matches, replacing the older one).
// Per-launch timers need the direct path.
int mixed_phase_a(Plan* p, const double* rho, double* phi, cudaStream_t s, MixedRun& R) {
  if (!p->graphs || p->timing || !p->phase_a_warm) {
    const int st = phase_a_direct(p, rho, phi, s, R);
    if (st == SP_OK) p->phase_a_warm = true;
    return st;
  }
  Plan::PhaseGraph* g = nullptr;
  for (auto& c : p->ga)
    if (c.exec && c.rho == rho && c.phi == phi && c.ws == p->ws) g = &c;
  if (!g) {
    int k = -1;
    for (int i = 0; i < Plan::kPhaseGraphs && k < 0; ++i)
      if (!p->ga[i].exec) k = i;
    if (k < 0) {
      k = p->ga_victim;
      p->ga_victim = (k + 1) % Plan::kPhaseGraphs;
      cudaGraphExecDestroy(p->ga[k].exec);
      p->ga[k] = Plan::PhaseGraph{};
    }
    if (!capture_phase_a(p, rho, phi, p->ga[k])) return phase_a_direct(p, rho, phi, s, R);
    g = &p->ga[k];
  }
  SP_CUDA(cudaGraphLaunch(g->exec, s));
  // host bookkeeping of what the graph did: its reductions sit in the first host slots,
  // and the iterate is in the state its one correction leaves
  R.pending = g->pending;
  R.next_slot = g->pending & 1;
  p->phi64_written = (p->max_iter >= 1 || p->mixed->resid64) ? phi : nullptr;
  p->mixed->lo_zero = false;
  p->mixed->iter64 = (first_correction_f64_only(*p) && !p->mixed->resid64) ? phi : nullptr;
  p->launches += g->launches;
  return SP_OK;
}

namespace {

// One low-precision solve's reductions: |e_k| measures the error of the previous iterate;
// the current one is smaller by the contraction factor of the refinement, taken as the
// larger of the observed ratio of successive corrections and a bound for the mode
// (largest ratio measured over the stellar, ragged, point-mass and random-source
// workloads at Nphi <= 256, times two: 1.9e-5 for 6 products, 1.2e-3 for 3 products;
// grown as (Nphi/256)^2 beyond).
void decide_one(Plan* p, MixedRun& R, const unsigned int* slot) {
  float v[2];
  std::memcpy(v, slot, sizeof(v));
  const double e_cur = v[0];
  R.pmax = v[1];
  if (!std::isfinite(e_cur) || !std::isfinite(R.pmax)) {   // a non-finite source or iterate
    R.done = R.nonfinite = true;
    R.est = R.last = std::numeric_limits<double>::infinity();
    if (R.iters < 8) R.hist[R.iters] = R.last;
    ++R.iters;
    return;
  }
  if (R.iters == 0) {
    R.e_prev = e_cur;
    R.hist[0] = R.pmax > 0.0 ? e_cur / R.pmax : 0.0;
    R.iters = 1;
    if (R.pmax == 0.0) {   // rho == 0
      R.done = true;
      R.est = R.last = 0.0;
    }
    return;
  }
  R.last = e_cur / R.pmax;
  if (R.iters < 8) R.hist[R.iters] = R.last;
  // the bounds were measured for Nphi <= 256; the low-precision solve's relative error
  // on the high phi modes grows with their eigenvalue range, so beyond that they grow as
  // (Nphi / 256)^2 (measured single-correction contractions of the 6-product mode:
  // ~2e-4 at Nphi = 1024, ~8e-4 at 2048)
  const double grow = p->nphi > 256 ? (p->nphi / 256.0) * (p->nphi / 256.0) : 1.0;
  const double bound = ((p->mixed->np == 3) ? 4e-5 : 2.5e-3) * grow;
  const double ratio = (R.iters >= 2 && R.e_prev > 0.0) ? e_cur / R.e_prev : 0.0;
  const double c = ratio > bound ? ratio : bound;
  R.est = c < 1.0 ? R.last * c / (1.0 - c) : R.last;
  // Precision floor of the refinement: the float-float iterate carries 48 bits, and its
  // representation error reaches the residual through the phi part of the operator,
  // whose largest eigenvalue grows as (Nphi / 2 pi)^2; the fixed point then differs
  // from the exact solution by up to floor = 8 x 2^-48 x (Nphi / 2 pi)^2 (8: the largest
  // measured ratio of error to 2^-48 (Nphi / 2 pi)^2 was 5.9, over Ntheta 8 and 64,
  // Nphi 128..4096).  Below the floor no further correction helps.
  const double floor = mixed_floor(*p, p->mixed->resid64);
  if (floor > R.est) R.est = floor;
  R.floor_limited = floor > p->tol;
  R.done = R.est <= p->tol || R.last <= 1e-15 || R.floor_limited;
  R.e_prev = e_cur;
  ++R.iters;
}

}  // namespace

void mixed_decide_slot(Plan* p, MixedRun& R, const unsigned int* slot) {
  if (!R.done) decide_one(p, R, slot);
}

// Read the pending slots in issue order; a solve queued behind one that already met the
// tolerance is not counted (its correction is below the tolerance by construction).
void mixed_decide(Plan* p, MixedRun& R) {
  int slot = (R.next_slot - R.pending) & 1;
  for (; R.pending > 0; --R.pending, slot ^= 1)
    if (!R.done) decide_one(p, R, p->h_red + 2 * slot);
}

// Float-float iterate -> float64 Phi and the copy of the device status word (asynchronous).
int mixed_finish_issue(Plan* p, double* phi, cudaStream_t s) {
  Plan& P = *p;
  int st;
  // the last correction's inverse FFT already wrote phi; otherwise convert the iterate
  if (P.phi64_written != phi &&
      (st = launch_status(timed_launch(P, kKUpdate, s, [&] { return finish_mixed(P, phi, s); }))))
    return st;
  SP_CUDA(post_words(reinterpret_cast<const unsigned int*>(P.d_err), P.h_red_dev + kRedErrWord, 1, s));
  ++P.launches;
  return SP_OK;
}

// After the stream has reached mixed_finish_issue: status and info.
int mixed_finish_status(Plan* p, const MixedRun& R, sp_solve_info* info) {
  Plan& P = *p;
  const int herr = (int)P.h_red[kRedErrWord];
  const int st = herr ? ((herr & kErrTimeout) ? SP_ERR_TIMEOUT : SP_ERR_DEVICE_CHECK)
                      : ((R.done && !R.floor_limited && !R.nonfinite) ? SP_OK : SP_ERR_NOT_CONVERGED);
  if (info) {
    info->iterations = R.iters;
    info->precision_used = P.precision;
    info->last_update = R.last;
    info->est_rel_error = R.est;
    info->status = st;
    for (int q = 0; q < 8; ++q) info->update_history[q] = R.hist[q];
  }
  return st;
}

int mixed_finish(Plan* p, double* phi, cudaStream_t s, const MixedRun& R, sp_solve_info* info) {
  int st = mixed_finish_issue(p, phi, s);
  if (st) return st;
  SP_CUDA(cudaStreamSynchronize(s));
  return mixed_finish_status(p, R, info);
}

int solve_fp64_async(Plan* p, const double* rho, double* phi, cudaStream_t s) { return solve_fp64(p, rho, phi, s); }
int ensure_plan_workspace(Plan* p) { return ensure_workspace(p); }

int fill_fp64_info(int st, sp_solve_info* info) {
  if (info) {
    info->iterations = 1;
    info->precision_used = SP_FP64;
    info->last_update = 0.0;
    info->est_rel_error = 0.0;
    info->status = st;
    for (int q = 0; q < 8; ++q) info->update_history[q] = 0.0;
  }
  return st;
}

}  // namespace sp

namespace {

// Mixed-precision solve with float-float iterative refinement (stops when the estimated
// max|Phi - Phi_exact|/max|Phi| <= tol).
int solve_mixed(Plan* p, const double* rho, double* phi, cudaStream_t s, sp_solve_info* info) {
  sp::MixedRun R;
  int st;
  // The first low-precision solve meets the tolerance only for rho == 0, so the first
  // correction is queued right behind it and both are read after one synchronisation.
  if ((st = sp::mixed_phase_a(p, rho, phi, s, R))) return st;
  int k = p->max_iter >= 1 ? 2 : 1;
  SP_CUDA(cudaStreamSynchronize(s));
  sp::mixed_decide(p, R);
  bool more = false;   // kernels queued after phase A (its status word copy is then stale)
  for (; k <= p->max_iter && !R.done; ++k) {
    if ((st = sp::mixed_correct(p, rho, phi, s))) return st;
    if ((st = sp::mixed_issue_read(p, s, R))) return st;
    more = true;
    SP_CUDA(cudaStreamSynchronize(s));
    sp::mixed_decide(p, R);
  }
  // stopped after phase A with the output already in float64: its status word is current
  if (!more && p->phi64_written == phi) return sp::mixed_finish_status(p, R, info);
  return sp::mixed_finish(p, phi, s, R, info);
}

int apply_laplacian_impl(Plan* p, const double* phi, double* out, cudaStream_t s) {
  Plan& P = *p;
  int st = launch_status(sp::timed_launch(P, sp::kKStencil, s, [&] { return sp::stencil_f64(P, phi, out, s); }));
  if (st) return st;
  if (P.outer_bc == SP_OUTER_MULTIPOLE) {
    // FFT of the last shell, kappa in the eigenbasis, inverse FFT accumulated: 3 launches
    st = launch_status(sp::timed_launch(P, sp::kKOuter, s, [&] { return sp::outer_term_f64(P, phi, out, s); }));
    P.launches += 2;
    if (st) return st;
  }
  if (P.inner_bc == SP_INNER_REGULAR) {
    // the same for the first shell with the regular-interior operator
    st = launch_status(sp::timed_launch(P, sp::kKOuter, s, [&] { return sp::inner_term_f64(P, phi, out, s); }));
    P.launches += 2;
  }
  return st;
}

}  // namespace

namespace sp {

size_t workspace_bytes(const Plan& p) {
  if (p.mixed) return mixed_workspace_bytes(p);
  const size_t spec = sizeof(double) * (size_t)p.mh * p.nr * 2 * p.nth;
  const size_t shell = sizeof(double) * (size_t)p.mh * 2 * p.nth;
  return align256(spec) * 2 + align256(shell) * 2;
}

void bind_workspace(Plan& p, void* base) {
  char* c = static_cast<char*>(base);
  if (p.mixed) {
    mixed_bind_workspace(p, c);
    return;
  }
  const size_t spec = align256(sizeof(double) * (size_t)p.mh * p.nr * 2 * p.nth);
  const size_t shell = align256(sizeof(double) * (size_t)p.mh * 2 * p.nth);
  p.specA = reinterpret_cast<double*>(c);
  c += spec;
  p.specB = reinterpret_cast<double*>(c);
  c += spec;
  p.shell = reinterpret_cast<double*>(c);
  c += shell;
  p.shell2 = reinterpret_cast<double*>(c);
}

}  // namespace sp

extern "C" {

const char* sp_status_string(int status) {
  switch (status) {
    case SP_OK: return "SP_OK";
    case SP_ERR_INVALID_ARG: return "SP_ERR_INVALID_ARG";
    case SP_ERR_GRID: return "SP_ERR_GRID";
    case SP_ERR_CUDA: return "SP_ERR_CUDA";
    case SP_ERR_OOM: return "SP_ERR_OOM";
    case SP_ERR_NOT_CONVERGED: return "SP_ERR_NOT_CONVERGED";
    case SP_ERR_TIMEOUT: return "SP_ERR_TIMEOUT";
    case SP_ERR_DEVICE_CHECK: return "SP_ERR_DEVICE_CHECK";
    case SP_ERR_UNSUPPORTED: return "SP_ERR_UNSUPPORTED";
    default: return "SP_ERR_UNKNOWN";
  }
}

int sp_plan_create(const double* r_if, int nr, const double* th_if_in, int nth, int nphi, int outer_bc,
                   double G, int precision, double tol, int max_iter, void* stream, sp_plan** out) {
  sp_plan_desc d = {};
  d.r_interfaces = r_if;
  d.Nr = nr;
  d.theta_interfaces = th_if_in;
  d.Ntheta = nth;
  d.Nphi = nphi;
  d.inner_bc = SP_INNER_ZERO_FLUX;
  d.outer_bc = outer_bc;
  d.G = G;
  d.precision = precision;
  d.tol = tol;
  d.max_iter = max_iter;
  return sp_plan_create_ex(&d, stream, out);
}

int sp_plan_create_ex(const sp_plan_desc* desc, void* stream, sp_plan** out) {
  if (!out || !desc || !desc->r_interfaces) return SP_ERR_INVALID_ARG;
  const double* r_if = desc->r_interfaces;
  const double* th_if_in = desc->theta_interfaces;
  const int nr = desc->Nr, nth = desc->Ntheta, nphi = desc->Nphi, outer_bc = desc->outer_bc;
  const int precision = desc->precision, max_iter = desc->max_iter;
  const double G = desc->G, tol = desc->tol;
  *out = nullptr;
  cudaGetLastError();   // an earlier failed call of this thread is not this call's error
  if (nr < 1 || nth < 1 || nphi < 1) return SP_ERR_GRID;
  if (outer_bc != SP_OUTER_MULTIPOLE && outer_bc != SP_OUTER_DIRICHLET) return SP_ERR_INVALID_ARG;
  if (desc->inner_bc != SP_INNER_ZERO_FLUX && desc->inner_bc != SP_INNER_REGULAR) return SP_ERR_INVALID_ARG;
  if (precision != SP_FP64 && precision != SP_MIXED_BF16X3 && precision != SP_MIXED_BF16X6) return SP_ERR_INVALID_ARG;
  if (!std::isfinite(G)) return SP_ERR_INVALID_ARG;
  if (nth > sp::kMaxNtheta || nphi > sp::kMaxNphi) return SP_ERR_UNSUPPORTED;
  if (precision != SP_FP64 && (nth > 128 || max_iter < 1 || !(tol > 0.0))) return SP_ERR_UNSUPPORTED;
  sp::FftSchedule sched;
  if (!make_schedule(nphi, &sched)) return SP_ERR_UNSUPPORTED;
  // --- validate the grid
  if (!(r_if[0] >= 0.0) || !std::isfinite(r_if[0])) return SP_ERR_GRID;
  for (int i = 0; i < nr; ++i)
    if (!(r_if[i + 1] > r_if[i]) || !std::isfinite(r_if[i + 1])) return SP_ERR_GRID;
  std::vector<double> th(nth + 1);
  if (th_if_in) {
    for (int j = 0; j <= nth; ++j) th[j] = th_if_in[j];
    if (th[0] != 0.0 || std::fabs(th[nth] - kPi) > 1e-12) return SP_ERR_GRID;
    for (int j = 0; j < nth; ++j)
      if (!(th[j + 1] > th[j])) return SP_ERR_GRID;
    th[nth] = kPi;
  } else {
    for (int j = 0; j <= nth; ++j) th[j] = kPi * j / nth;
    th[nth] = kPi;
  }
  // explicit centres strictly inside their cells
  if (desc->r_centres)
    for (int i = 0; i < nr; ++i)
      if (!(desc->r_centres[i] > r_if[i] && desc->r_centres[i] < r_if[i + 1])) return SP_ERR_GRID;
  if (desc->theta_centres)
    for (int j = 0; j < nth; ++j)
      if (!(desc->theta_centres[j] > th[j] && desc->theta_centres[j] < th[j + 1])) return SP_ERR_GRID;
  const bool inner_regular = desc->inner_bc == SP_INNER_REGULAR && r_if[0] > 0.0;
  if (inner_regular && precision != SP_FP64) return SP_ERR_UNSUPPORTED;

  Plan* p = new (std::nothrow) Plan();
  if (!p) return SP_ERR_OOM;
  p->table_refs = new (std::nothrow) std::atomic<int>(1);
  if (!p->table_refs) {
    delete p;
    return SP_ERR_OOM;
  }
  cudaGetDevice(&p->device);
  if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || p->num_sms < 1)
    p->num_sms = 1;
  p->nr = nr;
  p->nth = nth;
  p->nphi = nphi;
  p->mh = nphi / 2 + 1;
  p->outer_bc = outer_bc;
  p->precision = precision;
  p->G = G;
  p->tol = tol;
  p->max_iter = max_iter;
  p->sched = sched;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // --- Sect. 3.1 geometry (host, float64)
  std::vector<double> rc(nr), dv3(nr), R(nr);
  for (int i = 0; i < nr; ++i) {
    const double rm = r_if[i], rp = r_if[i + 1];
    rc[i] = desc->r_centres ? desc->r_centres[i] : 0.5 * (rm + rp);
    dv3[i] = rp * rp * rp - rm * rm * rm;
    R[i] = 3.0 * (rp * rp - rm * rm) / (2.0 * rc[i] * dv3[i]);
  }
  std::vector<sp::RadialRow> rad(nr);
  for (int i = 0; i < nr; ++i) {
    const double sub = (i > 0) ? 3.0 * r_if[i] * r_if[i] / ((rc[i] - rc[i - 1]) * dv3[i]) : 0.0;
    const double sup = (i < nr - 1) ? 3.0 * r_if[i + 1] * r_if[i + 1] / ((rc[i + 1] - rc[i]) * dv3[i]) : 0.0;
    rad[i] = {sub, sup, R[i], -(sub + sup)};
  }
  p->r_out = r_if[nr];
  p->r_last = rc[nr - 1];
  p->outer_coef = 3.0 * p->r_out * p->r_out / dv3[nr - 1];
  p->inner_bc = inner_regular ? SP_INNER_REGULAR : SP_INNER_ZERO_FLUX;
  p->r_in = r_if[0];
  p->r_first = rc[0];
  p->inner_coef = 3.0 * r_if[0] * r_if[0] / dv3[0];

  std::vector<double> thc(nth), w(nth), dth(nth), sinc(nth), sinf(nth + 1), tface(nth > 1 ? nth - 1 : 1, 0.0);
  for (int j = 0; j <= nth; ++j) sinf[j] = (j == 0 || j == nth) ? 0.0 : std::sin(th[j]);
  for (int j = 0; j < nth; ++j) {
    thc[j] = desc->theta_centres ? desc->theta_centres[j] : 0.5 * (th[j] + th[j + 1]);
    w[j] = std::cos(th[j]) - std::cos(th[j + 1]);
    dth[j] = th[j + 1] - th[j];
    sinc[j] = std::sin(thc[j]);
  }
  for (int j = 0; j + 1 < nth; ++j) tface[j] = sinf[j + 1] / (thc[j + 1] - thc[j]);
  // equatorially symmetric grid with even Ntheta: mirror the lower half exactly so the
  // operator commutes with the reflection (enables the parity-split eigensolve)
  bool symmetric = (nth % 2 == 0);
  for (int j = 0; symmetric && j <= nth; ++j)
    if (std::fabs(th[j] + th[nth - j] - kPi) > 1e-13) symmetric = false;
  for (int j = 0; symmetric && j < nth; ++j)   // explicit centres must be mirrored as well
    if (std::fabs(thc[j] + thc[nth - 1 - j] - kPi) > 1e-13) symmetric = false;
  if (symmetric) {
    for (int j = nth / 2; j < nth; ++j) {
      const int q = nth - 1 - j;
      w[j] = w[q];
      dth[j] = dth[q];
      sinc[j] = sinc[q];
      thc[j] = kPi - thc[q];
    }
    for (int j = nth / 2; j + 1 < nth; ++j) tface[j] = tface[nth - 2 - j];
  }
  p->parity = symmetric;
  const double dphi = 2.0 * kPi / nphi;
  std::vector<sp::ThetaRow> thr(nth);
  for (int j = 0; j < nth; ++j) {
    const double tp = (j + 1 < nth) ? tface[j] / w[j] : 0.0;
    const double tm = (j > 0) ? tface[j - 1] / w[j] : 0.0;
    const double S = dth[j] / (sinc[j] * w[j]);
    thr[j] = {tp, tm, (nphi > 1) ? S / (dphi * dphi) : 0.0, 0.0};
  }
  // face-gradient coefficients (the operator's own centres and spacings)
  std::vector<sp::FaceCoef> face_r(nr), face_t(nth);
  for (int i = 0; i < nr; ++i) face_r[i] = {i > 0 ? 1.0 / (rc[i] - rc[i - 1]) : 0.0, 1.0 / rc[i]};
  for (int j = 0; j < nth; ++j)
    face_t[j] = {j > 0 ? 1.0 / (thc[j] - thc[j - 1]) : 0.0, nphi > 1 ? 1.0 / (sinc[j] * dphi) : 0.0};
  // T_m = W^-1/2 B_m W^-1/2: diag (B_jj)/w_j, offdiag t_{j+1/2}/sqrt(w_j w_{j+1})
  const int mh = p->mh;
  std::vector<double> tdiag((size_t)mh * nth), toff(nth, 0.0), sqw(nth);
  for (int j = 0; j < nth; ++j) sqw[j] = std::sqrt(w[j]);
  for (int j = 0; j + 1 < nth; ++j) toff[j] = tface[j] / (sqw[j] * sqw[j + 1]);
  for (int m = 0; m < mh; ++m) {
    const double hs = std::sin(m * 0.5 * dphi) / (0.5 * dphi);
    const double lphi = -hs * hs;
    for (int j = 0; j < nth; ++j) {
      double b = lphi * dth[j] / sinc[j];
      if (j + 1 < nth) b -= tface[j];
      if (j > 0) b -= tface[j - 1];
      tdiag[(size_t)m * nth + j] = b / w[j];
    }
  }
  // twiddles exp(-2 pi i t/nphi) with exact symmetry at the quarter points
  std::vector<double> tw(2 * (size_t)nphi);
  std::vector<float> tw32(2 * (size_t)nphi);
  for (int t = 0; t < nphi; ++t) {
    const double a = 2.0 * kPi * t / nphi;
    double c = std::cos(a), sn = std::sin(a);
    if (4 * t == nphi || 4 * t == 3 * nphi) c = 0.0;
    if (2 * t == nphi) sn = 0.0;
    tw[2 * t] = c;
    tw[2 * t + 1] = -sn;
    tw32[2 * t] = (float)c;
    tw32[2 * t + 1] = (float)-sn;
  }

  int st = SP_OK;
  DeviceGuard guard(p->device);
  do {
    if ((st = upload(&p->d_rad, rad.data(), rad.size()))) break;
    if ((st = upload(&p->d_theta, thr.data(), thr.size()))) break;
    if ((st = upload(&p->d_twid, tw.data(), tw.size()))) break;
    if ((st = upload(&p->d_twid32, tw32.data(), tw32.size()))) break;
    if ((st = upload(&p->d_tdiag, tdiag.data(), tdiag.size()))) break;
    if ((st = upload(&p->d_toff, toff.data(), toff.size()))) break;
    if ((st = upload(&p->d_sqw, sqw.data(), sqw.size()))) break;
    if ((st = upload(&p->d_face_r, face_r.data(), face_r.size()))) break;
    if ((st = upload(&p->d_face_t, face_t.data(), face_t.size()))) break;
    const size_t tab = (size_t)mh * nth;
    const size_t mat = tab * nth;
    if (cudaMalloc(&p->d_lam, sizeof(double) * tab) != cudaSuccess ||
        cudaMalloc(&p->d_kappa, sizeof(double) * tab) != cudaSuccess ||
        cudaMalloc(&p->d_outer, sizeof(double) * tab) != cudaSuccess ||
        cudaMalloc(&p->d_inner, sizeof(double) * tab) != cudaSuccess ||
        cudaMalloc(&p->d_HtW, sizeof(double) * mat) != cudaSuccess ||
        cudaMalloc(&p->d_H, sizeof(double) * mat) != cudaSuccess ||
        cudaMalloc(&p->d_err, sizeof(int)) != cudaSuccess ||
        (p->parity && (cudaMalloc(&p->d_HtWp, sizeof(double) * mat / 2) != cudaSuccess ||
                       cudaMalloc(&p->d_Hp, sizeof(double) * mat / 2) != cudaSuccess))) {
      st = SP_ERR_OOM;
      break;
    }
    if (cudaMemsetAsync(p->d_err, 0, sizeof(int), s) != cudaSuccess) { st = SP_ERR_CUDA; break; }
    if ((st = launch_status(sp::theta_eigen(*p, s)))) break;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = SP_ERR_CUDA;
      break;
    }
    if (herr) { st = SP_ERR_DEVICE_CHECK; break; }
    if (outer_bc == SP_OUTER_MULTIPOLE) {
      if (cudaMalloc(&p->d_oshell, sizeof(double) * mat) != cudaSuccess) { st = SP_ERR_OOM; break; }
      if ((st = launch_status(sp::outer_operator_f64(*p, s)))) break;
    }
    if (inner_regular) {
      if (cudaMalloc(&p->d_ishell, sizeof(double) * mat) != cudaSuccess) { st = SP_ERR_OOM; break; }
      if ((st = launch_status(sp::shell_operator_f64(*p, p->d_inner, p->d_ishell, s)))) break;
    }
    if (precision == SP_FP64) {
      const size_t rad_tab = (size_t)mh * nr * nth;
      if (cudaMalloc(&p->d_tinv, sizeof(double) * rad_tab) != cudaSuccess ||
          cudaMalloc(&p->d_tcp, sizeof(double) * rad_tab) != cudaSuccess) {
        st = SP_ERR_OOM;
        break;
      }
      if ((st = launch_status(sp::radial_factors_f64(*p, s)))) break;
    }
    if (precision != SP_FP64 && (st = sp::mixed_create_tables(*p, s))) break;
    // the float-float residual's floor above the tolerance: float64 iterate and residual
    if (precision != SP_FP64) p->mixed->resid64 = sp::mixed_floor(*p, false) > tol;
    if (precision != SP_FP64 && (st = sp::alloc_host_words(8, &p->h_red, &p->h_red_dev))) break;
    if ((st = sp::create_side_stream(*p))) break;
  } while (0);
  if (st != SP_OK) {
    free_tables(p);
    delete p;
    return st;
  }
  *out = reinterpret_cast<sp_plan*>(p);
  return SP_OK;
}

int sp_plan_clone(const sp_plan* src_plan, sp_plan** out) {
  cudaGetLastError();   // an earlier failed call of this thread is not this call's error
  if (!src_plan || !out) return SP_ERR_INVALID_ARG;
  *out = nullptr;
  const Plan* src = reinterpret_cast<const Plan*>(src_plan);
  DeviceGuard guard(src->device);
  Plan* c = new (std::nothrow) Plan(*src);
  if (!c) return SP_ERR_OOM;
  // per-plan state starts fresh; the tables are shared
  c->table_refs->fetch_add(1);
  c->d_err = nullptr;
  c->ws = nullptr;
  c->ws_bytes = 0;
  c->ws_owned = false;
  c->specA = c->specB = c->shell = c->shell2 = nullptr;
  c->d_rho_io = c->d_phi_io = nullptr;
  c->h_red = nullptr;
  c->h_red_dev = nullptr;
  c->launches = 0;
  c->timing = false;
  c->n_timed = 0;
  for (int i = 0; i < 2 * sp::kMaxTimedLaunches; ++i) c->ev[i] = nullptr;
  for (int k = 0; k < sp::kNumKernelIds; ++k) { c->acc_ms[k] = 0.0; c->acc_n[k] = 0; }
  c->mixed = nullptr;
  int st = SP_OK;
  if (src->mixed) {
    c->mixed = new (std::nothrow) sp::MixedTables(*src->mixed);
    if (!c->mixed) st = SP_ERR_OOM;
    else sp::mixed_clear_workspace(*c->mixed);
    if (st == SP_OK) st = sp::alloc_host_words(8, &c->h_red, &c->h_red_dev);
  }
  c->side = nullptr;
  c->ev_fork = c->ev_join = nullptr;
  c->cap_stream = nullptr;
  for (auto& g : c->ga) g = sp::Plan::PhaseGraph{};
  c->ga_victim = 0;
  c->pipe = nullptr;
  c->phase_a_warm = false;
  if (st == SP_OK) st = sp::create_side_stream(*c);
  if (st == SP_OK && cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess) st = SP_ERR_OOM;
  if (st == SP_OK && cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) st = SP_ERR_CUDA;
  if (st != SP_OK) {
    free_tables(c);
    delete c;
    return st;
  }
  *out = reinterpret_cast<sp_plan*>(c);
  return SP_OK;
}

size_t sp_plan_workspace_bytes(const sp_plan* plan) {
  if (!plan) return 0;
  return sp::workspace_bytes(*reinterpret_cast<const Plan*>(plan));
}

int sp_plan_set_workspace(sp_plan* plan, void* dev, size_t bytes) {
  if (!plan || !dev) return SP_ERR_INVALID_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (bytes < sp::workspace_bytes(*p) || (reinterpret_cast<uintptr_t>(dev) & 255)) return SP_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  if (p->ws_owned) {
    cudaDeviceSynchronize();
    cudaFree(p->ws);
    sp::drop_phase_graph(*p);   // graphs captured on the freed workspace
  }
  // graphs are keyed by (rho, phi, workspace): those of a caller-owned workspace stay for
  // when it is bound again (the layout depends on the plan's shape only)
  p->ws = dev;
  p->ws_bytes = bytes;
  p->ws_owned = false;
  sp::bind_workspace(*p, dev);
  return SP_OK;
}

int sp_solve(sp_plan* plan, const double* rho, double* phi, void* stream, sp_solve_info* info) {
  cudaGetLastError();   // an earlier failed call of this thread is not this call's error
  if (!plan || !rho || !phi) return SP_ERR_INVALID_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  const size_t bytes = sizeof(double) * (size_t)p->nr * p->nth * p->nphi;
  if (overlaps(rho, phi, bytes)) return SP_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  int st = ensure_workspace(p);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->mixed) return solve_mixed(p, rho, phi, s, info);
  return sp::fill_fp64_info(solve_fp64(p, rho, phi, s), info);
}

int sp_solve_host(sp_plan* plan, const double* rho_host, double* phi_host, void* stream, sp_solve_info* info) {
  cudaGetLastError();   // an earlier failed call of this thread is not this call's error
  if (!plan || !rho_host || !phi_host) return SP_ERR_INVALID_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  const size_t bytes = sizeof(double) * (size_t)p->nr * p->nth * p->nphi;
  DeviceGuard guard(p->device);
  if (!p->d_rho_io) SP_CUDA(cudaMalloc(&p->d_rho_io, bytes));
  if (!p->d_phi_io) SP_CUDA(cudaMalloc(&p->d_phi_io, bytes));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SP_CUDA(cudaMemcpyAsync(p->d_rho_io, rho_host, bytes, cudaMemcpyHostToDevice, s));
  int st = sp_solve(plan, p->d_rho_io, p->d_phi_io, stream, info);
  if (st) return st;
  SP_CUDA(cudaMemcpyAsync(phi_host, p->d_phi_io, bytes, cudaMemcpyDeviceToHost, s));
  SP_CUDA(cudaStreamSynchronize(s));
  return SP_OK;
}

// Device buffers, copy streams and events of the pipelined host path (made on first use).
static int ensure_pipe(Plan* p, size_t bytes) {
  if (p->pipe) return SP_OK;
  p->pipe = new (std::nothrow) Plan::HostPipe;
  if (!p->pipe) return SP_ERR_OOM;
  Plan::HostPipe& q = *p->pipe;
  bool ok = cudaStreamCreateWithFlags(&q.h2d, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&q.d2h, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&q.join, cudaEventDisableTiming) == cudaSuccess;
  for (int b = 0; b < 2 && ok; ++b)
    ok = cudaEventCreateWithFlags(&q.in[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&q.solved[b], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&q.out[b], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    free_pipe(p);
    return SP_ERR_CUDA;
  }
  for (int b = 0; b < 2; ++b)
    if (cudaMalloc(&q.rho[b], bytes) != cudaSuccess || cudaMalloc(&q.phi[b], bytes) != cudaSuccess) {
      cudaGetLastError();
      free_pipe(p);
      return SP_ERR_OOM;
    }
  return SP_OK;
}

int sp_solve_host_pipelined(sp_plan* plan, int n, const double* const* rho_host, double* const* phi_host,
                            void* stream, sp_solve_info* infos) {
  cudaGetLastError();   // an earlier failed call of this thread is not this call's error
  if (!plan || n < 0 || (n > 0 && (!rho_host || !phi_host))) return SP_ERR_INVALID_ARG;
  for (int q = 0; q < n; ++q)
    if (!rho_host[q] || !phi_host[q]) return SP_ERR_INVALID_ARG;
  if (n == 0) return SP_OK;
  Plan* p = reinterpret_cast<Plan*>(plan);
  const size_t bytes = sizeof(double) * (size_t)p->nr * p->nth * p->nphi;
  DeviceGuard guard(p->device);
  int st = ensure_pipe(p, bytes);
  if (st) return st;
  Plan::HostPipe& P = *p->pipe;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Solve q uses buffer pair b = q mod 2.  The upload of q waits for solve q-2 (the last
  // reader of rho[b]); solve q waits for its upload and for the download of q-2 (the last
  // reader of phi[b]); the download of q waits for solve q.  Upload q+1 and download q-1
  // are queued before solve q, so both copy directions run while q computes, also across
  // the host waits of a mixed solve.
  auto upload = [&](int q) -> cudaError_t {
    const int b = q & 1;
    cudaError_t e = q >= 2 ? cudaStreamWaitEvent(P.h2d, P.solved[b], 0) : cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.rho[b], rho_host[q], bytes, cudaMemcpyHostToDevice, P.h2d);
    if (e == cudaSuccess) e = cudaEventRecord(P.in[b], P.h2d);
    return e;
  };
  int first_err = SP_OK, done = 0;
  if (upload(0) != cudaSuccess) first_err = SP_ERR_CUDA;
  for (int q = 0; q < n && first_err == SP_OK; ++q) {
    const int b = q & 1;
    if (q + 1 < n && upload(q + 1) != cudaSuccess) { first_err = SP_ERR_CUDA; break; }
    if (cudaStreamWaitEvent(s, P.in[b], 0) != cudaSuccess ||
        (q >= 2 && cudaStreamWaitEvent(s, P.out[b], 0) != cudaSuccess)) {
      first_err = SP_ERR_CUDA;
      break;
    }
    const int r = sp_solve(plan, P.rho[b], P.phi[b], stream, infos ? &infos[q] : nullptr);
    done = q + 1;
    if (r != SP_OK) {
      first_err = r;
      break;
    }
    if (cudaEventRecord(P.solved[b], s) != cudaSuccess || cudaStreamWaitEvent(P.d2h, P.solved[b], 0) != cudaSuccess ||
        cudaMemcpyAsync(phi_host[q], P.phi[b], bytes, cudaMemcpyDeviceToHost, P.d2h) != cudaSuccess ||
        cudaEventRecord(P.out[b], P.d2h) != cudaSuccess) {
      first_err = SP_ERR_CUDA;
      break;
    }
  }
  // join both copy streams into the caller's stream and wait for everything queued
  const bool joined = cudaEventRecord(P.join, P.h2d) == cudaSuccess && cudaStreamWaitEvent(s, P.join, 0) == cudaSuccess &&
                      cudaEventRecord(P.join, P.d2h) == cudaSuccess && cudaStreamWaitEvent(s, P.join, 0) == cudaSuccess;
  const cudaError_t se = cudaStreamSynchronize(s);
  if (!joined) {
    cudaStreamSynchronize(P.h2d);
    cudaStreamSynchronize(P.d2h);
  }
  if (first_err == SP_OK && (!joined || se != cudaSuccess)) first_err = SP_ERR_CUDA;
  if (infos)
    for (int q = done; q < n; ++q) {   // not solved: a call before them failed
      infos[q] = sp_solve_info{};
      infos[q].status = first_err;
    }
  return first_err;
}

int sp_apply_laplacian(sp_plan* plan, const double* phi, double* out, void* stream) {
  cudaGetLastError();   // an earlier failed call of this thread is not this call's error
  if (!plan || !phi || !out) return SP_ERR_INVALID_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  const size_t bytes = sizeof(double) * (size_t)p->nr * p->nth * p->nphi;
  if (overlaps(phi, out, bytes)) return SP_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  int st = ensure_workspace(p);
  if (st) return st;
  return apply_laplacian_impl(p, phi, out, static_cast<cudaStream_t>(stream));
}

int sp_face_gradients(sp_plan* plan, const double* phi, double* g_r, double* g_theta, double* g_phi, void* stream) {
  cudaGetLastError();   // an earlier failed call of this thread is not this call's error
  if (!plan || !phi || !g_r || !g_theta || !g_phi) return SP_ERR_INVALID_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  const size_t cells = (size_t)p->nr * p->nth * p->nphi;
  const size_t b = sizeof(double) * cells;
  const size_t br = sizeof(double) * (cells + (size_t)p->nth * p->nphi);
  const size_t bt = sizeof(double) * (cells + (size_t)p->nr * p->nphi);
  auto ov = [](const void* a, size_t na, const void* c, size_t nc) {
    const char* x = static_cast<const char*>(a);
    const char* y = static_cast<const char*>(c);
    return x < y + nc && y < x + na;
  };
  if (ov(phi, b, g_r, br) || ov(phi, b, g_theta, bt) || ov(phi, b, g_phi, b) || ov(g_r, br, g_theta, bt) ||
      ov(g_r, br, g_phi, b) || ov(g_theta, bt, g_phi, b))
    return SP_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  int st = ensure_workspace(p);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = launch_status(sp::timed_launch(*p, sp::kKStencil, s, [&] { return sp::face_gradients_f64(*p, phi, g_r, g_theta, g_phi, s); }));
  if (p->outer_bc == SP_OUTER_MULTIPOLE) p->launches += 3;   // the outer face's shell transforms
  if (p->inner_bc == SP_INNER_REGULAR) p->launches += 3;     // the inner face's
  return st;
}

int sp_plan_set_residual(sp_plan* plan, int mode) {
  if (!plan) return SP_ERR_INVALID_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (mode != SP_RESIDUAL_AUTO && mode != SP_RESIDUAL_FLOAT_FLOAT && mode != SP_RESIDUAL_FLOAT64) return SP_ERR_INVALID_ARG;
  if (!p->mixed) return SP_OK;   // float64 plans have no refinement
  DeviceGuard guard(p->device);
  const bool r64 = mode == SP_RESIDUAL_FLOAT64 || (mode == SP_RESIDUAL_AUTO && sp::mixed_floor(*p, false) > p->tol);
  if (r64 != p->mixed->resid64) {
    p->mixed->resid64 = r64;
    sp::drop_phase_graph(*p);
    p->phase_a_warm = false;
  }
  return SP_OK;
}

int sp_plan_set_graphs(sp_plan* plan, int enable) {
  if (!plan) return SP_ERR_INVALID_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  DeviceGuard guard(p->device);
  p->graphs = enable != 0;
  if (!p->graphs) sp::drop_phase_graph(*p);
  return SP_OK;
}

int sp_plan_set_timing(sp_plan* plan, int enable) {
  if (!plan) return SP_ERR_INVALID_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  DeviceGuard guard(p->device);
  if (enable && !p->ev[0]) {
    for (int i = 0; i < 2 * sp::kMaxTimedLaunches; ++i) SP_CUDA(cudaEventCreate(&p->ev[i]));
  }
  p->timing = enable != 0;
  p->n_timed = 0;
  for (int k = 0; k < sp::kNumKernelIds; ++k) { p->acc_ms[k] = 0.0; p->acc_n[k] = 0; }
  return SP_OK;
}

int sp_plan_collect_timing(sp_plan* plan) {
  if (!plan) return SP_ERR_INVALID_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  DeviceGuard guard(p->device);
  for (int i = 0; i < p->n_timed; ++i) {
    SP_CUDA(cudaEventSynchronize(p->ev[2 * i + 1]));
    float ms = 0.f;
    SP_CUDA(cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]));
    p->acc_ms[p->ev_kernel[i]] += ms;
    p->acc_n[p->ev_kernel[i]] += 1;
  }
  p->n_timed = 0;
  return SP_OK;
}

int sp_plan_get_timing(const sp_plan* plan, double* ms, long long* count, int n) {
  if (!plan || !ms || !count) return SP_ERR_INVALID_ARG;
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  for (int k = 0; k < n && k < sp::kNumKernelIds; ++k) {
    ms[k] = p->acc_ms[k];
    count[k] = p->acc_n[k];
  }
  return SP_OK;
}

long long sp_plan_launch_count(const sp_plan* plan) {
  if (!plan) return -1;
  return reinterpret_cast<const Plan*>(plan)->launches;
}

int sp_plan_get_eigen(const sp_plan* plan, double* lambda, double* H, double* kappa) {
  if (!plan) return SP_ERR_INVALID_ARG;
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  DeviceGuard guard(p->device);
  SP_CUDA(cudaDeviceSynchronize());
  const int nth = p->nth;
  const size_t tab = (size_t)p->mh * nth;
  std::vector<double> lam(tab), kap(tab), hm(H ? tab * nth : 0);
  SP_CUDA(cudaMemcpy(lam.data(), p->d_lam, sizeof(double) * tab, cudaMemcpyDeviceToHost));
  SP_CUDA(cudaMemcpy(kap.data(), p->d_kappa, sizeof(double) * tab, cudaMemcpyDeviceToHost));
  if (H) SP_CUDA(cudaMemcpy(hm.data(), p->d_H, sizeof(double) * tab * nth, cudaMemcpyDeviceToHost));
  // the plan's own mode order (even then odd modes on parity grids) -> descending lambda
  std::vector<int> order(nth);
  for (int m = 0; m < p->mh; ++m) {
    const double* lm = lam.data() + (size_t)m * nth;
    for (int l = 0; l < nth; ++l) order[l] = l;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lm[a] > lm[b]; });
    for (int l = 0; l < nth; ++l) {
      if (lambda) lambda[(size_t)m * nth + l] = lm[order[l]];
      if (kappa) kappa[(size_t)m * nth + l] = kap[(size_t)m * nth + order[l]];
    }
    if (H)
      for (int j = 0; j < nth; ++j)
        for (int l = 0; l < nth; ++l)
          H[((size_t)m * nth + j) * nth + l] = hm[((size_t)m * nth + j) * nth + order[l]];
  }
  return SP_OK;
}

int sp_plan_last_status(const sp_plan* plan) {
  if (!plan) return SP_ERR_INVALID_ARG;
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  DeviceGuard guard(p->device);
  int herr = 0;
  SP_CUDA(cudaDeviceSynchronize());
  SP_CUDA(cudaMemcpy(&herr, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr & sp::kErrEigenIter) return SP_ERR_DEVICE_CHECK;
  if (herr) return SP_ERR_DEVICE_CHECK;
  return SP_OK;
}

int sp_plan_destroy(sp_plan* plan) {
  if (!plan) return SP_OK;
  Plan* p = reinterpret_cast<Plan*>(plan);
  DeviceGuard guard(p->device);
  cudaDeviceSynchronize();
  free_tables(p);
  delete p;
  return SP_OK;
}

}  // extern "C"

namespace sp {

// Device bytes of the tables a plan shares with its clones.
size_t plan_table_bytes(const Plan& p) {
  const size_t tab = (size_t)p.mh * p.nth;
  size_t b = ((p.d_oshell ? 3 : 2) + (p.d_ishell ? 1 : 0) + (p.d_HtWp ? 1 : 0)) * tab * p.nth * sizeof(double) +
             (p.d_tinv ? 2 * (size_t)p.mh * p.nr * p.nth * sizeof(double) : 0) +
             4 * tab * sizeof(double) +
             (size_t)p.nr * sizeof(RadialRow) +
             (size_t)p.nth * sizeof(ThetaRow) + 2 * (size_t)p.nphi * (sizeof(double) + sizeof(float)) + tab * sizeof(double);
  if (p.mixed) {
    const MixedTables& x = *p.mixed;
    b += 2 * (size_t)x.np * tab * x.kstride * 2 + 2 * (size_t)p.mh * p.nr * p.nth * sizeof(float) +
         (size_t)p.nr * (sizeof(RadialRowF) + sizeof(RadialRowFF) + sizeof(float)) + (size_t)x.nlow * p.nr * 16 +
         (size_t)p.nr * p.nth * sizeof(ThetaRowFF);
  }
  return b;
}

}  // namespace sp

namespace sp {

int alloc_host_words(int n, unsigned int** host, unsigned int** dev) {
  *host = *dev = nullptr;
  if (cudaMallocHost(host, sizeof(unsigned int) * n) != cudaSuccess) {
    cudaGetLastError();
    *host = nullptr;
    return SP_ERR_OOM;
  }
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(dev), *host, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(*host);
    *host = *dev = nullptr;
    return SP_ERR_CUDA;
  }
  std::memset(*host, 0, sizeof(unsigned int) * n);
  return SP_OK;
}

cudaError_t allow_dynamic_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> allowed;   // kernel -> dynamic bytes allowed
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const void* key = reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(kernel) ^ ((uintptr_t)dev << 56));
  std::lock_guard<std::mutex> lock(mu);
  auto it = allowed.find(key);
  if (it == allowed.end()) {
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
    const size_t dyn = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)) != cudaSuccess)
      return e;
    it = allowed.emplace(key, dyn).first;
  }
  return bytes <= it->second ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace sp
