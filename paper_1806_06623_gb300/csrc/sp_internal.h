// Internal declarations shared by the host plan code and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <utility>

#include "ff.cuh"
#include "sphpoisson.h"

namespace sp {

constexpr int kMaxStages = 16;
constexpr int kMaxNtheta = 160;   // theta eigenvectors of one m are kept in shared memory
constexpr int kMaxNphi = 4096;

// Radix schedule of a length-n complex FFT, n = 2^a 3^b 5^c (radix 4 first, then 2, 3, 5).
// Per stage: Ns (product of the earlier radices), the twiddle-table step n/(Ns R), and
// the division b/Ns as a shift (power-of-two Ns) or a multiply-high by magic =
// floor(2^32/Ns)+1 (exact for b < 8192).
struct FftSchedule {
  int n;
  int nstages;
  int radix[kMaxStages];
  int ns[kMaxStages];
  int tstep[kMaxStages];
  int shift[kMaxStages];
  unsigned int magic[kMaxStages];
  int nshift;            // log2 n for powers of two, else -1
  unsigned int nmagic;   // ceil(2^32 / n) otherwise: floor(x/n) = umulhi(x, nmagic) for x < 32 n
};

// ---- ragged batches: one launch over the CTAs of several instances (plans).  start[q]
// is the first CTA of instance q (start[n] = all CTAs); a CTA finds its instance by
// binary search and runs that instance's kernel body as its local CTA.
__device__ __forceinline__ int rag_instance(const int* __restrict__ start, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Error bits written by kernels into the plan's device status word.
enum : int { kErrEigenIter = 1, kErrBounds = 2, kErrTimeout = 4 };

// Per-radius coefficients of the radial operator (Eq. fin_vol3 with the Sect. 3.1
// areas): row i of Delta_r + R_i lambda reads
//   sub_i f_{i-1} + (base_i + R_i lambda) f_i + sup_i f_{i+1}
// with base_i = -(sub_i + sup_i); the outer boundary term is added per mode.
struct RadialRow {
  double sub, sup, R, base;
};

// Per-polar-row coefficients of the angular stencil (Delta_hat_theta + S_j Delta_hat_phi):
//   tp = t_{j+1/2}/w_j, tm = t_{j-1/2}/w_j, t = sin(theta_face)/(theta_{j+1}-theta_j),
//   sp = S_j / dphi^2.
struct ThetaRow {
  double tp, tm, sphi, pad;
};

// Face-gradient coefficients (gravitational acceleration): radial row i holds
// 1/(r_i - r_{i-1}) (0 for i = 0) and 1/r_i; polar row j holds 1/(theta_j - theta_{j-1})
// (0 for j = 0) and 1/(sin(theta_j) dphi) (0 when Nphi = 1), centres as in the operator.
struct FaceCoef {
  double inv_d, inv_c;
};

// float copy of RadialRow for the float32 radial solves
struct RadialRowF {
  float sub, sup, R, base;
};

// float-float copies of the stencil coefficients for the refinement residual
struct RadialRowFF {
  ff sub, sup, R, pad;
};
struct ThetaRowFF {
  ff tp, tm, sphi, pad;
};

// Tables and workspace views of the mixed-precision (split-bf16) path.
struct MixedTables {
  int np = 2;                      // bf16 planes per operand: 2 (3 products) or 3 (6 products)
  int kstride = 0;                 // K row stride of the bf16 panels (Ntheta rounded up to 8)
  int nlow = 0;                    // radial modes solved in float64 (|lambda| < low_threshold)
  double low_threshold = 30.0;
  __nv_bfloat16* HtW[3] = {};      // planes of (H^T W)_m, [mh][l][kstride]
  __nv_bfloat16* Hm[3] = {};       // planes of H_m, [mh][j][kstride]
  RadialRowF* radf = nullptr;      // [nr]
  RadialRowFF* radff = nullptr;    // [nr]
  ThetaRowFF* thff = nullptr;      // [nr][nth] R_i x (t_j+1/2, t_j-1/2, phi coefficient) as float pairs
  ff four_pi_g{}, dir_coef{};      // s = 4 pi G rho; Dirichlet outer diagonal (3 r^2/dV3)/(r_N - r_out)
  int* low_idx = nullptr;          // [nlow] flat (m*Ntheta + l) of the float64 modes
  double2* low_fac = nullptr;      // [nlow][nr] (c'_i, 1/pivot_i) of the float64 modes
  // workspace views
  float* r32 = nullptr;            // [nr][nth][nphi] residual
  float* phi_hi = nullptr;         // [nr][nth][nphi] iterate as float-float
  float* phi_lo = nullptr;
  bool lo_zero = false;            // the iterate is a first solve's: its low word is zero and not stored
  bool resid64 = false;            // float64 iterate (in the caller's output) and float64 residual
  const double* iter64 = nullptr;  // non-null: the iterate is stored only there, in float64 (hi, lo stale)
  float* panel = nullptr;          // spectral panel [mh][2nr][kstride] float32 (s_tilde, then f)
  float* d32 = nullptr;            // [mh][2nr][nth] projection output (s_hat, then g)
  float* fcp = nullptr;            // [mh][nr][nth] radial elimination factors c'_i (plan tables)
  float* finv = nullptr;           // [mh][nr][nth] 1/pivot_i
  float* sub_r = nullptr;          // [nr] sub-diagonal of the radial rows
  double* low_ws = nullptr;        // [nlow][nr][3] float64 Thomas scratch
  double* outer_shell = nullptr;   // [nth][nphi] multipole outer term of the residual
  double* shell_phi = nullptr;     // [nth][nphi] float64 value of the iterate's last shell
  unsigned int* red = nullptr;     // [2] max|e|, max|Phi| (bit patterns of non-negative floats)
  // tensor maps (CUtensorMap, 128 bytes each) for the tcgen05 projections
  alignas(64) unsigned char map_Af[3][128], map_Ai[3][128];
};

// Per-instance arguments of the ragged batch kernels (the single-plan launchers' values).
struct FwdArgs {   // forward FFT into the float32 panel (or a float64 shell spectrum)
  FftSchedule sch;
  const void* in;
  void* spec;
  const void* twid;
  double scale;
  int nlines, nth, nrs, lpc, rs, ahead;
};
struct InvArgs {   // inverse FFT with the iterate update (or a float64 shell write)
  FftSchedule sch;
  const void* spec;
  void* out;
  float* phi_lo;
  unsigned int* red;
  double* phi64;
  const void* twid;
  int nlines, nth, nrs, lpc, first, lo_read, hilo, ahead;
};
struct ScanArgs {   // radial scan of the mixed path
  const float* sub_r;
  const double* lam;
  const float* x;
  const float* fcp;
  const float* finv;
  float* pl;
  const int* low_idx;
  const RadialRow* rad64;
  const double2* low_fac;
  double thr;
  int nr, nth, kstride, nlowblk, nlow;
};
struct ResArgs {   // float-float residual rows [row_begin, row_end)
  const double* rho;
  const float* ph;
  const float* pl;
  const double* outer_shell;
  float* r;
  const RadialRowFF* rad;
  const ThetaRowFF* ang;
  ff dir_coef, four_pi_g;
  int nr, nth, nphi, row_begin, row_end, dirichlet;
  int gx, gy;   // the single-plan grid: (Ntheta, row chunks, column blocks)
};
struct FinishArgs {   // float-float words -> float64 (hi, lo of n values; lo may be null)
  const float* ph;
  const float* pl;
  double* phi;
  size_t n;
};
struct ShellArgs {   // z_m = O_m x_m on one shell spectrum
  const double* O;
  const double* x;
  double* z;
  int nth, mh, gx;   // gx = row blocks per m
};

// Kernel identities for the optional per-launch CUDA-event timers.
enum KernelId : int {
  kKFftFwd = 0, kKGemmFwd, kKThomas, kKGemmInv, kKFftInv, kKStencil, kKOuter, kKResidual,
  kKSplit, kKUpdate, kKEigen,
  kKResidualRows,   // the residual's interior-row kernel alone, inside the kKResidual span
  kNumKernelIds
};
constexpr int kMaxTimedLaunches = 256;

struct Plan {
  // Read-only tables (geometry rows, eigenbasis, elimination factors, bf16 planes) are
  // shared by a plan and its clones and freed with the last of them; workspace, error
  // word, host-buffer staging and timers belong to each plan.
  std::atomic<int>* table_refs = nullptr;
  int device = 0;
  int num_sms = 1;                // streaming multiprocessors of the device
  int nr = 0, nth = 0, nphi = 0, mh = 0;
  int outer_bc = SP_OUTER_MULTIPOLE;
  int inner_bc = SP_INNER_ZERO_FLUX;   // SP_INNER_REGULAR only with r_{1/2} > 0 (set otherwise to zero flux)
  int precision = SP_FP64;
  double G = 1.0, tol = 1e-10;
  int max_iter = 8;
  bool parity = false;   // theta grid symmetric about the equator with even Ntheta
  double r_out = 0, r_last = 0, outer_coef = 0;  // outer_coef = 3 r_out^2 / dV3_N
  double r_in = 0, r_first = 0, inner_coef = 0;  // inner_coef = 3 r_in^2 / dV3_1 (regular interior)
  FftSchedule sched{};

  // device tables owned by the plan
  RadialRow* d_rad = nullptr;     // [nr]
  ThetaRow* d_theta = nullptr;    // [nth]
  double* d_twid = nullptr;       // [2*nphi] cos, -sin of 2 pi t / nphi
  float* d_twid32 = nullptr;      // [2*nphi]
  double* d_tdiag = nullptr;      // [mh][nth] diagonal of W^-1/2 B_m W^-1/2
  double* d_toff = nullptr;       // [nth]     off-diagonal of W^-1/2 B_m W^-1/2
  double* d_sqw = nullptr;        // [nth]     sqrt(w_j)
  double* d_lam = nullptr;        // [mh][nth] lambda_Omega,l,m (descending in l)
  double* d_kappa = nullptr;      // [mh][nth] outer-face gradient per unit f_N
  double* d_outer = nullptr;      // [mh][nth] outer diagonal term of the radial row N
  double* d_inner = nullptr;      // [mh][nth] inner diagonal term of the radial row 1 (0 with zero flux)
  double* d_ishell = nullptr;     // [mh][j][j'] H_m diag(inner_m) (H^T W)_m (regular interior only)
  double* d_HtW = nullptr;        // [mh][l][j] (H^T W)_m
  double* d_H = nullptr;          // [mh][j][l] H_m
  double* d_HtWp = nullptr;       // parity grids: [mh][2][h][h] (H^T W)_m,p[l][j], h = nth/2, p = even/odd
  double* d_Hp = nullptr;         // parity grids: [mh][2][h][h] H_m,p[j][l]
  double* d_oshell = nullptr;     // [mh][j][j'] H_m diag(outer_m) (H^T W)_m (multipole only)
  double* d_tinv = nullptr;       // [mh][nr][nth] 1/pivot of each (m,l) radial system (float64 plans)
  double* d_tcp = nullptr;        // [mh][nr][nth] c' = sup/pivot of the same elimination
  FaceCoef* d_face_r = nullptr;   // [nr] radial face-gradient coefficients
  FaceCoef* d_face_t = nullptr;   // [nth] polar face-gradient coefficients
  int* d_err = nullptr;           // device status word

  // workspace (plan-owned or caller-provided)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  double* specA = nullptr;        // [mh][nr][2][nth]
  double* specB = nullptr;        // [mh][nr][2][nth]
  double* shell = nullptr;        // [mh][1][2][nth] outer-shell spectrum
  double* shell2 = nullptr;       // [mh][1][2][nth]

  // host-buffer path
  double* d_rho_io = nullptr;
  double* d_phi_io = nullptr;
  // pipelined host-buffer path: two device (rho, Phi) pairs, copy streams and their events
  struct HostPipe {
    double* rho[2] = {nullptr, nullptr};
    double* phi[2] = {nullptr, nullptr};
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t in[2] = {nullptr, nullptr};       // rho[b] uploaded
    cudaEvent_t solved[2] = {nullptr, nullptr};   // the solve reading rho[b] / writing phi[b] done
    cudaEvent_t out[2] = {nullptr, nullptr};      // phi[b] downloaded
    cudaEvent_t join = nullptr;
  };
  HostPipe* pipe = nullptr;

  MixedTables* mixed = nullptr;
  unsigned int* h_red = nullptr;  // pinned host copy of the mixed-path reductions
  unsigned int* h_red_dev = nullptr;   // the same memory as the device addresses it
  const double* phi64_written = nullptr;   // output already holding the current iterate in float64
  // CUDA graphs of phase A of a mixed solve (first low-precision solve + first correction
  // with their host reads), captured on a private stream, each for one (rho, phi,
  // workspace); eight are kept, so that callers alternating buffer pairs (the pipelined
  // host path) or the solve server's slots (each with its own buffers) replay theirs
  bool graphs = true;
  bool phase_a_warm = false;      // one direct phase A ran (attributes set, workspace bound)
  cudaStream_t cap_stream = nullptr;
  struct PhaseGraph {
    cudaGraphExec_t exec = nullptr;
    const void* rho = nullptr;
    const void* phi = nullptr;
    const void* ws = nullptr;
    long long launches = 0;
    int pending = 0;
  };
  static constexpr int kPhaseGraphs = 8;
  PhaseGraph ga[kPhaseGraphs];
  int ga_victim = 0;              // the entry the next capture replaces when both are taken
  // side stream (high priority) and fork/join events: the multipole shell term of the
  // mixed residual runs beside the residual's interior rows
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // launch configuration chosen by sp_plan_autotune (0 = the built-in heuristic)
  struct Tune {
    int lpc = 0;           // phi lines per CTA of the float32 panel FFTs
    int radix_order = 0;   // 0: radix 4, 2, 3, 5 stages in that order; 1: reversed
    int tc_ctas = 0;       // persistent CTAs of the tensor-core projection
    int scan_nc = 0;       // components per CTA of the radial scan (1 or 2)
  } tune;

  // launch accounting and optional CUDA-event timers (one event pair per launch)
  long long launches = 0;
  bool timing = false;
  int n_timed = 0;
  cudaEvent_t ev[2 * kMaxTimedLaunches] = {};
  int ev_kernel[kMaxTimedLaunches] = {};
  double acc_ms[kNumKernelIds] = {};
  long long acc_n[kNumKernelIds] = {};
};

// Record a launch of kernel `id` issued by `launch()` on stream s.
// Programmatic dependent launch (mixed-path kernels): a kernel launched with
// launch_pdl may be scheduled while the previous kernel of its stream finishes; it
// signals pdl_trigger() early, runs only its independent prologue (shared memory,
// barriers, TMEM, plan-constant tables) and calls pdl_wait() -- which returns once the
// previous kernel has completed and its memory is visible -- before any other global
// access.  Launched the ordinary way both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename F>
cudaError_t timed_span(Plan& p, int id, cudaStream_t s, F&& launch) {
  // the event pair's slot is taken before the launch, so spans may nest
  const int k = (p.timing && p.n_timed < kMaxTimedLaunches) ? p.n_timed++ : -1;
  if (k >= 0) cudaEventRecord(p.ev[2 * k], s);
  cudaError_t e = launch();
  if (k >= 0) {
    cudaEventRecord(p.ev[2 * k + 1], s);
    p.ev_kernel[k] = id;
  }
  return e;
}
template <typename F>
cudaError_t timed_launch(Plan& p, int id, cudaStream_t s, F&& launch) {
  const cudaError_t e = timed_span(p, id, s, static_cast<F&&>(launch));
  ++p.launches;
  return e;
}

// Allow `kernel` up to `bytes` of dynamic shared memory.  The attribute is raised once
// per kernel to the device's opt-in maximum and never lowered, so concurrent launches of
// the same kernel for different plan sizes (several host threads) cannot undercut each
// other.  Returns cudaErrorInvalidValue when `bytes` exceeds what the device allows.
cudaError_t allow_dynamic_smem(const void* kernel, size_t bytes);
template <typename K>
cudaError_t allow_smem(K* kernel, size_t bytes) {
  return allow_dynamic_smem(reinterpret_cast<const void*>(kernel), bytes);
}

size_t workspace_bytes(const Plan& p);
void bind_workspace(Plan& p, void* base);

// ---- kernels (launchers return the launch error) ----
// Forward FFT of nlines real lines of length n (line g = i*nth + j, shell-major),
// writing the half spectrum scaled by `scale` into spec[m][i][c][j] (nrs shells).
cudaError_t fft_forward_f64(const Plan& p, const double* in, int nrs, double scale, double* spec,
                            cudaStream_t s);
// Inverse FFT of spec[m][i][c][j] into lines; accumulate adds into `out`.
cudaError_t fft_inverse_f64(const Plan& p, const double* spec, int nrs, double* out, bool accumulate,
                            cudaStream_t s);
// Batched NT GEMM: C[b][n][r] = sum_k A[b][r][k] B[b][n][k], b < nb.
cudaError_t gemm_nt_f64(const double* A, const double* B, double* C, int nb, int M, int ncol, int K,
                        cudaStream_t s);
// Parity-split projections (nth = 2h): forward folds B[n][j] +- B[n][nth-1-j] and writes
// C[n][p*h + l] = sum_{j<h} A[b][p][l][j] fold_p(j); inverse forms
// g_p[n][j] = sum_{l<h} A[b][p][j][l] B[n][p*h + l] and writes C[n][j] = g_0 + g_1,
// C[n][nth-1-j] = g_0 - g_1.
cudaError_t gemm_parity_f64(const double* A, const double* B, double* C, int nb, int h, int ncol, bool inverse,
                            cudaStream_t s);
// Radial Thomas solves for every (m,l), in place on x[m][i][c][l].
cudaError_t thomas_f64(const Plan& p, double* x, cudaStream_t s);
cudaError_t radial_factors_f64(const Plan& p, cudaStream_t s);   // d_tinv, d_tcp (plan set-up)
// Local part of the finite-volume operator (all interior fluxes, Dirichlet outer term).
cudaError_t stencil_f64(const Plan& p, const double* phi, double* out, cudaStream_t s);
// Multipole outer term on the last shell: out[nr-1] += outer_coef * kappa(A_Omega) phi[nr-1].
cudaError_t outer_term_f64(const Plan& p, const double* phi, double* out, cudaStream_t s);
// out[m] = H_m diag(outer[m]) (H^T W)_m in[m] for the two real columns of one shell spectrum.
cudaError_t shell_kappa_f64(const Plan& p, const double* in, double* out, cudaStream_t s);
// the same with the per-m shell operator O ([mh][j][j'])
cudaError_t shell_apply_f64(const Plan& p, const double* O, const double* in, double* out, cudaStream_t s);
// O = H diag(diag) H^T W per m, into dst
cudaError_t shell_operator_f64(const Plan& p, const double* diag, double* dst, cudaStream_t s);
cudaError_t outer_operator_f64(const Plan& p, cudaStream_t s);
// Regular-interior inner term on the first shell: out[0] += O_in phi[0].
cudaError_t inner_term_f64(const Plan& p, const double* phi, double* out, cudaStream_t s);
// Face gradients of phi (radial [nr+1][nth][nphi], polar [nr][nth+1][nphi], azimuthal
// [nr][nth][nphi]); the outer radial face carries the boundary condition's gradient.
cudaError_t face_gradients_f64(const Plan& p, const double* phi, double* gr, double* gt, double* gp, cudaStream_t s);
// theta eigensolve for every m; writes lam, kappa, outer, H, HtW.
cudaError_t theta_eigen(const Plan& p, cudaStream_t s);

// ---- mixed-precision path ----
size_t mixed_workspace_bytes(const Plan& p);
void mixed_bind_workspace(Plan& p, char* base);
int mixed_create_tables(Plan& p, cudaStream_t s);   // after theta_eigen; returns sp_status
void mixed_free_shared(MixedTables& x);     // tables shared with clones
void mixed_clear_workspace(MixedTables& x);  // forget workspace views (clone set-up)
struct Planes {
  __nv_bfloat16* p[3];
  int n;
};
cudaError_t fft_forward_panel(const Plan& p, const void* in, bool in_double, float scale, int kstride, float* out,
                              cudaStream_t s);
cudaError_t fft_inverse_update(const Plan& p, const float* spec, float* phi_hi, float* phi_lo, bool first, bool lo_read,
                               bool f64_only, unsigned int* red, double* phi64, cudaStream_t s);
cudaError_t finish_mixed(const Plan& p, double* phi, cudaStream_t s);   // float-float iterate -> float64 Phi
cudaError_t split_iterate(const Plan& p, const double* phi, cudaStream_t s);   // float64 iterate -> hi, lo
bool first_correction_f64_only(const Plan& p);   // the first correction stores the iterate in float64 only
cudaError_t tc_project(const Plan& p, bool inverse, cudaStream_t s);   // pan -> d32
cudaError_t thomas_mixed(const Plan& p, cudaStream_t s);   // d32 -> pan (f); float32 + float64 low modes
cudaError_t residual_ff(Plan& p, const double* rho, cudaStream_t s);  // iterate -> r32
// the float-float residual fused with its forward FFT (iterate -> panel), where
// residual_fft_supported: Nphi = 256, even Ntheta, 16-byte aligned rho, float-float residual
bool residual_fft_supported(const Plan& p, const double* rho);
cudaError_t residual_fft(Plan& p, const double* rho, cudaStream_t s);
cudaError_t residual_f64(const Plan& p, const double* rho, const double* phi, cudaStream_t s);  // float64 iterate -> r32
// inverse FFT adding the correction into a float64 iterate (first: phi = e), reductions into red
cudaError_t fft_inverse_update64(const Plan& p, const float* spec, double* phi, bool first, unsigned int* red,
                                 cudaStream_t s);
int create_side_stream(Plan& p);   // side stream and events of a mixed multipole plan; sp_status

// phi lines per CTA of the float32 panel FFTs (the tuned value when one is set)
int panel_lpc(const Plan& p, int nlines);
// radix schedule of a length-n FFT; order 1 reverses the default stage order
bool make_fft_schedule(int n, int order, FftSchedule* s);

// ---- ragged batch launches (kind: forward 0 = float32 panel from float64 rho,
// 1 = float32 panel from the float32 residual, 2 = float64 shell; inverse 0 = iterate
// update, 1 = float64 shell write)
void fft_fwd_panel_desc(const Plan& p, const void* in, float scale, int kstride, float* out, FwdArgs& a, int& ctas,
                        size_t& smem);
void fft_fwd_shell_desc(const Plan& p, const double* in, double* spec, FwdArgs& a, int& ctas, size_t& smem);
void fft_inv_update_desc(const Plan& p, const float* spec, float* phi_hi, float* phi_lo, bool first, bool lo_read,
                         bool f64_only, unsigned int* red, double* phi64, InvArgs& a, int& ctas, size_t& smem);
void fft_inv_shell_desc(const Plan& p, const double* spec, double* out, InvArgs& a, int& ctas, size_t& smem);
cudaError_t fft_fwd_rag(int kind, const FwdArgs* tab, const int* start, int n, int total, size_t smem, cudaStream_t s);
cudaError_t fft_inv_rag(int kind, const InvArgs* tab, const int* start, int n, int total, size_t smem, cudaStream_t s);
int fft_resident_ctas(const Plan& p, size_t smem);
void shell_apply_desc(const Plan& p, const double* O, const double* in, double* out, ShellArgs& a, int& ctas);
int scan_components(const Plan& p);
void scan_desc(const Plan& p, int nc, ScanArgs& a, int& ctas, size_t& smem);
cudaError_t scan_rag(int nc, const ScanArgs* tab, const int* start, int n, int total, size_t smem, cudaStream_t s);
bool residual_pairs(const Plan& p, const double* rho);
int residual_threads(const Plan& p);
void residual_desc(const Plan& p, const double* rho, int r0, int r1, int tpb, ResArgs& a, int& ctas);
cudaError_t residual_rag(bool lo_read, const ResArgs* tab, const int* start, int n, int total, int tpb,
                         cudaStream_t s);
void shell_finish_desc(const Plan& p, FinishArgs& a, int& ctas);
cudaError_t finish_rag(const FinishArgs* tab, const int* start, int n, int total, cudaStream_t s);
// n result words of the device -> page-locked host memory (`host_dst` a device-accessible
// pointer of a cudaMallocHost allocation), by one kernel's stores instead of a copy
cudaError_t post_words(const unsigned int* src, unsigned int* host_dst, int n, cudaStream_t s);
cudaError_t post_words2(const unsigned int* a, unsigned int* host_a, int na, const unsigned int* b,
                        unsigned int* host_b, int nb, cudaStream_t s);
// n page-locked host words and the device address of the same memory (SP_OK / SP_ERR_*)
int alloc_host_words(int n, unsigned int** host, unsigned int** dev);
cudaError_t shell_apply_rag(const ShellArgs* tab, const int* start, int n, int total, cudaStream_t s);

// ---- solve phases shared by sp_solve, sp_solve_batched and the server ----
// Refinement state of one mixed-precision solve.
struct MixedRun {
  double e_prev = 0.0, pmax = 0.0, est = 1.0, last = 1.0;
  double hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int iters = 0;       // low-precision solves read
  int pending = 0;     // reductions copied to host slots but not yet read (at most 2)
  int next_slot = 0;   // host slot of the next copy
  bool done = false;
  bool floor_limited = false;   // the iterate's precision floor is above the tolerance
  bool nonfinite = false;       // a correction or the iterate held a NaN or an infinity
};
constexpr int kRedErrWord = 4;   // h_red: two slots of (max|e|, max|Phi|), then the status word
int mixed_start(Plan* p, const double* rho, double* phi, cudaStream_t s);
double mixed_floor(const Plan& p, bool resid64);   // precision floor of the refinement
int mixed_correct(Plan* p, const double* rho, double* phi, cudaStream_t s);
int mixed_issue_read(Plan* p, cudaStream_t s, MixedRun& R);
// First low-precision solve and (max_iter >= 1) the first correction, each with the copy
// of its reductions to a host slot; replayed from a CUDA graph when the plan allows.
int mixed_phase_a(Plan* p, const double* rho, double* phi, cudaStream_t s, MixedRun& R);
void drop_phase_graph(Plan& p);
void mixed_decide(Plan* p, MixedRun& R);   // after the stream has reached the pending copies
// one solve's reductions (max|e|, max|Phi| bit patterns) read from `slot` (ragged batches)
void mixed_decide_slot(Plan* p, MixedRun& R, const unsigned int* slot);
// Ragged batched mixed solves (sp_batch.cu): every instance's steps as one launch per step.
// Returns false when the instances cannot form one ragged group (then nothing was issued).
bool ragged_supported(Plan* const* P, const double* const* rho, int n);
int ragged_groups(int n, int nstreams);   // ragged groups (stream pairs) used for n instances
int ragged_solve(Plan* const* P, const double* const* rho, double* const* phi, int n, const cudaStream_t* streams,
                 int nstreams, MixedRun* runs, int* status);
int mixed_finish(Plan* p, double* phi, cudaStream_t s, const MixedRun& R, sp_solve_info* info);
int mixed_finish_issue(Plan* p, double* phi, cudaStream_t s);
int mixed_finish_status(Plan* p, const MixedRun& R, sp_solve_info* info);
size_t plan_table_bytes(const Plan& p);
int fill_fp64_info(int st, sp_solve_info* info);
int solve_fp64_async(Plan* p, const double* rho, double* phi, cudaStream_t s);
int ensure_plan_workspace(Plan* p);

}  // namespace sp
