/*
 * sphpoisson.h -- C ABI of the GB300 exact spherical-polar Poisson solver.
 *
 * The library solves the finite-volume Poisson equation of Mueller & Chan (2018),
 * Sect. 3.1, Eq. (fin_vol0)-(fin_vol3):
 *
 *     (Delta_r + Delta_theta + Delta_phi) Phi_{ijk} = s_{ijk} = 4 pi G rho_{ijk}
 *
 * on a grid of Nr radial x Ntheta polar x Nphi azimuthal cells, exactly (to rounding),
 * by the separated algorithm of Sect. 3.2: an FFT along phi, a projection onto the
 * eigenvectors H_{l,m}(j) of the discrete theta operator for every azimuthal wavenumber
 * m, one tridiagonal radial solve per (l,m) that carries the multipole outer boundary
 * condition (last equation of Sect. 3.2), the back projection and the inverse FFT.
 *
 * Conventions shared by every entry point
 *  - Fields rho, Phi and (Delta Phi) are float64, C order [i][j][k] with k (phi) fastest:
 *    element (i,j,k) at offset (i*Ntheta + j)*Nphi + k.
 *  - "dev" pointers are CUDA device pointers on the plan's device; "host" pointers are
 *    CPU memory (page-locked memory gives the fastest copies).  The caller owns every
 *    buffer it passes; the library never frees caller memory.
 *  - Calls with a stream argument are asynchronous on that CUDA stream (a
 *    cudaStream_t passed as void*; NULL is the legacy default stream).  Results are
 *    ready when the stream reaches the work.
 *  - Every function returns an sp_status; nothing aborts or throws across the ABI.
 *    Errors found on the device (eigen-iteration limit, non-convergence) are
 *    recorded in the plan and returned by sp_plan_last_status() after the stream
 *    has been synchronised.
 *  - Cell centres are the midpoints of their interfaces; phi zones are uniform with
 *    centres (k+1/2) 2 pi/Nphi.  The inner radial face carries zero flux (its area
 *    vanishes when r_{1/2} = 0).
 */
#ifndef SPHPOISSON_H
#define SPHPOISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sp_plan sp_plan;

typedef enum {
    SP_OK = 0,
    SP_ERR_INVALID_ARG = 1,     /* null pointer, bad enum, aliasing, size mismatch */
    SP_ERR_GRID = 2,            /* interfaces not increasing, theta not spanning [0,pi] */
    SP_ERR_CUDA = 3,            /* a CUDA runtime call failed */
    SP_ERR_OOM = 4,             /* device allocation failed */
    SP_ERR_NOT_CONVERGED = 5,   /* mixed-precision refinement did not reach tol */
    SP_ERR_TIMEOUT = 6,         /* a bounded device wait gave up */
    SP_ERR_DEVICE_CHECK = 7,    /* a device-side check failed (eigen iteration limit) */
    SP_ERR_UNSUPPORTED = 8      /* size outside what the kernels support */
} sp_status;

/* Outer radial boundary.  SP_OUTER_MULTIPOLE is the paper's condition (Sect. 3.2):
 * the outer-face gradient of mode (l,m) is -p f_N (r_{N+1/2}/r_N)^(-p) / r_{N+1/2},
 * p = (1 + sqrt(1 - 4 lambda_Omega,l,m))/2.  SP_OUTER_DIRICHLET sets Phi(r_{N+1/2}) = 0
 * (the gradient is -f_N/(r_{N+1/2} - r_N)); it has no counterpart in the paper and
 * exists for tests and for bounded domains. */
enum { SP_OUTER_MULTIPOLE = 0, SP_OUTER_DIRICHLET = 1 };

/* Inner radial boundary (only meaningful when r_{1/2} > 0).  SP_INNER_ZERO_FLUX: no flux
 * through r_{1/2} (exact for the l = 0 part when no mass lies inside).  SP_INNER_REGULAR:
 * the region r < r_{1/2} is empty and holds the regular Laplace solution, so each mode
 * (l,m) is extrapolated as f ~ r^q from the innermost zone, q = (-1 + sqrt(1 - 4
 * lambda_Omega,l,m))/2: the inner-face gradient is q f_1 (r_{1/2}/r_1)^q / r_{1/2} (the
 * mirror image of the paper's outer condition, Sect. 3.2; the paper itself treats
 * r_{1/2} = 0 only). */
enum { SP_INNER_ZERO_FLUX = 0, SP_INNER_REGULAR = 1 };

/* Arithmetic of sp_solve.  SP_FP64: every step in float64.  The mixed modes run a
 * low-precision solve -- phi FFTs and radial solves in float32 (float64 for the
 * near-singular |lambda| < 30 radial modes), theta projections on the tensor cores
 * from bf16 split operands with float32 accumulation -- and refine it with the
 * residual of the finite-volume operator evaluated in float-float (~48-bit)
 * arithmetic until the estimated error is below tol:
 *   SP_MIXED_BF16X3  operands split into 2 bf16 planes, 3 products (~2^-16 per product)
 *   SP_MIXED_BF16X6  operands split into 3 bf16 planes, 6 products (~2^-24), which
 *                    needs fewer refinement steps. */
enum { SP_FP64 = 0, SP_MIXED_BF16X3 = 1, SP_MIXED_BF16X6 = 2 };

/* Arithmetic of the mixed modes' refinement residual (sp_plan_set_residual; no
 * counterpart in the paper).  SP_RESIDUAL_FLOAT_FLOAT: the iterate is kept as a pair of
 * floats (48 bits) and the residual evaluated in float-float arithmetic, with no
 * float64 instructions (GB300's float64 rate is 1/64 of float32); its precision floor
 * is 8 x 2^-48 x (Nphi / 2 pi)^2.  SP_RESIDUAL_FLOAT64: the iterate is float64 (held in
 * the caller's output) and the residual is the float64 finite-volume stencil; floor
 * 2^-40 (measured fixed points ~3e-14 up to Nphi = 4096), at several times the
 * residual's cost.  SP_RESIDUAL_AUTO (the default) takes float-float where its floor is
 * below tol and float64 otherwise: at tol 1e-10 float-float up to Nphi = 372. */
enum { SP_RESIDUAL_AUTO = 0, SP_RESIDUAL_FLOAT_FLOAT = 1, SP_RESIDUAL_FLOAT64 = 2 };

typedef struct {
    int iterations;        /* low-precision solves performed (1 for SP_FP64) */
    int precision_used;    /* SP_FP64, SP_MIXED_BF16X3 or SP_MIXED_BF16X6 */
    double last_update;    /* max|e|/max|Phi| of the last correction (0 for SP_FP64) */
    double est_rel_error;  /* estimated max|Phi - Phi_exact|/max|Phi| (0 for SP_FP64): the larger of
                              the refinement's contraction estimate and its precision floor
                              8 x 2^-48 x (Nphi / 2 pi)^2 with the float-float residual (the
                              48-bit iterate seen through the phi part of the operator;
                              4.7e-11 at Nphi = 256), 2^-40 with the float64 one.  When the
                              floor exceeds tol the solve stops and returns
                              SP_ERR_NOT_CONVERGED (with SP_RESIDUAL_AUTO only for tol below
                              2^-40 or a float-float residual chosen explicitly); a NaN or an
                              infinity in a correction or the iterate (a non-finite rho) stops
                              the refinement with SP_ERR_NOT_CONVERGED and an infinite
                              estimate */
    int status;            /* sp_status of the solve */
    double update_history[8]; /* max|e_k|/max|Phi| of the first 8 solves (k = 0 is the first solve) */
} sp_solve_info;

/* Create a plan (Sect. 3.1 geometry, Sect. 3.2 eigenbasis) on the current CUDA device.
 *  r_interfaces      host, Nr+1 values, strictly increasing, r_interfaces[0] >= 0
 *  theta_interfaces  host, Ntheta+1 values, strictly increasing from 0 to pi
 *                    (|last - pi| <= 1e-12); NULL = uniform theta
 *  Nr, Ntheta >= 1; Ntheta <= 160.  Nphi >= 1 with Nphi = 2^a 3^b 5^c, Nphi <= 4096.
 *  outer_bc          SP_OUTER_MULTIPOLE or SP_OUTER_DIRICHLET
 *  G                 gravitational constant (s = 4 pi G rho)
 *  precision         SP_FP64, SP_MIXED_BF16X3 or SP_MIXED_BF16X6 (mixed: Ntheta <= 128)
 *  tol, max_iter     refinement target max|Phi-Phi_exact|/max|Phi| and iteration cap
 *                    (mixed precision only; e.g. 1e-10 and 8).  tol below the mixed
 *                    modes' precision floor cannot be met (see sp_solve_info.est_rel_error
 *                    and SP_RESIDUAL_AUTO)
 *  stream            set-up work (theta eigensolve on the GPU) runs on this stream and
 *                    is complete when the call returns
 *  out               receives the plan; the plan owns its tables and, until
 *                    sp_plan_set_workspace is called, its own workspace.
 * Returns SP_ERR_GRID for invalid interfaces, SP_ERR_UNSUPPORTED for sizes outside the
 * limits above, SP_ERR_DEVICE_CHECK if the eigensolver hit its iteration limit. */
int sp_plan_create(const double* r_interfaces, int Nr,
                   const double* theta_interfaces, int Ntheta,
                   int Nphi, int outer_bc, double G, int precision,
                   double tol, int max_iter, void* stream, sp_plan** out);

/* Everything sp_plan_create takes, plus explicit cell centres and the inner boundary.
 *  r_centres      host, Nr values with r_interfaces[i] < r_centres[i] < r_interfaces[i+1],
 *                 or NULL for the midpoints; the operator's r_i (radial differences,
 *                 R_i and the boundary extrapolations) are these points
 *  theta_centres  host, Ntheta values strictly inside their cells, or NULL for the
 *                 midpoints (theta_j of the differences and of S_j = dtheta_j/(sin
 *                 theta_j w_j))
 *  inner_bc       SP_INNER_ZERO_FLUX or SP_INNER_REGULAR (float64 plans only)
 * Returns what sp_plan_create returns; SP_ERR_GRID for centres outside their cells,
 * SP_ERR_UNSUPPORTED for SP_INNER_REGULAR on a mixed-precision plan. */
typedef struct {
    const double* r_interfaces; int Nr;
    const double* theta_interfaces; int Ntheta;
    int Nphi;
    const double* r_centres;
    const double* theta_centres;
    int inner_bc;
    int outer_bc;
    double G;
    int precision;
    double tol;
    int max_iter;
} sp_plan_desc;
int sp_plan_create_ex(const sp_plan_desc* desc, void* stream, sp_plan** out);

/* A second plan for the same problem that shares the source plan's read-only tables
 * (geometry, theta eigenbasis, radial elimination factors) and has its own workspace,
 * so solves on the source and on its clones may run concurrently (for instance on
 * different streams or host threads).  The tables live until the last of the plans
 * sharing them is destroyed.  No counterpart in the paper. */
int sp_plan_clone(const sp_plan* src, sp_plan** out);

/* Bytes of device workspace sp_solve and sp_apply_laplacian need. */
size_t sp_plan_workspace_bytes(const sp_plan* plan);

/* Hand the plan a caller-owned device workspace of at least sp_plan_workspace_bytes
 * (256-byte aligned).  The plan frees its own workspace, if any, and uses this one
 * until destroyed.  The caller keeps ownership and must not free it while the plan
 * may still use it. */
int sp_plan_set_workspace(sp_plan* plan, void* dev_workspace, size_t bytes);

/* Phi = L^{-1} (4 pi G rho): the exact discrete solve of Sect. 3.2.
 *  rho_dev  device, Nr*Ntheta*Nphi float64, read only
 *  phi_dev  device, Nr*Ntheta*Nphi float64, written; must not overlap rho_dev
 *  info     host, may be NULL; filled when the call returns (for mixed precision
 *           this call synchronises the stream to test convergence)
 * SP_FP64 plans run asynchronously and fill info with iterations = 1. */
int sp_solve(sp_plan* plan, const double* rho_dev, double* phi_dev, void* stream,
             sp_solve_info* info);

/* Same as sp_solve with host buffers: copies rho to the device, solves, copies Phi
 * back, and synchronises the stream before returning.  Uses plan-owned device buffers
 * for rho and Phi (allocated on first use, freed with the plan). */
int sp_solve_host(sp_plan* plan, const double* rho_host, double* phi_host, void* stream,
                  sp_solve_info* info);

/* n solves of one plan from host buffers, q = 0..n-1 in order: rho_host[q] -> phi_host[q]
 * (Sect. 3.2 for each; no counterpart in the paper's design).  The same results as n calls
 * of sp_solve_host, but pipelined: the upload of q+1 and the download of q-1 run on two
 * copy streams of the plan while q is solved on `stream`, through two device (rho, Phi)
 * buffer pairs owned by the plan (4 x Nr x Ntheta x Nphi doubles, allocated on first use,
 * freed with the plan).  With page-locked host buffers the copies overlap the solves and
 * each other; with pageable ones the call is correct but the copies do not overlap.
 * The host arrays must stay valid, and phi_host[q] unread, until the call returns (it
 * synchronises `stream`); a phi_host pointer may repeat (later solves overwrite it in
 * order), none may overlap a rho_host buffer.
 *  n          number of solves (0: nothing to do)
 *  rho_host   n host pointers, each Nr x Ntheta x Nphi doubles
 *  phi_host   n host pointers, each Nr x Ntheta x Nphi doubles
 *  infos      host array of n entries or NULL
 * Returns SP_OK, SP_ERR_INVALID_ARG (a NULL plan, array or entry, or n < 0: nothing runs),
 * SP_ERR_OOM, SP_ERR_CUDA, or the first failing solve's status; solves after a failing
 * one are not run (their infos[q].status is the same error, iterations 0). */
int sp_solve_host_pipelined(sp_plan* plan, int n, const double* const* rho_host, double* const* phi_host,
                            void* stream, sp_solve_info* infos);

/* n independent solves (Sect. 3.2 for each), any mix of grids and precisions, as one
 * call: instance q solves plans[q] with rho[q] -> phi[q] (device buffers as for
 * sp_solve).  The plans must be distinct (use sp_plan_clone for several problems on one
 * grid).  Work runs on internal streams forked from `stream` and joined back into it;
 * mixed-precision instances refine in lock-step rounds with one host wait per round
 * for the whole batch, so this call synchronises when any plan is mixed.
 *  infos  host array of n entries or NULL.
 * Returns the first failing instance's status (each infos[q].status is set). */
int sp_solve_batched(sp_plan* const* plans, const double* const* rho_dev, double* const* phi_dev, int n,
                     void* stream, sp_solve_info* infos);

/* Whether sp_solve_batched issues its mixed-precision instances as ragged batches (off
 * by default; no counterpart in the paper).  When every mixed instance has the same
 * precision, the float-float residual, an even Nphi and a 16-byte aligned rho, each step
 * of the solve -- forward FFT, forward projection, radial scan, inverse projection,
 * inverse FFT, the residual and its multipole shell chain -- is ONE kernel launch for all
 * of them: the launch reads a table of per-instance arguments, and each CTA runs its
 * instance's share (the projection's persistent CTAs are split in proportion to the
 * instances' column tiles).  The instances form up to four groups (by angular grid) on
 * stream pairs of their own, so that the groups' steps overlap; a refinement round is
 * then about twenty operations per group instead of ~20 per instance, with results
 * bitwise those of the instances' own solves.  Turned off, or for other mixes, each
 * instance is its own launch sequence on the batch's 8 streams (measured faster on the
 * 64-instance ragged workload: 14.2 against 15.9 ms).  Applies to calls made after it
 * returns. */
int sp_batched_set_ragged(int enable);
/* Instances the calling thread's last sp_solve_batched solved as one ragged batch (0 when
 * it used per-instance launch sequences). */
int sp_batched_last_ragged(void);

/* out = (Delta Phi)_{ijk}, the finite-volume operator of Eq. (fin_vol0)-(fin_vol3)
 * with the plan's boundary conditions, in float64 (not divided by 4 pi G).
 *  phi_dev, out_dev  device, Nr*Ntheta*Nphi float64; must not overlap */
int sp_apply_laplacian(sp_plan* plan, const double* phi_dev, double* out_dev, void* stream);

/* sp_apply_laplacian without device allocation.  The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc where they need the operator -- code that
 * must not synchronise the device (cudaMalloc/cudaFree may), or that runs under a host
 * framework owning a fixed device-memory pool.  The plan itself is created (and
 * allocates its tables) beforehand; float64 and mixed-precision plans both work.
 *  - Result: bitwise identical to sp_apply_laplacian on the same plan and input (the
 *    same kernels in the same order); the launches count in sp_plan_launch_count and
 *    are timed by the plan's per-kernel timers like sp_apply_laplacian's.
 *  - Scratch: the outer-shell spectra of the multipole boundary term live in one
 *    fixed 4 MiB array inside the library's device image (every GPU that loads the
 *    library holds it until the process exits).  Plans needing more,
 *    2 x 256-byte-aligned (Nphi/2+1)*2*Ntheta doubles > 4 MiB, get SP_ERR_UNSUPPORTED.
 *  - Set-up: the first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call before
 *    any stream capture.
 *  - Sharing: every call uses the same array and leaves the last call's contents in
 *    it (all of it is rewritten before it is read).  Calls that overlap on the GPU --
 *    on different streams, or from different threads -- race and must be serialised
 *    by the caller.
 *  phi_dev, out_dev  device, Nr*Ntheta*Nphi float64; must not overlap */
int sp_apply_laplacian_noalloc(sp_plan* plan, const double* phi_dev, double* out_dev, void* stream);

/* Gradient of Phi on every cell face, in float64: the gradients whose fluxes make up the
 * finite-volume operator of Eq. (fin_vol0)-(fin_vol3), so that their discrete divergence
 * (outward face area x gradient, over the cell volume, Sect. 3.1) is exactly (Delta Phi).
 * The gravitational acceleration is minus these; taken from the exact potential of
 * sp_solve they give the momentum-conserving gravity source terms the paper's
 * introduction (Sect. 1) names as a use of an exact solver.
 *  g_r_dev      device, (Nr+1)*Ntheta*Nphi: face i (i = 0..Nr) between cells i-1 and i,
 *               (Phi_i - Phi_{i-1})/(r_i - r_{i-1}); face 0 is zero (zero flux through
 *               r_{1/2}); face Nr is the outer boundary condition's gradient (multipole:
 *               kappa applied to the last shell in the theta/phi eigenbasis; Dirichlet:
 *               -Phi_N/(r_{N+1/2} - r_N))
 *  g_theta_dev  device, Nr*(Ntheta+1)*Nphi: face j between polar cells j-1 and j,
 *               (Phi_j - Phi_{j-1})/(r_i (theta_j - theta_{j-1})); zero at the poles
 *  g_phi_dev    device, Nr*Ntheta*Nphi: face k+1/2 between k and k+1 (periodic),
 *               (Phi_{k+1} - Phi_k)/(r_i sin(theta_j) 2 pi/Nphi); zero when Nphi = 1
 * Cell centres r_i, theta_j as everywhere (midpoints of the interfaces).  phi_dev and the
 * three outputs must not overlap; uses the plan's workspace. */
int sp_face_gradients(sp_plan* plan, const double* phi_dev, double* g_r_dev, double* g_theta_dev,
                      double* g_phi_dev, void* stream);

/* Copy the plan's theta eigenbasis (Sect. 3.2) to host memory, any pointer may be NULL:
 *  lambda   (Nphi/2+1) x Ntheta: lambda_Omega,l,m, row m, descending in l
 *  H        (Nphi/2+1) x Ntheta x Ntheta: H[m][j][l] = H_{l,m}(j), W-orthonormal
 *  kappa    (Nphi/2+1) x Ntheta: outer-face gradient per unit f_N of mode (l,m)
 * Synchronises the plan's device. */
int sp_plan_get_eigen(const sp_plan* plan, double* lambda, double* H, double* kappa);

/* Per-kernel CUDA-event timers (tracing; no counterpart in the paper).  With timing
 * enabled every kernel launch of the plan is bracketed by two events on its stream
 * (at most 256 launches between collections).  sp_plan_collect_timing waits for the
 * recorded events and adds their durations to per-kernel totals;
 * sp_plan_get_timing copies the totals (milliseconds) and launch counts of the first
 * n kernel identities, in this order: forward FFT, forward projection, radial solve,
 * inverse projection, inverse FFT, stencil, outer-shell term, residual (with its shell
 * term on the side stream), split, update, eigensolve, and the residual's interior-row
 * kernel alone (inside the residual's span).  Enabling resets the totals. */
int sp_plan_set_timing(sp_plan* plan, int enable);
int sp_plan_collect_timing(sp_plan* plan);
int sp_plan_get_timing(const sp_plan* plan, double* ms, long long* count, int n);

/* Choose the refinement residual of a mixed-precision plan (SP_RESIDUAL_*; the default
 * is SP_RESIDUAL_AUTO).  A float64 plan ignores it.  Drops the plan's captured graph. */
int sp_plan_set_residual(sp_plan* plan, int mode);

/* CUDA-graph replay of a mixed solve's first phase (no counterpart in the paper; on by
 * default).  Phase A of sp_solve and sp_solve_batched -- the first low-precision solve,
 * the first correction and the copies of their reductions to host -- is captured on a
 * private stream of the plan at the second solve and replayed with one cudaGraphLaunch
 * on the caller's stream while rho, phi and the workspace stay the same (it is captured
 * again when one of them changes; sp_plan_set_workspace drops it).  Results are bitwise
 * those of the launch-by-launch path.  With per-kernel timing enabled the plan launches
 * kernel by kernel.  The capture runs in thread-local mode, but a device-wide
 * synchronisation made by another host thread during it (sp_plan_destroy does one) can
 * fail, so turn graphs off for plans solved while other threads create or destroy
 * plans; the solve server's slots run without graphs.  Returns SP_ERR_INVALID_ARG for
 * a NULL plan. */
int sp_plan_set_graphs(sp_plan* plan, int enable);

/* Autotune the plan's launch configuration (no counterpart in the paper): the phi lines
 * per CTA of the mixed path's float32 FFTs (which also decides whether Nphi = 256 takes
 * two radix-16 passes), the order of the FFT radix stages, the tensor-core projection's
 * persistent CTA count and the radial scan's components per CTA, one after the other,
 * each candidate timed as the median of three solves of rho_dev into phi_dev on `stream`.
 * The best configuration stays in the plan (and its later clones).  With cache_path
 * (a JSON file, created or updated; NULL for none) an entry for the same device, shape,
 * precision and outer condition is applied without timing (*from_cache = 1 then;
 * from_cache may be NULL) and a new result is added.  Different radix orders round
 * differently, so a tuned plan's results may differ from an untuned one's in the last
 * bits (both within the precision's tolerance).  Synchronises the stream. */
int sp_plan_autotune(sp_plan* plan, const double* rho_dev, double* phi_dev, const char* cache_path, void* stream,
                     int* from_cache);
/* The plan's tuned values (0 = built-in heuristic): values[0..3] = FFT lines per CTA,
 * radix order (0 default, 1 reversed), projection CTAs, scan components per CTA. */
int sp_plan_get_tuning(const sp_plan* plan, int* values);

/* Number of kernel launches this plan has issued since creation (host counter). */
long long sp_plan_launch_count(const sp_plan* plan);

/* ---- continuous-batching solve server (no counterpart in the paper) ----
 * Requests of any grid are queued and admitted into `slots` worker slots (one host
 * thread and one CUDA stream each) as slots and the device-memory budget allow; plans
 * are kept resident across requests of the same grid (least recently used plans are
 * evicted when memory runs short) and every slot solves on its own clone, so requests
 * that arrive while others run overlap with them on the device.  The device is the
 * current CUDA device at sp_server_create.  Slots capture the first phase of a mixed
 * solve into CUDA graphs (sp_plan_set_graphs) on their own threads, so while a server
 * runs, other threads should synchronise streams or events rather than the whole device:
 * a device-wide synchronisation (cudaDeviceSynchronize) that meets a capture fails with
 * cudaErrorStreamCaptureUnsupported. */
typedef struct sp_server sp_server;
typedef struct {
    long long completed, failed, queued;
    int running_peak;          /* most requests on the device at once */
    int resident_plans;
    long long evictions;
    double mem_peak_bytes;     /* peak device memory accounted to plans and buffers */
    double p50_ms, p99_ms, max_ms;   /* submit-to-completion latency of completed requests */
    double zones_per_s;        /* zones completed / (last completion - first submission) */
} sp_server_stats_t;

/* mem_budget_bytes > 0 device bytes for plans, workspaces and staging; 1 <= slots <= 64. */
int sp_server_create(size_t mem_budget_bytes, int slots, sp_server** out);
/* Queue one solve (arguments as sp_plan_create, plus host buffers of Nr*Ntheta*Nphi
 * doubles that must stay valid until sp_server_wait returns for the ticket). */
int sp_server_submit(sp_server* server, const double* r_interfaces, int Nr, const double* theta_interfaces,
                     int Ntheta, int Nphi, int outer_bc, double G, int precision, double tol, int max_iter,
                     const double* rho_host, double* phi_host, long long* ticket);
/* Wait for a ticket (timeout_s < 0: no limit); returns the solve's status or
 * SP_ERR_TIMEOUT (the ticket stays valid).  A completed ticket is released. */
int sp_server_wait(sp_server* server, long long ticket, double timeout_s, sp_solve_info* info);
int sp_server_stats(sp_server* server, sp_server_stats_t* out);
/* Forget the latency and throughput record (for instance after warming resident plans). */
int sp_server_reset_stats(sp_server* server);
/* Finishes queued and running requests, then releases everything. */
int sp_server_destroy(sp_server* server);

/* Status of the most recent device-side checks of this plan (synchronises). */
int sp_plan_last_status(const sp_plan* plan);

/* Release every resource the plan owns.  NULL is accepted. */
int sp_plan_destroy(sp_plan* plan);

/* Human-readable name of a status code (static storage). */
const char* sp_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* SPHPOISSON_H */
