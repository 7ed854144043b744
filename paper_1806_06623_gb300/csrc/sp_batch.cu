// Ragged batches of mixed-precision solves: the separated solve of Sect. 3.2 for many
// independent grids at once, every step issued as ONE launch over all instances.
//
// Each step's kernel reads a table of per-instance arguments (the values the single-plan
// launcher would pass) and a prefix array of per-instance CTA counts; a CTA finds its
// instance by binary search and runs that instance's kernel body as its local CTA
// (rag_instance in sp_internal.h).  The per-instance arithmetic is the single-plan
// kernel's, so every instance's result is bitwise that of its solo solve.  A round of
// the refinement -- first low-precision solve, or residual plus correction -- is about
// twenty operations for the whole batch: the table upload, the reduction reset and
// read-back, five solve steps each (forward FFT, forward projection, radial scan,
// inverse projection, inverse FFT with the iterate update) and the residual with its
// multipole shell chain on a side stream.  The projection's persistent CTAs are shared
// out in proportion to each instance's column tiles.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "sp_internal.h"
#include "tc_gemm.cuh"

namespace sp {
namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// Device and page-locked host buffers of one device's ragged batches: argument tables,
// CTA prefix arrays and the batch's reduction slots [2][n][2].
struct RagBuffers {
  std::mutex mu;
  char* dev = nullptr;
  size_t dcap = 0;
  char* host = nullptr;
  size_t hcap = 0;
  unsigned int* d_red = nullptr;
  unsigned int* h_red = nullptr;
  unsigned int* h_red_dev = nullptr;   // device address of h_red
  int red_n = 0;
  cudaEvent_t fork = nullptr, join = nullptr;
};

int ensure(RagBuffers& b, size_t bytes, int n) {
  if (bytes > b.dcap) {
    cudaFree(b.dev);
    cudaFreeHost(b.host);
    b.dev = nullptr;
    b.host = nullptr;
    b.dcap = b.hcap = 0;
    const size_t cap = std::max(bytes, (size_t)1 << 20);
    if (cudaMalloc(&b.dev, cap) != cudaSuccess) return SP_ERR_OOM;
    if (cudaMallocHost(&b.host, cap) != cudaSuccess) return SP_ERR_OOM;
    b.dcap = b.hcap = cap;
  }
  if (n > b.red_n) {
    cudaFree(b.d_red);
    cudaFreeHost(b.h_red);
    b.d_red = nullptr;
    b.h_red = b.h_red_dev = nullptr;
    b.red_n = 0;
    if (cudaMalloc(&b.d_red, sizeof(unsigned int) * 4 * n) != cudaSuccess) return SP_ERR_OOM;
    if (const int st = alloc_host_words(4 * n, &b.h_red, &b.h_red_dev)) return st;
    b.red_n = n;
  }
  return SP_OK;
}

int cuda_st(cudaError_t e) { return e == cudaSuccess ? SP_OK : (e == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA); }

// Host image of a round's tables; every table starts on a 64-byte boundary.
struct Image {
  std::vector<char> h;
  size_t put(const void* p, size_t bytes) {
    const size_t off = (h.size() + 63) & ~(size_t)63;
    h.resize(off + bytes);
    std::memcpy(h.data() + off, p, bytes);
    return off;
  }
};

// One ragged launch: its argument table and CTA prefix array in the image.
struct Step {
  size_t tab = 0, start = 0;
  int n = 0, total = 0;
  size_t smem = 0;
  int aux = 0;
};

template <typename A>
Step add_step(Image& im, const std::vector<A>& args, const std::vector<int>& ctas, size_t smem, int aux) {
  Step st;
  std::vector<int> start(ctas.size() + 1, 0);
  for (size_t q = 0; q < ctas.size(); ++q) start[q + 1] = start[q] + ctas[q];
  st.n = (int)ctas.size();
  st.total = start.back();
  st.tab = im.put(args.data(), sizeof(A) * std::max<size_t>(args.size(), 1));
  st.start = im.put(start.data(), sizeof(int) * start.size());
  st.smem = smem;
  st.aux = aux;
  return st;
}

// The tables of one low-precision solve over the instances `idx`.
struct SolveSteps {
  Step fwd, pfwd, scan, pinv, inv;
};

template <int NP>
void tc_args(const Plan& p, bool inverse, tc::TcArgs& a) {
  const MixedTables& x = *p.mixed;
  for (int q = 0; q < NP; ++q) std::memcpy(&a.maps.a[q], inverse ? x.map_Ai[q] : x.map_Af[q], sizeof(CUtensorMap));
  a.prm = tc::Params{x.d32, x.panel, p.nth, p.nth, x.kstride, 2 * p.nr, (p.nth + tc::kKBlk - 1) / tc::kKBlk, p.mh,
                     p.d_err};
}

// Persistent projection CTAs shared out over the instances: the smallest per-CTA tile
// count T for which the instances' ceil(tiles / T) CTAs fit one wave (one CTA per SM), so
// the slowest CTA carries at most T tiles.
std::vector<int> tc_ctas(Plan* const* P, const std::vector<int>& idx) {
  std::vector<long long> w(idx.size());
  long long wmax = 1;
  for (size_t k = 0; k < idx.size(); ++k) {
    const Plan& p = *P[idx[k]];
    w[k] = (long long)((2 * p.nr + tc::kM - 1) / tc::kM) * p.mh;
    wmax = std::max(wmax, w[k]);
  }
  const long long sms = std::max((long long)P[idx[0]]->num_sms, (long long)idx.size());
  auto ctas_for = [&](long long T) {
    long long c = 0;
    for (long long x : w) c += (x + T - 1) / T;
    return c;
  };
  long long lo = 1, hi = wmax;   // ctas_for(wmax) = number of instances <= sms
  while (lo < hi) {
    const long long mid = (lo + hi) / 2;
    if (ctas_for(mid) <= sms) hi = mid;
    else lo = mid + 1;
  }
  std::vector<int> c(idx.size());
  for (size_t k = 0; k < idx.size(); ++k) c[k] = (int)((w[k] + lo - 1) / lo);
  return c;
}

template <int NP>
SolveSteps solve_steps(Image& im, Plan* const* P, const std::vector<int>& idx, const double* const* rho, bool first,
                       int nc) {
  SolveSteps S;
  const int n = (int)idx.size();
  std::vector<FwdArgs> fa(n);
  std::vector<ScanArgs> sa(n);
  std::vector<tc::TcArgs> ta(n), tb(n);
  std::vector<int> cf(n), cs(n);
  size_t smf = 0, sms = 0;
  int resident = 0;
  for (int k = 0; k < n; ++k) {
    Plan& p = *P[idx[k]];
    MixedTables& x = *p.mixed;
    size_t sm;
    const void* in = first ? static_cast<const void*>(rho[idx[k]]) : static_cast<const void*>(x.r32);
    const float scale = first ? (float)(4.0 * kPi * p.G / p.nphi) : (float)(1.0 / p.nphi);
    fft_fwd_panel_desc(p, in, scale, x.kstride, x.panel, fa[k], cf[k], sm);
    smf = std::max(smf, sm);
    scan_desc(p, nc, sa[k], cs[k], sm);
    sms = std::max(sms, sm);
    tc_args<NP>(p, false, ta[k]);
    tc_args<NP>(p, true, tb[k]);
  }
  // the forward FFT's L2 prefetch of the same instance's CTA about one resident wave later
  resident = fft_resident_ctas(*P[idx[0]], smf);
  long long totf = 0;
  for (int k = 0; k < n; ++k) totf += cf[k];
  for (int k = 0; k < n; ++k)
    fa[k].ahead = resident > 0 ? std::max(1, (int)((long long)resident * cf[k] / std::max(totf, 1LL))) : 0;
  S.fwd = add_step(im, fa, cf, smf, first ? 0 : 1);
  const std::vector<int> ct = tc_ctas(P, idx);
  S.pfwd = add_step(im, ta, ct, tc::smem_bytes<NP>(), 0);
  S.scan = add_step(im, sa, cs, sms, nc);
  S.pinv = add_step(im, tb, ct, tc::smem_bytes<NP>(), 1);
  return S;
}

// inverse-FFT tables after the solve's flags are known (per instance: first solve, or a
// correction reading/writing the float-float words and float64 output)
Step inv_step(Image& im, Plan* const* P, const std::vector<int>& idx, double* const* phi, bool first,
              unsigned int* d_red_slot) {
  const int n = (int)idx.size();
  std::vector<InvArgs> ia(n);
  std::vector<int> ci(n);
  size_t smi = 0;
  for (int k = 0; k < n; ++k) {
    Plan& p = *P[idx[k]];
    MixedTables& x = *p.mixed;
    const bool lo_read = !first && !x.lo_zero;
    const bool f64_only = !first && x.lo_zero && first_correction_f64_only(p);
    size_t sm;
    fft_inv_update_desc(p, x.d32, x.phi_hi, x.phi_lo, first, lo_read, f64_only, d_red_slot + 2 * k,
                        first ? nullptr : phi[idx[k]], ia[k], ci[k], sm);
    smi = std::max(smi, sm);
  }
  return add_step(im, ia, ci, smi, 0);
}

// residual tables: interior rows, last shells, and the multipole shell chain
struct ResSteps {
  Step interior, last, finish, sfwd, apply, sinv;
  bool lo_read = false;
  int tpb = 32;
  bool any_multipole = false;
};

ResSteps residual_steps(Image& im, Plan* const* P, const std::vector<int>& idx, const double* const* rho) {
  ResSteps R;
  const int n = (int)idx.size();
  std::vector<ResArgs> ra(n), rl;
  std::vector<int> cr(n), cl;
  std::vector<FinishArgs> fa;
  std::vector<FwdArgs> sf;
  std::vector<ShellArgs> sa;
  std::vector<InvArgs> si;
  std::vector<int> cfin, csf, csa, csi;
  size_t smf = 0, smi = 0;
  R.lo_read = !P[idx[0]]->mixed->lo_zero;
  // one block size for the batch: the widest instance's; narrower ones idle the rest
  for (int k = 0; k < n; ++k) R.tpb = std::max(R.tpb, residual_threads(*P[idx[k]]));
  for (int k = 0; k < n; ++k) {
    Plan& p = *P[idx[k]];
    MixedTables& x = *p.mixed;
    const bool mp = p.outer_bc == SP_OUTER_MULTIPOLE;
    residual_desc(p, rho[idx[k]], 0, mp ? p.nr - 1 : p.nr, R.tpb, ra[k], cr[k]);
    if (mp) {
      R.any_multipole = true;
      ResArgs a;
      int c;
      residual_desc(p, rho[idx[k]], p.nr - 1, p.nr, R.tpb, a, c);
      rl.push_back(a);
      cl.push_back(c);
      FinishArgs f;
      shell_finish_desc(p, f, c);
      fa.push_back(f);
      cfin.push_back(c);
      FwdArgs w;
      size_t sm;
      fft_fwd_shell_desc(p, x.shell_phi, p.shell, w, c, sm);
      sf.push_back(w);
      csf.push_back(c);
      smf = std::max(smf, sm);
      ShellArgs s;
      shell_apply_desc(p, p.d_oshell, p.shell, p.shell2, s, c);
      sa.push_back(s);
      csa.push_back(c);
      InvArgs v;
      fft_inv_shell_desc(p, p.shell2, x.outer_shell, v, c, sm);
      si.push_back(v);
      csi.push_back(c);
      smi = std::max(smi, sm);
    }
  }
  R.interior = add_step(im, ra, cr, 0, 0);
  if (R.any_multipole) {
    R.last = add_step(im, rl, cl, 0, 0);
    R.finish = add_step(im, fa, cfin, 0, 0);
    R.sfwd = add_step(im, sf, csf, smf, 2);
    R.apply = add_step(im, sa, csa, 0, 0);
    R.sinv = add_step(im, si, csi, smi, 1);
  }
  return R;
}

template <typename T>
const T* dptr(const RagBuffers& b, size_t off) { return reinterpret_cast<const T*>(b.dev + off); }

template <int NP>
cudaError_t launch_tc(const RagBuffers& b, const Step& st, cudaStream_t s) {
  if (st.total <= 0) return cudaSuccess;
  cudaError_t e = allow_smem(tc::k_tc_gemm_split_rag<NP>, st.smem);
  if (e != cudaSuccess) return e;
  e = launch_pdl(tc::k_tc_gemm_split_rag<NP>, dim3(st.total), dim3(tc::kThreads), st.smem, s,
                 dptr<tc::TcArgs>(b, st.tab), dptr<int>(b, st.start), st.n);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int NP>
cudaError_t issue_solve(const RagBuffers& b, const SolveSteps& S, const Step& inv, cudaStream_t s) {
  cudaError_t e;
  if ((e = fft_fwd_rag(S.fwd.aux, dptr<FwdArgs>(b, S.fwd.tab), dptr<int>(b, S.fwd.start), S.fwd.n, S.fwd.total,
                       S.fwd.smem, s)) != cudaSuccess)
    return e;
  if ((e = launch_tc<NP>(b, S.pfwd, s)) != cudaSuccess) return e;
  if ((e = scan_rag(S.scan.aux, dptr<ScanArgs>(b, S.scan.tab), dptr<int>(b, S.scan.start), S.scan.n, S.scan.total,
                    S.scan.smem, s)) != cudaSuccess)
    return e;
  if ((e = launch_tc<NP>(b, S.pinv, s)) != cudaSuccess) return e;
  return fft_inv_rag(0, dptr<InvArgs>(b, inv.tab), dptr<int>(b, inv.start), inv.n, inv.total, inv.smem, s);
}

cudaError_t issue_residual(const RagBuffers& b, const ResSteps& R, cudaStream_t s, cudaStream_t side) {
  cudaError_t e;
  if (R.any_multipole) {
    if ((e = cudaEventRecord(b.fork, s)) != cudaSuccess || (e = cudaStreamWaitEvent(side, b.fork, 0)) != cudaSuccess)
      return e;
    if ((e = finish_rag(dptr<FinishArgs>(b, R.finish.tab), dptr<int>(b, R.finish.start), R.finish.n, R.finish.total,
                        side)) != cudaSuccess ||
        (e = fft_fwd_rag(2, dptr<FwdArgs>(b, R.sfwd.tab), dptr<int>(b, R.sfwd.start), R.sfwd.n, R.sfwd.total,
                         R.sfwd.smem, side)) != cudaSuccess ||
        (e = shell_apply_rag(dptr<ShellArgs>(b, R.apply.tab), dptr<int>(b, R.apply.start), R.apply.n, R.apply.total,
                             side)) != cudaSuccess ||
        (e = fft_inv_rag(1, dptr<InvArgs>(b, R.sinv.tab), dptr<int>(b, R.sinv.start), R.sinv.n, R.sinv.total,
                         R.sinv.smem, side)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(b.join, side)) != cudaSuccess) return e;
  }
  if ((e = residual_rag(R.lo_read, dptr<ResArgs>(b, R.interior.tab), dptr<int>(b, R.interior.start), R.interior.n,
                        R.interior.total, R.tpb, s)) != cudaSuccess)
    return e;
  if (R.any_multipole) {
    if ((e = cudaStreamWaitEvent(s, b.join, 0)) != cudaSuccess) return e;
    if ((e = residual_rag(R.lo_read, dptr<ResArgs>(b, R.last.tab), dptr<int>(b, R.last.start), R.last.n, R.last.total,
                          R.tpb, s)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

// Instance state after a low-precision solve, as lp_solve leaves it.
void after_solve(Plan& p, double* phi, bool first) {
  MixedTables& x = *p.mixed;
  const bool f64_only = !first && x.lo_zero && first_correction_f64_only(p);
  x.lo_zero = first;
  x.iter64 = f64_only ? phi : nullptr;
  if (!first) p.phi64_written = phi;
}

// One ragged group: its instances (indices into the batch), its streams and buffers.
struct Group {
  std::vector<int> idx;
  cudaStream_t s = nullptr, side = nullptr;
  RagBuffers* b = nullptr;
};

int upload(Group& g, const Image& im, int n) {
  int st = ensure(*g.b, im.h.size(), n);
  if (st) return st;
  std::memcpy(g.b->host, im.h.data(), im.h.size());
  return cuda_st(cudaMemcpyAsync(g.b->dev, g.b->host, im.h.size(), cudaMemcpyHostToDevice, g.s));
}

template <int NP>
int run(Plan* const* P, const double* const* rho, double* const* phi, std::vector<Group>& groups, MixedRun* runs,
        int* status) {
  int nc = 2;
  for (auto& g : groups)
    for (int q : g.idx) nc = std::min(nc, scan_components(*P[q]));
  int st;
  // ---- round 0 of every group: first solves, then the first corrections queued behind
  // them; the groups' streams run concurrently
  for (auto& g : groups) {
    const int n = (int)g.idx.size();
    if ((st = ensure(*g.b, 0, n))) return st;
    unsigned int* red0 = g.b->d_red;          // slot 0: [n][2]
    unsigned int* red1 = g.b->d_red + 2 * n;  // slot 1
    Image im;
    const SolveSteps s0 = solve_steps<NP>(im, P, g.idx, rho, true, nc);
    const Step i0 = inv_step(im, P, g.idx, phi, true, red0);
    for (int q : g.idx) {
      P[q]->phi64_written = nullptr;
      after_solve(*P[q], phi[q], true);
    }
    const ResSteps r1 = residual_steps(im, P, g.idx, rho);
    const SolveSteps s1 = solve_steps<NP>(im, P, g.idx, rho, false, nc);
    const Step i1 = inv_step(im, P, g.idx, phi, false, red1);
    for (int q : g.idx) after_solve(*P[q], phi[q], false);
    st = upload(g, im, n);
    const RagBuffers& b = *g.b;
    if (!st) st = cuda_st(cudaMemsetAsync(b.d_red, 0, sizeof(unsigned int) * 4 * n, g.s));
    if (!st) st = cuda_st(issue_solve<NP>(b, s0, i0, g.s));
    if (!st) st = cuda_st(issue_residual(b, r1, g.s, g.side));
    if (!st) st = cuda_st(issue_solve<NP>(b, s1, i1, g.s));
    if (!st) st = cuda_st(post_words(b.d_red, b.h_red_dev, 4 * n, g.s));
    if (st) return st;
  }
  for (auto& g : groups)
    if ((st = cuda_st(cudaStreamSynchronize(g.s)))) return st;
  for (auto& g : groups) {
    const int n = (int)g.idx.size();
    for (int k = 0; k < n; ++k) {
      mixed_decide_slot(P[g.idx[k]], runs[g.idx[k]], g.b->h_red + 2 * k);
      mixed_decide_slot(P[g.idx[k]], runs[g.idx[k]], g.b->h_red + 2 * n + 2 * k);
    }
  }
  // ---- further rounds: one residual + correction for each group's unfinished instances
  std::vector<std::vector<int>> act(groups.size());
  for (;;) {
    bool any = false;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      Group& g = groups[gi];
      act[gi].clear();
      for (int q : g.idx)
        if (!status[q] && !runs[q].done && runs[q].iters - 1 < P[q]->max_iter) act[gi].push_back(q);
      if (act[gi].empty()) continue;
      any = true;
      // a float64-only iterate is split back into float-float words first (per instance)
      for (int q : act[gi])
        if (P[q]->mixed->iter64) {
          if (cuda_st(split_iterate(*P[q], P[q]->mixed->iter64, g.s))) return SP_ERR_CUDA;
          P[q]->mixed->iter64 = nullptr;
        }
      Image jm;
      const ResSteps rr = residual_steps(jm, P, act[gi], rho);
      const SolveSteps ss = solve_steps<NP>(jm, P, act[gi], rho, false, nc);
      const Step ii = inv_step(jm, P, act[gi], phi, false, g.b->d_red);
      for (int q : act[gi]) after_solve(*P[q], phi[q], false);
      // (the previous round's tables were read before the synchronisation that ended it)
      st = upload(g, jm, (int)g.idx.size());
      const RagBuffers& b = *g.b;
      const size_t words = 2 * act[gi].size();
      if (!st) st = cuda_st(cudaMemsetAsync(b.d_red, 0, sizeof(unsigned int) * words, g.s));
      if (!st) st = cuda_st(issue_residual(b, rr, g.s, g.side));
      if (!st) st = cuda_st(issue_solve<NP>(b, ss, ii, g.s));
      if (!st) st = cuda_st(post_words(b.d_red, b.h_red_dev, words, g.s));
      if (st) return st;
    }
    if (!any) break;
    for (size_t gi = 0; gi < groups.size(); ++gi)
      if (!act[gi].empty() && (st = cuda_st(cudaStreamSynchronize(groups[gi].s)))) return st;
    for (size_t gi = 0; gi < groups.size(); ++gi)
      for (size_t k = 0; k < act[gi].size(); ++k)
        mixed_decide_slot(P[act[gi][k]], runs[act[gi][k]], groups[gi].b->h_red + 2 * k);
  }
  return SP_OK;
}

constexpr int kMaxGroups = 4;

std::mutex g_grp_mu;
std::map<int, RagBuffers*> g_grp;   // device -> kMaxGroups buffers

RagBuffers* group_buffers(int dev) {
  std::lock_guard<std::mutex> lock(g_grp_mu);
  auto it = g_grp.find(dev);
  if (it != g_grp.end()) return it->second;
  RagBuffers* b = new (std::nothrow) RagBuffers[kMaxGroups];
  if (!b) return nullptr;
  for (int k = 0; k < kMaxGroups; ++k)
    if (cudaEventCreateWithFlags(&b[k].fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b[k].join, cudaEventDisableTiming) != cudaSuccess)
      return nullptr;
  g_grp[dev] = b;
  return b;
}

}  // namespace

bool ragged_supported(Plan* const* P, const double* const* rho, int n) {
  if (n < 2) return false;
  const int np = P[0]->mixed ? P[0]->mixed->np : 0;
  for (int q = 0; q < n; ++q) {
    const Plan& p = *P[q];
    if (!p.mixed || p.mixed->np != np || p.mixed->resid64 || p.max_iter < 1 || p.device != P[0]->device) return false;
    if (scan_components(p) == 0 || !residual_pairs(p, rho[q])) return false;
  }
  return true;
}

int ragged_groups(int n, int nstreams) { return std::max(1, std::min({kMaxGroups, nstreams / 2, n / 4})); }

int ragged_solve(Plan* const* P, const double* const* rho, double* const* phi, int n, const cudaStream_t* streams,
                 int nstreams, MixedRun* runs, int* status) {
  RagBuffers* bufs = group_buffers(P[0]->device);
  if (!bufs) return SP_ERR_OOM;
  // Several ragged groups on their own streams, so that the steps of different groups
  // overlap on the device (a projection of one group beside FFTs of another).  Instances
  // of the same angular grid (Ntheta, Nphi) go to the same group where the group count
  // allows, so a group's launches share one block size, FFT shape and K-block count;
  // the angular grids are dealt to the least-loaded group by zones, largest first.
  const int G = ragged_groups(n, nstreams);
  std::vector<Group> groups(G);
  std::vector<double> load(G, 0.0);
  auto zones = [&](int q) { return (double)P[q]->nr * P[q]->nth * P[q]->nphi; };
  std::map<std::pair<int, int>, std::vector<int>> by_grid;
  for (int q = 0; q < n; ++q) by_grid[{P[q]->nth, P[q]->nphi}].push_back(q);
  std::vector<std::pair<double, std::vector<int>>> sets;
  for (auto& kv : by_grid) {
    double z = 0.0;
    for (int q : kv.second) z += zones(q);
    sets.push_back({z, kv.second});
  }
  // split angular-grid sets (largest first, in halves) until there is one per group
  while ((int)sets.size() < G) {
    std::stable_sort(sets.begin(), sets.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
    if (sets[0].second.size() < 2) break;
    std::vector<int> a = sets[0].second, lo, hi;
    std::stable_sort(a.begin(), a.end(), [&](int x, int y) { return zones(x) > zones(y); });
    double zl = 0.0, zh = 0.0;
    for (int q : a) {
      if (zl <= zh) { lo.push_back(q); zl += zones(q); }
      else { hi.push_back(q); zh += zones(q); }
    }
    sets[0] = {zl, lo};
    sets.push_back({zh, hi});
  }
  if ((int)sets.size() < G) {   // still fewer: one set per instance
    std::vector<int> order(n);
    for (int q = 0; q < n; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return zones(a) > zones(c); });
    sets.clear();
    for (int q : order) sets.push_back({zones(q), std::vector<int>{q}});
  }
  std::stable_sort(sets.begin(), sets.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
  for (auto& set : sets) {
    const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    for (int q : set.second) groups[g].idx.push_back(q);
    load[g] += set.first;
  }
  for (int g = 0; g < G; ++g) {
    std::sort(groups[g].idx.begin(), groups[g].idx.end());
    groups[g].s = streams[2 * g];
    groups[g].side = streams[2 * g + 1];
    groups[g].b = &bufs[g];
  }
  std::vector<std::unique_lock<std::mutex>> locks;   // one ragged batch per device at a time
  for (int g = 0; g < kMaxGroups; ++g) locks.emplace_back(bufs[g].mu);
  return P[0]->mixed->np == 3 ? run<3>(P, rho, phi, groups, runs, status) : run<2>(P, rho, phi, groups, runs, status);
}

}  // namespace sp
