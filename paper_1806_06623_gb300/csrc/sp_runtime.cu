// Batched solves and the continuous-batching solve server.
//
// sp_solve_batched runs independent problems (any mix of grids and precisions) on a pool
// of streams forked from the caller's stream.  Float64 solves are issued back to back;
// the mixed-precision refinements advance in lock-step rounds -- every unfinished
// instance issues its next correction, then one host wait per round reads all their
// update norms -- so the batch costs a few host synchronisations instead of a few per
// instance, and the instances' kernels overlap on the device.
//
// The server admits solve requests of any grid size from a queue into worker slots (one
// host thread and one stream each) while the device-memory budget allows, keeps plans
// (geometry, eigenbasis, elimination factors) resident across requests of the same grid
// and hands every slot its own clone of them (own workspace, shared tables), so requests
// that arrive while others run start as soon as a slot and memory are free and their
// kernels overlap on the device.  Latency is measured from submission to completion.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sp_internal.h"

using sp::Plan;

namespace {

constexpr int kBatchStreams = 8;

struct StreamPool {
  cudaStream_t s[kBatchStreams] = {};
  cudaEvent_t ev[kBatchStreams + 1] = {};
};

std::mutex g_pool_mu;
std::map<int, StreamPool*> g_pools;

StreamPool* pool_for(int dev) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  StreamPool* sp = new (std::nothrow) StreamPool();
  if (!sp) return nullptr;
  for (int k = 0; k < kBatchStreams; ++k)
    if (cudaStreamCreateWithFlags(&sp->s[k], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  for (int k = 0; k <= kBatchStreams; ++k)
    if (cudaEventCreateWithFlags(&sp->ev[k], cudaEventDisableTiming) != cudaSuccess) return nullptr;
  g_pools[dev] = sp;
  return sp;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? SP_OK : (e == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA); }

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// sp_solve_batched issues same-precision mixed instances as ragged batches when turned on
// (off by default: on the 64-instance ragged workload the per-instance streams measured
// 14.2 against 15.9 ms, the ragged form issuing ~30x fewer launches)
std::atomic<int> g_ragged{0};
thread_local int t_last_ragged = 0;   // instances of this thread's last call solved as a ragged batch

}  // namespace

extern "C" int sp_batched_set_ragged(int enable) {
  g_ragged.store(enable ? 1 : 0);
  return SP_OK;
}

extern "C" int sp_batched_last_ragged(void) { return t_last_ragged; }

extern "C" int sp_solve_batched(sp_plan* const* plans, const double* const* rho, double* const* phi, int n,
                                void* stream, sp_solve_info* infos) {
  cudaGetLastError();   // an earlier failed call of this thread is not this call's error
  if (n < 0) return SP_ERR_INVALID_ARG;
  if (n == 0) return SP_OK;
  if (!plans || !rho || !phi) return SP_ERR_INVALID_ARG;
  std::vector<Plan*> P(n);
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !rho[i] || !phi[i]) return SP_ERR_INVALID_ARG;
    P[i] = reinterpret_cast<Plan*>(plans[i]);
    if (P[i]->device != P[0]->device) return SP_ERR_INVALID_ARG;
    const size_t bytes = sizeof(double) * (size_t)P[i]->nr * P[i]->nth * P[i]->nphi;
    const char* a = reinterpret_cast<const char*>(rho[i]);
    const char* b = reinterpret_cast<const char*>(phi[i]);
    if (a < b + bytes && b < a + bytes) return SP_ERR_INVALID_ARG;
  }
  {
    std::vector<Plan*> sorted(P);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return SP_ERR_INVALID_ARG;   // shared workspace
  }
  DeviceScope dev(P[0]->device);
  StreamPool* pool = pool_for(P[0]->device);
  if (!pool) return SP_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    const int st = sp::ensure_plan_workspace(P[i]);
    if (st) return st;
  }
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  const int ns = std::min(n, kBatchStreams);
  int st = cuda_status(cudaEventRecord(pool->ev[kBatchStreams], user));
  for (int k = 0; k < ns && !st; ++k) st = cuda_status(cudaStreamWaitEvent(pool->s[k], pool->ev[kBatchStreams], 0));
  if (st) return st;

  std::vector<int> status(n, SP_OK);
  std::vector<sp::MixedRun> runs(n);
  // the mixed instances as one ragged batch on stream 0 (side stream 1) when they form one;
  // the rest keep one launch sequence each on the pool's streams
  std::vector<int> mixed_idx;
  for (int i = 0; i < n; ++i)
    if (P[i]->mixed) mixed_idx.push_back(i);
  std::vector<Plan*> MP;
  std::vector<const double*> MR;
  std::vector<double*> MF;
  for (int i : mixed_idx) {
    MP.push_back(P[i]);
    MR.push_back(rho[i]);
    MF.push_back(phi[i]);
  }
  const bool ragged = g_ragged.load() && ns >= 2 && sp::ragged_supported(MP.data(), MR.data(), (int)MP.size());
  t_last_ragged = ragged ? (int)MP.size() : 0;
  const int groups = ragged ? sp::ragged_groups((int)MP.size(), ns) : 0;
  // per-instance launch sequences: largest instances first, each to the stream with the
  // fewest zones so far, so that the streams end together and the small instances fill
  // the GPU beside the last large ones
  std::vector<int> order(n), lane(n, 0);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto zones = [&](int i) { return (double)P[i]->nr * P[i]->nth * P[i]->nphi; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return zones(a) > zones(b); });
  {
    std::vector<double> load(ns > 0 ? ns : 1, 0.0);
    for (int i : order) {
      int k = 0;
      for (int q = 1; q < ns; ++q)
        if (load[q] < load[k]) k = q;
      lane[i] = k;
      load[k] += zones(i);
    }
  }
  auto stream_of = [&](int i) { return ragged ? pool->s[2 * (i % groups)] : pool->s[lane[i]]; };
  if (ragged) {
    // float64 instances on the groups' main streams ahead of their ragged rounds
    for (int i = 0; i < n; ++i)
      if (!P[i]->mixed) status[i] = sp::solve_fp64_async(P[i], rho[i], phi[i], stream_of(i));
    std::vector<sp::MixedRun> mr(MP.size());
    std::vector<int> ms(MP.size(), SP_OK);
    const int st = sp::ragged_solve(MP.data(), MR.data(), MF.data(), (int)MP.size(), pool->s, ns, mr.data(), ms.data());
    for (size_t k = 0; k < mixed_idx.size(); ++k) {
      runs[mixed_idx[k]] = mr[k];
      status[mixed_idx[k]] = st ? st : ms[k];
    }
    for (size_t k = 0; k < mixed_idx.size(); ++k)
      if (!status[mixed_idx[k]])
        status[mixed_idx[k]] = sp::mixed_finish_issue(P[mixed_idx[k]], phi[mixed_idx[k]], pool->s[0]);
  }
  // round 0: float64 solves and the first low-precision solves, largest first
  for (int k = 0; k < n && !ragged; ++k) {
    const int i = order[k];
    if (P[i]->mixed) {
      // the first correction goes right behind the first solve (see solve_mixed)
      status[i] = sp::mixed_phase_a(P[i], rho[i], phi[i], stream_of(i), runs[i]);
    } else {
      status[i] = sp::solve_fp64_async(P[i], rho[i], phi[i], stream_of(i));
    }
  }
  // refinement rounds
  std::vector<char> more(n, 0);   // corrections queued after phase A (its status copy then stale)
  std::vector<int> active;
  for (int i = 0; i < n && !ragged; ++i)
    if (P[i]->mixed && !status[i]) active.push_back(i);
  while (!active.empty()) {
    for (int k = 0; k < ns; ++k)
      if (cudaStreamSynchronize(pool->s[k]) != cudaSuccess) return SP_ERR_CUDA;
    std::vector<int> next;
    for (int i : active) {
      sp::mixed_decide(P[i], runs[i]);
      if (!runs[i].done && runs[i].iters - 1 < P[i]->max_iter) next.push_back(i);
    }
    for (int i : next) {
      status[i] = sp::mixed_correct(P[i], rho[i], phi[i], stream_of(i));
      if (!status[i]) status[i] = sp::mixed_issue_read(P[i], stream_of(i), runs[i]);
      more[i] = 1;
    }
    active.clear();
    for (int i : next)
      if (!status[i]) active.push_back(i);
  }
  // float-float iterates -> float64 results (not for instances that stopped after phase A
  // with the float64 output written: its status word copy is current)
  for (int i = 0; i < n && !ragged; ++i)
    if (P[i]->mixed && !status[i] && (more[i] || P[i]->phi64_written != phi[i]))
      status[i] = sp::mixed_finish_issue(P[i], phi[i], stream_of(i));
  bool any_mixed = false;
  for (int i = 0; i < n; ++i) any_mixed = any_mixed || P[i]->mixed;
  if (any_mixed)
    for (int k = 0; k < ns; ++k)
      if (cudaStreamSynchronize(pool->s[k]) != cudaSuccess) return SP_ERR_CUDA;
  int first_err = SP_OK;
  for (int i = 0; i < n; ++i) {
    if (P[i]->mixed) {
      if (!status[i]) status[i] = sp::mixed_finish_status(P[i], runs[i], infos ? &infos[i] : nullptr);
      else if (infos) infos[i].status = status[i];
    } else {
      sp::fill_fp64_info(status[i], infos ? &infos[i] : nullptr);
    }
    if (status[i] && !first_err) first_err = status[i];
  }
  // join the pool back into the caller's stream
  for (int k = 0; k < ns; ++k) {
    if (cudaEventRecord(pool->ev[k], pool->s[k]) != cudaSuccess) return SP_ERR_CUDA;
    if (cudaStreamWaitEvent(user, pool->ev[k], 0) != cudaSuccess) return SP_ERR_CUDA;
  }
  return first_err;
}

// ======================================================================== server
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long ticket = 0;
  std::string key;
  std::vector<double> r_if, th_if;
  int nphi = 0, outer_bc = 0, precision = 0, max_iter = 8;
  double G = 1.0, tol = 1e-10;
  const double* rho = nullptr;
  double* phi = nullptr;
  size_t zones = 0;
  size_t io_bytes = 0;
  int status = SP_OK;
  sp_solve_info info{};
  bool done = false;
  Clock::time_point t_submit, t_done;
};

struct Resident {
  sp_plan* master = nullptr;
  size_t table_bytes = 0;
  size_t clone_bytes = 0;   // device memory of one clone beside its workspace (error word)
  size_t ws_bytes = 0;      // the grid's workspace, held by the slot that runs it
  size_t io_bytes = 0;      // the grid's device rho and Phi, held by the slot that runs it
  int active = 0;
  bool creating = false;
  int create_status = SP_OK;
  long long last_used = 0;
  std::vector<sp_plan*> idle;   // clones with a workspace, ready for reuse
};

std::string make_key(const Request& q) {
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
  const int hdr[5] = {(int)q.r_if.size(), (int)q.th_if.size(), q.nphi, q.outer_bc, q.precision};
  put(hdr, sizeof(hdr));
  put(&q.G, sizeof(double));
  put(&q.tol, sizeof(double));
  put(&q.max_iter, sizeof(int));
  put(q.r_if.data(), q.r_if.size() * sizeof(double));
  put(q.th_if.data(), q.th_if.size() * sizeof(double));
  return k;
}

}  // namespace

struct sp_server {
  int device = 0;
  size_t budget = 0;
  int slots = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<long long, Request*> requests;
  std::map<std::string, Resident> resident;
  size_t mem_used = 0, mem_peak = 0;
  long long next_ticket = 1, clock = 0;
  int running = 0, running_peak = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
  // statistics
  std::vector<double> latency_ms;
  double zones_done = 0.0;
  long long completed = 0, failed = 0, evictions = 0;
  bool have_first = false;
  Clock::time_point t_first, t_last;

  void worker(int slot);
  bool evict_for(size_t need);   // caller holds mu
};

bool sp_server::evict_for(size_t need) {
  // idle clones first (their workspaces), least recently used grids first
  while (mem_used + need > budget) {
    auto victim = resident.end();
    for (auto it = resident.begin(); it != resident.end(); ++it) {
      if (it->second.idle.empty()) continue;
      if (victim == resident.end() || it->second.last_used < victim->second.last_used) victim = it;
    }
    if (victim == resident.end()) break;
    sp_plan_destroy(victim->second.idle.back());
    victim->second.idle.pop_back();
    mem_used -= victim->second.clone_bytes;
  }
  // then whole plans nobody uses
  while (mem_used + need > budget) {
    auto victim = resident.end();
    for (auto it = resident.begin(); it != resident.end(); ++it) {
      if (it->second.active || it->second.creating || !it->second.master) continue;
      if (victim == resident.end() || it->second.last_used < victim->second.last_used) victim = it;
    }
    if (victim == resident.end()) return false;
    for (sp_plan* c : victim->second.idle) {
      sp_plan_destroy(c);
      mem_used -= victim->second.clone_bytes;
    }
    sp_plan_destroy(victim->second.master);
    mem_used -= victim->second.table_bytes;
    resident.erase(victim);
    ++evictions;
  }
  return true;
}

void sp_server::worker(int slot) {
  (void)slot;
  cudaSetDevice(device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  double* d_io = nullptr;
  size_t d_io_bytes = 0;
  void* ws = nullptr;        // this slot's workspace
  size_t ws_bytes = 0;
  std::unique_lock<std::mutex> lock(mu);
  while (true) {
    // admit the oldest request whose plan memory fits (or any request when nothing runs)
    Request* q = nullptr;
    size_t reserve = 0;
    cv_work.wait(lock, [&] { return stopping || !queue.empty(); });
    if (queue.empty()) {
      if (stopping) break;
      continue;
    }
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Request* c = *it;
      auto r = resident.find(c->key);
      const bool have = r != resident.end() && r->second.master;
      if (r != resident.end() && r->second.creating) continue;   // another slot builds its plan
      // rough need before the plan exists: tables + workspace of the float64 layout;
      // for a resident grid, a clone if none is idle and this slot's workspace growth
      size_t need = c->io_bytes;
      if (!have) need += 64u << 20;
      else {
        if (r->second.idle.empty()) need += r->second.clone_bytes;
        if (r->second.ws_bytes > ws_bytes) need += r->second.ws_bytes - ws_bytes;
      }
      if (mem_used + need <= budget || evict_for(need) || running == 0) {
        q = c;
        reserve = c->io_bytes;
        queue.erase(it);
        break;
      }
    }
    if (!q) {
      cv_work.wait_for(lock, std::chrono::milliseconds(2));
      continue;
    }
    ++running;
    running_peak = std::max(running_peak, running);
    mem_used += reserve;
    mem_peak = std::max(mem_peak, mem_used);
    // resident plan for this grid (built once, outside the lock)
    Resident& res = resident[q->key];
    while (res.creating) cv_done.wait(lock);
    int st = SP_OK;
    if (!res.master) {
      res.creating = true;
      lock.unlock();
      sp_plan* m = nullptr;
      cudaSetDevice(device);
      st = sp_plan_create(q->r_if.data(), (int)q->r_if.size() - 1, q->th_if.data(), (int)q->th_if.size() - 1,
                          q->nphi, q->outer_bc, q->G, q->precision, q->tol, q->max_iter, s, &m);
      lock.lock();
      res.creating = false;
      if (st == SP_OK) {
        res.master = m;
        const Plan* pm = reinterpret_cast<const Plan*>(m);
        res.table_bytes = sp::plan_table_bytes(*pm);
        res.clone_bytes = 256;
        res.ws_bytes = sp_plan_workspace_bytes(m);
        res.io_bytes = 2 * q->zones * sizeof(double);
        mem_used += res.table_bytes;
        mem_peak = std::max(mem_peak, mem_used);
      }
      cv_done.notify_all();
    }
    sp_plan* plan = nullptr;
    if (st == SP_OK) {
      res.active += 1;
      res.last_used = ++clock;
      if (!res.idle.empty()) {
        plan = res.idle.back();
        res.idle.pop_back();
      } else {
        mem_used += res.clone_bytes;
        mem_peak = std::max(mem_peak, mem_used);
      }
    }
    sp_plan* master = res.master;
    const size_t clone_bytes = res.clone_bytes;
    lock.unlock();
    // ---- run on this slot's stream (a clone replays the phase-A graph it captured for
    // this slot's buffers; a capture that fails leaves that clone launching directly)
    if (st == SP_OK && !plan) st = sp_plan_clone(master, &plan);
    // the plan runs in this slot's workspace (grown to the largest grid the slot has run),
    // so a clone allocates no workspace of its own and reusing one costs a pointer rebind
    if (st == SP_OK) {
      size_t need_ws = sp_plan_workspace_bytes(plan);
      if (need_ws > ws_bytes) {
        // grow once to the largest resident grid's workspace that the budget leaves room
        // for (a free synchronises the device, so repeated growth would stall every slot)
        lock.lock();
        size_t want = need_ws;
        for (const auto& kv : resident) want = std::max(want, kv.second.ws_bytes);
        if (want > need_ws && mem_used - ws_bytes + want > budget) want = need_ws;
        lock.unlock();
        need_ws = want;
        cudaFree(ws);
        ws = nullptr;
        const size_t old = ws_bytes;
        ws_bytes = 0;
        if (cudaMalloc(&ws, need_ws) != cudaSuccess) {
          cudaGetLastError();
          ws = nullptr;
          st = SP_ERR_OOM;
        } else {
          ws_bytes = need_ws;
        }
        lock.lock();
        mem_used = mem_used - old + ws_bytes;
        mem_peak = std::max(mem_peak, mem_used);
        lock.unlock();
      }
      if (st == SP_OK && reinterpret_cast<Plan*>(plan)->ws != ws) st = sp_plan_set_workspace(plan, ws, ws_bytes);
    }
    size_t need_io = 2 * q->zones * sizeof(double);
    if (st == SP_OK && d_io_bytes < need_io) {
      // as the workspace: once to the largest resident grid's (budget permitting)
      lock.lock();
      size_t want = need_io;
      for (const auto& kv : resident) want = std::max(want, kv.second.io_bytes);
      if (want > need_io && mem_used + want > budget) want = need_io;
      lock.unlock();
      need_io = want;
      cudaFree(d_io);
      d_io = nullptr;
      d_io_bytes = 0;
      if (cudaMalloc(&d_io, need_io) != cudaSuccess) {
        cudaGetLastError();
        st = SP_ERR_OOM;
      } else {
        d_io_bytes = need_io;
      }
    }
    sp_solve_info info{};
    if (st == SP_OK) {
      const size_t b = q->zones * sizeof(double);
      double* drho = d_io;
      double* dphi = d_io + q->zones;
      st = cuda_status(cudaMemcpyAsync(drho, q->rho, b, cudaMemcpyHostToDevice, s));
      if (!st) st = sp_solve(plan, drho, dphi, s, &info);
      if (!st) st = cuda_status(cudaMemcpyAsync(q->phi, dphi, b, cudaMemcpyDeviceToHost, s));
      if (!st) st = cuda_status(cudaStreamSynchronize(s));
    }
    lock.lock();
    --running;
    mem_used -= reserve;
    Resident& r2 = resident[q->key];
    if (plan) {
      r2.active -= 1;
      if (st == SP_OK || st == SP_ERR_NOT_CONVERGED) {
        r2.idle.push_back(plan);
      } else {
        sp_plan_destroy(plan);
        mem_used -= clone_bytes;
      }
    } else if (st != SP_OK && r2.master && master) {
      // clone failed: release the reservation made for it
      r2.active -= 1;
      mem_used -= clone_bytes;
    }
    q->status = st;
    q->info = info;
    q->info.status = st;
    q->t_done = Clock::now();
    q->done = true;
    if (st == SP_OK) {
      ++completed;
      latency_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count());
      zones_done += (double)q->zones;
      t_last = q->t_done;
    } else {
      ++failed;
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  mem_used -= ws_bytes;
  lock.unlock();
  cudaFree(d_io);
  cudaFree(ws);
  cudaStreamDestroy(s);
}

extern "C" int sp_server_create(size_t mem_budget_bytes, int slots, sp_server** out) {
  if (!out || slots < 1 || slots > 64 || mem_budget_bytes == 0) return SP_ERR_INVALID_ARG;
  *out = nullptr;
  sp_server* sv = new (std::nothrow) sp_server();
  if (!sv) return SP_ERR_OOM;
  cudaGetDevice(&sv->device);
  sv->budget = mem_budget_bytes;
  sv->slots = slots;
  try {
    for (int k = 0; k < slots; ++k) sv->workers.emplace_back(&sp_server::worker, sv, k);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    delete sv;
    return SP_ERR_OOM;
  }
  *out = sv;
  return SP_OK;
}

extern "C" int sp_server_submit(sp_server* sv, const double* r_interfaces, int nr, const double* theta_interfaces,
                                int ntheta, int nphi, int outer_bc, double G, int precision, double tol, int max_iter,
                                const double* rho_host, double* phi_host, long long* ticket) {
  if (!sv || !r_interfaces || !rho_host || !phi_host || !ticket || nr < 1 || ntheta < 1 || nphi < 1)
    return SP_ERR_INVALID_ARG;
  Request* q = new (std::nothrow) Request();
  if (!q) return SP_ERR_OOM;
  q->r_if.assign(r_interfaces, r_interfaces + nr + 1);
  if (theta_interfaces) {
    q->th_if.assign(theta_interfaces, theta_interfaces + ntheta + 1);
  } else {
    q->th_if.resize(ntheta + 1);
    for (int j = 0; j <= ntheta; ++j) q->th_if[j] = 3.14159265358979323846264338327950288 * j / ntheta;
  }
  q->nphi = nphi;
  q->outer_bc = outer_bc;
  q->precision = precision;
  q->max_iter = max_iter;
  q->G = G;
  q->tol = tol;
  q->rho = rho_host;
  q->phi = phi_host;
  q->zones = (size_t)nr * ntheta * nphi;
  q->io_bytes = 2 * q->zones * sizeof(double);
  q->key = make_key(*q);
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stopping) {
      delete q;
      return SP_ERR_INVALID_ARG;
    }
    q->ticket = sv->next_ticket++;
    if (!sv->have_first) {
      sv->have_first = true;
      sv->t_first = q->t_submit;
    }
    sv->requests[q->ticket] = q;
    sv->queue.push_back(q);
    *ticket = q->ticket;
  }
  sv->cv_work.notify_one();
  return SP_OK;
}

extern "C" int sp_server_wait(sp_server* sv, long long ticket, double timeout_s, sp_solve_info* info) {
  if (!sv) return SP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->requests.find(ticket);
  if (it == sv->requests.end()) return SP_ERR_INVALID_ARG;
  Request* q = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (!q->done) {
    if (timeout_s >= 0 && sv->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && !q->done)
      return SP_ERR_TIMEOUT;
    if (timeout_s < 0) sv->cv_done.wait(lock);
  }
  const int st = q->status;
  if (info) *info = q->info;
  sv->requests.erase(it);
  delete q;
  return st;
}

extern "C" int sp_server_stats(sp_server* sv, sp_server_stats_t* out) {
  if (!sv || !out) return SP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = sv->completed;
  out->failed = sv->failed;
  out->queued = (long long)sv->queue.size();
  out->running_peak = sv->running_peak;
  out->resident_plans = (int)sv->resident.size();
  out->evictions = sv->evictions;
  out->mem_peak_bytes = (double)sv->mem_peak;
  if (!sv->latency_ms.empty()) {
    std::vector<double> l(sv->latency_ms);
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
      const double pos = q * (double)(l.size() - 1);
      const size_t a = (size_t)pos;
      const size_t b = std::min(a + 1, l.size() - 1);
      return l[a] + (pos - (double)a) * (l[b] - l[a]);
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = l.back();
    const double span = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
    out->zones_per_s = span > 0 ? sv->zones_done / span : 0.0;
  }
  return SP_OK;
}

extern "C" int sp_server_reset_stats(sp_server* sv) {
  if (!sv) return SP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  sv->latency_ms.clear();
  sv->zones_done = 0.0;
  sv->completed = sv->failed = 0;
  sv->running_peak = sv->running;
  sv->have_first = false;
  return SP_OK;
}

extern "C" int sp_server_destroy(sp_server* sv) {
  if (!sv) return SP_OK;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stopping = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers) t.join();
  DeviceScope dev(sv->device);
  for (auto& kv : sv->resident) {
    for (sp_plan* c : kv.second.idle) sp_plan_destroy(c);
    if (kv.second.master) sp_plan_destroy(kv.second.master);
  }
  for (auto& kv : sv->requests) delete kv.second;
  delete sv;
  return SP_OK;
}
