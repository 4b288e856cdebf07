// Continuous-batching request loop for whole time-marching solves.
//
// A worker thread owns the device side.  Requests wait in a FIFO queue until the device-memory
// budget and the active-slot limit admit them; an admitted request gets its own stream and a
// tau_problem whose Krylov basis and solution stay on the device until its last step.  Every
// pass of the loop harvests finished requests (memory returns to the budget), admits waiting ones,
// and enqueues the next steps of the admitted requests.  Admitted mixed-precision requests of the
// same kind (d, residual precision, initial guess; line-pass routes, which the server selects for
// them) share their steps: one graph whose every kernel is a single launch over all of them
// (tau_batch's grouped execution), rebuilt when the set changes, each launch advancing every
// member by one step whatever step it stands at.  Other requests step on their own streams.
// Requests that arrive while others run join the next group or overlap on the GPU.  A request's
// last enqueued work is marked by its event, on whichever stream it ran, and every stream waits
// for a request's event before stepping it.  Host-side waits are bounded (condition variable with
// a timeout); the device is never polled in a spin loop.
#include "tau_rsfde.h"
#include "tau_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace tau {
struct GroupExec;
int64_t problem_group_key(const tau_problem* p);
tau_status group_exec_create(tau_problem* const* ps, int n, GroupExec** out, void** pool, size_t* pool_cap);
tau_status group_exec_launch(GroupExec* g, int64_t count, cudaStream_t st);
void group_exec_destroy(GroupExec* g);
}  // namespace tau

namespace {

using Clock = std::chrono::steady_clock;

// A group of admitted requests stepping together, its stream, and the event of its last launch.
struct Group {
  tau::GroupExec* ge = nullptr;
  std::vector<int64_t> ids;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  void* tables = nullptr;   // argument tables of the group's launches, reused across rebuilds
  size_t tables_cap = 0;
};

// Requests up to this many unknowns share launches: below it a request's own kernels leave much of
// the GPU idle (launch- and latency-bound); above it they fill the GPU by themselves.
constexpr int64_t GROUP_MAX_UNKNOWNS = (int64_t)1 << 20;

struct Req {
  int64_t id = 0;
  tau_problem_desc desc{};
  int re = 0, rf = 0, rp = 0;
  std::vector<double> e_tc, f_tc, psi_tc;
  std::vector<double> e_sp[3], f_sp[3], psi_sp[3];
  int64_t n_tot = 1, bytes_est = 0, bytes = 0;
  int state = TAU_REQ_QUEUED;
  tau_status status = TAU_OK;
  std::string msg;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  tau_problem* p = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  int64_t launched = 0;
  int64_t iters = 0;
  std::vector<double> result;
};

}  // namespace

struct tau_server {
  int64_t budget = 0;
  int max_active = 0;
  int chunk = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Req>> queue;
  std::vector<std::shared_ptr<Req>> active;
  std::unordered_map<int64_t, std::shared_ptr<Req>> all;
  std::vector<double> latencies;
  int64_t next_id = 1;
  int64_t used = 0;
  int64_t completed = 0, failed = 0;
  double unk_steps = 0, t_first = -1, t_last = 0;
  Clock::time_point t0;
  std::atomic<bool> stop{false};
  std::thread worker;
  std::map<int64_t, Group> groups;   // by group key (worker thread only)
  bool grouping = true;              // TAU_BATCH_GROUPS=0 at creation: every request steps alone
  int64_t group_launches = 0, group_rebuilds = 0, group_steps = 0;
};

namespace {

double now_s(const tau_server* s) {
  return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

// Device bytes a request will hold (Krylov basis and work vectors), known before tau_create.
int64_t estimate_bytes(const tau_problem_desc& d, int64_t n) {
  // d = 1: the long-line route's tables and scratch (length F = 2 K_T, up to ~128 F bytes with
  // the copies in the other element types and the setup's staging buffer)
  int64_t lng = 0;
  if (d.d == 1) {
    int64_t kt = 2;
    while (kt < n + 1) kt <<= 1;
    lng = 128 * 2 * kt;
  }
  if (d.precision == TAU_MIXED) {
    const int64_t k = d.inner_max_iter > 0 ? d.inner_max_iter : 30;
    return (2 * k + 4) * n * 4 + 12 * n * 8 + lng + (1 << 20);
  }
  // two-sided: two more vectors (the sine-basis diagonals of P^{-1/2} and P^{-1/2} B^{-1})
  return ((int64_t)d.max_iter + 11 + (d.method != TAU_OPGM ? 2 : 0)) * n * 8 + lng + (1 << 20);
}

void finish(tau_server* s, const std::shared_ptr<Req>& r, tau_status st, const char* msg) {
  r->status = st;
  if (msg) r->msg = msg;
  r->state = st == TAU_OK || st == TAU_ENOTCONV ? TAU_REQ_DONE : TAU_REQ_FAILED;
  r->t_finish = now_s(s);
  if (r->p) {
    tau_destroy(r->p);
    r->p = nullptr;
  }
  if (r->ev) cudaEventDestroy(r->ev);
  if (r->st) cudaStreamDestroy(r->st);
  r->ev = nullptr;
  r->st = nullptr;
  r->e_tc.clear();
  r->f_tc.clear();
  for (int i = 0; i < 3; ++i) {
    r->e_sp[i].clear();
    r->f_sp[i].clear();
    r->psi_sp[i].clear();
  }
}

// Create, fill and set up the request's problem on its own stream (worker thread).  Mixed-precision
// requests run their inner solve on the line passes (TAU_TC_OFF), whose kernels can be grouped.
tau_status admit(const std::shared_ptr<Req>& r) {
  if (r->desc.precision == TAU_MIXED) r->desc.tc = TAU_TC_OFF;
  // admission runs on the worker thread, between the launches that keep the GPU busy: no timing
  // runs unless the request asks for them; recorded choices still apply
  if (r->desc.autotune == TAU_TUNE_AUTO) r->desc.autotune = TAU_TUNE_RECORDED;
  if (cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess)
    return TAU_ECUDA;
  tau_status st = tau_create(&r->desc, r->st, &r->p);
  if (st != TAU_OK) return st;
  tau_field fe{}, ff{}, fp{};
  fe.rank = r->re;
  fe.n_times = r->desc.M;
  fe.time_coef = r->e_tc.data();
  ff.rank = r->rf;
  ff.n_times = r->desc.M;
  ff.time_coef = r->f_tc.data();
  fp.rank = r->rp;
  fp.n_times = 1;
  fp.time_coef = r->psi_tc.data();
  for (int i = 0; i < r->desc.d; ++i) {
    fe.space[i] = r->e_sp[i].data();
    ff.space[i] = r->f_sp[i].data();
    fp.space[i] = r->psi_sp[i].data();
  }
  st = tau_set_fields(r->p, &fe, &ff, &fp);
  if (st != TAU_OK) return st;
  st = tau_setup(r->p);
  if (st != TAU_OK) return st;
  tau_stats ss{};
  tau_get_stats(r->p, &ss);
  r->bytes = ss.device_bytes;
  return TAU_OK;
}

void worker_loop(tau_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    bool progress = false;
    // 1. harvest requests whose last step completed
    std::vector<std::shared_ptr<Req>> act;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      act = s->active;
    }
    for (auto& r : act) {
      if (r->launched < r->desc.M || cudaEventQuery(r->ev) != cudaSuccess) continue;
      tau_stats ss{};
      tau_status st = tau_get_stats(r->p, &ss);
      r->iters = ss.total_iters;
      r->result.resize((size_t)r->n_tot);
      tau_status st2 = tau_get_solution(r->p, r->result.data(), 0, nullptr);
      if (st2 != TAU_OK) st = st2;
      std::lock_guard<std::mutex> lk(s->mu);
      finish(s, r, st, st == TAU_OK ? nullptr : tau_last_error());
      s->used -= r->bytes_est;
      s->active.erase(std::find(s->active.begin(), s->active.end(), r));
      if (r->state == TAU_REQ_DONE) {
        s->completed++;
        s->latencies.push_back(r->t_finish - r->t_submit);
        s->unk_steps += (double)r->n_tot * (double)r->desc.M;
        s->t_last = std::max(s->t_last, r->t_finish);
      } else {
        s->failed++;
      }
      s->cv.notify_all();
      progress = true;
    }
    // 2. admit by device memory and slot count
    while (true) {
      std::shared_ptr<Req> r;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->queue.empty() || (int)s->active.size() >= s->max_active) break;
        if (s->used + s->queue.front()->bytes_est > s->budget) break;
        r = s->queue.front();
        s->queue.pop_front();
        s->used += r->bytes_est;
        r->state = TAU_REQ_RUNNING;
        r->t_admit = now_s(s);
      }
      tau_status st = admit(r);
      std::lock_guard<std::mutex> lk(s->mu);
      if (st != TAU_OK) {
        finish(s, r, st, tau_last_error());
        s->used -= r->bytes_est;
        s->failed++;
        s->cv.notify_all();
      } else {
        s->active.push_back(r);
      }
      progress = true;
    }
    // 3. steps: groups of mixed requests share launches; the others step on their own streams
    {
      std::lock_guard<std::mutex> lk(s->mu);
      act = s->active;
    }
    std::map<int64_t, std::vector<std::shared_ptr<Req>>> members;
    std::vector<std::shared_ptr<Req>> alone;
    for (auto& r : act) {
      if (r->launched >= r->desc.M) continue;
      const int64_t key = s->grouping && r->n_tot <= GROUP_MAX_UNKNOWNS ? tau::problem_group_key(r->p) : -1;
      if (key >= 0) members[key].push_back(r);
      else alone.push_back(r);
    }
    for (auto& kv : members)
      if (kv.second.size() < 2) {
        alone.push_back(kv.second[0]);
        kv.second.clear();
      }
    auto fail_req = [&](const std::shared_ptr<Req>& r, tau_status st) {
      std::lock_guard<std::mutex> lk(s->mu);
      finish(s, r, st, tau_last_error());
      s->used -= r->bytes_est;
      s->failed++;
      s->active.erase(std::find(s->active.begin(), s->active.end(), r));
      s->cv.notify_all();
    };
    for (auto& kv : s->groups) {   // groups whose launches completed
      Group& G = kv.second;
      if (G.busy && cudaEventQuery(G.ev) == cudaSuccess) G.busy = false;
    }
    for (auto& kv : members) {
      auto& mem = kv.second;
      if (mem.empty()) continue;
      Group& G = s->groups[kv.first];
      if (G.busy) continue;   // its last launch is still running
      std::vector<int64_t> ids;
      for (auto& r : mem) ids.push_back(r->id);
      if (ids != G.ids || !G.ge) {   // the set changed: a new graph for the new set
        tau::group_exec_destroy(G.ge);
        G.ge = nullptr;
        G.ids.clear();
        if (!G.st && (cudaStreamCreateWithFlags(&G.st, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming) != cudaSuccess)) {
          for (auto& r : mem) fail_req(r, TAU_ECUDA);
          continue;
        }
        std::vector<tau_problem*> ps;
        for (auto& r : mem) ps.push_back(r->p);
        const tau_status st = tau::group_exec_create(ps.data(), (int)ps.size(), &G.ge, &G.tables, &G.tables_cap);
        if (st != TAU_OK) {   // step them alone instead
          for (auto& r : mem) alone.push_back(r);
          continue;
        }
        G.ids = ids;
        s->group_rebuilds++;
      }
      int64_t c = s->chunk;
      for (auto& r : mem) c = std::min<int64_t>(c, r->desc.M - r->launched);
      cudaError_t e = cudaSuccess;
      for (auto& r : mem)
        if (e == cudaSuccess && r->launched > 0) e = cudaStreamWaitEvent(G.st, r->ev, 0);
      tau_status st = e == cudaSuccess ? tau::group_exec_launch(G.ge, c, G.st) : TAU_ECUDA;
      for (auto& r : mem)
        if (st == TAU_OK && cudaEventRecord(r->ev, G.st) != cudaSuccess) st = TAU_ECUDA;
      if (st == TAU_OK && cudaEventRecord(G.ev, G.st) != cudaSuccess) st = TAU_ECUDA;
      if (st != TAU_OK) {
        for (auto& r : mem) fail_req(r, st);
        continue;
      }
      G.busy = true;
      s->group_launches += c;
      s->group_steps += c * (int64_t)mem.size();
      for (auto& r : mem) r->launched += c;
      progress = true;
    }
    for (auto& r : alone) {
      if (r->launched > 0 && cudaEventQuery(r->ev) != cudaSuccess) continue;
      const int64_t c = std::min<int64_t>(s->chunk, r->desc.M - r->launched);
      tau_status st = TAU_OK;
      if (r->launched > 0 && cudaStreamWaitEvent(r->st, r->ev, 0) != cudaSuccess) st = TAU_ECUDA;
      if (st == TAU_OK) st = tau_step(r->p, c);
      if (st == TAU_OK && cudaEventRecord(r->ev, r->st) != cudaSuccess) st = TAU_ECUDA;
      if (st != TAU_OK) {
        fail_req(r, st);
        continue;
      }
      r->launched += c;
      progress = true;
    }
    bool idle;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      idle = s->queue.empty() && s->active.empty();
      if (s->stop && idle) break;
    }
    if (idle)
      for (auto& kv : s->groups) {   // nothing runs: free the groups' graphs
        tau::group_exec_destroy(kv.second.ge);
        kv.second.ge = nullptr;
        kv.second.ids.clear();
        kv.second.busy = false;
      }
    if (!progress) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::microseconds(idle ? 2000 : 50));
    }
  }
}

tau_status sfail(const char* msg) {
  tau::set_last_error(msg);
  return TAU_EINVAL;
}

}  // namespace

extern "C" {

tau_status tau_server_create(int64_t device_bytes_budget, int max_active, int steps_per_launch, tau_server** out) {
  if (!out || device_bytes_budget <= 0 || max_active < 1 || steps_per_launch < 1)
    return sfail("tau_server_create: budget > 0, max_active >= 1 and steps_per_launch >= 1 are required");
  tau_server* s = new (std::nothrow) tau_server();
  if (!s) return TAU_ENOMEM;
  s->budget = device_bytes_budget;
  s->max_active = max_active;
  s->chunk = steps_per_launch;
  s->t0 = Clock::now();
  const char* ge = std::getenv("TAU_BATCH_GROUPS");
  s->grouping = !(ge && ge[0] == '0');
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return sfail("tau_server_create: no CUDA device");
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return TAU_OK;
}

tau_status tau_server_submit(tau_server* s, const tau_problem_desc* desc, const tau_field* e, const tau_field* f,
                             const tau_field* psi, int64_t* id_out) {
  if (!s || !desc || !e || !f || !psi || !id_out) return sfail("tau_server_submit: NULL argument");
  if (desc->d < 1 || desc->d > 3 || desc->M < 1) return sfail("tau_server_submit: bad d or M");
  if (e->n_times != desc->M || f->n_times != desc->M || psi->n_times != 1)
    return sfail("tau_server_submit: n_times must be M for e and f, 1 for psi");
  auto r = std::make_shared<Req>();
  r->desc = *desc;
  r->re = e->rank;
  r->rf = f->rank;
  r->rp = psi->rank;
  r->e_tc.assign(e->time_coef, e->time_coef + (size_t)desc->M * e->rank);
  r->f_tc.assign(f->time_coef, f->time_coef + (size_t)desc->M * f->rank);
  r->psi_tc.assign(psi->time_coef, psi->time_coef + psi->rank);
  for (int i = 0; i < desc->d; ++i) {
    const size_t w = (size_t)desc->n[i] + 2;
    r->e_sp[i].assign(e->space[i], e->space[i] + w * e->rank);
    r->f_sp[i].assign(f->space[i], f->space[i] + w * f->rank);
    r->psi_sp[i].assign(psi->space[i], psi->space[i] + w * psi->rank);
    r->n_tot *= desc->n[i];
  }
  r->bytes_est = estimate_bytes(*desc, r->n_tot);
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  r->t_submit = now_s(s);
  if (s->t_first < 0) s->t_first = r->t_submit;
  s->all[r->id] = r;
  if (r->bytes_est > s->budget) {
    r->state = TAU_REQ_FAILED;
    r->status = TAU_ENOMEM;
    r->msg = "request needs more device memory than the whole budget";
    r->t_finish = r->t_submit;
    s->failed++;
  } else {
    s->queue.push_back(r);
  }
  *id_out = r->id;
  s->cv.notify_all();
  return TAU_OK;
}

static void fill_info(const Req& r, tau_request_info* info) {
  info->id = r.id;
  info->state = r.state;
  info->status = r.status;
  info->t_submit = r.t_submit;
  info->t_admit = r.t_admit;
  info->t_finish = r.t_finish;
  info->unknowns = r.n_tot;
  info->steps = r.desc.M;
  info->gmres_iters = r.iters;
  info->device_bytes = r.bytes;
}

tau_status tau_server_poll(tau_server* s, int64_t id, tau_request_info* info) {
  if (!s || !info) return sfail("tau_server_poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return sfail("tau_server_poll: unknown id");
  fill_info(*it->second, info);
  return TAU_OK;
}

tau_status tau_server_wait(tau_server* s, int64_t id, double timeout_s, tau_request_info* info) {
  if (!s || !info) return sfail("tau_server_wait: NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return sfail("tau_server_wait: unknown id");
  auto r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
  while (r->state == TAU_REQ_QUEUED || r->state == TAU_REQ_RUNNING) {
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout &&
        (r->state == TAU_REQ_QUEUED || r->state == TAU_REQ_RUNNING)) {
      fill_info(*r, info);
      tau::set_last_error("tau_server_wait: timed out");
      return TAU_ETIMEOUT;
    }
  }
  fill_info(*r, info);
  return TAU_OK;
}

tau_status tau_server_result(tau_server* s, int64_t id, double* u_host, int64_t n) {
  if (!s || !u_host) return sfail("tau_server_result: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return sfail("tau_server_result: unknown id");
  Req& r = *it->second;
  if (r.state != TAU_REQ_DONE) {
    tau::set_last_error("tau_server_result: request not finished");
    return TAU_ESTATE;
  }
  if (n != (int64_t)r.result.size()) return sfail("tau_server_result: n differs from the request's unknowns");
  memcpy(u_host, r.result.data(), sizeof(double) * (size_t)n);
  return r.status;
}

tau_status tau_server_release(tau_server* s, int64_t id) {
  if (!s) return sfail("tau_server_release: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return sfail("tau_server_release: unknown id");
  if (it->second->state != TAU_REQ_DONE && it->second->state != TAU_REQ_FAILED) {
    tau::set_last_error("tau_server_release: request still queued or running");
    return TAU_ESTATE;
  }
  s->all.erase(it);
  return TAU_OK;
}

tau_status tau_server_summary(tau_server* s, tau_server_stats* out) {
  if (!s || !out) return sfail("tau_server_summary: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = (int64_t)s->queue.size();
  out->active = (int64_t)s->active.size();
  out->device_bytes_in_use = s->used;
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  if (!l.empty()) {
    auto pct = [&](double q) {
      const double pos = q * (double)(l.size() - 1);
      const size_t i = (size_t)pos;
      const double fr = pos - (double)i;
      return i + 1 < l.size() ? l[i] * (1 - fr) + l[i + 1] * fr : l[i];
    };
    out->latency_p50_s = pct(0.50);
    out->latency_p99_s = pct(0.99);
    double sum = 0;
    for (double v : l) sum += v;
    out->latency_mean_s = sum / (double)l.size();
  }
  out->unknowns_steps = s->unk_steps;
  out->group_launches = s->group_launches;
  out->group_rebuilds = s->group_rebuilds;
  out->group_request_steps = s->group_steps;
  out->span_s = s->t_first >= 0 ? s->t_last - s->t_first : 0.0;
  out->throughput = out->span_s > 0 ? s->unk_steps / out->span_s : 0.0;
  return TAU_OK;
}

tau_status tau_server_destroy(tau_server* s) {
  if (!s) return TAU_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    // queued requests are cancelled; admitted ones run to completion
    for (auto& r : s->queue) {
      r->state = TAU_REQ_FAILED;
      r->status = TAU_ESTATE;
      r->msg = "cancelled: server destroyed";
    }
    s->queue.clear();
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->groups) {
    tau::group_exec_destroy(kv.second.ge);
    if (kv.second.st) cudaStreamSynchronize(kv.second.st);
    if (kv.second.tables) cudaFree(kv.second.tables);
    if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    if (kv.second.st) cudaStreamDestroy(kv.second.st);
  }
  delete s;
  return TAU_OK;
}

}  // extern "C"
