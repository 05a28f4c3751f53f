// A request server for CDR solves: continuous batching of transient requests,
// concurrent stationary solves, admission by a device-memory budget.
//
// Threads.
//  * admission (`builders` threads): take submitted requests in arrival order,
//    each as soon as the budget and the slot count allow one more, build its
//    problem (mesh, coefficients, Dirichlet data, assembly, initial data) on the
//    request's own stream, and hand it to the stepper (transient) or to the
//    stationary queue.  Several requests build at once, so that requests that
//    arrive close together reach the stepper close together and join one batch.
//  * stepper: keeps every admitted transient request resident on the device and
//    advances all of them together, one batched SSP step sequence (a "chunk" of
//    at most max_chunk steps) at a time, on a stream of the highest priority;
//    requests admitted meanwhile join at the next chunk boundary, finished ones
//    leave (their solution is copied to the host and their device memory released).
//  * stationary workers: each runs one damped fixed-point solve at a time on the
//    request's own stream, so several solves and the transient batch overlap on
//    the device.
//  * serial mode (the plain baseline): one worker runs the requests one at a
//    time in arrival order, each step through afc_step, with nothing overlapped.
//
// Every request is solved by the same library calls it would use alone (the
// batched step gives an instance the same bits as afc_step), so its result does
// not depend on what else is running.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "afc_internal.h"

struct afc_server_s;

namespace afc {

int batch_create_on_stream(const afc_problem* list, int count, cudaStream_t stream, afc_batch* out);

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  afc_request spec{};                         // pointers below replace the caller's
  std::vector<double> b, f, u_dir, u0;
  std::vector<uint8_t> mask;
  int64_t N = 0;
  int64_t bytes = 0;                          // reserved device memory
  int state = AFC_REQ_PENDING;
  int status = AFC_OK;
  afc_stats stats{};
  std::vector<double> u;                      // result
  std::string message;                        // error detail of a failed request
  double t_submit = 0, t_admit = 0, t_done = 0;
  bool cancel = false;
  // while admitted
  afc_problem p = nullptr;
  cudaStream_t stream = nullptr;
  double dt = 0.0;
  int steps_left = 0;
};

using ReqPtr = std::shared_ptr<Request>;

int64_t nodes_of(const afc_request& r) { return (int64_t)r.n[0] * r.n[1] * r.n[2]; }

}  // namespace
}  // namespace afc

struct afc_server_s {
  afc_serve_config cfg{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_admit;      // pending requests or freed budget
  std::condition_variable cv_step;       // transient arrivals
  std::condition_variable cv_stat;       // stationary arrivals
  std::condition_variable cv_done;       // completions
  bool stop = false;
  int64_t next_id = 1;
  std::deque<afc::ReqPtr> pending;
  std::vector<afc::ReqPtr> arrivals;     // admitted transient requests not yet in the batch
  std::deque<afc::ReqPtr> stat_queue;    // admitted stationary requests
  std::map<int64_t, afc::ReqPtr> all;    // every request not yet released
  int active = 0;                        // admitted and not finished
  int64_t bytes_in_use = 0;
  int64_t completed = 0, failed = 0, chunks = 0, batched_steps = 0, instance_steps = 0;
  int64_t max_batch = 0;
  std::vector<std::thread> threads;
};

namespace afc {
namespace {

double now_s(afc_server_s* s) { return std::chrono::duration<double>(Clock::now() - s->t0).count(); }

// Device bytes a request holds while admitted: the arrays of one problem of
// `elem` with N nodes (mesh, coefficients, the K-diagonal matrices, edge data,
// node vectors) plus the Krylov workspace of a stationary solve, with 10 % margin.
int64_t estimate_bytes(int elem, int64_t N, int kind, int precision, int restart) {
  const int64_t K = elem == AFC_P1 ? 15 : 27, Kup = K / 2;
  const int64_t per_cell_ints = elem == AFC_P1 ? 24 : 8;   // connectivity per node (one cell per node)
  double b = 0;
  b += N * (24.0 + 8.0 + 4.0 + 8.0 * per_cell_ints);        // xyz, mask, inc_ptr, conn + incidences
  b += N * (24.0 + 8.0 + 1.0 + 8.0);                         // b, f, Dirichlet mask and values
  b += N * 8.0 * K * 6.0;                                    // M, S, K, A, AA, stationary system
  b += N * 8.0 * Kup * 3.0;                                  // m_ij, d_ij, r_ij
  b += N * 8.0 * 32.0;                                       // node vectors
  if (kind == AFC_REQ_STATIONARY) {
    b += N * (8.0 * Kup * 3.0 + 8.0 * K + 4.0 + 12.0 * Kup + 16.0);   // MC pair data, unlimited operator
    b += N * (precision == AFC_MIXED ? 4.0 : 8.0) * (restart + 8.0); // GMRES basis and work vectors
    if (precision == AFC_MIXED) b += N * (4.0 * K + 4.0);
  } else if (precision == AFC_MIXED) {
    b += N * (4.0 * Kup * 3.0 + 8.0);                        // single-precision edge data and node copies
  }
  return (int64_t)(b * 1.1) + (1 << 20);
}

int64_t estimate_of(const afc_request& r) {
  return estimate_bytes(r.elem, nodes_of(r), r.kind, r.opts.precision, r.opts.gmres_restart);
}

void finish(afc_server_s* s, const ReqPtr& r, int state, int status) {
  // called without the lock, on the thread whose call failed (the error detail is per thread);
  // releases the device resources of the request
  if (state == AFC_REQ_FAILED) r->message = afc_last_error();
  if (r->p) {
    if (state == AFC_REQ_DONE) {
      r->u.resize(r->N);
      int st = afc_get_solution(r->p, r->u.data(), 0);
      if (st < 0) {
        state = AFC_REQ_FAILED;
        status = st;
      }
    }
    afc_destroy(r->p);
    r->p = nullptr;
  }
  if (r->stream) {
    cudaStreamDestroy(r->stream);
    r->stream = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  r->state = r->cancel && state != AFC_REQ_FAILED ? AFC_REQ_CANCELLED : state;
  r->status = status;
  r->t_done = now_s(s);
  s->bytes_in_use -= r->bytes;
  s->active--;
  if (r->state == AFC_REQ_DONE) s->completed++;
  else if (r->state == AFC_REQ_FAILED) s->failed++;
  s->cv_admit.notify_all();
  s->cv_done.notify_all();
}

// Mesh, coefficients, Dirichlet data, assembly and initial data of a request.
int build_problem(afc_server_s* s, Request& r) {
  if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "cudaStreamCreateWithFlags");
  const afc_request& q = r.spec;
  int st;
  if ((st = afc_create_structured(q.elem, q.n[0], q.n[1], q.n[2], q.lo, q.hi, s->device, r.stream, &r.p))) return st;
  if ((st = afc_set_coefficients(r.p, q.eps, r.b.data(), nullptr, nullptr, q.c, r.f.empty() ? nullptr : r.f.data())))
    return st;
  if ((st = afc_set_dirichlet(r.p, r.mask.data(), r.u_dir.data()))) return st;
  if ((st = afc_assemble(r.p, q.family, q.opts.precision))) return st;
  if ((st = afc_set_solution(r.p, r.u0.data(), 0))) return st;
  if (q.kind == AFC_REQ_TRANSIENT) {
    r.dt = q.opts.dt;
    if (!(r.dt > 0.0) && (st = afc_cfl_timestep(r.p, q.cfl, &r.dt))) return st;
    r.steps_left = q.steps;
  }
  AFC_CUDA(cudaStreamSynchronize(r.stream));
  return AFC_OK;
}

void admission_loop(afc_server_s* s) {
  cudaSetDevice(s->device);
  for (;;) {
    ReqPtr r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        // drop cancelled requests at the head
        while (!s->pending.empty() && s->pending.front()->cancel) {
          auto c = s->pending.front();
          s->pending.pop_front();
          c->state = AFC_REQ_CANCELLED;
          c->t_done = now_s(s);
          s->cv_done.notify_all();
        }
        if (!s->pending.empty()) {
          auto& h = s->pending.front();
          const bool fits = s->bytes_in_use + h->bytes <= s->cfg.hbm_budget && s->active < s->cfg.max_active;
          if (fits) {
            r = h;
            s->pending.pop_front();
            s->bytes_in_use += r->bytes;
            s->active++;
            r->state = AFC_REQ_RUNNING;
            r->t_admit = now_s(s);
            break;
          }
        }
        s->cv_admit.wait(lk);
      }
    }
    int st = r->cancel ? AFC_OK : build_problem(s, *r);
    if (st || r->cancel) {
      finish(s, r, st ? AFC_REQ_FAILED : AFC_REQ_CANCELLED, st);
      continue;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->spec.kind == AFC_REQ_TRANSIENT) {
      s->arrivals.push_back(r);
      s->cv_step.notify_all();
    } else {
      s->stat_queue.push_back(r);
      s->cv_stat.notify_all();
    }
  }
}

void stationary_loop(afc_server_s* s) {
  cudaSetDevice(s->device);
  for (;;) {
    ReqPtr r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_stat.wait(lk, [&] { return s->stop || !s->stat_queue.empty(); });
      if (s->stop) return;
      r = s->stat_queue.front();
      s->stat_queue.pop_front();
    }
    int st = AFC_OK;
    if (!r->cancel) st = afc_solve_stationary(r->p, &r->spec.opts, &r->stats);
    finish(s, r, st < 0 ? AFC_REQ_FAILED : AFC_REQ_DONE, st);
  }
}

// Transient requests grouped by the options a batched step shares.
struct Group {
  std::vector<ReqPtr> members;
  afc_batch batch = nullptr;
  bool dirty = true;
};

std::string group_key(const afc_request& q) {
  return std::to_string(q.opts.scheme) + "/" + std::to_string(q.opts.limiter) + "/" +
         std::to_string(q.opts.precision);
}

void stepper_loop(afc_server_s* s) {
  cudaSetDevice(s->device);
  // The batch runs at the highest stream priority: a chunk of batched steps is short
  // work that many requests wait on, so its kernels go ahead of the long stationary
  // solves (on default-priority streams) whenever both are queued on the device.
  cudaStream_t ws = nullptr;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
      cudaStreamCreateWithPriority(&ws, cudaStreamNonBlocking, greatest) != cudaSuccess)
    cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
  std::map<std::string, Group> groups;
  std::vector<afc_stats> stats;
  std::vector<double> dts;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      bool any = false;
      for (auto& kv : groups) any = any || !kv.second.members.empty();
      if (!any) s->cv_step.wait(lk, [&] { return s->stop || !s->arrivals.empty(); });
      if (s->stop) break;
      for (auto& r : s->arrivals) {
        Group& g = groups[group_key(r->spec)];
        g.members.push_back(r);
        g.dirty = true;
      }
      s->arrivals.clear();
    }
    for (auto& kv : groups) {
      Group& g = kv.second;
      // cancelled members leave before the chunk
      for (size_t q = 0; q < g.members.size();) {
        if (g.members[q]->cancel) {
          finish(s, g.members[q], AFC_REQ_CANCELLED, AFC_OK);
          g.members.erase(g.members.begin() + q);
          g.dirty = true;
        } else {
          ++q;
        }
      }
      if (g.members.empty()) {
        if (g.batch) afc_batch_destroy(g.batch);
        g.batch = nullptr;
        continue;
      }
      if (g.dirty) {
        if (g.batch) afc_batch_destroy(g.batch);
        g.batch = nullptr;
        std::vector<afc_problem> list;
        for (auto& r : g.members) list.push_back(r->p);
        int st = batch_create_on_stream(list.data(), (int)list.size(), ws, &g.batch);
        if (st) {
          for (auto& r : g.members) finish(s, r, AFC_REQ_FAILED, st);
          g.members.clear();
          continue;
        }
        g.dirty = false;
        std::lock_guard<std::mutex> lk(s->mu);
        s->max_batch = std::max<int64_t>(s->max_batch, (int64_t)list.size());
      }
      int chunk = s->cfg.max_chunk;
      for (auto& r : g.members) chunk = std::min(chunk, r->steps_left);
      dts.resize(g.members.size());
      stats.resize(g.members.size());
      for (size_t q = 0; q < g.members.size(); ++q) dts[q] = g.members[q]->dt;
      int st = chunk > 0 ? afc_batch_step(g.batch, &g.members[0]->spec.opts, dts.data(), chunk, stats.data()) : AFC_OK;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->chunks++;
        s->batched_steps += chunk;
        s->instance_steps += chunk * (int64_t)g.members.size();
      }
      std::vector<ReqPtr> keep;
      for (size_t q = 0; q < g.members.size(); ++q) {
        auto& r = g.members[q];
        r->steps_left -= chunk;
        if (st < 0) {
          finish(s, r, AFC_REQ_FAILED, st);
        } else if (r->steps_left <= 0) {
          r->stats.stages += stats[q].stages;
          r->stats.dmp_violation = std::max(r->stats.dmp_violation, stats[q].dmp_violation);
          r->stats.umin = stats[q].umin;
          r->stats.umax = stats[q].umax;
          r->stats.status = AFC_OK;
          finish(s, r, AFC_REQ_DONE, AFC_OK);
        } else {
          r->stats.stages += stats[q].stages;
          r->stats.dmp_violation = std::max(r->stats.dmp_violation, stats[q].dmp_violation);
          keep.push_back(r);
        }
      }
      if (keep.size() != g.members.size()) g.dirty = true;
      g.members.swap(keep);
    }
  }
  for (auto& kv : groups) {
    if (kv.second.batch) afc_batch_destroy(kv.second.batch);
    for (auto& r : kv.second.members) finish(s, r, AFC_REQ_CANCELLED, AFC_OK);
  }
  if (ws) cudaStreamDestroy(ws);
}

// Serial baseline: one request at a time, in arrival order, nothing overlapped.
void serial_loop(afc_server_s* s) {
  cudaSetDevice(s->device);
  for (;;) {
    ReqPtr r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_admit.wait(lk, [&] { return s->stop || !s->pending.empty(); });
      if (s->stop) return;
      r = s->pending.front();
      s->pending.pop_front();
      if (r->cancel) {
        r->state = AFC_REQ_CANCELLED;
        r->t_done = now_s(s);
        s->cv_done.notify_all();
        continue;
      }
      s->bytes_in_use += r->bytes;
      s->active++;
      r->state = AFC_REQ_RUNNING;
      r->t_admit = now_s(s);
    }
    int st = build_problem(s, *r);
    if (!st) {
      if (r->spec.kind == AFC_REQ_STATIONARY) {
        st = afc_solve_stationary(r->p, &r->spec.opts, &r->stats);
      } else {
        afc_opts o = r->spec.opts;
        o.dt = r->dt;
        afc_stats one{};
        for (int k = 0; k < r->spec.steps && st >= 0; ++k) {
          st = afc_step(r->p, &o, &one);
          r->stats.stages += one.stages;
          r->stats.dmp_violation = std::max(r->stats.dmp_violation, one.dmp_violation);
        }
        r->stats.umin = one.umin;
        r->stats.umax = one.umax;
        r->stats.status = st;
      }
    }
    finish(s, r, st < 0 ? AFC_REQ_FAILED : AFC_REQ_DONE, st);
  }
}

int check_request(const afc_request* r) {
  if (!r) { set_error("null request"); return AFC_E_INVALID; }
  if (r->kind != AFC_REQ_TRANSIENT && r->kind != AFC_REQ_STATIONARY) { set_error("bad request kind"); return AFC_E_INVALID; }
  if (r->elem != AFC_P1 && r->elem != AFC_Q1) { set_error("bad element type"); return AFC_E_INVALID; }
  if (r->n[0] < 2 || r->n[1] < 2 || r->n[2] < 2) { set_error("need >= 2 nodes per side"); return AFC_E_INVALID; }
  if (!r->b || !r->dir_mask || !r->u_dir || !r->u0) { set_error("request needs b, dir_mask, u_dir and u0"); return AFC_E_INVALID; }
  if (r->kind == AFC_REQ_TRANSIENT) {
    if (r->opts.scheme != AFC_SSP2 && r->opts.scheme != AFC_SSP3) {
      set_error("transient requests run AFC_SSP2 / AFC_SSP3");
      return AFC_E_INVALID;
    }
    if (r->steps < 0 || (!(r->opts.dt > 0.0) && !(r->cfl > 0.0))) {
      set_error("transient requests need steps >= 0 and opts.dt > 0 or cfl > 0");
      return AFC_E_INVALID;
    }
  }
  if (r->family != AFC_FAMILY_FCT && r->family != AFC_FAMILY_MC) { set_error("bad family"); return AFC_E_INVALID; }
  return AFC_OK;
}

}  // namespace
}  // namespace afc

using namespace afc;

extern "C" void afc_serve_default_config(afc_serve_config* c) {
  if (!c) return;
  c->mode = AFC_SERVE_BATCHED;
  c->max_active = 512;
  c->hbm_budget = (int64_t)64 << 30;
  c->stationary_workers = 4;
  c->max_chunk = 10;
  c->builders = 4;
}

extern "C" int64_t afc_serve_estimate_bytes(const afc_request* r) {
  if (!r) return -1;
  return estimate_of(*r);
}

extern "C" int afc_serve_create(int device, const afc_serve_config* cfg, afc_server* out) {
  if (!out) { set_error("null argument"); return AFC_E_INVALID; }
  *out = nullptr;
  afc_serve_config c;
  afc_serve_default_config(&c);
  if (cfg) c = *cfg;
  if ((c.mode != AFC_SERVE_BATCHED && c.mode != AFC_SERVE_SERIAL) || c.max_active < 1 || c.hbm_budget <= 0 ||
      c.stationary_workers < 1 || c.stationary_workers > 64 || c.max_chunk < 1 || c.builders < 1 ||
      c.builders > 64) {
    set_error("bad server configuration");
    return AFC_E_INVALID;
  }
  if (cudaSetDevice(device) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
  afc_server_s* s = new afc_server_s();
  s->cfg = c;
  s->device = device;
  s->t0 = Clock::now();
  if (c.mode == AFC_SERVE_SERIAL) {
    s->threads.emplace_back(serial_loop, s);
  } else {
    for (int w = 0; w < c.builders; ++w) s->threads.emplace_back(admission_loop, s);
    s->threads.emplace_back(stepper_loop, s);
    for (int w = 0; w < c.stationary_workers; ++w) s->threads.emplace_back(stationary_loop, s);
  }
  *out = s;
  return AFC_OK;
}

extern "C" int afc_serve_submit(afc_server s, const afc_request* r, int64_t* id) {
  if (!s || !id) { set_error("null argument"); return AFC_E_INVALID; }
  int st = check_request(r);
  if (st) return st;
  auto q = std::make_shared<Request>();
  q->spec = *r;
  q->N = nodes_of(*r);
  q->bytes = estimate_of(*r);
  if (q->bytes > s->cfg.hbm_budget) {
    set_error("request needs more device memory than the server's budget");
    return AFC_E_INVALID;
  }
  q->b.assign(r->b, r->b + 3 * q->N);
  if (r->f) q->f.assign(r->f, r->f + q->N);
  q->mask.assign(r->dir_mask, r->dir_mask + q->N);
  q->u_dir.assign(r->u_dir, r->u_dir + q->N);
  q->u0.assign(r->u0, r->u0 + q->N);
  q->spec.b = nullptr;
  q->spec.f = nullptr;
  q->spec.dir_mask = nullptr;
  q->spec.u_dir = nullptr;
  q->spec.u0 = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) { set_error("server is shutting down"); return AFC_E_STATE; }
  q->id = s->next_id++;
  q->t_submit = now_s(s);
  s->pending.push_back(q);
  s->all[q->id] = q;
  *id = q->id;
  s->cv_admit.notify_all();
  return AFC_OK;
}

namespace afc {
namespace {
void fill_result(const Request& r, afc_result* res, double* u_out) {
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->state = r.state;
    res->status = r.status;
    res->stats = r.stats;
    res->n_nodes = r.N;
    res->t_submit = r.t_submit;
    res->t_admit = r.t_admit;
    res->t_done = r.t_done;
    std::snprintf(res->message, sizeof res->message, "%s", r.message.c_str());
  }
  if (u_out && r.state == AFC_REQ_DONE && (int64_t)r.u.size() == r.N) std::memcpy(u_out, r.u.data(), r.N * sizeof(double));
}
}  // namespace
}  // namespace afc

extern "C" int afc_serve_poll(afc_server s, int64_t id, afc_result* res, double* u_out) {
  if (!s) { set_error("null server"); return AFC_E_INVALID; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) { set_error("unknown request id"); return AFC_E_INVALID; }
  fill_result(*it->second, res, u_out);
  return AFC_OK;
}

extern "C" int afc_serve_wait(afc_server s, int64_t id, double timeout_s, afc_result* res, double* u_out) {
  if (!s) { set_error("null server"); return AFC_E_INVALID; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) { set_error("unknown request id"); return AFC_E_INVALID; }
  ReqPtr r = it->second;
  auto done = [&] { return r->state != AFC_REQ_PENDING && r->state != AFC_REQ_RUNNING; };
  bool ok = timeout_s < 0 ? (s->cv_done.wait(lk, done), true)
                          : s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
  fill_result(*r, res, u_out);
  if (!ok) { set_error("request not finished within the timeout"); return AFC_E_TIMEOUT; }
  return AFC_OK;
}

extern "C" int afc_serve_cancel(afc_server s, int64_t id) {
  if (!s) { set_error("null server"); return AFC_E_INVALID; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) { set_error("unknown request id"); return AFC_E_INVALID; }
  it->second->cancel = true;
  s->cv_admit.notify_all();
  return AFC_OK;
}

extern "C" int afc_serve_release(afc_server s, int64_t id) {
  if (!s) { set_error("null server"); return AFC_E_INVALID; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) { set_error("unknown request id"); return AFC_E_INVALID; }
  const int st = it->second->state;
  if (st == AFC_REQ_PENDING || st == AFC_REQ_RUNNING) { set_error("request still in flight"); return AFC_E_STATE; }
  s->all.erase(it);
  return AFC_OK;
}

extern "C" int afc_serve_get_info(afc_server s, afc_serve_info* out) {
  if (!s || !out) { set_error("null argument"); return AFC_E_INVALID; }
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->pending = (int64_t)s->pending.size();
  out->active = s->active;
  out->bytes_in_use = s->bytes_in_use;
  out->completed = s->completed;
  out->failed = s->failed;
  out->chunks = s->chunks;
  out->batched_steps = s->batched_steps;
  out->max_batch = s->max_batch;
  out->instance_steps = s->instance_steps;
  out->clock = now_s(s);
  return AFC_OK;
}

extern "C" int afc_serve_destroy(afc_server s) {
  if (!s) return AFC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& r : s->pending) {
      r->state = AFC_REQ_CANCELLED;
      r->t_done = now_s(s);
    }
    s->pending.clear();
  }
  s->cv_admit.notify_all();
  s->cv_step.notify_all();
  s->cv_stat.notify_all();
  for (auto& t : s->threads) t.join();
  // admitted requests the threads did not reach
  for (auto& r : s->arrivals) finish(s, r, AFC_REQ_CANCELLED, AFC_OK);
  for (auto& r : s->stat_queue) finish(s, r, AFC_REQ_CANCELLED, AFC_OK);
  delete s;
  return AFC_OK;
}
