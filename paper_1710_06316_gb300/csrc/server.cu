// server.cu -- continuous-batching solve server (afmpb_server_*).
//
// Requests (a mesh, its charges and the solver parameters) are copied at submission and
// queued.  A fixed set of slot threads, each with its own CUDA stream, admits queued
// requests first-fit in arrival order whenever a slot is idle and the request's device
// memory reservation (afmpb_estimate_bytes) fits under the budget beside the requests
// already running.  An admitted request runs its whole life on its slot's stream: handle
// setup (tree, near field, FMM operators, captured product graph), GMRES solve with the
// Krylov basis on the device, energy, then the handle is freed and its reservation
// returned, which may admit the next request at once.  Requests on different slots
// overlap on the device (their kernels run on separate streams) and on the host (setup
// work runs on the slot threads).  Results are kept until a poll or wait hands them out.
//
// With batching (afmpb_server_create_batched, max_batch > 1) a slot only sets the request
// up; the finished handle (on a stream of its own) joins a ready list, and each of the
// solver threads takes the oldest ready request with the other ready requests of similar
// size (node counts within a factor of two), up to max_batch, into one
// afmpb_solve_batch: their GMRES steps run in lockstep with fused P2P and M2L launches.
// Under light load a batch holds one request; requests that pile up while solves run are
// solved together.  Grouping by size keeps a small request from waiting on a large one's
// steps.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t ticket = 0;
  std::vector<double> xyz, normals, atoms, q;
  std::vector<int32_t> tri;
  int64_t n_nodes = 0, n_tris = 0, n_atoms = 0;
  double eps_in = 1, eps_out = 1, kappa = 0, tol = 1e-6;
  int order = 6;
  afmpb_options opt{};
  double *f_out = nullptr, *h_out = nullptr;
  size_t reserve = 0;
  double t_submit = 0;
};

struct Done {
  afmpb_result res{};
  bool ready = false;
};

// A request whose handle is set up and waits for the batch solver.
struct Ready {
  std::unique_ptr<Job> job;
  afmpb_t *h = nullptr;
  afmpb_result r{};
};

}  // namespace

struct afmpb_server_t {
  size_t budget = 0;
  int max_slots = 0;
  int device = 0;                 // the creator's current device: every slot runs there
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Job>> queue;
  std::unordered_map<int64_t, Done> results;
  std::vector<std::thread> slots;
  int max_batch = 1;              // > 1: slots set up, one solver thread solves in batches
  std::deque<Ready> ready;
  std::condition_variable cv_ready;
  std::vector<std::thread> solvers;
  int setting_up = 0;             // batched: admitted requests still in setup on a slot
  int64_t batches = 0, batched = 0, max_batch_seen = 0;
  bool stop = false;
  int64_t next_ticket = 1;
  size_t in_use = 0, high_water = 0;
  int64_t submitted = 0, completed = 0, failed = 0, running = 0, max_running = 0;
  std::string err;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// First queued job (arrival order) whose reservation fits beside the running ones.
std::unique_ptr<Job> take_admissible(afmpb_server_t *s) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if (s->in_use + (*it)->reserve <= s->budget) {
      std::unique_ptr<Job> j = std::move(*it);
      s->queue.erase(it);
      return j;
    }
  }
  return nullptr;
}

// Handle setup of a request (nullptr with r.status set on failure).
afmpb_t *setup_job(afmpb_server_t *s, Job &j, cudaStream_t stream, afmpb_result &r) {
  afmpb_mesh mesh{j.n_nodes, j.n_tris, j.xyz.data(), j.tri.data(), j.normals.empty() ? nullptr : j.normals.data()};
  afmpb_charges ch{j.n_atoms, j.atoms.data(), j.q.data()};
  afmpb_options opt = j.opt;
  opt.stream = stream;
  afmpb_t *h = nullptr;
  r.status = afmpb_create(&mesh, j.n_atoms > 0 ? &ch : nullptr, j.eps_in, j.eps_out, j.kappa, j.order, j.tol, &opt, &h);
  if (r.status != AFMPB_OK) {
    std::strncpy(r.error, afmpb_last_error(nullptr), sizeof(r.error) - 1);
    return nullptr;
  }
  // Setup is done: shrink the reservation to what the handle holds at its peak, or now
  // plus the GMRES basis and work vectors still to come, whichever is larger.
  afmpb_info pre{};
  if (afmpb_get_info(h, &pre) == AFMPB_OK) {
    const size_t m = (size_t)(opt.restart > 0 ? opt.restart : opt.restart == AFMPB_RESTART_NONE ? AFMPB_RESTART_NONE_MAX : 80);
    const size_t n2 = 2 * (size_t)j.n_nodes;
    const size_t gmres = (m + 1) * n2 * 8 + 16 * n2 * 8 + (16u << 20);
    const size_t need = std::max((size_t)pre.device_bytes_peak, (size_t)pre.device_bytes + gmres);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use = s->in_use - j.reserve + need;
      s->high_water = std::max(s->high_water, s->in_use);
      j.reserve = need;
    }
    s->cv_work.notify_all();
  }
  return h;
}

// Energy (after a solve that reached the tolerance), memory high-water mark, handle freed.
void finish_job(afmpb_t *h, afmpb_result &r) {
  if (r.status == AFMPB_OK) r.status = afmpb_energy(h, &r.energy_kcal_mol);
  if (r.status != AFMPB_OK && !r.error[0]) std::strncpy(r.error, afmpb_last_error(h), sizeof(r.error) - 1);
  afmpb_info inf{};
  if (afmpb_get_info(h, &inf) == AFMPB_OK) r.bytes_used = inf.device_bytes_peak;
  afmpb_destroy(h);
}

void run_job(afmpb_server_t *s, Job &j, cudaStream_t stream, afmpb_result &r) {
  afmpb_t *h = setup_job(s, j, stream, r);
  if (!h) return;
  r.status = afmpb_solve(h, j.f_out, j.h_out, &r.info);
  if (r.status != AFMPB_OK) std::strncpy(r.error, afmpb_last_error(h), sizeof(r.error) - 1);
  finish_job(h, r);
}

// Hand a finished request's result out and return its reservation.
void complete(afmpb_server_t *s, Job &j, afmpb_result &r) {
  r.t_done = s->now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->in_use -= j.reserve;
    --s->running;
    ++s->completed;
    if (r.status != AFMPB_OK) ++s->failed;
    Done &d = s->results[j.ticket];
    d.res = r;
    d.ready = true;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();                              // freed memory may admit others
}

// Batched mode: take every ready request (up to max_batch) and solve them together.
void solver_main(afmpb_server_t *s) {
  const bool have_device = cudaSetDevice(s->device) == cudaSuccess;
  for (;;) {
    std::vector<Ready> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_ready.wait(lk, [&] { return !s->ready.empty() || (s->stop && s->setting_up == 0); });
      if (s->ready.empty()) break;                      // stopping and nothing left to solve
      // the oldest ready request, and ready ones within a factor of two of its size
      const int64_t n0 = s->ready.front().job->n_nodes;
      for (auto it = s->ready.begin(); it != s->ready.end() && (int)batch.size() < s->max_batch;) {
        const int64_t n = it->job->n_nodes;
        if (batch.empty() || (n <= 2 * n0 && 2 * n >= n0)) {
          batch.push_back(std::move(*it));
          it = s->ready.erase(it);
        } else {
          ++it;
        }
      }
      ++s->batches;
      s->batched += (int64_t)batch.size();
      s->max_batch_seen = std::max<int64_t>(s->max_batch_seen, (int64_t)batch.size());
    }
    const int k = (int)batch.size();
    std::vector<afmpb_t *> hs(k);
    std::vector<double *> fo(k), ho(k);
    std::vector<afmpb_solve_info> infos(k);
    std::vector<afmpb_status> st(k, AFMPB_ECUDA);
    for (int i = 0; i < k; ++i) {
      hs[i] = batch[i].h;
      fo[i] = batch[i].job->f_out;
      ho[i] = batch[i].job->h_out;
    }
    afmpb_status rc = AFMPB_ECUDA;
    std::string err;
    if (have_device) {
      try {
        rc = afmpb_solve_batch(hs.data(), k, fo.data(), ho.data(), infos.data(), st.data());
        if (rc != AFMPB_OK) err = afmpb_last_error(hs[0]);
      } catch (...) {
        rc = afmpb::current_exception_err().code;
      }
    } else {
      err = "solver thread device selection failed";
    }
    for (int i = 0; i < k; ++i) {
      afmpb_result &r = batch[i].r;
      r.info = infos[i];
      r.status = (rc == AFMPB_OK || rc == AFMPB_ENOCONV || rc == AFMPB_ETIMEOUT) ? st[i] : rc;
      if (r.status != AFMPB_OK) std::strncpy(r.error, err.empty() ? "batched solve failed" : err.c_str(), sizeof(r.error) - 1);
      try {
        finish_job(batch[i].h, r);
      } catch (...) {
        r.status = afmpb::current_exception_err().code;
      }
      complete(s, *batch[i].job, r);
    }
  }
}

void slot_main(afmpb_server_t *s, int slot) {
  // a new thread starts on device 0: take the creator's device before any CUDA call
  cudaStream_t stream = nullptr;
  const bool have_stream = cudaSetDevice(s->device) == cudaSuccess &&
                           cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    std::unique_ptr<Job> j;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || (!s->queue.empty() && (j = take_admissible(s)) != nullptr); });
      if (!j) break;                                    // stopping
      s->in_use += j->reserve;
      s->high_water = std::max(s->high_water, s->in_use);
      ++s->running;
      s->max_running = std::max(s->max_running, s->running);
      if (s->max_batch > 1) ++s->setting_up;
    }
    afmpb_result r{};
    r.t_submit = j->t_submit;
    r.t_admit = s->now();
    r.slot = slot;
    r.bytes_reserved = (int64_t)j->reserve;
    if (have_stream && s->max_batch > 1) {
      // batched: set the request up on a stream of its own, then hand it to the solver
      afmpb_t *h = nullptr;
      try {
        h = setup_job(s, *j, nullptr, r);
      } catch (...) {
        const afmpb::Err e = afmpb::current_exception_err();
        r.status = e.code;
        std::strncpy(r.error, e.msg.c_str(), sizeof(r.error) - 1);
      }
      if (h) {
        {
          std::lock_guard<std::mutex> lk(s->mu);
          Ready rd;
          rd.job = std::move(j);
          rd.h = h;
          rd.r = r;
          s->ready.push_back(std::move(rd));
          --s->setting_up;
        }
        s->cv_ready.notify_all();
        continue;
      }
      {
        std::lock_guard<std::mutex> lk(s->mu);
        --s->setting_up;
      }
      s->cv_ready.notify_all();
    } else if (have_stream) {
      try {
        run_job(s, *j, stream, r);
      } catch (...) {                                   // no exception may end a slot thread
        const afmpb::Err e = afmpb::current_exception_err();
        r.status = e.code;
        std::strncpy(r.error, e.msg.c_str(), sizeof(r.error) - 1);
      }
    } else {
      r.status = AFMPB_ECUDA;
      std::strncpy(r.error, "slot device selection or stream creation failed", sizeof(r.error) - 1);
      if (s->max_batch > 1) {
        std::lock_guard<std::mutex> lk(s->mu);
        --s->setting_up;
      }
    }
    complete(s, *j, r);
  }
  if (stream) cudaStreamDestroy(stream);
}

afmpb_status submit_job(afmpb_server_t *s, const afmpb_request *req, int64_t *ticket);

bool copy_array(std::vector<double> &dst, const double *src, int64_t n) {
  if (n < 0 || (n > 0 && !src)) return false;
  dst.assign(src, src + n);
  return true;
}

}  // namespace

extern "C" {

afmpb_status afmpb_server_create(size_t bytes_budget, int max_slots, afmpb_server_t **out) {
  return afmpb_server_create_batched(bytes_budget, max_slots, 1, 1, out);
}

afmpb_status afmpb_server_create_batched(size_t bytes_budget, int max_slots, int solvers, int max_batch,
                                         afmpb_server_t **out) {
  if (!out || bytes_budget == 0 || max_slots < 1 || max_slots > 256 || max_batch < 1 || max_batch > AFMPB_BATCH_MAX ||
      solvers < 1 || solvers > 256)
    return AFMPB_EINVAL;
  *out = nullptr;
  afmpb_server_t *s = new (std::nothrow) afmpb_server_t();
  if (!s) return AFMPB_ENOMEM;
  s->budget = bytes_budget;
  s->max_slots = max_slots;
  s->max_batch = max_batch;
  s->t0 = Clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess) {   // no device: every request fails at its slot
    cudaGetLastError();
    s->device = 0;
  }
  try {
    if (max_batch > 1)
      for (int i = 0; i < solvers; ++i) s->solvers.emplace_back(solver_main, s);
    for (int i = 0; i < max_slots; ++i) s->slots.emplace_back(slot_main, s, i);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_ready.notify_all();
    for (auto &t : s->slots) t.join();
    for (auto &t : s->solvers) t.join();
    delete s;
    return AFMPB_ENOMEM;
  }
  *out = s;
  return AFMPB_OK;
}

afmpb_status afmpb_server_submit(afmpb_server_t *s, const afmpb_request *req, int64_t *ticket) {
  if (!s || !req || !ticket) return AFMPB_EINVAL;
  try {
    return submit_job(s, req, ticket);
  } catch (...) {                                       // copying the request may run out of memory
    const afmpb::Err e = afmpb::current_exception_err();
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = e.msg;
    return e.code;
  }
}

}  // extern "C"

namespace {

afmpb_status submit_job(afmpb_server_t *s, const afmpb_request *req, int64_t *ticket) {
  const afmpb_mesh &m = req->mesh;
  if (m.n_nodes <= 0 || m.n_tris <= 0 || !m.xyz || !m.tri || req->charges.n < 0) return AFMPB_EINVAL;
  auto j = std::make_unique<Job>();
  j->n_nodes = m.n_nodes;
  j->n_tris = m.n_tris;
  j->n_atoms = req->charges.n;
  if (!copy_array(j->xyz, m.xyz, 3 * m.n_nodes)) return AFMPB_EINVAL;
  j->tri.assign(m.tri, m.tri + 3 * m.n_tris);
  if (m.normals) copy_array(j->normals, m.normals, 3 * m.n_nodes);
  if (!copy_array(j->atoms, req->charges.xyz, 3 * req->charges.n) || !copy_array(j->q, req->charges.q, req->charges.n))
    return AFMPB_EINVAL;
  j->eps_in = req->eps_in;
  j->eps_out = req->eps_out;
  j->kappa = req->kappa;
  j->tol = req->tol;
  j->order = req->fmm_order;
  j->opt = req->options;
  j->f_out = req->f_out;
  j->h_out = req->h_out;
  j->reserve = afmpb_estimate_bytes(m.n_nodes, req->charges.n, req->fmm_order, &req->options);
  if (j->reserve == 0) return AFMPB_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return AFMPB_ESTATE;
    if (j->reserve > s->budget) {
      s->err = "request needs more device memory than the whole budget";
      return AFMPB_ENOMEM;
    }
    j->ticket = s->next_ticket++;
    j->t_submit = s->now();
    *ticket = j->ticket;
    s->results[j->ticket];                              // pending entry
    s->queue.push_back(std::move(j));
    ++s->submitted;
  }
  s->cv_work.notify_one();
  return AFMPB_OK;
}

}  // namespace

extern "C" {

afmpb_status afmpb_server_poll(afmpb_server_t *s, int64_t ticket, afmpb_result *res) {
  if (!s || !res) return AFMPB_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return AFMPB_EINVAL;
  if (!it->second.ready) return AFMPB_EBUSY;
  *res = it->second.res;
  s->results.erase(it);
  return AFMPB_OK;
}

afmpb_status afmpb_server_wait(afmpb_server_t *s, int64_t ticket, double timeout_s, afmpb_result *res) {
  if (!s || !res || !(timeout_s >= 0)) return AFMPB_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return AFMPB_EINVAL;
  // The entry may be taken by another thread's poll or wait meanwhile: look it up, never
  // insert it, and report a ticket that disappeared as unknown.
  bool gone = false;
  auto ready = [&] {
    auto jt = s->results.find(ticket);
    gone = jt == s->results.end();
    return gone || jt->second.ready;
  };
  constexpr double kMaxWait = 1e6;                    // seconds; longer waits (or inf) wait without a limit
  if (timeout_s >= kMaxWait) {
    s->cv_done.wait(lk, ready);
  } else {
    const auto limit = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    if (!s->cv_done.wait_until(lk, limit, ready)) return AFMPB_ETIMEOUT;
  }
  if (gone) return AFMPB_EINVAL;
  it = s->results.find(ticket);
  *res = it->second.res;
  s->results.erase(it);
  return AFMPB_OK;
}

afmpb_status afmpb_server_get_info(afmpb_server_t *s, afmpb_server_info *st) {
  if (!s || !st) return AFMPB_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->running = s->running;
  st->queued = (int64_t)s->queue.size();
  st->bytes_in_use = (int64_t)s->in_use;
  st->bytes_high_water = (int64_t)s->high_water;
  st->bytes_budget = (int64_t)s->budget;
  st->max_running = s->max_running;
  st->slots = s->max_slots;
  st->batches = s->batches;
  st->batched_requests = s->batched;
  st->max_batch = (int)s->max_batch_seen;
  return AFMPB_OK;
}

afmpb_status afmpb_server_destroy(afmpb_server_t *s) {
  if (!s) return AFMPB_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();                                   // queued requests are dropped
  }
  s->cv_work.notify_all();
  for (auto &t : s->slots) t.join();                    // running requests finish first
  s->cv_ready.notify_all();
  for (auto &t : s->solvers) t.join();                  // then the requests set up for a batch
  delete s;
  return AFMPB_OK;
}

}  // extern "C"
