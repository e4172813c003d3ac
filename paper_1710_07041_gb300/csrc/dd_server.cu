// Serving loop for streamed solve requests (continuous batching).
//
// The paper runs one solve at a time on a partition of QPACE 3 (Sec. 4); a
// GB300 holds many lattices at once, so requests are served concurrently:
//   * a scheduler thread admits queued requests while the device-memory
//     budget and the worker count allow, FIFO;
//   * requests with the same solver parameters on operators with the same
//     smoother precision and Schwarz block shape share a worker - one host
//     thread, one CUDA stream and one BatchSolver whose slots hold individual
//     right-hand sides, on any of those operators and lattices: every
//     Arnoldi step runs the Schwarz smoother of all its slots as one launch
//     per colour phase, lattices of different sizes included (the two-level
//     preconditioner keeps one operator per worker);
//   * a slot retires its right-hand side as soon as it converges and takes
//     the next waiting one at the following Arnoldi step, so requests that
//     arrive while others run join the batch without waiting for it to end;
//   * a request joins a compatible worker that has free slots for it, else a
//     new worker starts (up to max_slots workers, which run on separate
//     streams and overlap on the device), else the least loaded compatible
//     worker queues it;
//   * a worker reserves its slot count times the workspace of the largest
//     lattice it has admitted; an idle worker frees its memory after a
//     short grace time.
// Each right-hand side's arithmetic does not depend on its batch mates, so a
// result is the same alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "dd_solver.cuh"
#include "dd_pool.cuh"

namespace dd {

using clk = std::chrono::steady_clock;
constexpr int MAGIC_SERVER = 0x53525631;

struct Request {
  uint64_t ticket = 0;
  Op *op = nullptr;
  int nrhs = 0;
  dd_solve_params params{};
  std::vector<double> b, x;
  std::vector<dd_solve_info> info;
  int state = DD_QUEUED;
  int remaining = 0, next_rhs = 0, worst = DD_OK;
  std::atomic<int> cancel{0};   // set by dd_cancel / shutdown, read by running solves
  clk::time_point t_submit, t_done;
};

struct Server;

struct Worker {
  Server *srv = nullptr;
  Op *op = nullptr;        // the operator of its first request (defines its class)
  dd_solve_params params{};
  int slots = 0;
  size_t per = 0;          // reserved device bytes per slot
  size_t bytes = 0;        // slots x per
  cudaStream_t stream = nullptr;
  // admitted requests with right-hand sides left to start: a request leaves
  // the queue when its last right-hand side is handed to a slot, so the queue
  // never points at a request that can finish (and be freed by dd_poll)
  std::deque<Request *> queue;
  std::thread th;
  bool exited = false;
};

struct Server {
  int magic = MAGIC_SERVER;
  dd_server_params p{};
  std::mutex mu;
  std::condition_variable cv;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::deque<Request *> pending;
  std::vector<std::unique_ptr<Worker>> workers;
  size_t budget = 0, in_use = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::thread scheduler;
  int device = 0;
  // statistics
  uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, rhs_done = 0;
  std::vector<double> latencies_ms;
  clk::time_point t_first, t_last;
  bool any = false;
};

// whether a worker created for operator a can take right-hand sides on b
static bool same_class(const Op *a, const Op *b, const dd_solve_params &p) {
  if (p.mg) return a == b;
  bool same = a->prec == b->prec;
  for (int mu = 0; mu < 4; mu++) same = same && a->lat->g.bd[mu] == b->lat->g.bd[mu];
  return same;
}

static bool same_params(const dd_solve_params &a, const dd_solve_params &b) {
  return a.tol == b.tol && a.restart == b.restart && a.max_iter == b.max_iter && a.sap.sweeps == b.sap.sweeps &&
         a.sap.mr_steps == b.sap.mr_steps && a.inner_reduction == b.inner_reduction && a.mg == b.mg &&
         a.outer_f64 == b.outer_f64;
}

// Called with srv->mu held: a right-hand side of r finished with `status`.
static void rhs_finished(Server *srv, Request *r, int status) {
  if (status != DD_OK && r->worst == DD_OK) r->worst = status;
  if (--r->remaining > 0) return;
  r->t_done = clk::now();
  double ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  for (auto &i : r->info) i.ms_total = ms;
  if (r->worst == DD_ECANCELLED || r->cancel) {
    r->state = DD_CANCELLED_STATE;
    srv->cancelled++;
  } else if (r->worst != DD_OK) {
    r->state = DD_FAILED;
    srv->failed++;
  } else {
    r->state = DD_DONE;
    srv->completed++;
    srv->latencies_ms.push_back(ms);
  }
  srv->rhs_done += r->nrhs;
  srv->t_last = r->t_done;
  srv->cv.notify_all();
}

static void worker_main(Worker *w) {
  Server *srv = w->srv;
  cudaSetDevice(srv->device);
  std::unique_ptr<BatchSolver> bs(new BatchSolver(w->op, w->params, w->slots, w->stream));
  bs->set_cache_workspace(false);   // the budget accounts for this memory: free it on exit
  int rc = bs->init();
  auto next = [&](RhsJob &job) -> bool {
    std::lock_guard<std::mutex> lk(srv->mu);
    while (!w->queue.empty()) {
      Request *r = w->queue.front();
      if (r->cancel || r->next_rhs >= r->nrhs) {
        if (r->cancel)
          while (r->next_rhs < r->nrhs) {
            r->info[r->next_rhs++].status = DD_ECANCELLED;
            rhs_finished(srv, r, DD_ECANCELLED);
          }
        w->queue.pop_front();
        continue;
      }
      int k = r->next_rhs++;
      r->state = DD_RUNNING;
      if (r->next_rhs >= r->nrhs) w->queue.pop_front();   // every right-hand side started
      const size_t fs = (size_t)r->op->lat->g.V * 24;
      job.op = r->op;
      job.b = r->b.data() + k * fs;
      job.x = r->x.data() + k * fs;
      job.b_on_device = job.x_on_device = 0;
      job.use_x0 = 0;
      job.info = &r->info[k];
      job.cancel = &r->cancel;
      job.done = [srv, r](int status) {
        std::lock_guard<std::mutex> lk2(srv->mu);
        rhs_finished(srv, r, status);
      };
      return true;
    }
    return false;
  };
  for (;;) {
    if (rc == DD_OK) {
      rc = bs->run(next);
      if (rc == DD_ENOTCONV) rc = DD_OK;  // recorded per right-hand side
    }
    std::unique_lock<std::mutex> lk(srv->mu);
    if (rc != DD_OK) {
      // a device error: fail everything assigned to this worker
      for (Request *r : w->queue)
        while (r->next_rhs < r->nrhs) {
          r->info[r->next_rhs++].status = rc;
          rhs_finished(srv, r, rc);
        }
      w->queue.clear();
    }
    auto has_work = [&] {
      for (Request *r : w->queue)
        if (r->next_rhs < r->nrhs) return true;
      return false;
    };
    if (!srv->cv.wait_for(lk, std::chrono::milliseconds(500), [&] { return srv->stop || has_work(); }) ||
        srv->stop || rc != DD_OK) {
      if (has_work() && !srv->stop && rc == DD_OK) continue;
      w->exited = true;   // takes no new work
      break;
    }
  }
  bs.reset();
  cudaStreamSynchronize(w->stream);
  // the budget gets the memory back only once it is freed
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->in_use -= w->bytes;
  w->bytes = 0;
  srv->cv.notify_all();
}

static void scheduler_main(Server *srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (!srv->stop) {
    // reap exited workers
    for (auto it = srv->workers.begin(); it != srv->workers.end();) {
      if ((*it)->exited) {
        Worker *w = it->get();
        lk.unlock();
        if (w->th.joinable()) w->th.join();
        cudaStreamDestroy(w->stream);
        lk.lock();
        it = srv->workers.erase(it);
      } else {
        ++it;
      }
    }
    // admit pending requests in arrival order
    for (auto it = srv->pending.begin(); it != srv->pending.end();) {
      Request *r = *it;
      if (r->cancel) {
        r->state = DD_CANCELLED_STATE;
        srv->cancelled++;
        it = srv->pending.erase(it);
        continue;
      }
      Worker *target = nullptr;
      const Geom &g = r->op->lat->g;
      size_t per = BatchSolver::bytes_per_slot(g, r->op->prec, r->params.restart);
      if (r->params.mg)
        per += MgWork::bytes(g, r->op->prec, ((Mg *)r->params.mg)->N, ((Mg *)r->params.mg)->p.coarse_max_iter);
      size_t room = srv->budget > srv->in_use ? srv->budget - srv->in_use : 0;
      // a compatible worker with free slots for this request's right-hand
      // sides takes it (its reservation grown to a larger lattice if the
      // budget allows); otherwise a new worker starts while the worker count
      // allows; otherwise the least loaded compatible worker queues it
      auto pending_rhs = [](const Worker *w) {
        int n = 0;
        for (const Request *q : w->queue) n += q->nrhs - q->next_rhs;
        return n;
      };
      auto take = [&](Worker *w) {
        if (per <= w->per) return true;
        const size_t extra = (size_t)w->slots * (per - w->per);
        if (extra > room) return false;
        srv->in_use += extra;   // a larger lattice: grow the worker's reservation to it
        room -= extra;
        w->bytes += extra;
        w->per = per;
        return true;
      };
      Worker *least = nullptr;
      for (auto &w : srv->workers) {
        if (w->exited || !same_class(w->op, r->op, r->params) || !same_params(w->params, r->params)) continue;
        if (pending_rhs(w.get()) + r->nrhs <= w->slots && take(w.get())) {
          target = w.get();
          break;
        }
        if (!least || pending_rhs(w.get()) < pending_rhs(least)) least = w.get();
      }
      if (!target && (int)srv->workers.size() >= srv->p.max_slots && least && take(least)) target = least;
      if (!target && (int)srv->workers.size() < srv->p.max_slots) {
        int slots = (int)std::min<size_t>((size_t)srv->p.max_batch_rhs, room / per);
        if (slots >= 1) {
          auto w = std::make_unique<Worker>();
          w->srv = srv;
          w->op = r->op;
          w->params = r->params;
          w->slots = slots;
          w->per = per;
          w->bytes = (size_t)slots * per;
          if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) == cudaSuccess) {
            srv->in_use += w->bytes;
            target = w.get();
            srv->workers.push_back(std::move(w));
            target->th = std::thread(worker_main, target);
          }
        }
      }
      if (target) {
        // the solution buffer is allocated on admission (pending requests
        // hold only their right-hand sides)
        try {
          r->x.assign((size_t)r->op->lat->g.V * 24 * r->nrhs, 0.0);
        } catch (...) {
          for (auto &i : r->info) i.status = DD_ENOMEM;
          r->remaining = 1;
          r->worst = DD_ENOMEM;
          rhs_finished(srv, r, DD_ENOMEM);
          it = srv->pending.erase(it);
          continue;
        }
        target->queue.push_back(r);
        it = srv->pending.erase(it);
        srv->cv.notify_all();
      } else {
        ++it;
      }
    }
    srv->cv.wait_for(lk, std::chrono::milliseconds(20));
  }
}

void destroy_server(void *h) {
  Server *srv = (Server *)h;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    for (auto &kv : srv->reqs) kv.second->cancel = 1;
    srv->cv.notify_all();
  }
  if (srv->scheduler.joinable()) srv->scheduler.join();
  for (auto &w : srv->workers) {
    if (w->th.joinable()) w->th.join();
    if (w->stream) cudaStreamDestroy(w->stream);
  }
  srv->magic = 0;
  delete srv;
}

}  // namespace dd

using namespace dd;

extern "C" {

int dd_server_create(const dd_server_params *p, dd_server_t *out) {
  if (!p || !out || p->max_slots < 1 || p->max_slots > 64 || p->max_batch_rhs < 1 || p->max_batch_rhs > MAX_RHS) {
    set_error("dd_server_create: bad parameters (1 <= max_slots <= 64, 1 <= max_batch_rhs <= %d)", MAX_RHS);
    return DD_EINVAL;
  }
  Server *srv = new (std::nothrow) Server;
  if (!srv) return DD_ENOMEM;
  srv->p = *p;
  cudaGetDevice(&srv->device);
  // the server budgets device memory itself: cached solver workspaces of
  // earlier dd_solve calls are released first
  pool_release();
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    delete srv;
    return cuda_fail(e, "dd_server_create");
  }
  srv->budget = p->hbm_budget_bytes ? p->hbm_budget_bytes : free_b / 10 * 8;
  srv->scheduler = std::thread(scheduler_main, srv);
  *out = (dd_server_t)srv;
  return DD_OK;
}

int dd_submit(dd_server_t sh, const dd_request *req, uint64_t *ticket) {
  Server *srv = (Server *)sh;
  if (!srv || srv->magic != MAGIC_SERVER || !req || !ticket || !req->b_host || req->nrhs < 1) {
    set_error("dd_submit: bad argument");
    return DD_EINVAL;
  }
  Op *op = (Op *)req->op;
  if (!op || op->magic != 0x4f505231) {
    set_error("dd_submit: bad operator handle");
    return DD_EINVAL;
  }
  int rc = check_solve_params(&req->params);
  if (rc) return rc;
  if (req->params.mg && (((Mg *)req->params.mg)->magic != MAGIC_MG || ((Mg *)req->params.mg)->op != op ||
                         op->prec == DD_F64)) {
    set_error("dd_submit: the multigrid object must belong to the request's operator (not FP64)");
    return DD_EINVAL;
  }
  const Geom &g = op->lat->g;
  size_t per = BatchSolver::bytes_per_slot(g, op->prec, req->params.restart);
  if (per > srv->budget) {
    set_error("dd_submit: one right-hand side needs %zu device bytes, the budget is %zu", per, srv->budget);
    return DD_EBUSY;
  }
  auto r = std::make_unique<Request>();
  const size_t fs = (size_t)g.V * 24;
  try {
    r->b.assign(req->b_host, req->b_host + fs * req->nrhs);
    r->info.assign(req->nrhs, dd_solve_info{});
  } catch (...) {
    set_error("dd_submit: out of host memory");
    return DD_ENOMEM;
  }
  r->op = op;
  r->nrhs = r->remaining = req->nrhs;
  r->params = req->params;
  r->params.where = DD_HOST;
  r->params.use_x0 = 0;
  r->t_submit = clk::now();
  std::lock_guard<std::mutex> lk(srv->mu);
  r->ticket = srv->next_ticket++;
  *ticket = r->ticket;
  if (!srv->any) {
    srv->any = true;
    srv->t_first = r->t_submit;
  }
  srv->submitted++;
  srv->pending.push_back(r.get());
  srv->reqs[r->ticket] = std::move(r);
  srv->cv.notify_all();
  return DD_OK;
}

int dd_poll(dd_server_t sh, uint64_t ticket, int *state, double *x_out, dd_solve_info *info) {
  Server *srv = (Server *)sh;
  if (!srv || srv->magic != MAGIC_SERVER || !state) {
    set_error("dd_poll: bad argument");
    return DD_EINVAL;
  }
  std::unique_ptr<Request> done;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) {
      set_error("dd_poll: unknown ticket %llu", (unsigned long long)ticket);
      return DD_ENOTFOUND;
    }
    Request *r = it->second.get();
    *state = r->state;
    if (r->state == DD_QUEUED || r->state == DD_RUNNING) return DD_OK;
    done = std::move(it->second);
    srv->reqs.erase(it);
  }
  if (x_out) memcpy(x_out, done->x.data(), done->x.size() * sizeof(double));
  if (info) memcpy(info, done->info.data(), done->info.size() * sizeof(dd_solve_info));
  return DD_OK;
}

int dd_cancel(dd_server_t sh, uint64_t ticket) {
  Server *srv = (Server *)sh;
  if (!srv || srv->magic != MAGIC_SERVER) {
    set_error("dd_cancel: bad argument");
    return DD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) {
    set_error("dd_cancel: unknown ticket %llu", (unsigned long long)ticket);
    return DD_ENOTFOUND;
  }
  it->second->cancel = 1;
  srv->cv.notify_all();
  return DD_OK;
}

int dd_server_get_stats(dd_server_t sh, dd_server_stats *out) {
  Server *srv = (Server *)sh;
  if (!srv || srv->magic != MAGIC_SERVER || !out) {
    set_error("dd_server_get_stats: bad argument");
    return DD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  memset(out, 0, sizeof *out);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->failed = srv->failed;
  out->cancelled = srv->cancelled;
  out->bytes_in_use = srv->in_use;
  if (!srv->latencies_ms.empty()) {
    std::vector<double> v = srv->latencies_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double span = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
    out->rhs_per_s = span > 0 ? srv->rhs_done / span : 0;
  }
  return DD_OK;
}

}  // extern "C"
