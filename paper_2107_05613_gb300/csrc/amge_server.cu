// Request server: continuous batching of PCG-AMGe solves on one GPU.
//
// Clients submit solves (a hierarchy, 1..32 right-hand sides in host memory, solve
// options) and get a ticket back immediately.  One scheduler thread owns all GPU work.
// Every right-hand side becomes one column solve that runs in a slot: a workspace
// view of its hierarchy (own vectors, Krylov state, reduction scratch and captured
// PCG graph), its own CUDA stream and staging buffers.  The scheduler admits queued
// columns whenever a slot of the right hierarchy is idle or a new slot fits the HBM
// budget, advances every running column without blocking (CUDA event queries), and
// retires columns as they finish, so requests that arrive while others run are
// admitted as slots and memory free up and their kernels overlap on the device.
// A column computes exactly what amge_pcg_solve computes for that right-hand side
// (same kernels, same order, its own workspace), whatever else is running.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "amge_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  amge_hier* hier = nullptr;
  int nrhs = 1;
  int64_t n = 0;
  double* bcol = nullptr;  // pinned [nrhs][n]: the right-hand sides, one column after another
  double* xcol = nullptr;  // pinned [nrhs][n]: the solutions, scattered into x_host on collection
  double* x_host = nullptr;
  amge_solve_opts opts{};
  std::vector<amge_info> info;
  int next_col = 0, cols_done = 0, running = 0;
  bool canceled = false, done = false;
  amge_status status = AMGE_OK;
  Clock::time_point t_submit;
};

struct Slot {
  amge_hier* view = nullptr;
  const amge_hier* base = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  double* b_dev = nullptr;
  double* x_dev = nullptr;
  size_t bytes = 0;
  PcgRun* run = nullptr;
  Request* req = nullptr;
  int col = -1;
  int phase = 0;  // 0 idle, 1 solving, 2 copying the solution back
  Clock::time_point last_used;
};

}  // namespace

struct amge_server {
  size_t budget = 0;
  int max_slots = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> reqs;
  uint64_t next_ticket = 1;
  std::vector<Slot*> slots;
  size_t used = 0;
  std::thread th;
  std::atomic<bool> stop{false};
  int64_t running_cols = 0;
};

namespace {

size_t slot_need(const amge_hier* base) {
  return amge::hier_workspace_bytes(base) + 2 * (size_t)amge::hier_dofs(base) * sizeof(double);
}

void free_slot(amge_server* sv, Slot* sl) {
  if (sl->view) amge_hier_free(sl->view);
  if (sl->b_dev) cudaFree(sl->b_dev);
  if (sl->x_dev) cudaFree(sl->x_dev);
  if (sl->ev) cudaEventDestroy(sl->ev);
  if (sl->stream) cudaStreamDestroy(sl->stream);
  sv->used -= sl->bytes;
  delete sl;
}

// Create a slot for `base` (scheduler thread; mutex held).  Returns nullptr if a
// CUDA call fails (memory is then given back).
Slot* make_slot(amge_server* sv, amge_hier* hier) {
  Slot* sl = new Slot;
  sl->base = amge::hier_base(hier);
  const int64_t n = amge::hier_dofs(hier);
  bool ok = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaMalloc(&sl->b_dev, n * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&sl->x_dev, n * sizeof(double)) == cudaSuccess;
  if (ok) ok = amge::hier_make_view(hier, sl->stream, &sl->view) == AMGE_OK;
  if (!ok) {
    cudaGetLastError();
    free_slot(sv, sl);  // bytes not yet counted
    return nullptr;
  }
  sl->bytes = slot_need(sl->base);
  sv->used += sl->bytes;
  sv->slots.push_back(sl);
  return sl;
}

void finish_request(amge_server* sv, Request* rq) {
  rq->done = true;
  const double ms = std::chrono::duration<double, std::milli>(Clock::now() - rq->t_submit).count();
  amge_status worst = rq->canceled ? AMGE_ECANCELED : AMGE_OK;
  for (auto& in : rq->info) {
    in.time_ms = ms;  // request latency: submission to completion
    if (worst == AMGE_OK && in.status == AMGE_ENONFINITE) worst = AMGE_ENONFINITE;
    if (worst == AMGE_OK && in.status == AMGE_ENOTCONV) worst = AMGE_ENOTCONV;
    if (in.status == AMGE_ECUDA) worst = AMGE_ECUDA;
  }
  if (rq->status == AMGE_OK || rq->status == AMGE_EAGAIN) rq->status = worst;
  sv->cv_done.notify_all();
}

// Start column `col` of `rq` in slot `sl` (mutex held).
bool start_column(amge_server* sv, Slot* sl, Request* rq, int col) {
  const int64_t n = rq->n;
  if (cudaMemcpyAsync(sl->b_dev, rq->bcol + (size_t)col * n, n * sizeof(double), cudaMemcpyHostToDevice,
                      sl->stream) != cudaSuccess)
    return false;
  if (amge::pcg_run_start(sl->view, sl->b_dev, sl->x_dev, rq->opts, sl->stream, &sl->run) != AMGE_OK) return false;
  sl->req = rq;
  sl->col = col;
  sl->phase = 1;
  rq->running++;
  sv->running_cols++;
  return true;
}

void fail_column(amge_server* sv, Slot* sl, amge_status st) {
  Request* rq = sl->req;
  rq->info[sl->col].status = st;
  rq->status = st;
  rq->running--;
  rq->cols_done++;
  sv->running_cols--;
  sl->req = nullptr, sl->run = nullptr, sl->phase = 0, sl->col = -1;
  if (rq->cols_done == rq->nrhs || (rq->canceled && rq->running == 0)) finish_request(sv, rq);
}

// Advance every running slot once (mutex held).  Returns true if anything changed.
bool advance_slots(amge_server* sv) {
  bool progressed = false;
  for (Slot* sl : sv->slots) {
    if (sl->phase == 1) {
      amge_status err;
      const int d = amge::pcg_run_advance(sl->run, &err);
      if (d < 0) {
        amge::pcg_run_free(sl->run);  // partially finished run
        fail_column(sv, sl, err);
        progressed = true;
      } else if (d == 1) {
        amge_info info{};
        amge::pcg_run_finish(sl->run, &info);
        sl->run = nullptr;
        sl->req->info[sl->col] = info;
        cudaMemcpyAsync(sl->req->xcol + (size_t)sl->col * sl->req->n, sl->x_dev, sl->req->n * sizeof(double),
                        cudaMemcpyDeviceToHost, sl->stream);
        cudaEventRecord(sl->ev, sl->stream);
        sl->phase = 2;
        progressed = true;
      }
    } else if (sl->phase == 2) {
      const cudaError_t q = cudaEventQuery(sl->ev);
      if (q == cudaErrorNotReady) continue;
      Request* rq = sl->req;
      if (q != cudaSuccess) {
        fail_column(sv, sl, AMGE_ECUDA);
        progressed = true;
        continue;
      }
      rq->running--;
      rq->cols_done++;
      sv->running_cols--;
      sl->req = nullptr, sl->phase = 0, sl->col = -1;
      sl->last_used = Clock::now();
      const bool all = rq->cols_done == rq->nrhs;
      const bool stopped = rq->canceled && rq->running == 0 && rq->next_col >= rq->nrhs;
      if (all || stopped) finish_request(sv, rq);
      progressed = true;
    }
  }
  return progressed;
}

// Admit queued columns into idle or new slots (mutex held).
bool admit(amge_server* sv) {
  bool progressed = false;
  while (!sv->queue.empty()) {
    Request* rq = sv->queue.front();
    if (rq->canceled) {
      rq->next_col = rq->nrhs;
      sv->queue.pop_front();
      if (rq->running == 0) finish_request(sv, rq);
      progressed = true;
      continue;
    }
    const amge_hier* base = amge::hier_base(rq->hier);
    const size_t need = slot_need(base);
    if (need > sv->budget) {  // can never run: fail instead of waiting forever
      rq->status = AMGE_ENOMEM;
      for (int c = rq->next_col; c < rq->nrhs; c++) rq->info[c].status = AMGE_ENOMEM;
      rq->cols_done += rq->nrhs - rq->next_col;
      rq->next_col = rq->nrhs;
      sv->queue.pop_front();
      if (rq->running == 0) finish_request(sv, rq);
      progressed = true;
      continue;
    }
    Slot* sl = nullptr;
    for (Slot* c : sv->slots)
      if (c->phase == 0 && c->base == base) {
        sl = c;
        break;
      }
    if (!sl) {
      // make room: drop least recently used idle slots of other hierarchies
      while ((int)sv->slots.size() >= sv->max_slots || sv->used + need > sv->budget) {
        Slot* victim = nullptr;
        for (Slot* c : sv->slots)
          if (c->phase == 0 && (!victim || c->last_used < victim->last_used)) victim = c;
        if (!victim) break;
        sv->slots.erase(std::find(sv->slots.begin(), sv->slots.end(), victim));
        free_slot(sv, victim);
      }
      if ((int)sv->slots.size() < sv->max_slots && sv->used + need <= sv->budget) sl = make_slot(sv, rq->hier);
    }
    if (!sl) break;  // wait for a running column to finish
    const int col = rq->next_col++;
    if (!start_column(sv, sl, rq, col)) {
      rq->info[col].status = AMGE_ECUDA;
      rq->status = AMGE_ECUDA;
      rq->cols_done++;
    }
    if (rq->next_col >= rq->nrhs) {
      sv->queue.pop_front();
      if (rq->running == 0 && rq->cols_done == rq->nrhs) finish_request(sv, rq);
    }
    progressed = true;
  }
  return progressed;
}

void scheduler(amge_server* sv) {
  cudaSetDevice(sv->device);
  while (!sv->stop.load()) {
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      bool progressed = advance_slots(sv);
      progressed |= admit(sv);
      if (!progressed) {
        if (sv->running_cols > 0) {
          lk.unlock();
          std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else {
          sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        }
      }
    }
  }
}

}  // namespace

extern "C" {

amge_status amge_server_create(size_t hbm_budget_bytes, int32_t max_slots, amge_server** out) {
  if (!out || max_slots < 1 || max_slots > 4096) {
    amge::set_error("amge_server_create: out must be non-NULL and max_slots in [1, 4096]");
    return AMGE_EINVAL;
  }
  *out = nullptr;
  amge_server* sv = new amge_server;
  cudaError_t e = cudaGetDevice(&sv->device);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    amge::set_error(std::string("amge_server_create: ") + cudaGetErrorString(e));
    delete sv;
    return AMGE_ECUDA;
  }
  sv->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
  sv->max_slots = max_slots;
  sv->th = std::thread(scheduler, sv);
  *out = sv;
  return AMGE_OK;
}

amge_status amge_submit(amge_server* sv, amge_hier* h, const double* b_host, double* x_host, int32_t nrhs,
                        const amge_solve_opts* opts, uint64_t* ticket) {
  if (!sv || !h || !b_host || !x_host || !opts || !ticket) {
    amge::set_error("amge_submit: NULL argument");
    return AMGE_EINVAL;
  }
  if (nrhs < 1 || nrhs > amge::kMaxRhs || !(opts->rtol > 0) || opts->maxit < 1 ||
      (opts->precision != AMGE_FP64 && opts->precision != AMGE_FP32_VCYCLE)) {
    amge::set_error("amge_submit: invalid nrhs or solve options");
    return AMGE_EINVAL;
  }
  Request* rq = new Request;
  rq->hier = h;
  rq->nrhs = nrhs;
  rq->n = amge::hier_dofs(h);
  const size_t bytes = (size_t)rq->n * nrhs * sizeof(double);
  if (cudaMallocHost(&rq->bcol, bytes) != cudaSuccess || cudaMallocHost(&rq->xcol, bytes) != cudaSuccess) {
    cudaGetLastError();
    if (rq->bcol) cudaFreeHost(rq->bcol);
    delete rq;
    amge::set_error("amge_submit: pinned staging allocation failed");
    return AMGE_ENOMEM;
  }
  std::memset(rq->xcol, 0, bytes);  // columns that never run (cancelled, failed) read as zero
  // column-major copy, done here in the caller's thread (the scheduler only issues copies)
  for (int64_t i = 0; i < rq->n; i++)
    for (int c = 0; c < nrhs; c++) rq->bcol[(size_t)c * rq->n + i] = b_host[(size_t)i * nrhs + c];
  rq->x_host = x_host;
  rq->opts = *opts;
  rq->info.assign(nrhs, amge_info{0, AMGE_EAGAIN, 0.0, 0.0});
  rq->status = AMGE_EAGAIN;
  rq->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    rq->ticket = sv->next_ticket++;
    sv->reqs[rq->ticket] = rq;
    sv->queue.push_back(rq);
  }
  sv->cv_work.notify_one();
  *ticket = rq->ticket;
  return AMGE_OK;
}

static void release(Request* rq) {
  if (rq->bcol) cudaFreeHost(rq->bcol);
  if (rq->xcol) cudaFreeHost(rq->xcol);
  delete rq;
}

// Detach a finished request (mutex held by the caller); the caller then finishes it
// with hand_back() after releasing the mutex.
static Request* detach(amge_server* sv, std::map<uint64_t, Request*>::iterator it) {
  Request* rq = it->second;
  sv->reqs.erase(it);
  return rq;
}

// Scatter the solution columns into the caller's x_host (in the caller's thread,
// without the server mutex) and release the request.
static amge_status hand_back(Request* rq, amge_info* info) {
  if (info)
    for (int c = 0; c < rq->nrhs; c++) info[c] = rq->info[c];
  for (int64_t i = 0; i < rq->n; i++)
    for (int c = 0; c < rq->nrhs; c++) rq->x_host[(size_t)i * rq->nrhs + c] = rq->xcol[(size_t)c * rq->n + i];
  const amge_status st = rq->status;
  release(rq);
  return st;
}

amge_status amge_poll(amge_server* sv, uint64_t ticket, amge_info* info) {
  if (!sv) {
    amge::set_error("amge_poll: NULL server");
    return AMGE_EINVAL;
  }
  Request* rq = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
      amge::set_error("amge_poll: unknown ticket");
      return AMGE_EINVAL;
    }
    if (!it->second->done) return AMGE_EAGAIN;
    rq = detach(sv, it);
  }
  return hand_back(rq, info);
}

amge_status amge_wait(amge_server* sv, uint64_t ticket, int32_t timeout_ms, amge_info* info) {
  if (!sv) {
    amge::set_error("amge_wait: NULL server");
    return AMGE_EINVAL;
  }
  Request* rq = nullptr;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
      amge::set_error("amge_wait: unknown ticket");
      return AMGE_EINVAL;
    }
    Request* r0 = it->second;
    const auto pred = [&] { return r0->done; };
    if (timeout_ms < 0) {
      sv->cv_done.wait(lk, pred);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
      return AMGE_ETIMEOUT;
    }
    rq = detach(sv, sv->reqs.find(ticket));
  }
  return hand_back(rq, info);
}

amge_status amge_cancel(amge_server* sv, uint64_t ticket) {
  if (!sv) {
    amge::set_error("amge_cancel: NULL server");
    return AMGE_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end() || it->second->done) {
      amge::set_error("amge_cancel: unknown or finished ticket");
      return AMGE_EINVAL;
    }
    it->second->canceled = true;
  }
  sv->cv_work.notify_one();
  return AMGE_OK;
}

amge_status amge_server_stats(amge_server* sv, int64_t* queued, int64_t* running_columns, size_t* bytes_in_use,
                              int32_t* slots) {
  if (!sv) {
    amge::set_error("amge_server_stats: NULL server");
    return AMGE_EINVAL;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if (queued) *queued = (int64_t)sv->queue.size();
  if (running_columns) *running_columns = sv->running_cols;
  if (bytes_in_use) *bytes_in_use = sv->used;
  if (slots) *slots = (int32_t)sv->slots.size();
  return AMGE_OK;
}

void amge_server_destroy(amge_server* sv) {
  if (!sv) return;
  sv->stop.store(true);
  sv->cv_work.notify_all();
  if (sv->th.joinable()) sv->th.join();
  cudaDeviceSynchronize();
  for (Slot* sl : sv->slots) {
    if (sl->run) amge::pcg_run_free(sl->run);
    free_slot(sv, sl);
  }
  for (auto& kv : sv->reqs) release(kv.second);
  delete sv;
}

}  // extern "C"
