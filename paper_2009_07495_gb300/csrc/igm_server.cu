// igm_server.cu -- serving runtime: continuous batching of independent
// refinement solves (Fig. 1 with int-GMRES) on one GPU.
//
// Requests are queued on the host.  An admission thread takes them in
// arrival order while the device memory held by admitted systems stays
// within the budget and sets each up on the device on its own stream, so
// set-up overlaps the rounds; a set-up system waits in the ready list.  The
// round thread runs rounds: each round runs the convergence test of Fig. 1
// and one inner solve of Fig. 2 for all active systems in the same kernels
// (a batch over their tiles); ready systems join at the next round,
// converged systems are finalised and release their memory after the round.
// Every system's state stays resident on the device from set-up to its
// last round.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "igm_host.h"

using namespace igm;

namespace {

using clk = std::chrono::steady_clock;

struct Request {
  long long id = 0;
  int n = 0, nnz = 0;
  std::vector<int> rowptr, col;
  std::vector<double> val, b, x;
  igm_params prm{};
  clk::time_point t_submit, t_done;
  igm_report rep{};
  igm_status status = IGM_OK;
  bool done = false;
  igm_handle h = nullptr;
  long long bytes = 0;
};

}  // namespace

struct igm_server_s {
  igm_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::map<long long, Request *> all;
  std::vector<Request *> active;   // in the rounds (round thread only)
  std::vector<Request *> ready;    // set up, joining at the next round
  int admitting = 0;               // requests in set-up, ready or active
  double est_scale = 1.0;          // largest footprint / estimate seen so far
  long long next_id = 1, used = 0;
  igm_server_stats st{};
  bool stop = false;
  std::thread worker, admitter;
  cudaStream_t stream = nullptr;   // rounds
  cudaStream_t astream = nullptr;  // set-up
  int dev = 0;
  Batch *batch = nullptr;
  bool dirty = true;
  int4 *d_state = nullptr, *h_state = nullptr;
  int state_cap = 0;
};

namespace {

// a request's device memory and admission slot are free again
void release(igm_server_s *S, Request *r) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= r->bytes;
    S->admitting--;
  }
  S->cv_work.notify_all();
}

void finish(igm_server_s *S, Request *r, igm_status st) {
  std::lock_guard<std::mutex> lk(S->mu);
  r->status = st;
  r->rep.status = st;
  r->t_done = clk::now();
  r->done = true;
  if (st == IGM_OK || st == IGM_ENOCONV) S->st.completed++;
  else S->st.failed++;
  S->cv_done.notify_all();
}

// set-up and Fig. 1 initialisation of one admitted request (admission
// thread, on its stream)
igm_status admit(igm_server_s *S, Request *r) {
  IGM_RANGE("serve: admit one request (set-up)");
  igm_status st = int_gmres_setup(r->n, r->nnz, r->rowptr.data(), r->col.data(), r->val.data(),
                                  &r->prm, S->astream, &r->h);
  if (st) return st;
  r->bytes = int_gmres_device_bytes(r->h);
  st = load_vec(r->h, r->h->hs.bh, r->b.data(), S->astream);
  if (st) return st;
  st = ir_init_host(r->h->solo, S->astream);
  if (st) return st;
  CK(cudaStreamSynchronize(S->astream));
  // the host copies of the matrix are no longer needed
  std::vector<int>().swap(r->rowptr);
  std::vector<int>().swap(r->col);
  std::vector<double>().swap(r->val);
  return IGM_OK;
}

igm_status ensure_state(igm_server_s *S, int n) {
  if (n <= S->state_cap) return IGM_OK;
  if (S->d_state) cudaFree(S->d_state);
  if (S->h_state) cudaFreeHost(S->h_state);
  S->state_cap = n * 2;
  CK(cudaMalloc((void **)&S->d_state, sizeof(int4) * S->state_cap));
  CK(cudaMallocHost((void **)&S->h_state, sizeof(int4) * S->state_cap));
  return IGM_OK;
}

// one round over the active set; finished requests are finalised after it
igm_status round(igm_server_s *S) {
  if (S->dirty) {
    delete S->batch;
    S->batch = nullptr;
    std::vector<igm_handle> hs;
    for (Request *r : S->active) hs.push_back(r->h);
    igm_status st = build_batch(hs, &S->batch);
    if (st) return st;
    S->dirty = false;
  }
  Batch *b = S->batch;
  const BatchDev &B = b->bd;
  cudaStream_t s = S->stream;
  igm_status st = ensure_state(S, B.nsys);
  if (st) return st;
  // convergence test of Fig. 1 for everyone, then one inner solve
  launch_resid(B, 0, s);
  launch_norm(B, VEC_R, ACT_RHO, 1, s);
  launch_gather_state(B, S->d_state, s);
  CKL();
  g_launches += 3;
  CK(cudaMemcpyAsync(S->h_state, S->d_state, sizeof(int4) * B.nsys, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  bool any = false;
  for (int i = 0; i < B.nsys; ++i) any |= S->h_state[i].x != 0;
  if (any) {
    launch_rhs(B, s);
    enqueue_inner_host(b, s);
    CKL();
    CK(cudaStreamSynchronize(s));
  }
  S->st.rounds++;
  // finalise the systems that left the refinement loop
  std::vector<Request *> keep;
  for (int i = 0; i < B.nsys; ++i) {
    Request *r = S->active[i];
    if (S->h_state[i].x != 0) {
      keep.push_back(r);
      continue;
    }
    igm_status fs = ir_finish_host(r->h->solo, s);
    if (!fs) {
      r->x.resize(r->n);
      store_vec(r->h, r->x.data(), r->h->hs.xt, s);
      fs = collect_host(r->h, &r->rep, s);
    }
    int_gmres_destroy(r->h);
    r->h = nullptr;
    release(S, r);
    finish(S, r, fs);
    S->dirty = true;
  }
  S->active.swap(keep);
  return IGM_OK;
}

// a request's device footprint before set-up: the host estimate, scaled by
// the largest footprint / estimate ratio of the systems set up so far
// (called with the lock held)
long long estimate(const igm_server_s *S, const Request *r) {
  return (long long)((double)handle_bytes_estimate(r->n, r->nnz, &r->prm) * S->est_scale) + 1;
}

// Admission thread: in arrival order, while the budget (and max_active)
// allows; the first request is admitted whenever nothing else is resident.
void admit_main(igm_server_s *S) {
  cudaSetDevice(S->dev);
  cudaStreamCreateWithFlags(&S->astream, cudaStreamNonBlocking);
  for (;;) {
    Request *r = nullptr;
    long long est = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->stop) return true;
        if (S->queue.empty()) return false;
        if (S->cfg.max_active > 0 && S->admitting >= S->cfg.max_active) return false;
        const Request *q = S->queue.front();
        return S->admitting == 0 ||
               S->used + estimate(S, q) <= S->cfg.budget_bytes;
      });
      if (S->stop) break;
      r = S->queue.front();
      S->queue.pop_front();
      est = estimate(S, r);
      S->used += est;
      S->admitting++;
    }
    igm_status st = admit(S, r);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->used += (st ? 0 : r->bytes) - est;
      if (S->used > S->st.peak_bytes) S->st.peak_bytes = S->used;
      const double raw = (double)handle_bytes_estimate(r->n, r->nnz, &r->prm);
      if (!st && r->bytes > raw * S->est_scale) S->est_scale = r->bytes / raw;
      if (!st) S->ready.push_back(r);
    }
    if (st) {
      if (r->h) int_gmres_destroy(r->h);
      r->h = nullptr;
      r->bytes = 0;
      release(S, r);
      finish(S, r, st);
      continue;
    }
    S->cv_work.notify_all();
  }
  cudaStreamSynchronize(S->astream);
  cudaStreamDestroy(S->astream);
}

// Round thread: ready systems join, then one round over the active set.
void worker_main(igm_server_s *S) {
  cudaSetDevice(S->dev);
  cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->active.empty())
        S->cv_work.wait(lk, [&] { return S->stop || !S->ready.empty(); });
      if (S->stop) break;
      if (!S->ready.empty()) {
        for (Request *r : S->ready) S->active.push_back(r);
        S->ready.clear();
        S->dirty = true;
      }
    }
    auto t0 = clk::now();
    IGM_RANGE("serve: one round over the active requests");
    igm_status st = round(S);
    S->st.busy_s += std::chrono::duration<double>(clk::now() - t0).count();
    if (st) {  // a failed round fails every active request
      for (Request *r : S->active) {
        if (r->h) int_gmres_destroy(r->h);
        r->h = nullptr;
        release(S, r);
        finish(S, r, st);
      }
      S->active.clear();
      S->dirty = true;
    }
  }
  for (Request *r : S->active)
    if (r->h) int_gmres_destroy(r->h);
  S->active.clear();
  delete S->batch;
  S->batch = nullptr;
  if (S->d_state) cudaFree(S->d_state);
  if (S->h_state) cudaFreeHost(S->h_state);
  cudaStreamDestroy(S->stream);
}

}  // namespace

extern "C" {

igm_status igm_server_create(const igm_server_config *cfg, igm_server *out) {
  g_err.clear();
  if (!cfg || !out) return fail(IGM_EINVAL, "NULL argument");
  if (cfg->budget_bytes <= 0 || cfg->m < 1 || cfg->m > IGM_MAX_M || cfg->max_active < 0 ||
      (cfg->inner != 0 && cfg->inner != 1))
    return fail(IGM_EINVAL, "bad server configuration");
  igm_server_s *S = new igm_server_s();
  S->cfg = *cfg;
  cudaGetDevice(&S->dev);
  S->worker = std::thread(worker_main, S);
  S->admitter = std::thread(admit_main, S);
  *out = S;
  return IGM_OK;
}

igm_status igm_server_submit(igm_server S, int n, int nnz, const int *rowptr, const int *col,
                             const double *val, const double *bhat, const igm_params *params,
                             long long *id) {
  g_err.clear();
  if (!S || !rowptr || !bhat || !params || !id || n < 1 || nnz < 0 ||
      (nnz > 0 && (!col || !val)))
    return fail(IGM_EINVAL, "bad arguments");
  if (params->m != S->cfg.m || params->inner != S->cfg.inner)
    return fail(IGM_EINVAL, "params.m / inner must match the server");
  if (rowptr[0] != 0 || rowptr[n] != nnz) return fail(IGM_EINVAL, "rowptr[0] / rowptr[n]");
  if (handle_bytes_estimate(n, nnz, params) > S->cfg.budget_bytes)
    return fail(IGM_EOOM, "request needs more than the whole budget");
  Request *r = new Request();
  r->n = n;
  r->nnz = nnz;
  r->rowptr.assign(rowptr, rowptr + n + 1);
  r->col.assign(col, col + nnz);
  r->val.assign(val, val + nnz);
  r->b.assign(bhat, bhat + n);
  r->prm = *params;
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    S->all[r->id] = r;
    S->queue.push_back(r);
    S->st.submitted++;
  }
  S->cv_work.notify_all();
  *id = r->id;
  return IGM_OK;
}

igm_status igm_server_poll(igm_server S, long long id, int wait_ms, double *xhat,
                           igm_report *rep, double *lat_s, int *done) {
  g_err.clear();
  if (!S || !done) return fail(IGM_EINVAL, "NULL argument");
  *done = 0;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return fail(IGM_EINVAL, "unknown request %lld", id);
  Request *r = it->second;
  if (!r->done && wait_ms != 0) {
    if (wait_ms < 0) S->cv_done.wait(lk, [&] { return r->done; });
    else S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return r->done; });
  }
  if (!r->done) return IGM_OK;
  *done = 1;
  if (xhat && !r->x.empty()) memcpy(xhat, r->x.data(), sizeof(double) * r->n);
  if (rep) *rep = r->rep;
  if (lat_s) *lat_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  igm_status st = r->status;
  S->all.erase(it);
  delete r;
  if (st) return fail(st, "request %lld: status %d", id, (int)st);
  return IGM_OK;
}

igm_status igm_server_get_stats(igm_server S, igm_server_stats *st) {
  if (!S || !st) return fail(IGM_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->st;
  return IGM_OK;
}

void igm_server_destroy(igm_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->admitter.joinable()) S->admitter.join();
  if (S->worker.joinable()) S->worker.join();
  for (Request *r : S->ready)
    if (r->h) int_gmres_destroy(r->h);
  S->ready.clear();
  for (auto &kv : S->all) delete kv.second;
  delete S;
}

}  // extern "C"
