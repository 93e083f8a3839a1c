// Serving loop of the library (efie_server_*): scattering requests of different geometries,
// sizes and wavenumbers are admitted into slots as slots and device memory free up (least
// estimated work first among the 8 oldest that fit), and run concurrently on the GPU, each in
// its own context and CUDA stream.  Host-side
// scheduling only; every numerical step is the ordinary per-context path.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/efie.h"
#include "admission.h"

namespace efie {
efie_status pool_ref(int dev);  // devmem.cpp
void pool_unref(int dev);
}  // namespace efie

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  // deep copies of the request
  int np = 0;
  std::vector<int> deg, ncp;
  std::vector<double> knots, cp, w;
  efie_options opt{};
  int nrhs = 0, ndir = 0;
  std::vector<double> dir, pol, ffdirs;
  double *w_out = nullptr, *e_inf_out = nullptr;  // caller-owned
  size_t footprint = 0;
  double cost = 0.0;  // relative work estimate, for the admission order
  int passed = 0;     // admissions that went to a request behind this one
  int64_t ndof = 0;
  // progress
  Clock::time_point t_submit, t_start, t_done;
  efie_result res{};
  bool done = false;
};

struct Server {
  int device = 0;
  size_t budget = 0, in_use = 0;
  int max_slots = 1, busy = 0;
  std::mutex mu;
  std::condition_variable cv_work;
  std::deque<std::shared_ptr<Job>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<std::thread> workers;
  std::atomic<uint64_t> next{1};
  bool stop = false;
};

size_t estimate_footprint(const Job &j) {
  return efie::request_footprint(j.np, j.opt.level_m, j.opt.p, j.opt.q, j.opt.gmres_restart, j.opt.gmres_maxit,
                                 j.opt.precision == EFIE_MIXED_FP32, j.nrhs, j.ndir, j.opt.m2l_store,
                                 j.opt.leaf_dense);
}

void run_job(Server *S, Job &j) {
  cudaSetDevice(S->device);
  efie_ctx *ctx = nullptr;
  efie_result &r = j.res;
  efie_status st = efie_create(&ctx, &j.opt, nullptr);
  if (st == EFIE_OK) st = efie_set_geometry(ctx, j.np, j.deg.data(), j.ncp.data(), j.knots.data(), j.cp.data(),
                                            j.w.data());
  auto t0 = Clock::now();
  if (st == EFIE_OK) st = efie_setup(ctx);
  auto t1 = Clock::now();
  efie_solve_info info{};
  if (st == EFIE_OK) {
    int64_t nd = 0;
    efie_num_dofs(ctx, &nd);
    r.ndof = nd;
    if (nd != j.ndof) st = EFIE_EGEOMETRY;  // the caller sized w_out for 2 N (n + p - 1)^2
  }
  if (st == EFIE_OK)
    st = efie_solve_plane_waves(ctx, j.nrhs, j.dir.data(), j.pol.data(), j.w_out, EFIE_PTR_HOST, &info);
  auto t2 = Clock::now();
  if (st >= 0 && j.ndir > 0 && j.e_inf_out) {
    efie_status s2 = efie_far_field(ctx, j.nrhs, j.w_out, j.ndir, j.ffdirs.data(), j.e_inf_out, EFIE_PTR_HOST);
    if (s2 < 0) st = s2;
  }
  int64_t peak = 0;
  if (ctx) efie_device_bytes(ctx, nullptr, &peak);
  efie_destroy(ctx);
  r.device_peak_bytes = peak;
  r.footprint_bytes = (int64_t)j.footprint;
  r.status = st;
  r.iterations = info.iterations;
  r.residual = info.residual;
  r.setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  r.solve_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
}

void worker(Server *S) {
  for (;;) {
    std::shared_ptr<Job> job;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) return;
        // among the kLookahead oldest queued requests whose footprint fits the remaining
        // budget, admit the one with the least estimated work; the oldest request goes first
        // once kLookahead admissions have passed it while it was the oldest
        const size_t left = S->budget > S->in_use ? S->budget - S->in_use : 0;
        constexpr int kLookahead = 8;
        size_t fp[kLookahead];
        double cost[kLookahead];
        const int nq = (int)std::min<size_t>(S->queue.size(), kLookahead);
        for (int i = 0; i < nq; ++i) {
          fp[i] = S->queue[i]->footprint;
          cost[i] = S->queue[i]->cost;
        }
        const int pick = efie::pick_admission(nq, fp, cost, nq ? S->queue.front()->passed : 0, left, S->busy == 0,
                                              kLookahead);
        if (pick >= 0) {
          if (pick > 0) ++S->queue.front()->passed;
          job = S->queue[pick];
          S->queue.erase(S->queue.begin() + pick);
        }
        if (job) break;
        S->cv_work.wait(lk);
      }
      S->in_use += job->footprint;
      ++S->busy;
      job->t_start = Clock::now();
    }
    run_job(S, *job);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_use -= job->footprint;
      --S->busy;
      job->t_done = Clock::now();
      job->res.queue_ms = std::chrono::duration<double, std::milli>(job->t_start - job->t_submit).count();
      job->res.latency_ms = std::chrono::duration<double, std::milli>(job->t_done - job->t_submit).count();
      job->res.ndof = job->ndof;
      job->done = true;
    }
    S->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

efie_status efie_server_create(efie_server **out, size_t hbm_budget_bytes, int max_slots) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) return EFIE_EINVAL;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EFIE_ECUDA;
  Server *S = new (std::nothrow) Server();
  if (!S) return EFIE_ENOMEM;
  S->device = dev;
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  // the device's memory pool lives as long as the server, so that memory a finished request
  // returns is reused by the next one without going back to the driver
  if (efie::pool_ref(dev) != EFIE_OK) {
    delete S;
    return EFIE_ECUDA;
  }
  for (int i = 0; i < max_slots; ++i) S->workers.emplace_back(worker, S);
  *out = reinterpret_cast<efie_server *>(S);
  return EFIE_OK;
}

efie_status efie_server_submit(efie_server *srv, const efie_request *q, uint64_t *ticket) {
  Server *S = reinterpret_cast<Server *>(srv);
  if (!S || !q || !ticket || q->n_patches <= 0 || !q->deg || !q->ncp || !q->knots || !q->cp || !q->w ||
      q->nrhs <= 0 || !q->dir || !q->pol || !q->w_out || q->ndir < 0 || (q->ndir > 0 && (!q->ff_dirs || !q->e_inf_out)))
    return EFIE_EINVAL;
  // the options are checked here as efie_create checks them (the sizes below depend on them)
  if (q->opt.level_m < 0 || q->opt.level_m > 10 || q->opt.p < 1 || q->opt.p > 4 || q->opt.q < 1 || q->opt.q > 16 ||
      q->opt.gmres_restart < 1 || q->opt.gmres_maxit < 1)
    return EFIE_EINVAL;
  auto j = std::make_shared<Job>();
  j->np = q->n_patches;
  j->deg.assign(q->deg, q->deg + 2 * q->n_patches);
  j->ncp.assign(q->ncp, q->ncp + 2 * q->n_patches);
  size_t nk = 0, nc = 0;
  for (int i = 0; i < q->n_patches; ++i) {
    if (j->deg[2 * i] < 1 || j->deg[2 * i + 1] < 1 || j->ncp[2 * i] < 1 || j->ncp[2 * i + 1] < 1) return EFIE_EINVAL;
    nk += j->ncp[2 * i] + j->deg[2 * i] + 1 + j->ncp[2 * i + 1] + j->deg[2 * i + 1] + 1;
    nc += (size_t)j->ncp[2 * i] * j->ncp[2 * i + 1];
  }
  j->knots.assign(q->knots, q->knots + nk);
  j->cp.assign(q->cp, q->cp + 3 * nc);
  j->w.assign(q->w, q->w + nc);
  j->opt = q->opt;
  j->nrhs = q->nrhs;
  j->ndir = q->ndir;
  j->dir.assign(q->dir, q->dir + 3 * q->nrhs);
  j->pol.assign(q->pol, q->pol + 3 * q->nrhs);
  if (q->ndir > 0) j->ffdirs.assign(q->ff_dirs, q->ff_dirs + 3 * q->ndir);
  j->w_out = q->w_out;
  j->e_inf_out = q->e_inf_out;
  const int64_t n = int64_t(1) << q->opt.level_m;
  j->ndof = 2 * int64_t(q->n_patches) * (n + q->opt.p - 1) * (n + q->opt.p - 1);
  j->footprint = estimate_footprint(*j);
  // work ~ directions x DOFs x (basis functions per element) x interpolation nodes
  j->cost = double(j->nrhs) * double(j->ndof) * double((q->opt.p + 1) * (q->opt.p + 1)) *
            double((q->opt.q + 1) * (q->opt.q + 1));
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return EFIE_ESTATE;
  j->ticket = S->next++;
  *ticket = j->ticket;
  S->jobs[j->ticket] = j;
  S->queue.push_back(j);
  S->cv_work.notify_all();
  return EFIE_OK;
}

efie_status efie_server_poll(efie_server *srv, uint64_t ticket, efie_result *res) {
  Server *S = reinterpret_cast<Server *>(srv);
  if (!S || !res) return EFIE_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return EFIE_EINVAL;
  if (!it->second->done) return EFIE_PENDING;
  *res = it->second->res;
  S->jobs.erase(it);
  return EFIE_OK;
}

efie_status efie_server_destroy(efie_server *srv) {
  Server *S = reinterpret_cast<Server *>(srv);
  if (!S) return EFIE_OK;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // let queued and running requests finish
    while (!S->queue.empty() || S->busy > 0) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::milliseconds(1));
      lk.lock();
    }
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto &t : S->workers) t.join();
  efie::pool_unref(S->device);
  delete S;
  return EFIE_OK;
}

}  // extern "C"
