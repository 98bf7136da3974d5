// Serving loop of the C ABI (include/stfem.h): requests (one march each) are
// admitted by HBM footprint and run concurrently, one handle and one CUDA
// stream per request.  Independent mode: each worker thread sets up and
// marches its request.  Batched mode: workers set requests up and hand them
// to a stepper thread per class (temporal and spatial degree, precision, mesh), whose group
// marches its members in lockstep with fused smoother launches; requests join
// the group between steps as they become ready and leave when done.
#include "../../include/stfem.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace {

struct Request {
  long long id = 0;
  stfem_request req{};
  std::vector<double> lam, mu, kap, K; // copies of the per-cell arrays
  long long footprint = 0;
  stfem_result info{};
  std::vector<double> end_state;
  std::vector<double> slab_ms;
  bool done = false;
};

// A request whose handle is set up and waits for (or runs in) a group.
struct Ready {
  std::shared_ptr<Request> R;
  stfem_h h = nullptr;
  cudaStream_t stream = nullptr;
  double *state = nullptr;
  long long n_state = 0;
  long long member = 0;
};

// The requests of one class (temporal and spatial degree, precision, mesh) marching in lockstep
// on one stepper thread.
struct Lane {
  std::deque<Ready> queue;    // set up, waiting for a place in the group
  std::vector<Ready> running; // members of the group
  stfem_group group = nullptr;
  std::thread thread;
  std::condition_variable cv;
};

} // namespace

struct stfem_server_ctx {
  long long budget = 0, used = 0;
  int n_workers = 1, running = 0;
  bool stop = false;
  // batched mode: set-up workers hand handles to per-class groups
  bool batched = false;
  int max_members = 8;
  // lanes by class: temporal degree, precision, spatial degree and mesh size,
  // so that the members of a group cost about the same per step
  std::map<std::array<int, 5>, std::unique_ptr<Lane>> lanes;
  long long next_id = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::map<long long, std::shared_ptr<Request>> all;
  std::vector<std::thread> workers;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Runs one request on this thread's own stream and handle.
void run_request(stfem_server s, Request &R) {
  stfem_request q = R.req;
  q.mat.lambda_cell_host = R.lam.empty() ? nullptr : R.lam.data();
  q.mat.mu_cell_host = R.mu.empty() ? nullptr : R.mu.data();
  q.mat.kappa_cell_host = R.kap.empty() ? nullptr : R.kap.data();
  q.mat.K_cell_host = R.K.empty() ? nullptr : R.K.data();
  int status = STFEM_OK;
  cudaStream_t stream = nullptr;
  stfem_h h = nullptr;
  double *state = nullptr;
  long long n_slab = 0, n_state = 0;
  std::string msg;
  R.slab_ms.assign(q.n_slabs, 0.0);
  do {
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
      status = STFEM_ERR_CUDA;
      break;
    }
    status = stfem_setup(&q.mesh, &q.deg, &q.mat, &q.bcs, q.tau, &h);
    if (status < 0) {
      msg = stfem_last_error(nullptr);
      break;
    }
    stfem_set_stream(h, stream);
    if ((status = stfem_gmg_setup(h, &q.gmg)) < 0) break;
    stfem_level_info(h, -1, &n_slab, &n_state, nullptr, nullptr);
    if (cudaMalloc((void **)&state, n_state * sizeof(double)) != cudaSuccess) {
      status = STFEM_ERR_OOM;
      break;
    }
    if ((status = stfem_initial_state(h, state)) < 0) break;
    R.info.t_ready = s->now();
    int worst = STFEM_OK, iters_total = 0;
    for (int n = 0; n < q.n_slabs; ++n) {
      const double t = s->now();
      int it = 0;
      const int rc = march(h, n, 1, state, q.tol, q.restart, q.max_it, &it);
      R.slab_ms[n] = 1000.0 * (s->now() - t);
      iters_total += it;
      if (rc < 0) {
        worst = rc;
        break;
      }
      worst = std::max(worst, rc);
    }
    status = worst;
    R.info.iters_total = iters_total;
    R.end_state.assign(n_state, 0.0);
    if (cudaMemcpyAsync(R.end_state.data(), state, n_state * sizeof(double), cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      status = STFEM_ERR_CUDA;
    long long bytes = 0;
    stfem_footprint_bytes(h, &bytes);
    R.info.device_bytes = bytes + n_state * (long long)sizeof(double);
  } while (false);
  if (status < 0 && msg.empty()) msg = h ? stfem_last_error(h) : "CUDA stream or state allocation failed";
  std::snprintf(R.info.error, sizeof(R.info.error), "%s", status < 0 ? msg.c_str() : "");
  if (state) cudaFree(state);
  if (h) stfem_destroy(h);
  if (stream) cudaStreamDestroy(stream);
  R.info.status = status;
  R.info.n_slabs = q.n_slabs;
  R.info.n_state = n_state;
}

// The lane of a request in batched mode: requests of one lane share the
// temporal degree and the precision (a group's requirement), the spatial
// degree and the mesh (so they advance at about the same pace).
std::array<int, 5> lane_class(const stfem_request &q) {
  return {q.deg.k, q.gmg.precision, q.deg.r, q.mesh.n_cells[0], q.mesh.dim == 3 ? q.mesh.n_cells[2] : 1};
}

// Batched mode, set-up part: handle, stream and initial state of a request.
// Returns false on a failure (recorded in the request).
bool setup_request(stfem_server s, const std::shared_ptr<Request> &Rp, Ready *out) {
  Request &R = *Rp;
  stfem_request q = R.req;
  q.mat.lambda_cell_host = R.lam.empty() ? nullptr : R.lam.data();
  q.mat.mu_cell_host = R.mu.empty() ? nullptr : R.mu.data();
  q.mat.kappa_cell_host = R.kap.empty() ? nullptr : R.kap.data();
  q.mat.K_cell_host = R.K.empty() ? nullptr : R.K.data();
  Ready rd;
  rd.R = Rp;
  int status = STFEM_OK;
  std::string msg;
  long long n_slab = 0;
  do {
    if (cudaStreamCreateWithFlags(&rd.stream, cudaStreamNonBlocking) != cudaSuccess) {
      status = STFEM_ERR_CUDA;
      break;
    }
    status = stfem_setup(&q.mesh, &q.deg, &q.mat, &q.bcs, q.tau, &rd.h);
    if (status < 0) {
      msg = stfem_last_error(nullptr);
      break;
    }
    stfem_set_stream(rd.h, rd.stream);
    if ((status = stfem_gmg_setup(rd.h, &q.gmg)) < 0) break;
    stfem_level_info(rd.h, -1, &n_slab, &rd.n_state, nullptr, nullptr);
    if (cudaMalloc((void **)&rd.state, rd.n_state * sizeof(double)) != cudaSuccess) {
      status = STFEM_ERR_OOM;
      break;
    }
    if ((status = stfem_initial_state(rd.h, rd.state)) < 0) break;
  } while (false);
  R.info.n_slabs = q.n_slabs;
  if (status < 0) {
    if (msg.empty()) msg = rd.h ? stfem_last_error(rd.h) : "CUDA stream or state allocation failed";
    std::snprintf(R.info.error, sizeof(R.info.error), "%s", msg.c_str());
    R.info.status = status;
    if (rd.state) cudaFree(rd.state);
    if (rd.h) stfem_destroy(rd.h);
    if (rd.stream) cudaStreamDestroy(rd.stream);
    return false;
  }
  R.info.t_ready = s->now();
  R.info.n_state = rd.n_state;
  R.slab_ms.assign(q.n_slabs, 0.0);
  *out = rd;
  return true;
}

// Ends a batched request: result and end state into the request record,
// resources released, budget returned.
void finish_request(stfem_server s, Ready &rd, int status, const std::vector<int> &iters,
                    const std::vector<double> &slab_ms) {
  Request &R = *rd.R;
  R.info.status = status;
  R.info.iters_total = 0;
  for (int it : iters) R.info.iters_total += it;
  for (size_t i = 0; i < slab_ms.size() && i < R.slab_ms.size(); ++i) R.slab_ms[i] = slab_ms[i];
  R.end_state.assign(rd.n_state, 0.0);
  if (cudaMemcpyAsync(R.end_state.data(), rd.state, rd.n_state * sizeof(double), cudaMemcpyDeviceToHost,
                      rd.stream) != cudaSuccess ||
      cudaStreamSynchronize(rd.stream) != cudaSuccess)
    R.info.status = STFEM_ERR_CUDA;
  long long bytes = 0;
  stfem_footprint_bytes(rd.h, &bytes);
  R.info.device_bytes = bytes + rd.n_state * (long long)sizeof(double);
  if (R.info.status < 0) std::snprintf(R.info.error, sizeof(R.info.error), "%s", stfem_last_error(rd.h));
  cudaFree(rd.state);
  stfem_destroy(rd.h);
  cudaStreamDestroy(rd.stream);
  std::lock_guard<std::mutex> lock(s->mu);
  R.info.t_done = s->now();
  R.done = true;
  s->used -= R.footprint;
  --s->running;
}

// Batched mode, stepping part: the group of one class.  Set-up requests join
// between steps (continuous batching) and leave when their march ends.
void stepper(stfem_server s, Lane *lane) {
  cudaSetDevice(s->device);
  stfem_group_create(&lane->group);
  for (;;) {
    std::vector<Ready> failed;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      lane->cv.wait(lock, [&] { return s->stop || !lane->queue.empty() || !lane->running.empty(); });
      if (lane->queue.empty() && lane->running.empty()) {
        if (s->stop) break;
        continue;
      }
      while (!lane->queue.empty() && (int)lane->running.size() < s->max_members) {
        Ready rd = lane->queue.front();
        lane->queue.pop_front();
        const stfem_request &q = rd.R->req;
        if (stfem_group_add(lane->group, rd.h, 0, q.n_slabs, rd.state, q.tol, q.restart, q.max_it, &rd.member) < 0)
          failed.push_back(rd);
        else
          lane->running.push_back(rd);
      }
    }
    for (Ready &rd : failed) finish_request(s, rd, STFEM_ERR_ARG, {}, {});
    if (!failed.empty()) {
      s->cv_done.notify_all();
      s->cv_work.notify_all();
    }
    if (lane->running.empty()) continue;
    int active = 0;
    const int rc = stfem_group_step(lane->group, &active);
    // members that are done (or every member after a device error) leave
    std::vector<Ready> keep;
    bool freed = false;
    for (Ready &rd : lane->running) {
      const int n = rd.R->req.n_slabs;
      int done = 0, status = 0;
      std::vector<int> its(std::max(n, 1), 0);
      std::vector<double> ms(std::max(n, 1), 0.0);
      stfem_group_member(lane->group, rd.member, &done, &status, its.data(), ms.data());
      if (rc < 0 && !done) {
        done = 1;
        status = rc;
      }
      if (!done) {
        keep.push_back(rd);
        continue;
      }
      stfem_group_remove(lane->group, rd.member);
      its.resize(n);
      ms.resize(n);
      finish_request(s, rd, status, its, ms);
      freed = true;
    }
    {
      std::lock_guard<std::mutex> lock(s->mu);
      lane->running.swap(keep);
    }
    if (freed) {
      s->cv_done.notify_all();
      s->cv_work.notify_all();
    }
  }
  stfem_group_destroy(lane->group);
}

void worker(stfem_server s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::shared_ptr<Request> R;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      for (;;) {
        if (s->stop && s->pending.empty()) return;
        // first request in arrival order that fits the remaining budget
        auto it = std::find_if(s->pending.begin(), s->pending.end(), [&](const std::shared_ptr<Request> &r) {
          return s->used + r->footprint <= s->budget;
        });
        if (it != s->pending.end()) {
          R = *it;
          s->pending.erase(it);
          s->used += R->footprint;
          ++s->running;
          R->info.t_admit = s->now();
          break;
        }
        s->cv_work.wait(lock);
      }
    }
    if (s->batched) {
      // set up here, march in the lockstep group of the request's class
      Ready rd;
      if (setup_request(s, R, &rd)) {
        const std::array<int, 5> cls = lane_class(R->req);
        std::lock_guard<std::mutex> lock(s->mu);
        Lane *lane = s->lanes.at(cls).get();
        lane->queue.push_back(rd);
        lane->cv.notify_one();
        continue;
      }
    } else {
      run_request(s, *R);
    }
    {
      std::lock_guard<std::mutex> lock(s->mu);
      R->info.t_done = s->now();
      R->done = true;
      s->used -= R->footprint;
      --s->running;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
}

} // namespace

extern "C" {

int stfem_server_create(long long hbm_budget, int n_workers, stfem_server *out) {
  if (!out || hbm_budget <= 0 || n_workers < 1 || n_workers > 256) return STFEM_ERR_ARG;
  stfem_server s = new stfem_server_ctx();
  s->budget = hbm_budget;
  s->n_workers = n_workers;
  s->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&s->device);
  for (int i = 0; i < n_workers; ++i) s->workers.emplace_back(worker, s);
  *out = s;
  return STFEM_OK;
}

int stfem_server_create_batched(long long hbm_budget, int n_workers, int max_members, stfem_server *out) {
  if (!out || hbm_budget <= 0 || n_workers < 1 || n_workers > 256 || max_members < 1 || max_members > 256)
    return STFEM_ERR_ARG;
  stfem_server s = new stfem_server_ctx();
  s->budget = hbm_budget;
  s->n_workers = n_workers;
  s->batched = true;
  s->max_members = max_members;
  s->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&s->device);
  for (int i = 0; i < n_workers; ++i) s->workers.emplace_back(worker, s);
  *out = s;
  return STFEM_OK;
}

int stfem_server_submit(stfem_server s, const stfem_request *req, long long *id) {
  if (!s || !req || !id || req->n_slabs < 0) return STFEM_ERR_ARG;
  auto R = std::make_shared<Request>();
  R->req = *req;
  long ncell = 1;
  for (int i = 0; i < req->mesh.dim && i < 3; ++i) ncell *= req->mesh.n_cells[i];
  if (req->mat.lambda_cell_host) R->lam.assign(req->mat.lambda_cell_host, req->mat.lambda_cell_host + ncell);
  if (req->mat.mu_cell_host) R->mu.assign(req->mat.mu_cell_host, req->mat.mu_cell_host + ncell);
  if (req->mat.kappa_cell_host) R->kap.assign(req->mat.kappa_cell_host, req->mat.kappa_cell_host + ncell);
  if (req->mat.K_cell_host)
    R->K.assign(req->mat.K_cell_host, req->mat.K_cell_host + ncell * req->mesh.dim * req->mesh.dim);
  const int rc = stfem_estimate_bytes(&req->mesh, &req->deg, &req->gmg, req->restart, &R->footprint);
  if (rc < 0) return rc;
  R->info.footprint = R->footprint;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (R->footprint > s->budget) return STFEM_ERR_ARG;
    if (s->batched) { // the stepper of the request's class
      const std::array<int, 5> cls = lane_class(*req);
      if (!s->lanes.count(cls)) {
        auto lane = std::make_unique<Lane>();
        lane->thread = std::thread(stepper, s, lane.get());
        s->lanes[cls] = std::move(lane);
      }
    }
    R->id = s->next_id++;
    R->info.t_submit = s->now();
    s->all[R->id] = R;
    s->pending.push_back(R);
    *id = R->id;
  }
  s->cv_work.notify_one();
  return STFEM_OK;
}

int stfem_server_result(stfem_server s, long long id, double timeout_s, stfem_result *info, double *end_state_host,
                        double *slab_ms_host) {
  if (!s) return STFEM_ERR_ARG;
  std::shared_ptr<Request> R;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return STFEM_ERR_ARG;
    R = it->second;
    auto ready = [&] { return R->done; };
    if (timeout_s < 0)
      s->cv_done.wait(lock, ready);
    else if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ready))
      return STFEM_NOT_CONVERGED;
  }
  if (info) *info = R->info;
  if (end_state_host) std::copy(R->end_state.begin(), R->end_state.end(), end_state_host);
  if (slab_ms_host) std::copy(R->slab_ms.begin(), R->slab_ms.end(), slab_ms_host);
  return STFEM_OK;
}

void stfem_server_destroy(stfem_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto &kv : s->lanes) kv.second->cv.notify_all();
  }
  for (auto &kv : s->lanes) kv.second->thread.join();
  delete s;
}

} // extern "C"
