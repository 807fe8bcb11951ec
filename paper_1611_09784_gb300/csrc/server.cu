// server.cu - a request loop over the level sampler: requests (level,
// n_samples, seed, first sample) arrive at any time from any host thread; a
// scheduler thread admits them in arrival order onto a pool of worker streams
// (each with its own workspace and float64 accumulators) while the summed
// workspace of the requests in flight stays within an HBM budget, so requests
// of different sizes and levels overlap on the device; completion is found by
// polling each worker's event.  A request's result is the float64 sum of Y and
// Y^2 over its samples (the level terms of eq. (2.6)); its launch shapes depend
// only on the request, so it is the same whether it runs alone or in a mix.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace idos {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  int level = 0;
  int64_t n = 0;
  uint64_t seed = 0;
  int64_t first = 0;
  size_t footprint = 0;
  Clock::time_point t_submit;
  // results
  int status = IDOS_OK;
  std::string error;
  double latency = 0.0;
  double device_ms = 0.0;
  std::vector<double> sum, sumsq;
  bool done = false;
};

struct Worker {
  cudaStream_t stream = nullptr;
  Arena ws;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int* err = nullptr;
  double* acc = nullptr;   // device [kAccRows][n_E]
  int64_t ticket = -1;     // request in flight, -1 = free
};

}  // namespace

struct Server {
  idos_model* model = nullptr;
  int n_E = 0;
  size_t budget = 0;
  std::vector<Worker> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::map<int64_t, Request> reqs;
  int64_t next_ticket = 1;
  size_t in_flight_bytes = 0;
  size_t peak_bytes = 0;
  int64_t completed = 0;
  bool stop = false;
  std::thread loop;
  int device = 0;
};

namespace {

// Moves a finished worker's request to done (holding the lock).
void harvest(Server* S, Worker& w) {
  Request& r = S->reqs[w.ticket];
  r.sum.assign(S->n_E, 0.0);
  r.sumsq.assign(S->n_E, 0.0);
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(r.sum.data(), w.acc, sizeof(double) * S->n_E, cudaMemcpyDeviceToHost, w.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r.sumsq.data(), w.acc + S->n_E, sizeof(double) * S->n_E, cudaMemcpyDeviceToHost, w.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, w.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w.stream);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, w.ev0, w.ev1);
  if (e != cudaSuccess) {
    r.status = IDOS_ERR_CUDA;
    r.error = cudaGetErrorString(e);
  } else if (herr) {
    r.status = status_of_word(herr);
    r.error = get_error();
  }
  r.device_ms = ms;
  r.latency = std::chrono::duration<double>(Clock::now() - r.t_submit).count();
  r.done = true;
  S->in_flight_bytes -= r.footprint;
  ++S->completed;
  w.ticket = -1;
}

// Starts request `t` on worker w (holding the lock).
void start(Server* S, Worker& w, int64_t t) {
  Request& r = S->reqs[t];
  w.ticket = t;
  S->in_flight_bytes += r.footprint;
  S->peak_bytes = std::max(S->peak_bytes, S->in_flight_bytes);
  cudaError_t e = cudaMemsetAsync(w.acc, 0, sizeof(double) * kAccRows * S->n_E, w.stream);
  int st = e == cudaSuccess ? IDOS_OK : IDOS_ERR_CUDA;
  if (st == IDOS_OK)
    st = level_run_async(S->model, r.level, r.n, r.seed, r.first, w.stream, w.ws, w.ev0, w.ev1, w.err, w.acc);
  if (st != IDOS_OK) {
    // the request fails; record ev1 so that the loop harvests it
    r.status = st;
    r.error = get_error();
    cudaEventRecord(w.ev0, w.stream);
    cudaEventRecord(w.ev1, w.stream);
  }
}

void scheduler(Server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (true) {
    bool busy = false;
    for (Worker& w : S->workers) {
      if (w.ticket < 0) continue;
      if (cudaEventQuery(w.ev1) == cudaSuccess) {
        harvest(S, w);   // keeps a launch error recorded by start()
        S->cv_done.notify_all();
      } else {
        busy = true;
      }
    }
    // admit in arrival order while a worker is free and the budget allows
    // (the oldest request always runs when nothing else is in flight)
    while (!S->queue.empty()) {
      Worker* free_w = nullptr;
      for (Worker& w : S->workers)
        if (w.ticket < 0) { free_w = &w; break; }
      if (!free_w) break;
      Request& r = S->reqs[S->queue.front()];
      if (S->in_flight_bytes > 0 && S->in_flight_bytes + r.footprint > S->budget) break;
      const int64_t t = S->queue.front();
      S->queue.pop_front();
      start(S, *free_w, t);
      busy = true;
    }
    if (S->stop && S->queue.empty() && !busy) break;
    if (busy) {
      lock.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lock.lock();
    } else {
      S->cv_work.wait_for(lock, std::chrono::milliseconds(50));
    }
  }
}

}  // namespace
}  // namespace idos

using namespace idos;

struct idos_server : public idos::Server {};

extern "C" int idos_server_create(const idos_model_desc* d, int n_workers, int64_t hbm_budget_bytes,
                                  idos_server** out) {
  if (!out || !d) { set_error("null argument"); return IDOS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (n_workers < 1 || n_workers > 64 || hbm_budget_bytes < 0) {
    set_error("n_workers must lie in 1..64 and hbm_budget_bytes must not be negative");
    return IDOS_ERR_INVALID_ARG;
  }
  idos_model_desc dd = *d;
  dd.sm_split = 0;   // requests share all SMs through the worker streams
  idos_model* m = nullptr;
  IDOS_TRY(idos_create_model(&dd, nullptr, &m));
  idos_server* S = new idos_server();
  S->model = m;
  S->n_E = d->n_E;
  S->budget = hbm_budget_bytes > 0 ? (size_t)hbm_budget_bytes : (size_t(8) << 30);
  cudaGetDevice(&S->device);
  S->workers.resize(n_workers);
  cudaError_t e = cudaSuccess;
  for (Worker& w : S->workers) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&w.ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&w.ev1);
    if (e == cudaSuccess) e = cudaMalloc(&w.err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&w.acc, sizeof(double) * kAccRows * S->n_E);
  }
  if (e != cudaSuccess) {
    set_error(std::string("server resources: ") + cudaGetErrorString(e));
    idos_server_destroy(S);
    return IDOS_ERR_CUDA;
  }
  S->loop = std::thread(scheduler, S);
  *out = S;
  return IDOS_OK;
}

extern "C" int idos_server_submit(idos_server* S, int level, int64_t n_samples, uint64_t seed, int64_t first_sample,
                                  int64_t* ticket) {
  if (!S || !ticket) { set_error("null argument"); return IDOS_ERR_INVALID_ARG; }
  const idos_model_desc& d = S->model->d;
  if (level < 0 || level >= d.n_levels || n_samples < 1 || first_sample < 0) {
    set_error("level out of range, n_samples < 1 or first_sample < 0");
    return IDOS_ERR_INVALID_ARG;
  }
  Request r;
  r.level = level;
  r.n = n_samples;
  r.seed = seed;
  r.first = first_sample;
  r.footprint = level_footprint(S->model, level, n_samples);
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    r.ticket = S->next_ticket++;
    *ticket = r.ticket;
    S->reqs[r.ticket] = std::move(r);
    S->queue.push_back(*ticket);
  }
  S->cv_work.notify_one();
  return IDOS_OK;
}

extern "C" int idos_server_wait(idos_server* S, int64_t ticket, double* sum, double* sumsq, double* latency_s,
                                double* device_ms) {
  if (!S) { set_error("null server"); return IDOS_ERR_INVALID_ARG; }
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) { set_error("unknown ticket"); return IDOS_ERR_INVALID_ARG; }
  S->cv_done.wait(lock, [&] { return it->second.done; });
  Request& r = it->second;
  const int st = r.status;
  if (st == IDOS_OK) {
    if (sum) std::copy(r.sum.begin(), r.sum.end(), sum);
    if (sumsq) std::copy(r.sumsq.begin(), r.sumsq.end(), sumsq);
  } else {
    set_error(r.error);
  }
  if (latency_s) *latency_s = r.latency;
  if (device_ms) *device_ms = r.device_ms;
  S->reqs.erase(it);
  return st;
}

extern "C" int idos_server_info(const idos_server* S, int64_t* completed, int64_t* queued,
                                int64_t* in_flight_bytes, int64_t* peak_bytes) {
  if (!S) { set_error("null server"); return IDOS_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lock(const_cast<idos_server*>(S)->mu);
  if (completed) *completed = S->completed;
  if (queued) *queued = (int64_t)S->queue.size();
  if (in_flight_bytes) *in_flight_bytes = (int64_t)S->in_flight_bytes;
  if (peak_bytes) *peak_bytes = (int64_t)S->peak_bytes;
  return IDOS_OK;
}

extern "C" void idos_server_destroy(idos_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->loop.joinable()) S->loop.join();
  for (Worker& w : S->workers) {
    if (w.stream) cudaStreamSynchronize(w.stream);
    if (w.err) cudaFree(w.err);
    if (w.acc) cudaFree(w.acc);
    if (w.ev0) cudaEventDestroy(w.ev0);
    if (w.ev1) cudaEventDestroy(w.ev1);
    if (w.stream) cudaStreamDestroy(w.stream);
    w.ws.release();
  }
  if (S->model) idos_destroy_model(S->model);
  delete S;
}
