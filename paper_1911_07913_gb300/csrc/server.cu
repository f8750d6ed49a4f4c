// Continuous-batching step server: step requests for resident scenes are
// queued, admitted as worker slots and memory free up, and run concurrently
// (each scene on its own CUDA stream, so their kernels overlap on the GPU).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <set>
#include <thread>

#include "internal.h"

namespace hot {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id;
  Scene *scene;
  Clock::time_point t_submit;
};

struct Finished {
  int64_t id;
  mpm_status code;
  mpm_step_stats stats;
  double latency_s;
  double queue_s;
};

}  // namespace

struct Server {
  int64_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::deque<Finished> done;
  std::set<Scene *> busy;
  int64_t in_flight_bytes = 0;
  int64_t peak_in_flight_bytes = 0;
  int in_flight = 0;
  bool stop = false;
  std::vector<std::thread> workers;

  // first queued request whose scene is idle and whose footprint fits next
  // to the work already in flight (FIFO otherwise); a lone request is always
  // admitted so that an over-budget footprint cannot stall the queue
  bool take(Request &out, int64_t &bytes) {
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      if (busy.count(it->scene)) continue;
      int64_t b = (int64_t)it->scene->bytes();
      if (in_flight > 0 && in_flight_bytes + b > budget) continue;
      out = *it;
      bytes = b;
      queue.erase(it);
      return true;
    }
    return false;
  }

  void work() {
    cudaSetDevice(device);
    while (true) {
      Request r;
      int64_t bytes = 0;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || take(r, bytes); });
        if (stop) return;
        busy.insert(r.scene);
        in_flight_bytes += bytes;
        in_flight += 1;
        peak_in_flight_bytes = std::max(peak_in_flight_bytes, in_flight_bytes);
      }
      const auto t_start = Clock::now();
      mpm_step_stats st;
      std::memset(&st, 0, sizeof(st));
      mpm_status code = mpm_step(reinterpret_cast<mpm_scene_t>(r.scene), &st);
      const auto t_end = Clock::now();
      {
        std::lock_guard<std::mutex> lk(mu);
        busy.erase(r.scene);
        in_flight_bytes -= bytes;
        in_flight -= 1;
        done.push_back(Finished{r.id, code, st, std::chrono::duration<double>(t_end - r.t_submit).count(),
                                std::chrono::duration<double>(t_start - r.t_submit).count()});
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

}  // namespace hot

using hot::Server;

extern "C" {

mpm_status mpm_server_create(int64_t budget_bytes, int32_t n_workers, mpm_server_t *out) {
  if (!out || budget_bytes <= 0 || n_workers < 1 || n_workers > 256) return MPM_ERR_INVALID_ARG;
  Server *s = new Server();
  s->budget = budget_bytes;
  cudaGetDevice(&s->device);
  for (int k = 0; k < n_workers; ++k) s->workers.emplace_back([s] { s->work(); });
  *out = reinterpret_cast<mpm_server_t>(s);
  return MPM_OK;
}

mpm_status mpm_server_submit(mpm_server_t sv, mpm_scene_t scene, int64_t request_id) {
  Server *s = reinterpret_cast<Server *>(sv);
  if (!s || !scene) return MPM_ERR_INVALID_ARG;
  hot::Scene *sc = reinterpret_cast<hot::Scene *>(scene);
  if ((int64_t)sc->bytes() > s->budget) return MPM_ERR_ADMISSION;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->queue.push_back(hot::Request{request_id, sc, hot::Clock::now()});
  }
  s->cv_work.notify_one();
  return MPM_OK;
}

mpm_status mpm_server_poll(mpm_server_t sv, int32_t wait, int64_t *request_id, mpm_step_stats *stats,
                           double *latency_s, double *queue_s, int32_t *step_status) {
  Server *s = reinterpret_cast<Server *>(sv);
  if (!s || !request_id) return MPM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (wait) {
    s->cv_done.wait(lk, [&] { return !s->done.empty() || (s->queue.empty() && s->in_flight == 0); });
  }
  if (s->done.empty()) {
    *request_id = -1;
    return MPM_OK;
  }
  hot::Finished f = s->done.front();
  s->done.pop_front();
  *request_id = f.id;
  if (stats) *stats = f.stats;
  if (latency_s) *latency_s = f.latency_s;
  if (queue_s) *queue_s = f.queue_s;
  if (step_status) *step_status = (int32_t)f.code;
  return MPM_OK;
}

mpm_status mpm_server_info(mpm_server_t sv, int64_t *queued, int64_t *in_flight, int64_t *in_flight_bytes,
                           int64_t *peak_in_flight_bytes) {
  Server *s = reinterpret_cast<Server *>(sv);
  if (!s) return MPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int64_t)s->queue.size();
  if (in_flight) *in_flight = s->in_flight;
  if (in_flight_bytes) *in_flight_bytes = s->in_flight_bytes;
  if (peak_in_flight_bytes) *peak_in_flight_bytes = s->peak_in_flight_bytes;
  return MPM_OK;
}

mpm_status mpm_server_destroy(mpm_server_t sv) {
  Server *s = reinterpret_cast<Server *>(sv);
  if (!s) return MPM_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // let queued and running requests finish
    s->cv_done.wait(lk, [&] { return s->queue.empty() && s->in_flight == 0; });
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  delete s;
  return MPM_OK;
}

}  // extern "C"
