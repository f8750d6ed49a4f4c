// Continuous-batching step server with residency admission.
//
// Step requests for scenes are queued and admitted as worker slots and device
// memory free up; admitted requests run concurrently (each scene on its own
// CUDA stream, so their kernels overlap on the GPU).  The server decides which
// scenes hold device memory: the device footprint of every scene it manages
// that is resident (buffers allocated) stays within the budget.  A request
// whose scene is parked (particle state on the host, no device buffers) needs
// the scene's largest footprint so far; to make room, idle resident scenes are
// parked, least recently stepped first.  A request that cannot be given room
// while other work is in flight waits in the queue; a request that finds
// nothing in flight is always admitted, so that the queue cannot stall.  Only
// the particle state survives parking -- the grid, the hierarchy and the
// L-BFGS history are rebuilt by the next step anyway (Alg. 3 builds them per
// step).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
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
  bool deferred;   // waited at least once for device memory
};

struct Finished {
  int64_t id;
  mpm_status code;
  mpm_step_stats stats;
  double latency_s;
  double queue_s;
};

// What the server knows of a managed scene, updated under its lock only by
// the thread that owns the scene at that moment (submission, or the worker
// that stepped or parked it): the scene's own fields change while a worker
// runs it.
struct Resid {
  int64_t bytes = 0;   // device bytes now (0 while parked)
  int64_t peak = 0;    // largest footprint seen: what it needs when brought back
  bool parked = false;
};

Resid snapshot(const Scene *s) {
  Resid r;
  r.parked = s->parked;
  r.bytes = s->parked ? 0 : (int64_t)s->bytes();
  r.peak = (int64_t)std::max(s->peak_bytes, s->parked ? (size_t)0 : s->bytes());
  return r;
}

}  // namespace

struct Server {
  int64_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::deque<Finished> done;
  std::set<Scene *> busy;        // being stepped or parked by a worker
  std::list<Scene *> lru;        // scenes the server manages, least recently stepped first
  std::map<Scene *, Resid> info;
  int64_t in_flight_bytes = 0;
  int64_t peak_in_flight_bytes = 0;
  int64_t reserved = 0;          // growth admitted for requests in flight (peak of a parked scene, etc.)
  int64_t peak_resident_bytes = 0;
  int64_t parks = 0, unparks = 0, deferred = 0;
  int in_flight = 0;
  bool stop = false;
  std::vector<std::thread> workers;

  int64_t resident_bytes() const {
    int64_t r = 0;
    for (const auto &kv : info) r += kv.second.bytes;
    return r;
  }

  // idle resident scenes to park, oldest first, until `need` more bytes fit
  // next to `resident`; false if they cannot be found
  bool victims_for(int64_t need, int64_t resident, const Scene *keep, std::vector<Scene *> &out) {
    out.clear();
    int64_t r = resident;
    for (Scene *v : lru) {
      if (r + need <= budget) break;
      const Resid &ri = info.at(v);
      if (v == keep || ri.parked || busy.count(v)) continue;
      out.push_back(v);
      r -= ri.bytes;
    }
    return r + need <= budget;
  }

  // first queued request (FIFO) whose scene is idle and for which room can
  // be made; its victims are returned marked busy
  bool take(Request &out, int64_t &bytes, int64_t &grow, std::vector<Scene *> &victims) {
    const int64_t resident = resident_bytes() + reserved;
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Scene *sc = it->scene;
      if (busy.count(sc)) continue;
      const Resid &ri = info.at(sc);
      // a parked scene needs its peak footprint; a resident one may grow back
      // to its peak during the step (unknown before its first step)
      const int64_t need = ri.parked ? ri.peak : std::max<int64_t>(0, ri.peak - ri.bytes);
      const bool fits = victims_for(need, resident, sc, victims);
      if (!fits && in_flight > 0) {
        if (!it->deferred) {
          it->deferred = true;
          ++deferred;
        }
        continue;
      }
      if (!fits) victims_for(need, resident, sc, victims);   // lone request: park what is idle, run anyway
      out = *it;
      bytes = std::max(ri.peak, ri.bytes);
      grow = need;
      queue.erase(it);
      for (Scene *v : victims) {   // counted as parked from now on (the worker parks them first)
        busy.insert(v);
        Resid &rv = info[v];
        rv.bytes = 0;
        rv.parked = true;
      }
      return true;
    }
    return false;
  }

  void touch(Scene *s) {
    lru.remove(s);
    lru.push_back(s);
  }

  void work() {
    cudaSetDevice(device);
    while (true) {
      Request r;
      int64_t bytes = 0, grow = 0;
      std::vector<Scene *> victims;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || take(r, bytes, grow, victims); });
        if (stop) return;
        reserved += grow;
        busy.insert(r.scene);
        in_flight_bytes += bytes;
        in_flight += 1;
        peak_in_flight_bytes = std::max(peak_in_flight_bytes, in_flight_bytes);
      }
      const auto t_start = Clock::now();
      for (Scene *v : victims) {
        try {
          park_scene(*v);
        } catch (const Error &) {
          cudaGetLastError();   // the victim stays resident
        }
      }
      const bool was_parked = r.scene->parked;
      mpm_step_stats st;
      std::memset(&st, 0, sizeof(st));
      mpm_status code = mpm_step(reinterpret_cast<mpm_scene_t>(r.scene), &st);
      r.scene->peak_bytes = std::max(r.scene->peak_bytes, r.scene->bytes());
      const auto t_end = Clock::now();
      std::vector<Resid> vsnap;
      for (Scene *v : victims) vsnap.push_back(snapshot(v));
      const Resid ssnap = snapshot(r.scene);
      {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t k = 0; k < victims.size(); ++k) {
          busy.erase(victims[k]);
          info[victims[k]] = vsnap[k];
          if (vsnap[k].parked) ++parks;
        }
        info[r.scene] = ssnap;
        reserved -= grow;
        if (was_parked && !ssnap.parked) ++unparks;
        busy.erase(r.scene);
        touch(r.scene);
        in_flight_bytes -= bytes;
        in_flight -= 1;
        peak_resident_bytes = std::max(peak_resident_bytes, resident_bytes() + reserved);
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
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->info.find(sc);
    if (it == s->info.end()) {
      // managed from now on; the caller must not step it concurrently
      const hot::Resid r = hot::snapshot(sc);
      if (std::max(r.peak, r.bytes) > s->budget) return MPM_ERR_ADMISSION;
      s->info[sc] = r;
      s->lru.push_front(sc);   // never stepped here: first in line to park
    } else if (std::max(it->second.peak, it->second.bytes) > s->budget) {
      return MPM_ERR_ADMISSION;
    }
    s->queue.push_back(hot::Request{request_id, sc, hot::Clock::now(), false});
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

mpm_status mpm_server_residency(mpm_server_t sv, int64_t *resident_bytes, int64_t *peak_resident_bytes,
                                int64_t *parks, int64_t *unparks, int64_t *deferred) {
  Server *s = reinterpret_cast<Server *>(sv);
  if (!s) return MPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (resident_bytes) *resident_bytes = s->resident_bytes();
  if (peak_resident_bytes) *peak_resident_bytes = s->peak_resident_bytes;
  if (parks) *parks = s->parks;
  if (unparks) *unparks = s->unparks;
  if (deferred) *deferred = s->deferred;
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
