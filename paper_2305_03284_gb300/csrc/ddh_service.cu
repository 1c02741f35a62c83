// Native continuous-batching scheduler of libddh (declarations in include/ddh.h).
//
// One scheduler thread per service.  Sensors (ddh_state each, admitted against a memory
// budget) own FIFOs of submitted frames.  The thread loops: (1) resolve the oldest in-flight
// batches whose completion event has fired (completion timestamp, latency from arrival);
// (2) if the batch-formation policy (ddh_sched_pick, a pure function of the queue state) says
// so, launch one batch holding the next queued frame of every sensor that has one.  A batch
// holds at most one frame per sensor; frames n and n+1 of a sensor are dependent, and they may
// sit in consecutive batches on the device at the same time because every batch runs in order
// on the service's one stream (a batch's side-stream branches fork from and join back into
// it).  Host code only: the batch itself is enqueue_batch() of ddh_api.cu.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ddh.h"
#include "ddh_internal.h"
#include "ddh_kernels.cuh"

namespace {

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

struct Pending {
  const void* y;
  double arrival;
  uint64_t tag;
};

struct Sensor {
  int id;
  ddh_state* state;
  size_t bytes;
  std::deque<Pending> queue;
  int in_flight = 0;  // frames of this sensor in batches on the device
  bool closing = false;
  int64_t done = 0;
};

struct Batch {
  cudaEvent_t ev;
  std::vector<std::pair<Sensor*, Pending>> items;
};

}  // namespace

struct ddh_service {
  int device;
  cudaStream_t stream;
  size_t budget;
  size_t used = 0;
  int max_in_flight;
  unsigned flags;
  std::mutex mu;
  std::map<int, Sensor*> sensors;
  std::deque<Batch> in_flight;
  std::vector<cudaEvent_t> free_events;
  std::deque<ddh_completion> completed;
  std::thread thread;
  std::atomic<bool> running{false};
  std::atomic<int> error{DDH_OK};
  int64_t batches = 0;
  int64_t frames_launched = 0;
  std::vector<ddh_state*> scratch_states;
  std::vector<const void*> scratch_ys;
  std::vector<ddh_sched_sensor> view;  // the policy's view of the sensors (map order)
  std::vector<unsigned char> pick;
  double age_limit_s = 1e-3;
  unsigned sched_flags = DDH_SCHED_BACKLOG | DDH_SCHED_AGE;
};

namespace {

void reap_locked(ddh_service* s) {
  for (auto it = s->sensors.begin(); it != s->sensors.end();) {
    Sensor* se = it->second;
    if (se->closing && se->queue.empty() && se->in_flight == 0) {
      ddh_free(se->state);
      s->used -= se->bytes;
      delete se;
      it = s->sensors.erase(it);
    } else {
      ++it;
    }
  }
}

// One scheduler iteration; returns the number of frames launched (or a negative error).  The
// batch is formed under the service lock (frames popped, their sensors' in-flight counts
// raised, so that no release frees those states) and launched outside it, so that callers
// submitting frames never wait for a launch sequence.  Only one thread runs this function.
int service_step(ddh_service* s) {
  Batch b;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    while (!s->in_flight.empty()) {
      Batch& done = s->in_flight.front();
      const cudaError_t q = cudaEventQuery(done.ev);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) return ddh_internal_cuda_fail(q);
      const double t = now_s();
      for (auto& it : done.items) {
        Sensor* se = it.first;
        se->in_flight -= 1;
        se->done += 1;
        ddh_completion c{};
        c.tag = it.second.tag;
        c.sensor = se->id;
        c.frame_index = se->done;
        c.arrival_s = it.second.arrival;
        c.done_s = t;
        s->completed.push_back(c);
      }
      s->free_events.push_back(done.ev);
      s->in_flight.pop_front();
    }
    reap_locked(s);
    s->view.clear();
    for (auto& kv : s->sensors) {
      const Sensor* se = kv.second;
      ddh_sched_sensor v{};
      v.queued = static_cast<int>(se->queue.size());
      v.oldest_arrival_s = se->queue.empty() ? 0.0 : se->queue.front().arrival;
      s->view.push_back(v);
    }
    s->pick.assign(s->view.size(), 0);
    const int picked = ddh_sched_pick(s->view.data(), static_cast<int>(s->view.size()),
                                      static_cast<int>(s->in_flight.size()), s->max_in_flight, now_s(),
                                      s->age_limit_s, s->sched_flags, s->pick.data());
    if (picked <= 0) return picked < 0 ? picked : 0;
    s->scratch_states.clear();
    s->scratch_ys.clear();
    size_t k = 0;
    for (auto& kv : s->sensors) {
      Sensor* se = kv.second;
      if (!s->pick[k++] || se->queue.empty()) continue;
      Pending p = se->queue.front();
      se->queue.pop_front();
      se->in_flight += 1;
      s->scratch_states.push_back(se->state);
      s->scratch_ys.push_back(p.y);
      b.items.emplace_back(se, p);
    }
    if (b.items.empty()) return 0;
    if (s->free_events.empty()) {
      cudaEvent_t ev;
      const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return ddh_internal_cuda_fail(e);
      s->free_events.push_back(ev);
    }
    b.ev = s->free_events.back();
    s->free_events.pop_back();
  }
  DdhNvtxRange nv("ddh_service_batch");
  int rc = DDH_OK;
  if (s->flags & DDH_SERVICE_PER_FRAME_LAUNCH) {
    for (size_t i = 0; i < b.items.size() && rc == DDH_OK; ++i) rc = ddh_step(s->scratch_states[i], s->scratch_ys[i]);
  } else {
    rc = ddh_step_batch(s->scratch_states.data(), s->scratch_ys.data(), static_cast<int>(b.items.size()));
  }
  if (rc == DDH_OK) {
    const cudaError_t e = cudaEventRecord(b.ev, s->stream);
    if (e != cudaSuccess) rc = ddh_internal_cuda_fail(e);
  }
  std::lock_guard<std::mutex> lock(s->mu);
  if (rc != DDH_OK) {
    for (auto& it : b.items) it.first->in_flight -= 1;  // the frames are lost with the error
    s->free_events.push_back(b.ev);
    return rc;
  }
  const int launched = static_cast<int>(b.items.size());
  s->in_flight.push_back(std::move(b));
  s->batches += 1;
  s->frames_launched += launched;
  return launched;
}

void service_loop(ddh_service* s) {
  cudaSetDevice(s->device);
  while (s->running.load(std::memory_order_relaxed)) {
    const int rc = service_step(s);
    if (rc < 0) {
      s->error.store(rc);
      break;
    }
    if (rc == 0) std::this_thread::yield();
  }
}

}  // namespace

extern "C" {

double ddh_service_now(void) { return now_s(); }

int ddh_sched_pick(const ddh_sched_sensor* sensors, int count, int batches_in_flight, int max_in_flight,
                   double now, double age_limit_s, unsigned flags, unsigned char* pick) {
  if (count < 0 || (count > 0 && (sensors == nullptr || pick == nullptr)) || max_in_flight < 1) return DDH_EINVAL;
  int ready = 0;
  bool backlog = false, aged = false;
  for (int i = 0; i < count; ++i) {
    pick[i] = 0;
    if (sensors[i].queued <= 0) continue;
    ++ready;
    backlog = backlog || sensors[i].queued >= 2;
    aged = aged || now - sensors[i].oldest_arrival_s >= age_limit_s;
  }
  if (ready == 0 || batches_in_flight >= max_in_flight) return 0;
  // behind a running batch a new one goes out only if it holds at least half of the sensors
  // (light traffic gathers into full batches instead of spending a launch sequence on a few
  // frames), or a sensor has frames waiting beyond the one this batch takes (its frames
  // arrive faster than batches complete: it advances one frame per batch, so the next batch
  // must not wait for the running one), or a frame has waited longer than the age limit
  if (batches_in_flight > 0 && 2 * ready < count && !((flags & DDH_SCHED_BACKLOG) && backlog) &&
      !((flags & DDH_SCHED_AGE) && aged))
    return 0;
  for (int i = 0; i < count; ++i) pick[i] = sensors[i].queued > 0 ? 1 : 0;
  return ready;
}

int ddh_service_set_policy(ddh_service* s, unsigned flags, double age_limit_s) {
  if (s == nullptr || (flags & ~static_cast<unsigned>(DDH_SCHED_BACKLOG | DDH_SCHED_AGE)) || !(age_limit_s > 0.0))
    return DDH_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  s->sched_flags = flags;
  s->age_limit_s = age_limit_s;
  return DDH_OK;
}

int ddh_service_create(ddh_service** out, void* cuda_stream, size_t mem_budget_bytes, int max_in_flight,
                       unsigned flags) {
  if (out == nullptr || max_in_flight < 1 || max_in_flight > 64) return DDH_EINVAL;
  if (flags & ~static_cast<unsigned>(DDH_SERVICE_PER_FRAME_LAUNCH)) return DDH_EINVAL;
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ddh_internal_cuda_fail(e);
  ddh_service* s = new ddh_service();
  s->device = dev;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  s->max_in_flight = max_in_flight;
  s->flags = flags;
  if (mem_budget_bytes == 0) {
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
      delete s;
      return ddh_internal_cuda_fail(e);
    }
    const size_t reserve = size_t(1) << 30;
    mem_budget_bytes = free_b > reserve ? free_b - reserve : 0;
  }
  s->budget = mem_budget_bytes;
  *out = s;
  return DDH_OK;
}

size_t ddh_state_bytes(int n) {
  if (n != 32 && n != 64 && n != 128 && n != 256 && n != 512) return 0;
  ddh_params p{};
  p.n = n;
  p.exec_path = DDH_PATH_DEFAULT;
  return ddh_internal_state_bytes(&p);
}

int ddh_service_admit(ddh_service* s, int sensor_id, const ddh_params* p) {
  if (s == nullptr || p == nullptr) return DDH_EINVAL;
  const size_t need = ddh_internal_state_bytes(p);
  if (need == 0) return DDH_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->sensors.count(sensor_id)) return DDH_EINVAL;
  if (s->used + need > s->budget) return DDH_EBUDGET;
  ddh_state* st = nullptr;
  const int rc = ddh_init(&st, p, s->stream);
  if (rc != DDH_OK) return rc;
  Sensor* se = new Sensor();
  se->id = sensor_id;
  se->state = st;
  se->bytes = need;
  s->sensors[sensor_id] = se;
  s->used += need;
  return DDH_OK;
}

int ddh_service_release(ddh_service* s, int sensor_id) {
  if (s == nullptr) return DDH_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->sensors.find(sensor_id);
  if (it == s->sensors.end()) return DDH_EINVAL;
  it->second->closing = true;
  reap_locked(s);
  return DDH_OK;
}

ddh_state* ddh_service_state(ddh_service* s, int sensor_id) {
  if (s == nullptr) return nullptr;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->sensors.find(sensor_id);
  return it == s->sensors.end() ? nullptr : it->second->state;
}

int ddh_service_submit(ddh_service* s, int sensor_id, const void* y_c64_dev, double arrival_s, uint64_t tag) {
  if (s == nullptr || y_c64_dev == nullptr || reinterpret_cast<uintptr_t>(y_c64_dev) % 16 != 0) return DDH_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->sensors.find(sensor_id);
  if (it == s->sensors.end() || it->second->closing) return DDH_EINVAL;
  it->second->queue.push_back(Pending{y_c64_dev, arrival_s < 0 ? now_s() : arrival_s, tag});
  return DDH_OK;
}

int ddh_service_poll(ddh_service* s, ddh_completion* out, int max_out, int* n_out) {
  if (s == nullptr || n_out == nullptr || (max_out > 0 && out == nullptr)) return DDH_EINVAL;
  *n_out = 0;
  const int err = s->error.load();
  if (err != DDH_OK) return err;
  if (!s->running.load()) {
    const int rc = service_step(s);  // no background thread: the caller drives the loop
    if (rc < 0) return rc;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  int n = 0;
  while (n < max_out && !s->completed.empty()) {
    out[n++] = s->completed.front();
    s->completed.pop_front();
  }
  *n_out = n;
  return DDH_OK;
}

int64_t ddh_service_pending(ddh_service* s) {
  if (s == nullptr) return -1;
  std::lock_guard<std::mutex> lock(s->mu);
  int64_t n = static_cast<int64_t>(s->completed.size());
  for (auto& kv : s->sensors) n += static_cast<int64_t>(kv.second->queue.size()) + kv.second->in_flight;
  return n;
}

int ddh_service_stats(ddh_service* s, int64_t* batches, int64_t* frames, size_t* used_bytes) {
  if (s == nullptr) return DDH_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (batches) *batches = s->batches;
  if (frames) *frames = s->frames_launched;
  if (used_bytes) *used_bytes = s->used;
  return DDH_OK;
}

int ddh_service_start(ddh_service* s) {
  if (s == nullptr || s->running.load()) return DDH_EINVAL;
  s->running.store(true);
  s->thread = std::thread(service_loop, s);
  return DDH_OK;
}

int ddh_service_stop(ddh_service* s) {
  if (s == nullptr) return DDH_EINVAL;
  if (s->running.exchange(false) && s->thread.joinable()) s->thread.join();
  return s->error.load();
}

int ddh_service_free(ddh_service* s) {
  if (s == nullptr) return DDH_OK;
  ddh_service_stop(s);  // the scheduler thread has exited: nothing else touches `s`
  DdhDeviceGuard dg(s->device);
  cudaStreamSynchronize(s->stream);
  for (auto& kv : s->sensors) {
    ddh_free(kv.second->state);
    delete kv.second;
  }
  for (auto& b : s->in_flight) cudaEventDestroy(b.ev);
  for (cudaEvent_t ev : s->free_events) cudaEventDestroy(ev);
  delete s;
  return DDH_OK;
}

}  // extern "C"
