// Serving loop: scan requests of different sizes arrive at any time; the
// server keeps scene BVHs resident on the device within an HBM budget,
// admits requests as memory frees up, and runs them through the batched
// kernel in ticks (continuous batching).  Each tick packs up to `tick_rays`
// rays taken from every admitted request (large requests advance over several
// ticks), so requests that arrive while others are on the GPU join the next
// tick and their work overlaps on the device.  Results come back to the
// caller's host buffers; per-request latency is measured from submission to
// results-in-host-memory.
//
// Per-environment pose state stays on the device: the server owns a table of
// environment slots (48-byte poses, created by fgl_server_add_envs), and a
// request may scan a range of slots as they are, or first overwrite them from
// host or device memory.  Updates happen in admission order on the compute
// stream; a request that writes slots is admitted only once no admitted
// request uses them, and one that reads slots waits for admitted writers of
// them, so every request scans the poses that the requests before it left.
//
// The paper runs batched environments on one GPU (Sec. IV-C, last paragraph
// of "GPU-accelerated ray-casting"; Table I) but describes no request
// serving; this layer only schedules the same casts.
//
// Threads: a worker admits requests, launches ticks on the compute stream and
// right behind each tick enqueues the result copies of the requests it
// finishes on the copy stream (after the tick's event), one copy per output
// array; a completion thread waits for one event per tick (its copies done),
// moves results staged for pageable caller buffers, and wakes waiters.  Faults are
// reported per request; nothing here waits on the GPU without a host-side
// timeout on the caller's side (fgl_server_wait takes one).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fgl.h"
#include "nvtx_range.h"

namespace fgl {
void record_error(int status, const char* msg);  // api.cu
}

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct SceneEntry {
  fgl_scene scene = nullptr;
  int64_t bytes = 0;
  bool resident = false;
  int64_t active = 0;        // admitted requests using it
  uint64_t last_use = 0;     // LRU stamp
};

struct SensorEntry {
  fgl_sensor sensor = nullptr;
  int32_t n_rays = 0;
};

enum ReqState { PENDING, ACTIVE, DONE };

// Page-locked host buffers by power-of-two size class, reused across
// requests (a copy from pageable memory would wait for the whole stream).
struct PinnedPool {
  std::map<size_t, std::vector<void*>> free_;
  void* get(size_t bytes, size_t* cls) {
    size_t c = 256;
    while (c < bytes) c <<= 1;
    *cls = c;
    auto& v = free_[c];
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      return p;
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, c) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t cls) {
    if (p) free_[cls].push_back(p);
  }
  void release_all() {
    for (auto& kv : free_)
      for (void* p : kv.second) cudaFreeHost(p);
    free_.clear();
  }
};

// Results of at most this many bytes bound for pageable caller memory are
// staged in page-locked memory (larger ones are copied synchronously by the
// completion thread).
constexpr int64_t kStageMax = (int64_t)256 << 20;

struct Request {
  int64_t ticket = 0;
  fgl_request r{};
  float* poses = nullptr;      // page-locked host copy of host poses taken at submit
  size_t poses_cls = 0;
  void* stage = nullptr;       // page-locked result staging for pageable outputs
  size_t stage_cls = 0;
  bool pageable = false;       // an output buffer is pageable host memory
  int32_t n_rays = 0;
  int64_t bytes = 0;           // device bytes while active
  ReqState state = PENDING;
  int status = FGL_OK;
  bool cancel = false;
  Clock::time_point t_submit, t_admit, t_done;
  void* d_buf = nullptr;       // device allocation: [poses |] ranges | ids
  const float* d_poses = nullptr;  // poses the casts read (own buffer or the slot table)
  float* d_range = nullptr;
  int32_t* d_tri = nullptr;
  int32_t env_next = 0;        // next environment to schedule
  int64_t last_tick = -1;      // last tick that holds one of its chunks
  bool slots = false;          // scans resident environment slots
  bool writes = false;         // overwrites them first
  bool copy_queued = false;    // its result copies are enqueued
};

struct Tick {
  int64_t id = 0;
  cudaEvent_t done = nullptr;    // compute stream: the tick's casts
  cudaEvent_t copied = nullptr;  // copy stream: after `done` and the result copies
  std::vector<int64_t> finishing;  // tickets whose last chunk is in this tick
};

}  // namespace

struct fgl_server_s {
  fgl_server_opts o{};
  int device = 0;
  cudaStream_t compute = nullptr, copy = nullptr;

  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_tick;
  bool stop = false;

  std::vector<SceneEntry> scenes;
  std::vector<SensorEntry> sensors;
  std::map<int64_t, std::unique_ptr<Request>> reqs;  // by ticket
  std::deque<int64_t> pending;                        // FIFO
  std::vector<int64_t> active;                        // admission order
  std::deque<Tick> ticks;                             // in flight, in order
  int64_t next_ticket = 1, next_tick = 0;
  uint64_t lru_clock = 0;
  int64_t used_bytes = 0;
  int inject_alloc_fail = 0;
  int inject_worker_fault = 0;
  PinnedPool pinned;

  // resident environment slots: poses on the device, per-slot use counts
  float* d_env = nullptr;           // [env_capacity][12]
  int32_t n_envs = 0;
  std::vector<int32_t> env_readers;  // admitted requests using the slot
  std::vector<uint8_t> env_writer;   // an admitted request overwrote it

  // stats
  int64_t submitted = 0, completed = 0, rejected = 0, cancelled = 0, evictions = 0, uploads = 0,
          n_ticks = 0, rays_done = 0;
  std::vector<double> latencies;
  bool have_first = false;
  Clock::time_point t_first, t_last;

  std::thread worker, completer;
};

namespace {

fgl_status set_err(int status, const std::string& m) {
  fgl::record_error(status, m.c_str());
  return (fgl_status)status;
}

// Device bytes a request holds while admitted: its poses (unless it scans
// resident slots) and its results.
int64_t request_bytes(int32_t n_env, int32_t n_rays, bool slots) {
  return (slots ? 0 : (int64_t)n_env * 48) + (int64_t)n_env * n_rays * 8;
}

bool uses_slots(int32_t src) { return src >= FGL_POSES_SLOTS && src <= FGL_POSES_SLOTS_SET_DEVICE; }

// Make room for `need` bytes by evicting idle resident scenes (least recently
// used first), never the scene `keep`.  Caller holds the lock.
bool make_room(fgl_server_s& S, int64_t need, int keep) {
  while (S.used_bytes + need > S.o.hbm_budget_bytes) {
    int victim = -1;
    for (int i = 0; i < (int)S.scenes.size(); ++i) {
      const SceneEntry& e = S.scenes[i];
      if (i == keep || !e.resident || e.active > 0) continue;
      if (victim < 0 || e.last_use < S.scenes[victim].last_use) victim = i;
    }
    if (victim < 0) return false;
    fgl_scene_evict(S.scenes[victim].scene);
    S.scenes[victim].resident = false;
    S.used_bytes -= S.scenes[victim].bytes;
    ++S.evictions;
  }
  return true;
}

void finish_request(fgl_server_s& S, Request& q, int status) {
  q.status = status;
  q.state = DONE;
  q.t_done = Clock::now();
  S.t_last = q.t_done;
  if (status == FGL_OK) {
    ++S.completed;
    S.rays_done += (int64_t)q.r.n_env * q.n_rays;
    S.latencies.push_back(ms_between(q.t_submit, q.t_done));
  } else if (status == FGL_ERR_CANCELLED) {
    ++S.cancelled;
  } else {
    ++S.rejected;
  }
  S.cv_done.notify_all();
}

// Take an admitted request out of the scheduling list (the worker never
// touches it again).  Caller holds the lock.
void detach_request(fgl_server_s& S, Request& q) {
  S.active.erase(std::remove(S.active.begin(), S.active.end(), q.ticket), S.active.end());
}

// Free an admitted request's device buffers and its share of the budget.
// Caller holds the lock; the request is already detached.
void free_request(fgl_server_s& S, Request& q) {
  if (q.d_buf) {
    cudaFreeAsync(q.d_buf, S.copy);
    q.d_buf = nullptr;
    q.d_poses = nullptr;
    q.d_range = nullptr;
    q.d_tri = nullptr;
  }
  if (q.slots) {
    for (int32_t e = q.r.env_first; e < q.r.env_first + q.r.n_env; ++e) {
      S.env_readers[e] -= 1;
      if (q.writes) S.env_writer[e] = 0;
    }
    q.slots = false;
  }
  S.used_bytes -= q.bytes;
  q.bytes = 0;
  S.scenes[q.r.scene_id].active -= 1;
}

// May `q` be admitted now as far as its environment slots go?  A writer
// needs slots no admitted request uses; a reader needs slots no admitted
// request overwrote.  Caller holds the lock.
bool slots_free(const fgl_server_s& S, const Request& q) {
  const bool writes = q.r.pose_source != FGL_POSES_SLOTS;
  for (int32_t e = q.r.env_first; e < q.r.env_first + q.r.n_env; ++e) {
    if (S.env_writer[e]) return false;
    if (writes && S.env_readers[e] > 0) return false;
  }
  return true;
}

// Admit pending requests in arrival order while memory and slots allow.
// Caller holds the lock.
void admit(fgl_server_s& S) {
  while (!S.pending.empty() && (int)S.active.size() < S.o.max_active) {
    Request& q = *S.reqs[S.pending.front()];
    if (q.cancel) {
      S.pending.pop_front();
      finish_request(S, q, FGL_ERR_CANCELLED);
      continue;
    }
    const bool slots = uses_slots(q.r.pose_source);
    if (slots && !slots_free(S, q)) break;  // FIFO: wait for the slots' earlier users
    SceneEntry& se = S.scenes[q.r.scene_id];
    const int64_t need = q.bytes + (se.resident ? 0 : se.bytes);
    if (!make_room(S, need, q.r.scene_id)) break;  // wait for memory to free up
    if (!se.resident) {
      if (fgl_scene_upload(se.scene) != FGL_OK) {
        S.pending.pop_front();
        finish_request(S, q, FGL_ERR_OOM);
        continue;
      }
      se.resident = true;
      S.used_bytes += se.bytes;
      ++S.uploads;
    }
    // device buffers: [poses |] ranges | ids (stream-ordered allocation)
    void* base = nullptr;
    cudaError_t e = cudaErrorMemoryAllocation;
    if (S.inject_alloc_fail > 0) {
      --S.inject_alloc_fail;
    } else {
      e = cudaMallocAsync(&base, (size_t)q.bytes, S.compute);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      S.pending.pop_front();
      finish_request(S, q, FGL_ERR_OOM);
      continue;
    }
    S.pending.pop_front();
    q.d_buf = base;
    const size_t n_env = (size_t)q.r.n_env;
    float* own_poses = slots ? nullptr : (float*)base;
    q.d_range = (float*)base + (slots ? 0 : n_env * 12);
    q.d_tri = (int32_t*)(q.d_range + n_env * q.n_rays);
    if (!slots) {
      q.d_poses = own_poses;
      cudaMemcpyAsync(own_poses, q.poses, n_env * 48, cudaMemcpyHostToDevice, S.compute);
    } else {
      float* slot = S.d_env + (size_t)q.r.env_first * 12;
      q.d_poses = slot;
      if (q.r.pose_source == FGL_POSES_SLOTS_SET_HOST)
        cudaMemcpyAsync(slot, q.poses, n_env * 48, cudaMemcpyHostToDevice, S.compute);
      else if (q.r.pose_source == FGL_POSES_SLOTS_SET_DEVICE)
        cudaMemcpyAsync(slot, q.r.poses, n_env * 48, cudaMemcpyDeviceToDevice, S.compute);
      q.slots = true;
      q.writes = q.r.pose_source != FGL_POSES_SLOTS;
      for (int32_t k = q.r.env_first; k < q.r.env_first + q.r.n_env; ++k) {
        S.env_readers[k] += 1;
        if (q.writes) S.env_writer[k] = 1;
      }
    }
    S.used_bytes += q.bytes;
    se.active += 1;
    se.last_use = ++S.lru_clock;
    q.state = ACTIVE;
    q.t_admit = Clock::now();
    S.active.push_back(q.ticket);
  }
}

// Enqueue the device-to-host copies of a finished request's results on the
// copy stream (which already waits for the tick): straight into the caller's
// buffers when they are page-locked, else into the request's page-locked
// staging.  Large results bound for pageable memory are left to the
// completion thread.  Returns false when a copy could not be enqueued.
bool enqueue_result_copies(fgl_server_s& S, Request& q) {
  const size_t nr = (size_t)q.r.n_env * q.n_rays;
  if (q.pageable && !q.stage) return true;  // copied synchronously on completion
  float* dr = q.pageable ? (float*)q.stage : q.r.out_range;
  int32_t* dt = q.pageable ? (int32_t*)((float*)q.stage + nr) : q.r.out_tri;
  if (cudaMemcpyAsync(dr, q.d_range, nr * 4, cudaMemcpyDeviceToHost, S.copy) != cudaSuccess ||
      cudaMemcpyAsync(dt, q.d_tri, nr * 4, cudaMemcpyDeviceToHost, S.copy) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  q.copy_queued = true;
  return true;
}

void worker_main(fgl_server_s* Sp) {
  fgl_server_s& S = *Sp;
  cudaSetDevice(S.device);
  std::vector<fgl_cast_item> items;
  for (;;) {
    std::unique_lock<std::mutex> lk(S.mu);
    // at most two ticks in flight: the batched table of one is being built
    // while the other runs
    S.cv_tick.wait(lk, [&] { return S.stop || S.ticks.size() < 2; });
    if (S.stop) break;
    fgl::NvtxRange range("fgl_server tick");
    Tick t;
    t.id = S.next_tick;
    bool counted = false;  // the tick id is taken (next_tick advanced)
    int status = FGL_OK;
    // An exception while a tick is packed or launched (an allocation that
    // fails, or one injected by fgl_server_inject_worker_faults) fails the
    // requests with chunks in this tick, and only them; the tick is still
    // queued, without a launch, so that their buffers are freed once the
    // ticks before it (which may write into them) are done.
    try {
      admit(S);
      items.clear();
      int64_t budget = S.o.tick_rays;
      if (S.o.mode == 0) {
        for (int64_t tk : S.active) {
          Request& q = *S.reqs[tk];
          if (q.cancel || q.env_next >= q.r.n_env || budget <= 0) continue;
          int64_t fit = budget / std::max<int32_t>(1, q.n_rays);
          int32_t chunk = (int32_t)std::min<int64_t>(q.r.n_env - q.env_next, std::max<int64_t>(1, fit));
          fgl_cast_item it{};
          it.scene = S.scenes[q.r.scene_id].scene;
          it.sensor = S.sensors[q.r.sensor_id].sensor;
          it.poses = q.d_poses + (size_t)q.env_next * 12;
          it.n_env = chunk;
          it.max_range = q.r.max_range;
          it.min_range = q.r.min_range;
          it.out_range = q.d_range + (size_t)q.env_next * q.n_rays;
          it.out_tri = q.d_tri + (size_t)q.env_next * q.n_rays;
          items.push_back(it);
          q.env_next += chunk;
          q.last_tick = t.id;
          if (q.env_next >= q.r.n_env) t.finishing.push_back(tk);
          budget -= (int64_t)chunk * q.n_rays;
        }
      } else {
        // per-environment launches, one request at a time in arrival order
        for (int64_t tk : S.active) {
          Request& q = *S.reqs[tk];
          if (q.cancel || q.env_next >= q.r.n_env) continue;
          for (int32_t e = 0; e < q.r.n_env; ++e) {
            fgl_cast_item it{};
            it.scene = S.scenes[q.r.scene_id].scene;
            it.sensor = S.sensors[q.r.sensor_id].sensor;
            it.poses = q.d_poses + (size_t)e * 12;
            it.n_env = 1;
            it.max_range = q.r.max_range;
            it.min_range = q.r.min_range;
            it.out_range = q.d_range + (size_t)e * q.n_rays;
            it.out_tri = q.d_tri + (size_t)e * q.n_rays;
            items.push_back(it);
          }
          q.env_next = q.r.n_env;
          q.last_tick = t.id;
          t.finishing.push_back(tk);
          break;
        }
      }
      // cancelled active requests with nothing in flight complete right away
      for (size_t i = 0; i < S.active.size();) {
        Request& q = *S.reqs[S.active[i]];
        if (q.cancel && (q.last_tick < 0 || q.last_tick < S.next_tick - (int64_t)S.ticks.size())) {
          detach_request(S, q);
          free_request(S, q);
          finish_request(S, q, FGL_ERR_CANCELLED);
          continue;
        }
        ++i;
      }
      if (items.empty()) {
        S.cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      ++S.next_tick;
      ++S.n_ticks;
      counted = true;
      if (S.inject_worker_fault > 0) {
        --S.inject_worker_fault;
        throw std::runtime_error("injected worker fault");
      }
      lk.unlock();
      if (S.o.mode == 0) {
        status = fgl_cast_batched(items.data(), (int32_t)items.size(), &S.o.opts, S.compute);
      } else {
        for (const fgl_cast_item& it : items) {
          status = it.min_range > 0.f
                       ? fgl_cast_batched(&it, 1, &S.o.opts, S.compute)
                       : fgl_cast(it.scene, it.sensor, it.poses, 1, it.max_range, it.out_range,
                                  it.out_tri, S.compute);
          if (status != FGL_OK) break;
        }
      }
      lk.lock();
    } catch (const std::exception& ex) {
      if (!lk.owns_lock()) lk.lock();
      status = dynamic_cast<const std::bad_alloc*>(&ex) ? FGL_ERR_OOM : FGL_ERR_INTERNAL;
      if (!counted) {
        ++S.next_tick;
        ++S.n_ticks;
      }
      // every request with a chunk in this tick ends here, with the error
      t.finishing.clear();
      for (int64_t tk : S.active) {
        Request& q = *S.reqs[tk];
        if (q.last_tick != t.id) continue;
        q.env_next = q.r.n_env;
        t.finishing.push_back(tk);
      }
    }
    cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&t.copied, cudaEventDisableTiming);
    cudaEventRecord(t.done, S.compute);
    // the copy stream follows the tick; the results of the requests it
    // finishes go back right behind it, with no host round trip in between
    cudaStreamWaitEvent(S.copy, t.done, 0);
    if (status != FGL_OK) {
      // every request with a chunk in a failed tick carries the error; the
      // ones that continue still run their later chunks (their buffers are
      // freed only after their last tick) and end with it
      for (int64_t tk : S.active) {
        Request& q = *S.reqs[tk];
        if (q.last_tick == t.id && q.status == FGL_OK) q.status = status;
      }
    }
    for (int64_t tk : t.finishing) {
      Request& q = *S.reqs[tk];
      if (status != FGL_OK) {
        q.status = status;
      } else if (q.status == FGL_OK && !q.cancel && !enqueue_result_copies(S, q)) {
        q.status = FGL_ERR_CUDA;
      }
    }
    cudaEventRecord(t.copied, S.copy);
    S.ticks.push_back(std::move(t));
    S.cv_work.notify_all();
  }
}

void completer_main(fgl_server_s* Sp) {
  fgl_server_s& S = *Sp;
  cudaSetDevice(S.device);
  for (;;) {
    std::unique_lock<std::mutex> lk(S.mu);
    S.cv_work.wait(lk, [&] { return S.stop || !S.ticks.empty(); });
    if (S.ticks.empty() && S.stop) break;
    if (S.ticks.empty()) continue;
    // one wait per tick: its casts and the result copies queued behind them
    cudaEvent_t ev = S.ticks.front().copied;
    lk.unlock();
    cudaError_t e = cudaEventSynchronize(ev);
    lk.lock();
    Tick t = std::move(S.ticks.front());
    S.ticks.pop_front();
    cudaEventDestroy(t.done);
    cudaEventDestroy(t.copied);
    S.cv_tick.notify_all();
    S.cv_done.notify_all();
    // detach the requests that finished in this tick first, so the worker
    // cannot cancel or free them meanwhile
    std::vector<Request*> fin;
    for (int64_t tk : t.finishing) {
      Request* q = S.reqs[tk].get();
      detach_request(S, *q);
      fin.push_back(q);
    }
    lk.unlock();
    for (Request* q : fin) {
      int st = (e == cudaSuccess) ? q->status : FGL_ERR_CUDA;
      if (q->cancel) {
        st = FGL_ERR_CANCELLED;
      } else if (st == FGL_OK) {
        const size_t nr = (size_t)q->r.n_env * q->n_rays;
        if (q->copy_queued && q->pageable) {
          std::memcpy(q->r.out_range, q->stage, nr * 4);
          std::memcpy(q->r.out_tri, (const float*)q->stage + nr, nr * 4);
        } else if (!q->copy_queued) {  // large results for pageable memory
          if (cudaMemcpy(q->r.out_range, q->d_range, nr * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
              cudaMemcpy(q->r.out_tri, q->d_tri, nr * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            st = FGL_ERR_CUDA;
          }
        }
      }
      q->status = st;
    }
    lk.lock();
    for (Request* q : fin) {
      free_request(S, *q);
      finish_request(S, *q, q->status);
    }
    S.cv_work.notify_all();
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  double pos = p * (v.size() - 1);
  size_t i = (size_t)pos;
  double f = pos - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

fgl_status fgl_server_create(const fgl_server_opts* opts, fgl_server* out) {
  if (!out) return set_err(FGL_ERR_INVALID, "out is null");
  *out = nullptr;
  std::unique_ptr<fgl_server_s> S(new fgl_server_s());
  if (opts) S->o = *opts;
  if (S->o.hbm_budget_bytes <= 0) S->o.hbm_budget_bytes = (int64_t)150 << 30;
  if (S->o.tick_rays <= 0) S->o.tick_rays = (int64_t)16 << 20;
  if (S->o.max_active <= 0) S->o.max_active = 4096;
  if (S->o.mode != 0 && S->o.mode != 1) return set_err(FGL_ERR_INVALID, "mode must be 0 or 1");
  if (S->o.env_capacity < 0 || S->o.env_capacity > (1 << 24))
    return set_err(FGL_ERR_INVALID, "env_capacity must be in [0, 2^24]");
  if (S->o.env_capacity == 0) S->o.env_capacity = 65536;
  S->o.opts.use_graph = 0;
  if (cudaGetDevice(&S->device) != cudaSuccess) return set_err(FGL_ERR_CUDA, "no CUDA device");
  const int64_t env_bytes = (int64_t)S->o.env_capacity * 48;
  if (env_bytes >= S->o.hbm_budget_bytes)
    return set_err(FGL_ERR_BUDGET, "the environment slot table does not fit the budget");
  if (cudaMalloc(&S->d_env, (size_t)env_bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_err(FGL_ERR_OOM, "cannot allocate the environment slot table");
  }
  S->used_bytes = env_bytes;
  S->env_readers.assign(S->o.env_capacity, 0);
  S->env_writer.assign(S->o.env_capacity, 0);
  if (cudaStreamCreateWithFlags(&S->compute, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(S->d_env);
    return set_err(FGL_ERR_CUDA, "cannot create streams");
  }
  fgl_server_s* raw = S.release();
  raw->worker = std::thread(worker_main, raw);
  raw->completer = std::thread(completer_main, raw);
  *out = raw;
  return FGL_OK;
}

fgl_status fgl_server_add_scene(fgl_server S, fgl_scene scene, int32_t* scene_id) {
  if (!S || !scene || !scene_id) return set_err(FGL_ERR_INVALID, "null argument");
  fgl_scene_stats st;
  fgl_status s = fgl_scene_get_stats(scene, &st);
  if (s != FGL_OK) return s;
  std::lock_guard<std::mutex> lk(S->mu);
  SceneEntry e;
  e.scene = scene;
  e.bytes = st.node_bytes + st.tri_bytes;
  e.resident = st.resident != 0;
  if (e.resident) {
    if (!make_room(*S, e.bytes, -1)) {
      fgl_scene_evict(scene);
      e.resident = false;
    } else {
      S->used_bytes += e.bytes;
    }
  }
  S->scenes.push_back(e);
  *scene_id = (int32_t)S->scenes.size() - 1;
  return FGL_OK;
}

fgl_status fgl_server_add_sensor(fgl_server S, fgl_sensor sensor, int32_t* sensor_id) {
  if (!S || !sensor || !sensor_id) return set_err(FGL_ERR_INVALID, "null argument");
  SensorEntry e;
  e.sensor = sensor;
  fgl_status s = fgl_sensor_n_rays(sensor, &e.n_rays);
  if (s != FGL_OK) return s;
  std::lock_guard<std::mutex> lk(S->mu);
  S->sensors.push_back(e);
  *sensor_id = (int32_t)S->sensors.size() - 1;
  return FGL_OK;
}

fgl_status fgl_server_add_envs(fgl_server S, int32_t n_env, const float* poses, int32_t* env_first) {
  if (!S || !poses || !env_first) return set_err(FGL_ERR_INVALID, "null argument");
  if (n_env < 1) return set_err(FGL_ERR_INVALID, "n_env must be >= 1");
  for (int64_t i = 0; i < 12 * (int64_t)n_env; ++i)
    if (!std::isfinite(poses[i])) return set_err(FGL_ERR_INVALID, "non-finite pose");
  std::lock_guard<std::mutex> lk(S->mu);
  if ((int64_t)S->n_envs + n_env > S->o.env_capacity)
    return set_err(FGL_ERR_CAPACITY, "environment slots exhausted (raise env_capacity)");
  const int32_t first = S->n_envs;
  // New slots: no admitted request can name them yet, so a synchronous copy
  // (on no stream of the server's) finishes before any later request reads them.
  cudaError_t e = cudaMemcpy(S->d_env + (size_t)first * 12, poses, (size_t)n_env * 48,
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(FGL_ERR_CUDA, std::string("uploading environment poses: ") + cudaGetErrorString(e));
  }
  S->n_envs += n_env;
  *env_first = first;
  return FGL_OK;
}

fgl_status fgl_server_read_poses(fgl_server S, int32_t env_first, int32_t n_env, float* out) {
  if (!S || !out) return set_err(FGL_ERR_INVALID, "null argument");
  size_t cls = 0;
  void* stage = nullptr;
  cudaEvent_t ev = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (n_env < 1 || env_first < 0 || (int64_t)env_first + n_env > S->n_envs)
      return set_err(FGL_ERR_INVALID, "slot range outside the registered environments");
    stage = S->pinned.get((size_t)n_env * 48, &cls);
    if (!stage) return set_err(FGL_ERR_OOM, "cannot allocate page-locked staging");
    // behind every update of the requests admitted so far
    if (cudaMemcpyAsync(stage, S->d_env + (size_t)env_first * 12, (size_t)n_env * 48,
                        cudaMemcpyDeviceToHost, S->compute) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, S->compute) != cudaSuccess) {
      cudaGetLastError();
      if (ev) cudaEventDestroy(ev);
      S->pinned.put(stage, cls);
      return set_err(FGL_ERR_CUDA, "reading environment poses");
    }
  }
  cudaError_t e = cudaEventSynchronize(ev);
  cudaEventDestroy(ev);
  if (e == cudaSuccess) std::memcpy(out, stage, (size_t)n_env * 48);
  std::lock_guard<std::mutex> lk(S->mu);
  S->pinned.put(stage, cls);
  if (e != cudaSuccess) return set_err(FGL_ERR_CUDA, cudaGetErrorString(e));
  return FGL_OK;
}

fgl_status fgl_server_submit(fgl_server S, const fgl_request* r, int64_t* ticket) {
  if (!S || !r || !ticket) return set_err(FGL_ERR_INVALID, "null argument");
  std::unique_ptr<Request> q(new Request());
  q->r = *r;
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->scene_id < 0 || r->scene_id >= (int32_t)S->scenes.size())
      return set_err(FGL_ERR_INVALID, "unknown scene id");
    if (r->sensor_id < 0 || r->sensor_id >= (int32_t)S->sensors.size())
      return set_err(FGL_ERR_INVALID, "unknown sensor id");
    q->n_rays = S->sensors[r->sensor_id].n_rays;
    if (r->n_env < 1) return set_err(FGL_ERR_INVALID, "n_env must be >= 1");
    if (r->pose_source < FGL_POSES_REQUEST || r->pose_source > FGL_POSES_SLOTS_SET_DEVICE)
      return set_err(FGL_ERR_INVALID, "unknown pose_source");
    if (uses_slots(r->pose_source) &&
        (r->env_first < 0 || (int64_t)r->env_first + r->n_env > S->n_envs))
      return set_err(FGL_ERR_INVALID, "slot range outside the registered environments");
    const bool needs_poses = r->pose_source != FGL_POSES_SLOTS;
    if ((needs_poses && !r->poses) || !r->out_range || !r->out_tri)
      return set_err(FGL_ERR_INVALID, "null buffer");
    if (!(std::isfinite(r->max_range) && r->max_range > 0.f))
      return set_err(FGL_ERR_INVALID, "max_range must be finite and > 0");
    if (!(r->min_range >= 0.f && r->min_range < r->max_range))
      return set_err(FGL_ERR_INVALID, "min_range must satisfy 0 <= min_range < max_range");
    q->bytes = request_bytes(r->n_env, q->n_rays, uses_slots(r->pose_source));
    if (q->bytes + S->scenes[r->scene_id].bytes + (int64_t)S->o.env_capacity * 48 >
        S->o.hbm_budget_bytes) {
      ++S->rejected;
      return set_err(FGL_ERR_BUDGET, "request needs more device memory than the whole budget");
    }
  }
  const bool host_poses = r->pose_source == FGL_POSES_REQUEST || r->pose_source == FGL_POSES_SLOTS_SET_HOST;
  if (host_poses) {
    for (int64_t i = 0; i < 12 * (int64_t)r->n_env; ++i)
      if (!std::isfinite(r->poses[i])) return set_err(FGL_ERR_INVALID, "non-finite pose");
  }
  // pageable output buffers get page-locked staging, so the copies behind a
  // tick never wait on the host
  bool pageable = false;
  for (const void* p : {(const void*)r->out_range, (const void*)r->out_tri}) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      pageable = true;
    } else if (a.type != cudaMemoryTypeHost) {
      pageable = true;
    }
  }
  const size_t res_bytes = (size_t)r->n_env * q->n_rays * 8;
  std::lock_guard<std::mutex> lk(S->mu);
  if (host_poses) {
    q->poses = (float*)S->pinned.get((size_t)r->n_env * 48, &q->poses_cls);
    if (!q->poses) return set_err(FGL_ERR_OOM, "cannot allocate page-locked pose staging");
    std::memcpy(q->poses, r->poses, (size_t)r->n_env * 48);
  }
  q->pageable = pageable;
  if (pageable && (int64_t)res_bytes <= kStageMax) {
    q->stage = S->pinned.get(res_bytes, &q->stage_cls);  // NULL: copied synchronously instead
  }
  q->ticket = S->next_ticket++;
  *ticket = q->ticket;
  if (!S->have_first) {
    S->have_first = true;
    S->t_first = q->t_submit;
  }
  ++S->submitted;
  S->pending.push_back(q->ticket);
  S->reqs[q->ticket] = std::move(q);
  S->cv_work.notify_all();
  return FGL_OK;
}

fgl_status fgl_server_wait(fgl_server S, int64_t ticket, int32_t timeout_ms, fgl_request_info* info) {
  if (!S) return set_err(FGL_ERR_INVALID, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return set_err(FGL_ERR_INVALID, "unknown ticket");
  Request& q = *it->second;
  auto done = [&] { return q.state == DONE; };
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, done);
  } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    return set_err(FGL_ERR_TIMEOUT, "request not finished within the timeout");
  }
  if (info) {
    info->status = q.status;
    info->queue_ms = q.t_admit.time_since_epoch().count() ? ms_between(q.t_submit, q.t_admit) : 0.0;
    info->latency_ms = ms_between(q.t_submit, q.t_done);
    info->rays = (int64_t)q.r.n_env * q.n_rays;
  }
  int st = q.status;
  S->pinned.put(q.poses, q.poses_cls);
  q.poses = nullptr;
  S->pinned.put(q.stage, q.stage_cls);
  q.stage = nullptr;
  S->reqs.erase(it);
  if (st != FGL_OK) {
    return set_err(st, st == FGL_ERR_CANCELLED ? "request cancelled"
                       : st == FGL_ERR_OOM ? "device allocation for the request failed"
                       : st == FGL_ERR_INTERNAL ? "a host exception in the server's worker failed the request"
                                           : "request failed");
  }
  return FGL_OK;
}

fgl_status fgl_server_cancel(fgl_server S, int64_t ticket) {
  if (!S) return set_err(FGL_ERR_INVALID, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return set_err(FGL_ERR_INVALID, "unknown ticket");
  it->second->cancel = true;
  S->cv_work.notify_all();
  return FGL_OK;
}

fgl_status fgl_server_inject_alloc_failures(fgl_server S, int32_t n) {
  if (!S || n < 0) return set_err(FGL_ERR_INVALID, "bad argument");
  std::lock_guard<std::mutex> lk(S->mu);
  S->inject_alloc_fail = n;
  return FGL_OK;
}

fgl_status fgl_server_inject_worker_faults(fgl_server S, int32_t n) {
  if (!S || n < 0) return set_err(FGL_ERR_INVALID, "bad argument");
  std::lock_guard<std::mutex> lk(S->mu);
  S->inject_worker_fault = n;
  return FGL_OK;
}

fgl_status fgl_server_get_stats(fgl_server S, fgl_server_stats* o) {
  if (!S || !o) return set_err(FGL_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(o, 0, sizeof(*o));
  o->submitted = S->submitted;
  o->completed = S->completed;
  o->rejected = S->rejected;
  o->cancelled = S->cancelled;
  o->evictions = S->evictions;
  o->uploads = S->uploads;
  o->ticks = S->n_ticks;
  o->rays = S->rays_done;
  o->p50_ms = percentile(S->latencies, 0.50);
  o->p99_ms = percentile(S->latencies, 0.99);
  double sum = 0;
  for (double v : S->latencies) sum += v;
  o->mean_ms = S->latencies.empty() ? 0.0 : sum / S->latencies.size();
  o->busy_s = S->have_first ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
  o->rays_per_s = o->busy_s > 0 ? S->rays_done / o->busy_s : 0.0;
  o->device_bytes = S->used_bytes;
  o->pending = (int64_t)S->pending.size();
  o->active = (int64_t)S->active.size();
  return FGL_OK;
}

fgl_status fgl_server_reset_stats(fgl_server S) {
  if (!S) return set_err(FGL_ERR_INVALID, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  S->submitted = S->completed = S->rejected = S->cancelled = S->evictions = S->uploads = 0;
  S->n_ticks = S->rays_done = 0;
  S->latencies.clear();
  S->have_first = false;
  return FGL_OK;
}

fgl_status fgl_server_destroy(fgl_server S) {
  if (!S) return FGL_OK;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // let in-flight ticks finish, then stop both threads
    S->cv_done.wait_for(lk, std::chrono::seconds(60), [&] { return S->ticks.empty(); });
    S->stop = true;
    S->cv_work.notify_all();
    S->cv_tick.notify_all();
  }
  S->worker.join();
  S->completer.join();
  cudaStreamSynchronize(S->compute);
  cudaStreamSynchronize(S->copy);
  for (auto& kv : S->reqs) {
    Request& q = *kv.second;
    if (q.d_buf) cudaFree(q.d_buf);
  }
  for (SceneEntry& e : S->scenes) e.active = 0;
  for (auto& kv : S->reqs) {
    if (kv.second->poses) cudaFreeHost(kv.second->poses);
    if (kv.second->stage) cudaFreeHost(kv.second->stage);
  }
  cudaFree(S->d_env);
  S->pinned.release_all();
  cudaStreamDestroy(S->compute);
  cudaStreamDestroy(S->copy);
  delete S;
  return FGL_OK;
}

}  // extern "C"
