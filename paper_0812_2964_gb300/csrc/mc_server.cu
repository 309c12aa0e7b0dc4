// Serving (include/mc_server.h): continuous batching of weight-estimation
// jobs.  A host thread admits queued jobs into free slots (one CUDA stream
// each) while their device memory fits the budget, keeps every admitted
// job at most two weight iterations ahead of the GPU, and collects jobs
// as they finish.  Each job is driven only through the mc.h calls on its
// slot's stream, so its results are those of the same job run alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mc_server.h"
#include "mc_internal.h"

namespace {

constexpr int kAhead = 2;  // iterations a slot may have queued beyond the GPU

enum class State { Queued, Active, Done };

struct Rec {
  uint64_t id = 0;
  mc_jobspec spec{};
  State state = State::Queued;
  mc_job* job = nullptr;
  int slot = -1;
  int it_enq = 0, it_done = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  uint64_t bytes = 0;
  int status = MC_OK;
  std::string err;
  std::vector<double> W;
  int64_t joined = 0;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev[kAhead] = {};
  Rec* rec = nullptr;
};

}  // namespace

struct mc_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<uint64_t, std::unique_ptr<Rec>> recs;
  std::deque<Rec*> queue;
  std::vector<Slot> slots;
  uint64_t budget = 0, in_use = 0, peak = 0;
  int active = 0, peak_active = 0, finished = 0;
  uint64_t next_id = 1, admitted = 0, completed = 0;
  bool stopping = false;
  int device = 0, num_sms = 0;
  std::chrono::steady_clock::time_point t0;
  std::thread worker;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

bool spec_ok(const mc_jobspec& s) {
  return s.L >= 4 && s.L <= 128 && s.L % 4 == 0 && s.n_chains >= 1 && s.n_chains <= (1 << 24) &&
         (s.start == 0 || s.start == 1) && s.iterations >= 1 && s.sweeps >= 1 &&
         s.sweeps < (int64_t(1) << 34) / (static_cast<int64_t>(s.L) * s.L);
}

// Called with the lock held: the job ends (status set by the caller).
void finish_locked(mc_server* srv, Rec* r) {
  r->state = State::Done;
  r->t_done = srv->now();
  if (r->slot >= 0) {
    srv->slots[r->slot].rec = nullptr;
    srv->in_use -= r->bytes;
    srv->active -= 1;
    srv->completed += 1;
  }
  srv->finished += 1;
  srv->cv_done.notify_all();
}

// Without the lock: create the job's device state on its slot's stream.
int admit_job(mc_server* srv, Rec* r) {
  const mc_jobspec& s = r->spec;
  mc_job* j = nullptr;
  int rc = mc_init(s.L, s.n_chains, s.seed, s.start, &j);
  if (rc == MC_OK) rc = mc_set_stream(j, srv->slots[r->slot].st);
  if (rc == MC_OK) {
    // fullest warps: the job's rounds take as long as alone, on fewer warps
    const mcgpu::LaunchShape d = mcgpu::dense_shape(s.L, s.n_chains, srv->num_sms);
    rc = mc_set_launch_shape(j, d.placement, d.cpw, d.wpb);
  }
  if (rc != MC_OK) {
    r->err = mc_last_error();
    if (j) mc_free(j);
    return rc;
  }
  r->job = j;
  return MC_OK;
}

// Without the lock: queue one weight iteration (round, joint, update).
int enqueue_iteration(mc_server* srv, Rec* r) {
  Slot& sl = srv->slots[r->slot];
  int rc = mc_run_sweeps(r->job, r->spec.sweeps);
  if (rc == MC_OK) rc = mc_join(r->job, nullptr);
  if (rc == MC_OK) rc = mc_update_weights(r->job);
  if (rc == MC_OK) {
    const cudaError_t e = cudaEventRecord(sl.ev[r->it_enq % kAhead], sl.st);
    if (e != cudaSuccess) {
      r->err = cudaGetErrorString(e);
      return MC_ECUDA;
    }
  } else {
    r->err = mc_last_error();
  }
  return rc;
}

// Without the lock: read the result and release the job's device state.
int collect_job(Rec* r) {
  const int N = r->spec.L * r->spec.L;
  r->W.assign(N + 1, 0.0);
  int rc = mc_get_weights(r->job, r->W.data(), N + 1);
  mc_info info;
  if (rc == MC_OK) rc = mc_get_info(r->job, &info);
  if (rc == MC_OK) r->joined = info.total_joined;
  else r->err = mc_last_error();
  mc_free(r->job);
  r->job = nullptr;
  return rc;
}

void worker_main(mc_server* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    bool progressed = false;
    // admission: first fit in arrival order
    std::vector<Rec*> admit;
    for (auto it = srv->queue.begin(); it != srv->queue.end();) {
      Rec* r = *it;
      int free_slot = -1;
      for (int s = 0; s < static_cast<int>(srv->slots.size()); ++s)
        if (!srv->slots[s].rec) {
          free_slot = s;
          break;
        }
      if (free_slot < 0) break;
      if (srv->in_use + r->bytes > srv->budget) {
        ++it;
        continue;
      }
      r->slot = free_slot;
      r->state = State::Active;
      r->t_admit = srv->now();
      srv->slots[free_slot].rec = r;
      srv->in_use += r->bytes;
      srv->peak = std::max(srv->peak, srv->in_use);
      srv->active += 1;
      srv->peak_active = std::max(srv->peak_active, srv->active);
      srv->admitted += 1;
      admit.push_back(r);
      it = srv->queue.erase(it);
    }
    std::vector<Rec*> running;
    for (auto& sl : srv->slots)
      if (sl.rec && sl.rec->job) running.push_back(sl.rec);
    lk.unlock();

    std::vector<std::pair<Rec*, int>> ended;
    for (Rec* r : admit) {
      const int rc = admit_job(srv, r);
      progressed = true;
      if (rc != MC_OK) ended.push_back({r, rc});
      else running.push_back(r);
    }
    for (Rec* r : running) {
      Slot& sl = srv->slots[r->slot];
      int rc = MC_OK;
      while (r->it_done < r->it_enq) {
        const cudaError_t q = cudaEventQuery(sl.ev[r->it_done % kAhead]);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) {
          r->err = cudaGetErrorString(q);
          rc = MC_ECUDA;
          break;
        }
        r->it_done += 1;
        progressed = true;
      }
      while (rc == MC_OK && r->it_enq < r->spec.iterations && r->it_enq - r->it_done < kAhead) {
        rc = enqueue_iteration(srv, r);
        if (rc == MC_OK) r->it_enq += 1;
        progressed = true;
      }
      if (rc == MC_OK && r->it_done == r->spec.iterations) {
        rc = collect_job(r);
        ended.push_back({r, rc});
        progressed = true;
      } else if (rc != MC_OK) {
        if (r->job) {
          mc_free(r->job);
          r->job = nullptr;
        }
        ended.push_back({r, rc});
      }
    }

    lk.lock();
    for (auto& e : ended) {
      e.first->status = e.second;
      finish_locked(srv, e.first);
    }
    if (srv->stopping && srv->queue.empty() && srv->active == 0) break;
    if (!progressed) srv->cv_work.wait_for(lk, std::chrono::microseconds(100));
  }
}

}  // namespace

extern "C" {

int mc_server_create(uint64_t budget_bytes, int max_slots, mc_server** out) {
  if (!out) return MC_EINVAL;
  *out = nullptr;
  if (max_slots < 1 || max_slots > 64 || budget_bytes == 0) {
    mcgpu::set_last_error("mc_server_create: need 1 <= max_slots <= 64 and a nonzero budget");
    return MC_EINVAL;
  }
  mc_server* srv = new (std::nothrow) mc_server();
  if (!srv) return MC_ENOMEM;
  srv->budget = budget_bytes;
  srv->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&srv->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&srv->num_sms, cudaDevAttrMultiProcessorCount, srv->device);
  srv->slots.resize(max_slots);
  for (auto& sl : srv->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    for (int k = 0; k < kAhead && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&sl.ev[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    mcgpu::set_last_error(cudaGetErrorString(e));
    for (auto& sl : srv->slots) {
      for (auto& ev : sl.ev)
        if (ev) cudaEventDestroy(ev);
      if (sl.st) cudaStreamDestroy(sl.st);
    }
    delete srv;
    return e == cudaErrorMemoryAllocation ? MC_ENOMEM : MC_ECUDA;
  }
  try {
    srv->worker = std::thread(worker_main, srv);
  } catch (...) {  // no thread: release everything, nothing crosses the ABI
    for (auto& sl : srv->slots) {
      for (auto& ev : sl.ev)
        if (ev) cudaEventDestroy(ev);
      if (sl.st) cudaStreamDestroy(sl.st);
    }
    delete srv;
    mcgpu::set_last_error("mc_server_create: could not start the server thread");
    return MC_ENOMEM;
  }
  *out = srv;
  return MC_OK;
}

int mc_server_submit(mc_server* srv, const mc_jobspec* spec, uint64_t* id) {
  if (!srv || !spec || !id) return MC_EINVAL;
  if (!spec_ok(*spec)) {
    mcgpu::set_last_error("mc_server_submit: bad job spec");
    return MC_EINVAL;
  }
  const uint64_t bytes = mc_job_device_bytes(spec->L, spec->n_chains, spec->sweeps);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stopping) return MC_ESTATE;
  if (bytes > srv->budget) {
    mcgpu::set_last_error("mc_server_submit: the job alone exceeds the device-memory budget");
    return MC_ENOMEM;
  }
  std::unique_ptr<Rec> r(new (std::nothrow) Rec());
  if (!r) return MC_ENOMEM;
  r->id = srv->next_id++;
  r->spec = *spec;
  r->bytes = bytes;
  r->t_submit = srv->now();
  *id = r->id;
  try {
    srv->queue.push_back(r.get());
    srv->recs.emplace(r->id, std::move(r));
  } catch (...) {
    if (!srv->queue.empty() && r && srv->queue.back() == r.get()) srv->queue.pop_back();
    return MC_ENOMEM;
  }
  srv->cv_work.notify_one();
  return MC_OK;
}

int mc_server_poll(mc_server* srv, uint64_t id, int* done) {
  if (!srv || !done) return MC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->recs.find(id);
  if (it == srv->recs.end()) return MC_EINVAL;
  *done = it->second->state == State::Done ? 1 : 0;
  return MC_OK;
}

int mc_server_wait(mc_server* srv, uint64_t id, double* W_out, int n, mc_jobstats* stats) {
  if (!srv) return MC_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->recs.find(id);
  if (it == srv->recs.end()) {
    mcgpu::set_last_error("mc_server_wait: unknown id");
    return MC_EINVAL;
  }
  Rec* r = it->second.get();
  const int np1 = r->spec.L * r->spec.L + 1;
  if ((W_out && n != np1) || (!W_out && n != 0)) {
    mcgpu::set_last_error("mc_server_wait: W_out needs N+1 entries");
    return MC_EINVAL;
  }
  srv->cv_done.wait(lk, [r] { return r->state == State::Done; });
  if (W_out && r->status == MC_OK) std::copy(r->W.begin(), r->W.end(), W_out);
  if (stats) {
    const int64_t N = static_cast<int64_t>(r->spec.L) * r->spec.L;
    stats->status = r->status;
    stats->slot = r->slot;
    stats->t_submit = r->t_submit;
    stats->t_admit = r->t_admit;
    stats->t_done = r->t_done;
    stats->attempts = static_cast<int64_t>(r->spec.n_chains) * r->spec.iterations * r->spec.sweeps * N;
    stats->joined = r->joined;
    stats->device_bytes = r->bytes;
  }
  const int status = r->status;
  if (status != MC_OK) mcgpu::set_last_error(r->err.c_str());
  srv->finished -= 1;
  srv->recs.erase(it);
  return status;
}

int mc_server_get_info(mc_server* srv, mc_server_info* info) {
  if (!srv || !info) return MC_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  info->max_slots = static_cast<int>(srv->slots.size());
  info->queued = static_cast<int>(srv->queue.size());
  info->active = srv->active;
  info->finished = srv->finished;
  info->budget_bytes = srv->budget;
  info->bytes_in_use = srv->in_use;
  info->peak_bytes = srv->peak;
  info->peak_active = srv->peak_active;
  info->admitted = srv->admitted;
  info->completed = srv->completed;
  return MC_OK;
}

double mc_server_clock(mc_server* srv) { return srv ? srv->now() : 0.0; }

void mc_server_free(mc_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stopping = true;
    while (!srv->queue.empty()) {
      Rec* r = srv->queue.front();
      srv->queue.pop_front();
      r->status = MC_ESTATE;
      r->err = "cancelled: server stopped before admission";
      finish_locked(srv, r);
    }
    srv->cv_work.notify_one();
  }
  if (srv->worker.joinable()) srv->worker.join();
  for (auto& sl : srv->slots) {
    for (auto& ev : sl.ev)
      if (ev) cudaEventDestroy(ev);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  delete srv;
}

}  // extern "C"
