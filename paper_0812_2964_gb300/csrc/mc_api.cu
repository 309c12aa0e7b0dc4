// C ABI (include/mc.h): job lifetime, device memory, stream ordering and
// argument checking around the kernels of mc_kernels.cu.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mc.h"
#include "../../include/mc_server.h"
#include "mc_batch.h"
#include "mc_internal.h"

using mcgpu::DevJob;
using mcgpu::LaunchShape;

namespace {
thread_local std::string g_err;
}  // namespace

void mcgpu::set_last_error(const char* msg) { g_err = msg; }

namespace {

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? MC_ENOMEM : MC_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e),
              cudaGetErrorString(e));
}

#define MC_CUDA(call, what)                  \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

}  // namespace

struct mc_job {
  DevJob d;
  int L, N, p, wd, start;
  uint64_t seed;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  int device = 0, num_sms = 0;
  uint64_t t = 0;       // attempts per chain so far
  uint32_t r = 0;       // joints done
  int64_t last_S = 0;
  int64_t last_M = 0;           // attempts per chain of the last round
  bool attempts_round = false;  // the last round was not whole sweeps from a sweep start
  bool attempts_recorded = false;  // ... and its samples' levels are in d.plv
  size_t plv_cap = 0;           // int32 entries of d.plv
  long long plv_max = mcgpu::kPartialLevelsMax;  // largest p * M recorded
  uint16_t* rec_buf = nullptr;  // record of whole-sweep rounds (d.rec points here when used)
  size_t rec_cap = 0;           // uint16 entries of rec_buf
  long long rec_max = 0;                         // largest p * M recorded (set by mc_init)
  bool pending = false;
  bool trace_on = false;
  bool trace_valid = false;
  size_t trace_cap = 0;  // int32 elements
  LaunchShape shape;
  LaunchShape bshape{};          // shape in a fused batch launch (mc_batch_autotune)
  bool bshape_valid = false;
  int64_t seg_samples = 0;  // target samples per checkpoint segment (0: default)
  size_t bytes = 0;
  std::vector<void*> allocs;
};

namespace {

// Device memory of a job comes from the device's stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync on the job's stream): freeing a job does
// not wait for work of other jobs, which a server running many jobs at once
// relies on.  The pool keeps freed memory for later jobs.
//
// Failure injection (mc_inject_alloc_failure): with g_fail_after = n >= 0,
// n more allocations succeed and the next one fails on the host, before any
// CUDA call, as an out-of-memory would.  g_live counts the allocations held.
std::atomic<long long> g_fail_after{-1};
std::atomic<long long> g_live{0};

void raw_free(mc_job* j, void* v) {
  if (v) {
    cudaFreeAsync(v, j->stream);
    g_live.fetch_sub(1);
  }
}

cudaError_t raw_alloc(mc_job* j, void** v, size_t bytes) {
  long long n = g_fail_after.load();
  while (n >= 0 && !g_fail_after.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 0) {
    *v = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMallocAsync(v, bytes ? bytes : 1, j->stream);
  if (e == cudaSuccess) g_live.fetch_add(1);
  return e;
}

template <class T>
int dalloc(mc_job* j, T** p, size_t count) {
  void* v = nullptr;
  const size_t b = sizeof(T) * (count ? count : 1);
  cudaError_t e = raw_alloc(j, &v, b);
  if (e != cudaSuccess) return cuda_fail(e, "device allocation");
  j->allocs.push_back(v);
  j->bytes += b;
  *p = static_cast<T*>(v);
  return MC_OK;
}

void free_all(mc_job* j) {
  if (j->stream) {
    for (void* v : j->allocs) raw_free(j, v);
    raw_free(j, j->d.ckpt);
    raw_free(j, j->d.ckm);
    raw_free(j, j->d.plist);
    raw_free(j, j->d.trace);
    raw_free(j, j->d.plv);
    raw_free(j, j->rec_buf);
  }
  j->d.plv = nullptr;
  j->rec_buf = nullptr;
  j->d.rec = nullptr;
  j->allocs.clear();
  j->d.plist = nullptr;
  j->d.ckpt = nullptr;
  j->d.ckm = nullptr;
  j->d.trace = nullptr;
  if (j->own_stream) cudaStreamDestroy(j->own_stream);
  j->own_stream = nullptr;
  j->stream = nullptr;
}

// Once per device: the pool behind raw_alloc keeps what jobs free.
cudaError_t pool_setup(int device) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lk(mu);
  if (std::find(done.begin(), done.end(), device) != done.end()) return cudaSuccess;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = cudaDeviceGetDefaultMemPool(&pool, device);
  uint64_t keep = ~0ull;
  if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  if (e == cudaSuccess) done.push_back(device);
  return e;
}

int check_job(mc_job* j) {
  if (!j) return fail(MC_EINVAL, "null job");
  return MC_OK;
}

int sync(mc_job* j, const char* what) {
  MC_CUDA(cudaStreamSynchronize(j->stream), what);
  return MC_OK;
}

}  // namespace

extern "C" {

const char* mc_last_error(void) { return g_err.c_str(); }

int mc_inject_alloc_failure(int64_t after) {
  g_fail_after.store(after < 0 ? -1 : after);
  return MC_OK;
}

int64_t mc_live_allocations(void) { return g_live.load(); }

uint64_t mc_kernel_launches(void) { return mcgpu::launches_add(0); }

static int mc_init_impl(int L, int n_chains, uint64_t seed, int start, mc_job** out) {
  if (!out) return fail(MC_EINVAL, "out is null");
  *out = nullptr;
  if (L < 4 || L > 128 || (L % 4) != 0) return fail(MC_EINVAL, "L=%d: need 4 <= L <= 128, L %% 4 == 0", L);
  if (n_chains < 1 || n_chains > (1 << 24)) return fail(MC_EINVAL, "n_chains=%d out of range", n_chains);
  if (start != 0 && start != 1) return fail(MC_EINVAL, "start=%d: 0 (all up) or 1 (random)", start);
  mc_job* j = new (std::nothrow) mc_job();
  if (!j) return fail(MC_ENOMEM, "host allocation");
  j->L = L;
  j->N = L * L;
  j->p = n_chains;
  j->wd = (L + 31) / 32;
  j->start = start;
  j->seed = seed;
  int rc = MC_OK;
  cudaError_t e = cudaGetDevice(&j->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&j->num_sms, cudaDevAttrMultiProcessorCount, j->device);
  if (e == cudaSuccess) e = pool_setup(j->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&j->own_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "device setup");
    free_all(j);
    delete j;
    return rc;
  }
  j->stream = j->own_stream;
  DevJob& d = j->d;
  std::memset(&d, 0, sizeof d);
  d.L = L;
  d.N = j->N;
  d.np1 = j->N + 1;
  d.wd = j->wd;
  d.p = n_chains;
  d.key0 = static_cast<uint32_t>(seed);
  d.key1 = static_cast<uint32_t>(seed >> 32);
  d.passes_scan = mcgpu::kGridPassesScan;
  d.passes_plain = mcgpu::kGridPasses;
  d.scan_max_samples = mcgpu::kScanMaxSamples;
  const size_t lat = static_cast<size_t>(n_chains) * L * j->wd;
  const size_t np1 = static_cast<size_t>(d.np1);
  if ((rc = dalloc(j, &d.spins, lat)) || (rc = dalloc(j, &d.spins0, lat)) || (rc = dalloc(j, &d.m, n_chains)) ||
      (rc = dalloc(j, &d.m0, n_chains)) || (rc = dalloc(j, &d.W, np1)) || (rc = dalloc(j, &d.T, 5 * np1)) ||
      (rc = dalloc(j, &d.h, np1)) || (rc = dalloc(j, &d.hgen, np1)) || (rc = dalloc(j, &d.dpre, np1)) ||
      (rc = dalloc(j, &d.k, n_chains)) ||
      (rc = dalloc(j, &d.xused, n_chains)) || (rc = dalloc(j, &d.tj, static_cast<size_t>(n_chains) * np1)) ||
      (rc = dalloc(j, &d.offsets, n_chains)) || (rc = dalloc(j, &d.work, n_chains)) ||
      (rc = dalloc(j, &d.work2, n_chains)) ||
      (rc = dalloc(j, &d.lastacc, n_chains)) || (rc = dalloc(j, &d.summ, 5ull * n_chains)) || (rc = dalloc(j, &d.visited, np1)) ||
      (rc = dalloc(j, &d.perm, n_chains)) || (rc = dalloc(j, &d.lvcnt, np1)) || (rc = dalloc(j, &d.kmin, n_chains)) ||
      (rc = dalloc(j, &d.stats, mcgpu::kStatCount))) {
    free_all(j);
    delete j;
    return rc;
  }
  cudaStream_t st = j->stream;
  e = cudaMemsetAsync(d.W, 0, sizeof(double) * np1, st);  // w^(1) = 1
  if (e == cudaSuccess) e = cudaMemsetAsync(d.h, 0, sizeof(long long) * np1, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.visited, 0, np1, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.hgen, 0, sizeof(unsigned long long) * np1, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.dpre, 0, sizeof(unsigned long long) * np1, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.stats, 0, sizeof(long long) * mcgpu::kStatCount, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.k, 0, sizeof(int64_t) * n_chains, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.offsets, 0, sizeof(int64_t) * n_chains, st);
  if (e == cudaSuccess) e = mcgpu::k_init_lattice(d, start, st);
  if (e == cudaSuccess) e = mcgpu::k_levels(d, st);
  if (e == cudaSuccess) e = mcgpu::k_order(d, st);   // identity until ordered joining is chosen
  if (e == cudaSuccess) e = mcgpu::k_build_table(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "job initialisation");
    free_all(j);
    delete j;
    return rc;
  }
  j->shape = mcgpu::default_shape(L, n_chains, j->num_sms);
  j->rec_max = mcgpu::default_record_max(L);
  *out = j;
  return MC_OK;
}

// (host allocations inside may throw; nothing crosses the ABI)
int mc_init(int L, int n_chains, uint64_t seed, int start, mc_job** out) {
  try {
    return mc_init_impl(L, n_chains, seed, start, out);
  } catch (const std::bad_alloc&) {
    return fail(MC_ENOMEM, "mc_init: host allocation failed");
  } catch (...) {
    return fail(MC_EINVAL, "mc_init: unexpected host error");
  }
}

void mc_free(mc_job* job) {
  if (!job) return;
  if (job->stream) cudaStreamSynchronize(job->stream);
  free_all(job);
  delete job;
}

int mc_set_stream(mc_job* job, void* cuda_stream) {
  if (int rc = check_job(job)) return rc;
  MC_CUDA(cudaStreamSynchronize(job->stream), "stream switch");
  job->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : job->own_stream;
  return MC_OK;
}

int mc_set_trace(mc_job* job, int enabled) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending");
  job->trace_on = enabled != 0;
  return MC_OK;
}

int mc_set_launch_shape(mc_job* job, int placement, int cpw, int wpb) {
  if (int rc = check_job(job)) return rc;
  LaunchShape s{placement, cpw, wpb};
  if (!mcgpu::shape_supported(job->L, s))
    return fail(MC_EINVAL, "launch shape (%d, %d, %d) not supported for L=%d", placement, cpw, wpb, job->L);
  job->shape = s;
  return MC_OK;
}

}  // extern "C"

namespace {

// Segments of a round for the joint's parallel replays.  Every replay of
// the joint (search, summary, discarded prefixes) runs one segment per lane,
// so the segment length bounds the joint's critical path: segments of about
// `target` samples (whole sweeps), at least 32 of them (or S), at most 2^24
// samples each (the prefix pass relies on that bound), and no more segments
// than kCheckpointBytes of checkpoints allow.
constexpr int64_t kSegmentSamples = int64_t(1) << 16;   // default target
constexpr int64_t kCheckpointBytes = int64_t(4) << 30;   // per job

// Bytes of the checkpoint buffers per segment: lattices, levels, prefix work list.
size_t bytes_per_segment(int L, int p) {
  const size_t lw = static_cast<size_t>(L) * ((L + 31) / 32);
  return static_cast<size_t>(p) * (lw * 4 + 4 + 8);
}

void round_segments(int L, int p, int64_t n_sweeps, int64_t target, int* K, int* C) {
  const int64_t N = static_cast<int64_t>(L) * L;
  if (target <= 0) target = kSegmentSamples;
  int64_t c = std::max<int64_t>(1, target / N);                      // sweeps per segment
  const int64_t kmem = std::max<int64_t>(1, kCheckpointBytes / static_cast<int64_t>(bytes_per_segment(L, p)));
  if ((n_sweeps + c - 1) / c > kmem) c = (n_sweeps + kmem - 1) / kmem;  // fewer, longer segments
  const int64_t kmin = std::min<int64_t>(32, n_sweeps);
  if ((n_sweeps + c - 1) / c < kmin) c = (n_sweeps + kmin - 1) / kmin; // enough segments to spread
  c = std::min<int64_t>(c, std::max<int64_t>(1, (int64_t(1) << 24) / N));
  *C = static_cast<int>(c);
  *K = static_cast<int>((n_sweeps + c - 1) / c);
}

// Bytes of the checkpoint buffers for K segments.
size_t segment_bytes(const mc_job* job, int K) { return static_cast<size_t>(K) * bytes_per_segment(job->L, job->p); }

// Checkpoint buffers for at least K segments.
int ensure_segments(mc_job* job, int K) {
  DevJob& d = job->d;
  if (K <= d.kcap && d.ckpt) return MC_OK;
  const size_t lw = static_cast<size_t>(job->L) * job->wd;
  const size_t p = static_cast<size_t>(job->p);
  if (d.ckpt) {
    raw_free(job, d.ckpt);
    raw_free(job, d.ckm);
    raw_free(job, d.plist);
    job->bytes -= segment_bytes(job, d.kcap);
    d.ckpt = nullptr;
    d.ckm = nullptr;
    d.plist = nullptr;
    d.kcap = 0;
  }
  void *a = nullptr, *b = nullptr, *w = nullptr;
  cudaError_t e = raw_alloc(job, &a, static_cast<size_t>(K) * lw * p * 4);
  if (e == cudaSuccess) e = raw_alloc(job, &b, static_cast<size_t>(K) * p * 4);
  if (e == cudaSuccess) e = raw_alloc(job, &w, static_cast<size_t>(K) * p * 8);
  if (e != cudaSuccess) {
    raw_free(job, a);
    raw_free(job, b);
    raw_free(job, w);
    return cuda_fail(e, "checkpoint allocation");
  }
  d.ckpt = static_cast<uint32_t*>(a);
  d.ckm = static_cast<int32_t*>(b);
  d.plist = static_cast<int2*>(w);
  d.kcap = K;
  job->bytes += segment_bytes(job, K);
  return MC_OK;
}

// Device trace buffer big enough for n_sweeps sweeps of every chain.
int ensure_trace(mc_job* job, int64_t n_sweeps) {
  DevJob& d = job->d;
  const size_t need = static_cast<size_t>(n_sweeps) * job->p;
  if (need <= job->trace_cap) return MC_OK;
  if (d.trace) {
    raw_free(job, d.trace);
    job->bytes -= job->trace_cap * sizeof(int32_t);
    d.trace = nullptr;
    job->trace_cap = 0;
  }
  void* v = nullptr;
  MC_CUDA(raw_alloc(job, &v, need * sizeof(int32_t)), "trace allocation");
  d.trace = static_cast<int32_t*>(v);
  job->trace_cap = need;
  job->bytes += need * sizeof(int32_t);
  return MC_OK;
}

// Record buffer for a whole-sweep round of p * M samples (uint16 each, the
// chains padded to whole tiles of the layout), or none when the round is
// larger than the job's limit (the joint replays).
int ensure_record(mc_job* job, int64_t M, bool allow) {
  DevJob& d = job->d;
  d.rec = nullptr;
  if (!allow || static_cast<long long>(job->p) * M > job->rec_max) return MC_OK;
  const long long samples = mcgpu::rec_entries(job->p, M);
  if (static_cast<size_t>(samples) > job->rec_cap) {
    if (job->rec_buf) {
      raw_free(job, job->rec_buf);
      job->bytes -= job->rec_cap * sizeof(uint16_t);
      job->rec_buf = nullptr;
      job->rec_cap = 0;
    }
    void* v = nullptr;
    MC_CUDA(raw_alloc(job, &v, static_cast<size_t>(samples) * sizeof(uint16_t)), "round record allocation");
    job->rec_buf = static_cast<uint16_t*>(v);
    job->rec_cap = static_cast<size_t>(samples);
    job->bytes += job->rec_cap * sizeof(uint16_t);
  }
  d.rec = job->rec_buf;
  return MC_OK;
}

// Start a round: checks, round-start copies (for the joint's replays) and the
// host bookkeeping; *t0 = attempts each chain made before this round.  With
// allow_record the round's levels are recorded when it is small enough (the
// fused batch launch writes no record).
int round_prepare(mc_job* job, int64_t n_sweeps, uint64_t* t0, bool allow_record = true) {
  if (job->pending) return fail(MC_ESTATE, "previous round not joined");
  if (n_sweeps < 1) return fail(MC_EINVAL, "n_sweeps=%lld", static_cast<long long>(n_sweeps));
  const int64_t M = n_sweeps * job->N;
  if (n_sweeps > (int64_t(1) << 34) / job->N || M >= (int64_t(1) << 34))
    return fail(MC_EINVAL, "n_sweeps * N must stay below 2^34");
  if (job->trace_on)
    if (int rc = ensure_trace(job, n_sweeps)) return rc;
  int K = 0, C = 0;
  round_segments(job->L, job->p, n_sweeps, job->seg_samples, &K, &C);
  if (int rc = ensure_segments(job, K)) return rc;
  if (int rc = ensure_record(job, M, allow_record)) return rc;
  DevJob& d = job->d;
  d.ck_K = K;
  d.ck_C = C;
  d.seg_len = static_cast<int64_t>(C) * job->N;
  const size_t lat = static_cast<size_t>(job->p) * job->L * job->wd;
  MC_CUDA(cudaMemcpyAsync(d.spins0, d.spins, lat * sizeof(uint32_t), cudaMemcpyDeviceToDevice, job->stream),
          "round-start copy");
  MC_CUDA(cudaMemcpyAsync(d.m0, d.m, job->p * sizeof(int32_t), cudaMemcpyDeviceToDevice, job->stream),
          "round-start copy");
  *t0 = job->t;
  job->t += static_cast<uint64_t>(M);
  job->last_S = n_sweeps;
  job->last_M = M;
  job->attempts_round = false;
  job->pending = true;
  job->trace_valid = job->trace_on;
  return MC_OK;
}

// A round of n attempts that does not start or end on a sweep: the level of
// every sample is recorded for the joint when p * n is small enough
// (kPartialLevelsMax), else round-start copies serve the serial joint's
// replays; no checkpoints, no trace.
int attempts_prepare(mc_job* job, int64_t n, uint64_t* t0) {
  if (job->pending) return fail(MC_ESTATE, "previous round not joined");
  if (n < 1 || n >= (int64_t(1) << 34)) return fail(MC_EINVAL, "n_attempts=%lld", static_cast<long long>(n));
  DevJob& d = job->d;
  d.rec = nullptr;   // (their levels go to plv)
  const long long entries = static_cast<long long>(job->p) * n;
  job->attempts_recorded = entries <= job->plv_max;
  if (job->attempts_recorded && static_cast<size_t>(entries) > job->plv_cap) {
    if (d.plv) {
      raw_free(job, d.plv);
      job->bytes -= job->plv_cap * sizeof(int32_t);
      d.plv = nullptr;
      job->plv_cap = 0;
    }
    void* v = nullptr;
    MC_CUDA(raw_alloc(job, &v, static_cast<size_t>(entries) * sizeof(int32_t)), "level record allocation");
    d.plv = static_cast<int32_t*>(v);
    job->plv_cap = static_cast<size_t>(entries);
    job->bytes += job->plv_cap * sizeof(int32_t);
  }
  const size_t lat = static_cast<size_t>(job->p) * job->L * job->wd;
  MC_CUDA(cudaMemcpyAsync(d.spins0, d.spins, lat * sizeof(uint32_t), cudaMemcpyDeviceToDevice, job->stream),
          "round-start copy");
  MC_CUDA(cudaMemcpyAsync(d.m0, d.m, job->p * sizeof(int32_t), cudaMemcpyDeviceToDevice, job->stream),
          "round-start copy");
  *t0 = job->t;
  job->t += static_cast<uint64_t>(n);
  job->last_S = n / job->N;
  job->last_M = n;
  job->attempts_round = true;
  job->pending = true;
  job->trace_valid = false;
  return MC_OK;
}

}  // namespace

extern "C" {

int mc_run_attempts(mc_job* job, int64_t n_attempts) {
  if (int rc = check_job(job)) return rc;
  const int64_t N = job->N;
  if (n_attempts >= 1 && n_attempts % N == 0 && job->t % static_cast<uint64_t>(N) == 0)
    return mc_run_sweeps(job, n_attempts / N);
  uint64_t t0 = 0;
  if (int rc = attempts_prepare(job, n_attempts, &t0)) return rc;
  MC_CUDA(mcgpu::k_generate_attempts(job->d, t0, n_attempts, job->attempts_recorded, job->stream), "generation");
  return MC_OK;
}

int mc_run_sweeps(mc_job* job, int64_t n_sweeps) {
  if (int rc = check_job(job)) return rc;
  if (job->t % static_cast<uint64_t>(job->N) != 0) {   // chains are inside a sweep
    if (n_sweeps < 1 || n_sweeps > (int64_t(1) << 34) / job->N)
      return fail(MC_EINVAL, "n_sweeps=%lld", static_cast<long long>(n_sweeps));
    return mc_run_attempts(job, n_sweeps * job->N);
  }
  uint64_t t0 = 0;
  if (int rc = round_prepare(job, n_sweeps, &t0)) return rc;
  MC_CUDA(mcgpu::k_generate(job->d, job->shape, t0, n_sweeps, job->trace_on, job->stream), "generation");
  return MC_OK;
}

static int join_common(mc_job* job, int64_t* joined_len, bool naive) {
  if (int rc = check_job(job)) return rc;
  if (!job->pending) return fail(MC_ESTATE, "no round to join");
  const int64_t M = job->last_M;
  if (job->attempts_round)
    MC_CUDA(mcgpu::k_join_attempts(job->d, job->t - static_cast<uint64_t>(M), M, job->r, naive,
                                   job->attempts_recorded, job->stream),
            "joint");
  else
    MC_CUDA(mcgpu::k_join(job->d, job->shape, job->t - static_cast<uint64_t>(M), job->last_S, job->r, naive,
                          job->stream),
            "joint");
  job->r += 1;
  job->pending = false;
  if (joined_len) {
    long long v = 0;
    MC_CUDA(cudaMemcpyAsync(&v, job->d.stats + mcgpu::kStatJoined, sizeof v, cudaMemcpyDeviceToHost, job->stream),
            "read joined length");
    if (int rc = sync(job, "joint")) return rc;
    *joined_len = v;
  }
  return MC_OK;
}

int mc_join(mc_job* job, int64_t* joined_len) { return join_common(job, joined_len, false); }
int mc_join_naive(mc_job* job, int64_t* joined_len) { return join_common(job, joined_len, true); }

int mc_histogram(mc_job* job, int64_t* out, int n_bins) {
  if (int rc = check_job(job)) return rc;
  if (!out || n_bins != job->N + 1) return fail(MC_EINVAL, "histogram needs N+1 = %d bins", job->N + 1);
  MC_CUDA(cudaMemcpyAsync(out, job->d.h, sizeof(int64_t) * n_bins, cudaMemcpyDeviceToHost, job->stream),
          "histogram copy");
  return sync(job, "histogram");
}

// Step 6 of Sec. 2 and the update of Sec. 3.1 in one call: rounds of
// n_sweeps until h holds m_total samples (at least one round), then the
// weight update.  adapt != 0: after a short round the next one has
// ceil(remaining * S_last / joined_last) sweeps, within [1, n_sweeps]
// (n_sweeps when the last round kept nothing).
int mc_iteration(mc_job* job, int64_t n_sweeps, int64_t m_total, int adapt, int max_rounds, int64_t* joined,
                 int* rounds) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending: join first");
  if (n_sweeps < 1 || m_total < 0 || max_rounds < 1) return fail(MC_EINVAL, "need n_sweeps >= 1, m_total >= 0, max_rounds >= 1");
  int64_t total = 0, s_cur = n_sweeps;
  int r = 0;
  for (;;) {
    if (int rc = mc_run_sweeps(job, s_cur)) return rc;
    int64_t got = 0;
    if (int rc = mc_join(job, &got)) return rc;
    total += got;
    ++r;
    if (total >= m_total || r >= max_rounds) break;
    int64_t nxt = n_sweeps;
    if (adapt && got > 0) {
      nxt = ((m_total - total) * s_cur + got - 1) / got;
      nxt = std::max<int64_t>(1, std::min<int64_t>(nxt, n_sweeps));
    }
    s_cur = nxt;
  }
  if (int rc = mc_update_weights(job)) return rc;
  if (joined) *joined = total;
  if (rounds) *rounds = r;
  return MC_OK;
}

int mc_update_weights(mc_job* job) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending: join first");
  MC_CUDA(mcgpu::k_update_weights(job->d, job->stream), "weight update");
  return MC_OK;
}

// ------------------------------------------------------------------ batches
// Fused-launch shape by rule.  A round takes as long as its slowest chain, so
// the blocks of all jobs should be resident at once: full warps (few blocks
// per job), the lattice where a single job runs fastest.  (Lane groups for
// the shared-memory jobs -- 8 chains a warp, 4 lanes each -- shorten their
// chains' critical path but need four times the blocks: measured 1.04e11
// against 1.10e11 kept attempts/s on the uneven batch.)
static LaunchShape batch_rule_shape(int L, int p) {
  LaunchShape s{(L <= 32 && L != 24 && L != 32) ? mcgpu::kPlaceReg : mcgpu::kPlaceSmem, std::min(32, p),
                mcgpu::kBatchWarps};
  while (s.cpw > 1 && !mcgpu::batch_supported(L, s)) s.cpw >>= 1;
  return s;
}

// `iterations` weight iterations of several independent jobs, everything on
// the first job's stream: per iteration every job runs one round of n_sweeps
// sweeps, is joined and updates its weight.  mode 0: one generation launch
// per job; 1: one fused generation launch for all jobs that fit it (others
// keep their own launch); 2: as 1, with the whole loop captured once as a
// CUDA graph and launched.  Results are identical in all modes.
static int mc_batch_run_impl(mc_job** jobs, int n_jobs, int iterations, int64_t n_sweeps, int mode) {
  if (!jobs || n_jobs < 1) return fail(MC_EINVAL, "no jobs");
  if (mode < 0 || mode > 2) return fail(MC_EINVAL, "mode=%d: 0 per-job, 1 fused, 2 fused + graph", mode);
  if (iterations < 1) return fail(MC_EINVAL, "iterations=%d", iterations);
  if (mode > 0 && n_jobs > mcgpu::kMaxBatch) return fail(MC_EINVAL, "at most %d jobs per fused batch", mcgpu::kMaxBatch);
  for (int i = 0; i < n_jobs; ++i) {
    if (!jobs[i]) return fail(MC_EINVAL, "job %d is null", i);
    if (jobs[i]->pending) return fail(MC_ESTATE, "job %d has a round pending", i);
    if (jobs[i]->t % static_cast<uint64_t>(jobs[i]->N) != 0)
      return fail(MC_EINVAL, "job %d is inside a sweep: batches run whole sweeps", i);
    if (jobs[i]->device != jobs[0]->device) return fail(MC_EINVAL, "jobs on different devices");
    for (int k = 0; k < i; ++k)
      if (jobs[k] == jobs[i]) return fail(MC_EINVAL, "job %d listed twice", i);
  }
  cudaStream_t st = jobs[0]->stream;
  std::vector<cudaStream_t> saved(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    MC_CUDA(cudaStreamSynchronize(jobs[i]->stream), "batch start");
    saved[i] = jobs[i]->stream;
    jobs[i]->stream = st;
  }
  // shapes for the fused launch: the autotuned ones (mc_batch_autotune), else
  // the rule of batch_rule_shape
  std::vector<LaunchShape> bshape(n_jobs);
  std::vector<char> fused(n_jobs, 0);
  for (int i = 0; i < n_jobs && mode > 0; ++i) {
    const LaunchShape s = jobs[i]->bshape_valid ? jobs[i]->bshape : batch_rule_shape(jobs[i]->L, jobs[i]->p);
    bshape[i] = s;
    fused[i] = mcgpu::batch_supported(jobs[i]->L, s) ? 1 : 0;
  }
  // fused blocks in order of decreasing work per chain (N), so that the
  // longest chains start first
  std::vector<int> order(n_jobs);
  for (int i = 0; i < n_jobs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a]->N > jobs[b]->N; });
  int rc = MC_OK;
  for (int i = 0; i < n_jobs && rc == MC_OK; ++i) {  // no allocation inside a capture
    if (jobs[i]->trace_on) rc = ensure_trace(jobs[i], n_sweeps);
    int K = 0, C = 0;
    round_segments(jobs[i]->L, jobs[i]->p, n_sweeps, jobs[i]->seg_samples, &K, &C);
    if (rc == MC_OK) rc = ensure_segments(jobs[i], K);
  }
  bool capturing = false;
  if (rc == MC_OK && mode == 2) {
    const cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = cuda_fail(e, "graph capture");
    else capturing = true;
  }
  for (int it = 0; it < iterations && rc == MC_OK; ++it) {
    mcgpu::BatchParams P;
    P.n = 0;
    size_t smem = 0;
    int blocks = 0;
    for (int oi = 0; oi < n_jobs && rc == MC_OK; ++oi) {
      const int i = order[oi];
      uint64_t t0 = 0;
      if ((rc = round_prepare(jobs[i], n_sweeps, &t0, false))) break;
      cudaError_t e = cudaSuccess;
      if (mode > 0 && fused[i]) {
        mcgpu::BatchItem& item = P.items[P.n++];
        size_t b = 0;
        int nb = 0;
        mcgpu::batch_item(jobs[i]->d, bshape[i], t0, n_sweeps, jobs[i]->trace_on, &item, &b, &nb);
        item.first_block = blocks;
        blocks += nb;
        smem = std::max(smem, b);
      } else {
        e = mcgpu::k_generate(jobs[i]->d, jobs[i]->shape, t0, n_sweeps, jobs[i]->trace_on, st);
      }
      if (e != cudaSuccess) rc = cuda_fail(e, "generation");
    }
    if (rc == MC_OK && P.n > 0) {
      const cudaError_t e = mcgpu::k_generate_batched(P, smem, blocks, st);
      if (e != cudaSuccess) rc = cuda_fail(e, "batched generation");
    }
    for (int i = 0; i < n_jobs && rc == MC_OK; ++i) {
      mc_job* j = jobs[i];
      const int64_t M = j->last_S * j->N;
      cudaError_t e = mcgpu::k_join(j->d, j->shape, j->t - static_cast<uint64_t>(M), j->last_S, j->r, false, st);
      if (e == cudaSuccess) e = mcgpu::k_update_weights(j->d, st);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "joint / weight update");
        break;
      }
      j->r += 1;
      j->pending = false;
    }
  }
  if (capturing) {
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc == MC_OK && e != cudaSuccess) rc = cuda_fail(e, "graph capture");
    if (rc == MC_OK) {
      cudaGraphExec_t ge = nullptr;
      cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
      if (e2 == cudaSuccess) e2 = cudaGraphLaunch(ge, st);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
      if (ge) cudaGraphExecDestroy(ge);
      if (e2 != cudaSuccess) rc = cuda_fail(e2, "graph launch");
    }
    if (g) cudaGraphDestroy(g);
  }
  for (int i = 0; i < n_jobs; ++i) jobs[i]->stream = saved[i];
  if (rc != MC_OK) {
    for (int i = 0; i < n_jobs; ++i) jobs[i]->pending = false;
    return rc;
  }
  MC_CUDA(cudaStreamSynchronize(st), "batch");
  return MC_OK;
}

// (host allocations inside may throw; nothing crosses the ABI)
int mc_batch_run(mc_job** jobs, int n_jobs, int iterations, int64_t n_sweeps, int mode) {
  try {
    return mc_batch_run_impl(jobs, n_jobs, iterations, n_sweeps, mode);
  } catch (const std::bad_alloc&) {
    return fail(MC_ENOMEM, "mc_batch_run: host allocation failed");
  } catch (...) {
    return fail(MC_EINVAL, "mc_batch_run: unexpected host error");
  }
}

int mc_get_weights(mc_job* job, double* out, int n) {
  if (int rc = check_job(job)) return rc;
  if (!out || n != job->N + 1) return fail(MC_EINVAL, "weights need N+1 = %d entries", job->N + 1);
  MC_CUDA(cudaMemcpyAsync(out, job->d.W, sizeof(double) * n, cudaMemcpyDeviceToHost, job->stream), "weights copy");
  return sync(job, "weights");
}

int mc_set_weights(mc_job* job, const double* w, int n) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending");
  if (!w || n != job->N + 1) return fail(MC_EINVAL, "weights need N+1 = %d entries", job->N + 1);
  MC_CUDA(cudaMemcpyAsync(job->d.W, w, sizeof(double) * n, cudaMemcpyHostToDevice, job->stream), "weights copy");
  MC_CUDA(mcgpu::k_build_table(job->d, job->stream), "table");
  return sync(job, "set weights");
}

int mc_get_visited(mc_job* job, uint8_t* out, int n) {
  if (int rc = check_job(job)) return rc;
  if (!out || n != job->N + 1) return fail(MC_EINVAL, "visited mask needs N+1 = %d entries", job->N + 1);
  MC_CUDA(cudaMemcpyAsync(out, job->d.visited, n, cudaMemcpyDeviceToHost, job->stream), "visited copy");
  return sync(job, "visited");
}

static int mc_set_visited_impl(mc_job* job, const uint8_t* in, int n) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending");
  if (!in || n != job->N + 1) return fail(MC_EINVAL, "visited mask needs N+1 = %d entries", job->N + 1);
  std::vector<uint8_t> v(in, in + n);
  for (auto& x : v) x = x ? 1 : 0;
  MC_CUDA(cudaMemcpyAsync(job->d.visited, v.data(), n, cudaMemcpyHostToDevice, job->stream), "visited copy");
  return sync(job, "visited");
}

// (host allocations inside may throw; nothing crosses the ABI)
int mc_set_visited(mc_job* job, const uint8_t* in, int n) {
  try {
    return mc_set_visited_impl(job, in, n);
  } catch (const std::bad_alloc&) {
    return fail(MC_ENOMEM, "mc_set_visited: host allocation failed");
  } catch (...) {
    return fail(MC_EINVAL, "mc_set_visited: unexpected host error");
  }
}

// ------------------------------------------------------------------ save / load
// File: "MCJOB01" + NUL, then int32 L, n_chains, start, join order; uint64
// seed, attempts per chain; uint32 rounds joined; int32 carry valid, carry
// level; int64 samples joined so far; then the bit-packed spins (u32), W
// (f64), h (i64) and the visited mask (u8), all little-endian as in memory.
namespace {
constexpr char kMagic[8] = {'M', 'C', 'J', 'O', 'B', '0', '1', '\0'};

struct FileHeader {
  char magic[8];
  int32_t L, p, start, order;
  uint64_t seed, t;
  uint32_t r;
  int32_t carry_valid, carry;
  int64_t joined_total;
};
}  // namespace

static int mc_save_impl(mc_job* job, const char* path) {
  if (int rc = check_job(job)) return rc;
  if (!path) return fail(MC_EINVAL, "path is null");
  if (job->pending) return fail(MC_ESTATE, "round pending: join first");
  const size_t lat = static_cast<size_t>(job->p) * job->L * job->wd, np1 = static_cast<size_t>(job->N) + 1;
  std::vector<uint32_t> spins(lat);
  std::vector<double> W(np1);
  std::vector<long long> h(np1);
  std::vector<uint8_t> vis(np1);
  long long st[mcgpu::kStatCount];
  MC_CUDA(cudaMemcpyAsync(spins.data(), job->d.spins, lat * 4, cudaMemcpyDeviceToHost, job->stream), "save");
  MC_CUDA(cudaMemcpyAsync(W.data(), job->d.W, np1 * 8, cudaMemcpyDeviceToHost, job->stream), "save");
  MC_CUDA(cudaMemcpyAsync(h.data(), job->d.h, np1 * 8, cudaMemcpyDeviceToHost, job->stream), "save");
  MC_CUDA(cudaMemcpyAsync(vis.data(), job->d.visited, np1, cudaMemcpyDeviceToHost, job->stream), "save");
  MC_CUDA(cudaMemcpyAsync(st, job->d.stats, sizeof st, cudaMemcpyDeviceToHost, job->stream), "save");
  if (int rc = sync(job, "save")) return rc;
  FileHeader hd;
  std::memcpy(hd.magic, kMagic, 8);
  hd.L = job->L;
  hd.p = job->p;
  hd.start = job->start;
  hd.order = job->d.ordered;
  hd.seed = job->seed;
  hd.t = job->t;
  hd.r = job->r;
  hd.carry_valid = static_cast<int32_t>(st[mcgpu::kStatCarryValid]);
  hd.carry = static_cast<int32_t>(st[mcgpu::kStatCarry]);
  hd.joined_total = st[mcgpu::kStatJoinedTotal];
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(MC_EINVAL, "cannot open %s for writing", path);
  bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 && std::fwrite(spins.data(), 4, lat, f) == lat &&
            std::fwrite(W.data(), 8, np1, f) == np1 && std::fwrite(h.data(), 8, np1, f) == np1 &&
            std::fwrite(vis.data(), 1, np1, f) == np1;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? MC_OK : fail(MC_EINVAL, "write to %s failed", path);
}

// (host allocations inside may throw; nothing crosses the ABI)
int mc_save(mc_job* job, const char* path) {
  try {
    return mc_save_impl(job, path);
  } catch (const std::bad_alloc&) {
    return fail(MC_ENOMEM, "mc_save: host allocation failed");
  } catch (...) {
    return fail(MC_EINVAL, "mc_save: unexpected host error");
  }
}

static int mc_load_impl(const char* path, mc_job** out) {
  if (!out) return fail(MC_EINVAL, "out is null");
  *out = nullptr;
  if (!path) return fail(MC_EINVAL, "path is null");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(MC_EINVAL, "cannot open %s", path);
  FileHeader hd;
  if (std::fread(&hd, sizeof hd, 1, f) != 1 || std::memcmp(hd.magic, kMagic, 8) != 0 || hd.L < 4 || hd.L > 128 ||
      hd.L % 4 != 0 || hd.p < 1 || hd.p > (1 << 24) || (hd.order != 0 && hd.order != 1)) {
    std::fclose(f);
    return fail(MC_EINVAL, "%s is not a saved job", path);
  }
  const int wd = (hd.L + 31) / 32;
  const size_t lat = static_cast<size_t>(hd.p) * hd.L * wd, np1 = static_cast<size_t>(hd.L) * hd.L + 1;
  std::vector<uint32_t> spins(lat);
  std::vector<double> W(np1);
  std::vector<long long> h(np1);
  std::vector<uint8_t> vis(np1);
  const bool ok = std::fread(spins.data(), 4, lat, f) == lat && std::fread(W.data(), 8, np1, f) == np1 &&
                  std::fread(h.data(), 8, np1, f) == np1 && std::fread(vis.data(), 1, np1, f) == np1;
  std::fclose(f);
  if (!ok) return fail(MC_EINVAL, "%s is truncated", path);
  mc_job* j = nullptr;
  int rc = mc_init(hd.L, hd.p, hd.seed, hd.start, &j);
  if (rc) return rc;
  rc = mc_set_spins(j, spins.data(), lat);
  if (!rc) rc = mc_set_weights(j, W.data(), static_cast<int>(np1));
  if (!rc) rc = mc_set_visited(j, vis.data(), static_cast<int>(np1));
  if (!rc) {
    long long st[mcgpu::kStatCount] = {};
    st[mcgpu::kStatCarryValid] = hd.carry_valid;
    st[mcgpu::kStatCarry] = hd.carry;
    st[mcgpu::kStatJoinedTotal] = hd.joined_total;
    cudaError_t e = cudaMemcpyAsync(j->d.h, h.data(), np1 * 8, cudaMemcpyHostToDevice, j->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(j->d.stats, st, sizeof st, cudaMemcpyHostToDevice, j->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(j->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "load");
  }
  if (rc) {
    mc_free(j);
    return rc;
  }
  j->t = hd.t;
  j->r = hd.r;
  j->d.ordered = hd.order;
  *out = j;
  return MC_OK;
}

// (host allocations inside may throw; nothing crosses the ABI)
int mc_load(const char* path, mc_job** out) {
  try {
    return mc_load_impl(path, out);
  } catch (const std::bad_alloc&) {
    return fail(MC_ENOMEM, "mc_load: host allocation failed");
  } catch (...) {
    return fail(MC_EINVAL, "mc_load: unexpected host error");
  }
}

int mc_set_join_policy(mc_job* job, int64_t scan_max_samples, int passes_before_scan, int passes_without_scan) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending");
  if (passes_before_scan < 0 || passes_before_scan > 64 || passes_without_scan < 0 || passes_without_scan > 64)
    return fail(MC_EINVAL, "passes must be in 0..64");
  job->d.scan_max_samples = scan_max_samples < 0 ? mcgpu::kScanMaxSamples : scan_max_samples;
  job->d.passes_scan = passes_before_scan;
  job->d.passes_plain = passes_without_scan;
  return MC_OK;
}

int mc_set_round_record(mc_job* job, int64_t max_samples) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending");
  job->rec_max = max_samples < 0 ? mcgpu::default_record_max(job->L) : max_samples;
  return MC_OK;
}

int mc_set_partial_record(mc_job* job, int64_t max_entries) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending");
  job->plv_max = max_entries < 0 ? mcgpu::kPartialLevelsMax : max_entries;
  return MC_OK;
}

int mc_set_segment_samples(mc_job* job, int64_t samples) {
  if (int rc = check_job(job)) return rc;
  if (samples < 0) return fail(MC_EINVAL, "segment samples %lld < 0", static_cast<long long>(samples));
  if (job->pending) return fail(MC_ESTATE, "round pending");
  job->seg_samples = samples;
  return MC_OK;
}

int mc_set_join_order(mc_job* job, int mode) {
  if (int rc = check_job(job)) return rc;
  if (mode != 0 && mode != 1) return fail(MC_EINVAL, "join order %d: 0 chain index, 1 ascending final energy", mode);
  if (job->pending) return fail(MC_ESTATE, "round pending");
  job->d.ordered = mode;
  return MC_OK;
}

int mc_get_order(mc_job* job, int32_t* out, int n) {
  if (int rc = check_job(job)) return rc;
  if (!out || n != job->p) return fail(MC_EINVAL, "order needs n_chains entries");
  MC_CUDA(cudaMemcpyAsync(out, job->d.perm, 4ull * n, cudaMemcpyDeviceToHost, job->stream), "order copy");
  return sync(job, "order");
}

int mc_thermo(mc_job* job, const double* betas, int n_beta, double* out) {
  if (int rc = check_job(job)) return rc;
  if (!betas || !out || n_beta < 1 || n_beta > 65535) return fail(MC_EINVAL, "need 1..65535 betas and an output");
  for (int b = 0; b < n_beta; ++b)
    if (!(betas[b] > 0.0) || !(betas[b] < 1e300)) return fail(MC_EINVAL, "beta[%d] must be positive and finite", b);
  void* dev = nullptr;
  MC_CUDA(raw_alloc(job, &dev, sizeof(double) * 5 * n_beta), "thermo buffer");
  double* db = static_cast<double*>(dev);
  double* dout = db + n_beta;
  cudaError_t e = cudaMemcpyAsync(db, betas, sizeof(double) * n_beta, cudaMemcpyHostToDevice, job->stream);
  if (e == cudaSuccess) e = mcgpu::k_thermo(job->d, db, n_beta, dout, job->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, dout, sizeof(double) * 4 * n_beta, cudaMemcpyDeviceToHost, job->stream);
  raw_free(job, dev);
  if (e != cudaSuccess) return cuda_fail(e, "thermo");
  return sync(job, "thermo");
}

int mc_get_table(mc_job* job, uint32_t* out, int n) {
  if (int rc = check_job(job)) return rc;
  if (!out || n != 5 * (job->N + 1)) return fail(MC_EINVAL, "table needs 5*(N+1) entries");
  MC_CUDA(cudaMemcpyAsync(out, job->d.T, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, job->stream), "table copy");
  return sync(job, "table");
}

int mc_get_spins(mc_job* job, uint32_t* out, size_t n_words) {
  if (int rc = check_job(job)) return rc;
  const size_t need = static_cast<size_t>(job->p) * job->L * job->wd;
  if (!out || n_words != need) return fail(MC_EINVAL, "spins need %zu words", need);
  MC_CUDA(cudaMemcpyAsync(out, job->d.spins, need * 4, cudaMemcpyDeviceToHost, job->stream), "spins copy");
  return sync(job, "spins");
}

static int mc_set_spins_impl(mc_job* job, const uint32_t* in, size_t n_words) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending");
  const size_t need = static_cast<size_t>(job->p) * job->L * job->wd;
  if (!in || n_words != need) return fail(MC_EINVAL, "spins need %zu words", need);
  const int lw = job->L - 32 * (job->wd - 1);
  const uint32_t last_mask = lw == 32 ? 0xFFFFFFFFu : ((1u << lw) - 1u);
  std::vector<uint32_t> tmp(in, in + need);
  for (size_t i = job->wd - 1; i < need; i += job->wd) tmp[i] &= last_mask;
  MC_CUDA(cudaMemcpyAsync(job->d.spins, tmp.data(), need * 4, cudaMemcpyHostToDevice, job->stream), "spins copy");
  MC_CUDA(mcgpu::k_levels(job->d, job->stream), "levels");
  return sync(job, "set spins");
}

// (host allocations inside may throw; nothing crosses the ABI)
int mc_set_spins(mc_job* job, const uint32_t* in, size_t n_words) {
  try {
    return mc_set_spins_impl(job, in, n_words);
  } catch (const std::bad_alloc&) {
    return fail(MC_ENOMEM, "mc_set_spins: host allocation failed");
  } catch (...) {
    return fail(MC_EINVAL, "mc_set_spins: unexpected host error");
  }
}

int mc_get_energies(mc_job* job, int32_t* out, int n) {
  if (int rc = check_job(job)) return rc;
  if (!out || n != job->p) return fail(MC_EINVAL, "energies need n_chains entries");
  MC_CUDA(cudaMemcpyAsync(out, job->d.m, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, job->stream), "levels copy");
  if (int rc = sync(job, "energies")) return rc;
  for (int i = 0; i < n; ++i) out[i] = 4 * out[i] - 2 * job->N;
  return MC_OK;
}

int mc_get_trace(mc_job* job, int32_t* out, size_t n) {
  if (int rc = check_job(job)) return rc;
  if (!job->trace_valid || !job->d.trace) return fail(MC_ESTATE, "no trace recorded for the last round");
  const size_t need = static_cast<size_t>(job->last_S) * job->p;
  if (!out || n < need) return fail(MC_EINVAL, "trace needs %zu entries", need);
  MC_CUDA(cudaMemcpyAsync(out, job->d.trace, need * 4, cudaMemcpyDeviceToHost, job->stream), "trace copy");
  return sync(job, "trace");
}

int mc_get_trace_chain(mc_job* job, int chain, int32_t* out, size_t n) {
  if (int rc = check_job(job)) return rc;
  if (!job->trace_valid || !job->d.trace) return fail(MC_ESTATE, "no trace recorded for the last round");
  if (chain < 0 || chain >= job->p) return fail(MC_EINVAL, "chain %d out of range", chain);
  const size_t S = static_cast<size_t>(job->last_S);
  if (!out || n < S) return fail(MC_EINVAL, "trace of one chain needs %zu entries", S);
  MC_CUDA(cudaMemcpy2DAsync(out, 4, job->d.trace + chain, 4ull * job->p, 4, S, cudaMemcpyDeviceToHost, job->stream),
          "trace column copy");
  return sync(job, "trace");
}

int mc_get_join(mc_job* job, int64_t* k, int64_t* offsets, int n) {
  if (int rc = check_job(job)) return rc;
  if (n != job->p) return fail(MC_EINVAL, "need n_chains entries");
  if (k) MC_CUDA(cudaMemcpyAsync(k, job->d.k, 8ull * n, cudaMemcpyDeviceToHost, job->stream), "k copy");
  if (offsets)
    MC_CUDA(cudaMemcpyAsync(offsets, job->d.offsets, 8ull * n, cudaMemcpyDeviceToHost, job->stream), "offsets copy");
  return sync(job, "join results");
}

int mc_get_info(mc_job* job, mc_info* info) {
  if (int rc = check_job(job)) return rc;
  if (!info) return fail(MC_EINVAL, "info is null");
  long long st[mcgpu::kStatCount];
  MC_CUDA(cudaMemcpyAsync(st, job->d.stats, sizeof st, cudaMemcpyDeviceToHost, job->stream), "stats copy");
  if (int rc = sync(job, "info")) return rc;
  std::memset(info, 0, sizeof *info);
  info->L = job->L;
  info->N = job->N;
  info->n_chains = job->p;
  info->words_per_row = job->wd;
  info->seed = job->seed;
  info->attempts_per_chain = job->t;
  info->rounds_joined = job->r;
  info->last_sweeps = job->last_S;
  info->round_pending = job->pending ? 1 : 0;
  info->carry_valid = static_cast<int>(st[mcgpu::kStatCarryValid]);
  info->carry_energy = info->carry_valid ? static_cast<int>(4 * st[mcgpu::kStatCarry] - 2 * job->N) : 0;
  info->last_joined = st[mcgpu::kStatJoined];
  info->last_rejected = st[mcgpu::kStatRejected];
  info->last_mismatch = st[mcgpu::kStatMismatch];
  info->last_passes = st[mcgpu::kStatPasses];
  info->last_searched = st[mcgpu::kStatSearched];
  info->total_joined = st[mcgpu::kStatJoinedTotal];
  info->placement = job->shape.placement;
  info->chains_per_warp = job->shape.cpw;
  info->warps_per_block = job->shape.wpb;
  info->device_bytes = job->bytes;
  info->last_scanned = st[mcgpu::kStatScanned];
  info->segments = job->d.ck_K;
  info->segment_sweeps = job->d.ck_C;
  return MC_OK;
}

// ------------------------------------------------------------------ autotuner
// Candidate launch shapes are timed on a scratch copy of the job's lattices
// and levels (so the job's own chains are not advanced), with CUDA events on
// the job's stream; the fastest is kept for the job and cached per
// (device, L, n_chains) for later jobs.  Every shape gives identical results.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, LaunchShape> g_tune_cache;
}  // namespace

static int mc_autotune_impl(mc_job* job, int64_t probe_sweeps, int use_cache, int* placement, int* cpw, int* wpb) {
  if (int rc = check_job(job)) return rc;
  if (job->pending) return fail(MC_ESTATE, "round pending");
  if (probe_sweeps < 1 || probe_sweeps * job->N >= (int64_t(1) << 34)) return fail(MC_EINVAL, "bad probe_sweeps");
  const auto key = std::make_tuple(job->device, job->L, job->p);
  if (use_cache) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      job->shape = it->second;
      if (placement) *placement = job->shape.placement;
      if (cpw) *cpw = job->shape.cpw;
      if (wpb) *wpb = job->shape.wpb;
      return MC_OK;
    }
  }
  // candidate shapes
  std::vector<LaunchShape> cands;
  const int sub = job->num_sms * 4;
  std::vector<int> cpws = {1, 2, 4, 8, 16, 32};
  for (int w = 1; w <= 4; w *= 2) {
    cpws.push_back((job->p + sub - 1) / sub);
    cpws.push_back((job->p + job->num_sms * w - 1) / (job->num_sms * w));
    cpws.push_back((job->p + 2 * sub - 1) / (2 * sub));
  }
  for (int pl = 0; pl < 3; ++pl)
    for (int w = 1; w <= 4; w *= 2)
      for (int c : cpws) {
        LaunchShape s{pl, std::min(32, std::max(1, c)), w};
        if (!mcgpu::shape_supported(job->L, s)) continue;
        bool dup = false;
        for (const auto& q : cands) dup = dup || (q.placement == s.placement && q.cpw == s.cpw && q.wpb == s.wpb);
        if (!dup) cands.push_back(s);
      }
  // scratch copy of the chain state
  DevJob d = job->d;
  const size_t lat = static_cast<size_t>(job->p) * job->L * job->wd;
  void *sp = nullptr, *sm = nullptr, *sh = nullptr;
  cudaError_t e = cudaMalloc(&sp, lat * 4);
  if (e == cudaSuccess) e = cudaMalloc(&sm, static_cast<size_t>(job->p) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&sh, static_cast<size_t>(d.np1) * 8);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  LaunchShape best = job->shape;
  float best_ms = 1e30f;
  if (e == cudaSuccess) {
    d.spins = static_cast<uint32_t*>(sp);
    d.m = static_cast<int32_t*>(sm);
    d.hgen = static_cast<unsigned long long*>(sh);
    d.trace = nullptr;
    d.ckpt = nullptr;  // probes write no checkpoints
    d.rec = nullptr;   // nor records
    for (const auto& s : cands) {
      float ms = 0.f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first run warms up
        e = cudaMemcpyAsync(d.spins, job->d.spins, lat * 4, cudaMemcpyDeviceToDevice, job->stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d.m, job->d.m, static_cast<size_t>(job->p) * 4, cudaMemcpyDeviceToDevice, job->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, job->stream);
        if (e == cudaSuccess) e = mcgpu::k_generate(d, s, job->t, probe_sweeps, false, job->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, job->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      }
      if (e != cudaSuccess) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = s;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sp) cudaFree(sp);
  if (sm) cudaFree(sm);
  if (sh) cudaFree(sh);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  job->shape = best;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  if (placement) *placement = best.placement;
  if (cpw) *cpw = best.cpw;
  if (wpb) *wpb = best.wpb;
  return MC_OK;
}

// (host allocations inside may throw; nothing crosses the ABI)
int mc_autotune(mc_job* job, int64_t probe_sweeps, int use_cache, int* placement, int* cpw, int* wpb) {
  try {
    return mc_autotune_impl(job, probe_sweeps, use_cache, placement, cpw, wpb);
  } catch (const std::bad_alloc&) {
    return fail(MC_ENOMEM, "mc_autotune: host allocation failed");
  } catch (...) {
    return fail(MC_EINVAL, "mc_autotune: unexpected host error");
  }
}

// Fused-batch autotuner: greedy over each job's candidate shapes (placement,
// chains per warp; lane groups follow from them), every candidate timed as a
// whole fused generation launch of all jobs on scratch copies of their
// chains (CUDA events; the jobs' own chains do not move), keeping only
// combinations whose blocks are all resident at once.  Jobs are visited from
// the longest chains (largest N) down; a candidate is kept if it shortens the
// launch by more than 1 %.  Cached per (device, the jobs' (L, p) in order).
namespace {
std::map<std::vector<int>, std::vector<LaunchShape>> g_btune_cache;
}  // namespace

static int mc_batch_autotune_impl(mc_job** jobs, int n_jobs, int64_t probe_sweeps, int use_cache) {
  if (!jobs || n_jobs < 1 || n_jobs > mcgpu::kMaxBatch) return fail(MC_EINVAL, "need 1..%d jobs", mcgpu::kMaxBatch);
  if (probe_sweeps < 1) return fail(MC_EINVAL, "bad probe_sweeps");
  for (int i = 0; i < n_jobs; ++i) {
    if (!jobs[i]) return fail(MC_EINVAL, "job %d is null", i);
    if (jobs[i]->pending) return fail(MC_ESTATE, "job %d has a round pending", i);
    if (jobs[i]->device != jobs[0]->device) return fail(MC_EINVAL, "jobs on different devices");
    if (probe_sweeps * jobs[i]->N >= (int64_t(1) << 34)) return fail(MC_EINVAL, "bad probe_sweeps");
    for (int k = 0; k < i; ++k)
      if (jobs[k] == jobs[i]) return fail(MC_EINVAL, "job %d listed twice", i);
  }
  std::vector<int> key{jobs[0]->device};
  for (int i = 0; i < n_jobs; ++i) {
    key.push_back(jobs[i]->L);
    key.push_back(jobs[i]->p);
  }
  if (use_cache) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_btune_cache.find(key);
    if (it != g_btune_cache.end()) {
      for (int i = 0; i < n_jobs; ++i) {
        jobs[i]->bshape = it->second[i];
        jobs[i]->bshape_valid = true;
      }
      return MC_OK;
    }
  }
  // candidates per job (the rule first); jobs without a fused form keep it
  std::vector<std::vector<LaunchShape>> cands(n_jobs);
  std::vector<LaunchShape> cur(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    cur[i] = batch_rule_shape(jobs[i]->L, jobs[i]->p);
    cands[i].push_back(cur[i]);
    if (!mcgpu::batch_supported(jobs[i]->L, cur[i])) continue;
    for (int pl = 0; pl < 2; ++pl)
      for (int c : {32, 16, 8, 4}) {
        const LaunchShape s{pl, std::min(c, jobs[i]->p), mcgpu::kBatchWarps};
        if (!mcgpu::batch_supported(jobs[i]->L, s)) continue;
        bool dup = false;
        for (const auto& q : cands[i]) dup = dup || (q.placement == s.placement && q.cpw == s.cpw);
        if (!dup) cands[i].push_back(s);
      }
  }
  std::vector<int> order(n_jobs);
  for (int i = 0; i < n_jobs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a]->N > jobs[b]->N; });
  // scratch copies of every job's chains
  cudaStream_t st = jobs[0]->stream;
  std::vector<DevJob> d(n_jobs);
  std::vector<void*> mem;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n_jobs && e == cudaSuccess; ++i) {
    e = cudaStreamSynchronize(jobs[i]->stream);
    d[i] = jobs[i]->d;
    const size_t lat = static_cast<size_t>(jobs[i]->p) * jobs[i]->L * jobs[i]->wd;
    void *sp = nullptr, *sm = nullptr, *sh = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sp, lat * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sm, static_cast<size_t>(jobs[i]->p) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sh, static_cast<size_t>(d[i].np1) * 8);
    for (void* v : {sp, sm, sh})
      if (v) mem.push_back(v);
    d[i].spins = static_cast<uint32_t*>(sp);
    d[i].m = static_cast<int32_t*>(sm);
    d[i].hgen = static_cast<unsigned long long*>(sh);
    d[i].trace = nullptr;
    d[i].ckpt = nullptr;   // probes write no checkpoints
    d[i].rec = nullptr;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // time of one fused launch with these shapes (1e30 if its blocks would not all be resident)
  auto probe = [&](const std::vector<LaunchShape>& sh) -> float {
    mcgpu::BatchParams P;
    P.n = 0;
    size_t smem = 0;
    int blocks = 0;
    for (int oi = 0; oi < n_jobs; ++oi) {
      const int i = order[oi];
      if (!mcgpu::batch_supported(jobs[i]->L, sh[i])) continue;
      mcgpu::BatchItem& item = P.items[P.n++];
      size_t b = 0;
      int nb = 0;
      mcgpu::batch_item(d[i], sh[i], jobs[i]->t, probe_sweeps, false, &item, &b, &nb);
      item.first_block = blocks;
      blocks += nb;
      smem = std::max(smem, b);
    }
    if (P.n == 0 || blocks > mcgpu::batch_resident_blocks(smem)) return 1e30f;
    float ms = 1e30f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up
      for (int i = 0; i < n_jobs && e == cudaSuccess; ++i) {
        const size_t lat = static_cast<size_t>(jobs[i]->p) * jobs[i]->L * jobs[i]->wd;
        e = cudaMemcpyAsync(d[i].spins, jobs[i]->d.spins, lat * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d[i].m, jobs[i]->d.m, static_cast<size_t>(jobs[i]->p) * 4, cudaMemcpyDeviceToDevice, st);
      }
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = mcgpu::k_generate_batched(P, smem, blocks, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    return e == cudaSuccess ? ms : 1e30f;
  };
  if (e == cudaSuccess) {
    float best = probe(cur);
    for (int oi = 0; oi < n_jobs && e == cudaSuccess; ++oi) {
      const int i = order[oi];
      for (const auto& c : cands[i]) {
        if (c.placement == cur[i].placement && c.cpw == cur[i].cpw) continue;
        std::vector<LaunchShape> trial = cur;
        trial[i] = c;
        const float t = probe(trial);
        if (e != cudaSuccess) break;
        if (t < 0.99f * best) {
          best = t;
          cur = trial;
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (void* v : mem) cudaFree(v);
  if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
  for (int i = 0; i < n_jobs; ++i) {
    jobs[i]->bshape = cur[i];
    jobs[i]->bshape_valid = true;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_btune_cache[key] = cur;
  }
  return MC_OK;
}

// (host allocations inside may throw; nothing crosses the ABI)
int mc_batch_autotune(mc_job** jobs, int n_jobs, int64_t probe_sweeps, int use_cache) {
  try {
    return mc_batch_autotune_impl(jobs, n_jobs, probe_sweeps, use_cache);
  } catch (const std::bad_alloc&) {
    return fail(MC_ENOMEM, "mc_batch_autotune: host allocation failed");
  } catch (...) {
    return fail(MC_EINVAL, "mc_batch_autotune: unexpected host error");
  }
}

int mc_batch_shape(mc_job* job, int* placement, int* chains_per_warp, int* warps_per_block) {
  if (int rc = check_job(job)) return rc;
  const LaunchShape s = job->bshape_valid ? job->bshape : batch_rule_shape(job->L, job->p);
  if (placement) *placement = s.placement;
  if (chains_per_warp) *chains_per_warp = s.cpw;
  if (warps_per_block) *warps_per_block = s.wpb;
  return mcgpu::batch_supported(job->L, s) ? 1 : 0;
}

uint64_t mc_job_device_bytes(int L, int n_chains, int64_t sweeps) {
  if (L < 4 || L > 128 || (L % 4) != 0 || n_chains < 1 || sweeps < 1) return 0;
  const uint64_t N = static_cast<uint64_t>(L) * L, np1 = N + 1, wd = (L + 31) / 32;
  const uint64_t p = static_cast<uint64_t>(n_chains), lw = static_cast<uint64_t>(L) * wd, lat = p * lw;
  // as allocated by mc_init: spins, spins0, m, m0, W, T, h, hgen, dpre, k,
  // xused, tj, offsets, work, work2, lastacc, summ, visited, perm, lvcnt, kmin, stats
  uint64_t b = lat * 4 * 2 + p * 4 * 2 + np1 * 8 + 5 * np1 * 4 + np1 * 8 * 3 + p * 8 + p * 4 + p * np1 * 4 +
               p * 8 + p * 4 + p * 4 + p * 4 + p * 20 + np1 + p * 4 + np1 * 4 + p * 8 + mcgpu::kStatCount * 8;
  int K = 0, C = 0;
  round_segments(L, n_chains, sweeps, 0, &K, &C);
  (void)lw;
  const uint64_t samples = p * static_cast<uint64_t>(sweeps) * N;   // record of the round, if small
  const uint64_t rec = samples <= static_cast<uint64_t>(mcgpu::default_record_max(L))
                           ? static_cast<uint64_t>(mcgpu::rec_entries(n_chains, sweeps * static_cast<int64_t>(N))) * 2
                           : 0;
  return b + static_cast<uint64_t>(K) * bytes_per_segment(L, n_chains) + rec;
}

int mc_sync(mc_job* job) {
  if (int rc = check_job(job)) return rc;
  return sync(job, "sync");
}

}  // extern "C"
