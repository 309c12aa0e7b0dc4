// mc_generate_noalloc: one round of chain generation on caller-owned device
// buffers, with no device memory allocation at all.
//
// Who needs this: callers that cannot call cudaMalloc while they run, for
// instance code executing inside a memory pool that forbids foreign
// allocations, a host function that must not synchronise the device (an
// allocation can), or an embedding that has reserved all device memory up
// front.  They hand in every input and output buffer; the only scratch the
// call needs -- the acceptance-threshold table built from the weight -- lives
// in the fixed array below, which every GPU that loads this library holds
// until the process exits.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mc.h"
#include "mc_internal.h"

namespace {

// Largest lattice the scratch covers: L = 128, 5 * (128*128 + 1) thresholds
// (320 KiB).
constexpr int kNoAllocMaxL = 128;
constexpr size_t kNoAllocTableWords = 5u * (static_cast<size_t>(kNoAllocMaxL) * kNoAllocMaxL + 1u);

static __device__ __align__(256) uint32_t g_noalloc_table[kNoAllocTableWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_table_ptr[kMaxDevices] = {};  // device address of the table, per device
int g_num_sms[kMaxDevices] = {};

thread_local char g_msg[256];

int fail(int code, const char* msg) {
  std::snprintf(g_msg, sizeof g_msg, "%s", msg);
  mcgpu::set_last_error(g_msg);
  return code;
}

}  // namespace

extern "C" int mc_generate_noalloc(int L, int n_chains, uint64_t seed, uint64_t t0, int64_t n_sweeps,
                                   uint32_t* d_spins, int32_t* d_levels, const double* d_weights,
                                   int64_t* d_hist, void* cuda_stream) {
  if (L < 4 || L > kNoAllocMaxL || (L % 4) != 0)
    return fail(MC_EINVAL, "mc_generate_noalloc: need 4 <= L <= 128 with L % 4 == 0 (scratch holds L <= 128)");
  if (n_chains < 1 || n_chains > (1 << 24)) return fail(MC_EINVAL, "mc_generate_noalloc: n_chains out of range");
  const int64_t N = static_cast<int64_t>(L) * L;
  if (n_sweeps < 1 || n_sweeps > (int64_t(1) << 34) / N) return fail(MC_EINVAL, "mc_generate_noalloc: bad n_sweeps");
  if (t0 % 4 != 0) return fail(MC_EINVAL, "mc_generate_noalloc: t0 must be a multiple of 4");
  if (!d_spins || !d_levels || !d_weights || !d_hist)
    return fail(MC_EINVAL, "mc_generate_noalloc: null buffer");
  if (static_cast<size_t>(5 * (N + 1)) > kNoAllocTableWords)
    return fail(MC_EINVAL, "mc_generate_noalloc: threshold table exceeds the fixed scratch");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(MC_ECUDA, "mc_generate_noalloc: no usable current device");
  uint32_t* table = nullptr;
  int sms = 0;
  {
    // once per device, with that device current: the table's device address
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_table_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_table);
      if (e != cudaSuccess || !p) {
        std::snprintf(g_msg, sizeof g_msg, "mc_generate_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
        mcgpu::set_last_error(g_msg);
        return MC_ECUDA;
      }
      int n = 0;
      if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(MC_ECUDA, "mc_generate_noalloc: device attribute query failed");
      g_table_ptr[dev] = static_cast<uint32_t*>(p);
      g_num_sms[dev] = n;
    }
    table = g_table_ptr[dev];
    sms = g_num_sms[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  mcgpu::DevJob d;
  std::memset(&d, 0, sizeof d);
  d.L = L;
  d.N = static_cast<int>(N);
  d.np1 = static_cast<int>(N + 1);
  d.wd = (L + 31) / 32;
  d.p = n_chains;
  d.key0 = static_cast<uint32_t>(seed);
  d.key1 = static_cast<uint32_t>(seed >> 32);
  d.spins = d_spins;
  d.m = d_levels;
  d.W = const_cast<double*>(d_weights);
  d.T = table;
  d.hgen = reinterpret_cast<unsigned long long*>(d_hist);
  cudaError_t e = cudaMemsetAsync(d_hist, 0, sizeof(int64_t) * static_cast<size_t>(N + 1), st);
  if (e == cudaSuccess) e = mcgpu::k_build_table(d, st);
  if (e == cudaSuccess) e = mcgpu::k_generate(d, mcgpu::default_shape(L, n_chains, sms), t0, n_sweeps, false, st);
  if (e != cudaSuccess) {
    std::snprintf(g_msg, sizeof g_msg, "mc_generate_noalloc: %s", cudaGetErrorString(e));
    mcgpu::set_last_error(g_msg);
    return MC_ECUDA;
  }
  return MC_OK;
}
