// Kernels of the hot path: initial lattices, threshold table, generation of
// p independent chains (Sec. 2 step 2), the joint by detailed balance (steps
// 3-5) as speculation + resolution + segmented scan, and the weight update
// (Sec. 3.1 Eq. new_weight in logarithms, Sec. 4.2).
#include <atomic>
#include <algorithm>
#include <math_constants.h>

#include "mc_chain_kernels.cuh"
#include "mc_scan_fsm.cuh"

namespace mcgpu {

static std::atomic<uint64_t> g_launches{0};
uint64_t launches_add(uint64_t n) { return g_launches.fetch_add(n) + n; }


// ------------------------------------------------------------------ init
// Step 1: C_1 all up, or random: bit (site & 31) of Philox word q & 3 at
// counter (q >> 2, 0, chain, 2), q = site >> 5, site = y L + x.
__global__ void init_lattice_kernel(const DevJob j, const int start) {
  const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  const long long total = static_cast<long long>(j.p) * j.L * j.wd;
  if (idx >= total) return;
  const int w = static_cast<int>(idx % j.wd);
  const long long cy = idx / j.wd;
  const int y = static_cast<int>(cy % j.L);
  const uint32_t c = static_cast<uint32_t>(cy / j.L);
  const int x0 = 32 * w, x1 = min(j.L, x0 + 32);
  uint32_t word = 0u;
  if (start == 0) {
    word = (x1 - x0 == 32) ? 0xFFFFFFFFu : ((1u << (x1 - x0)) - 1u);
  } else {
    uint32_t cached = 0xFFFFFFFFu, R = 0u;
    for (int x = x0; x < x1; ++x) {
      const uint32_t site = static_cast<uint32_t>(y * j.L + x);
      const uint32_t q = site >> 5;
      if (q != cached) {
        const uint4 v = philox4x32_10(make_uint4(q >> 2, 0u, c, kTagInit), j.key0, j.key1);
        R = uint4_word(v, q & 3u);
        cached = q;
      }
      word |= ((R >> (site & 31u)) & 1u) << (x - x0);
    }
  }
  j.spins[idx] = word;
}

__device__ __forceinline__ uint32_t site_bit(const uint32_t* lat, int wd, int L, int x, int y) {
  x = (x + L) % L;
  y = (y + L) % L;
  return (lat[y * wd + (x >> 5)] >> (x & 31)) & 1u;
}

// Level m = (E + 2N)/4 of each chain's lattice, E = -sum s (s_right + s_down).
__global__ void levels_kernel(const DevJob j) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= j.p) return;
  const uint32_t* lat = j.spins + static_cast<size_t>(c) * j.L * j.wd;
  int E = 0;
  for (int y = 0; y < j.L; ++y)
    for (int x = 0; x < j.L; ++x) {
      const int s = site_bit(lat, j.wd, j.L, x, y) ? 1 : -1;
      const int r = site_bit(lat, j.wd, j.L, x + 1, y) ? 1 : -1;
      const int d = site_bit(lat, j.wd, j.L, x, y + 1) ? 1 : -1;
      E -= s * (r + d);
    }
  j.m[c] = (E + 2 * j.N) / 4;
}

// T[a][m] = thr(W[m + a - 2] - W[m]); moves outside [0, N] never occur.
__global__ void table_kernel(const DevJob j) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 5 * j.np1) return;
  const int a = idx / j.np1, m = idx % j.np1;
  const int mp = m + a - 2;
  j.T[idx] = (mp < 0 || mp > j.N) ? 0u : threshold_det(__dsub_rn(j.W[mp], j.W[m]));
}

// Eq. (new_weight) in logarithms: W -= ln h where h > 0; h cleared.
__global__ void weights_kernel(const DevJob j) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= j.np1) return;
  const long long h = j.h[m];
  if (h > 0) {
    j.W[m] = __dsub_rn(j.W[m], log_det(static_cast<double>(h)));
    j.visited[m] = 1;
  }
  j.h[m] = 0;
}

// ------------------------------------------------------------------ part (ii)
// Statistical averages at inverse temperature beta (Sec. 3.2, Eq.
// reweighting2, with E, C, F, S of Sec. 4.1), one block per beta.  D(E) is
// proportional to 1/w(E) = e^{-W(E)} over the levels the weight iteration
// has visited; every sum is taken relative to its largest exponent (the
// logarithmic evaluation of Sec. 4.2).  D counts all 2^N states:
// ln Z = N ln 2 + ln sum e^{-W - beta E} - ln sum e^{-W}.
// C = beta^2 <(H - <H>)^2>, F = -ln Z / beta, S = beta (E - F).
// Reductions are fixed-shape trees, so repeated calls agree bit for bit.
constexpr int kThermoThreads = 256;

__device__ double block_max(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = kThermoThreads / 2; o > 0; o >>= 1) {
    if (t < o) sh[t] = fmax(sh[t], sh[t + o]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ double block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = kThermoThreads / 2; o > 0; o >>= 1) {
    if (t < o) sh[t] = sh[t] + sh[t + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThermoThreads) thermo_kernel(const DevJob j, const double* __restrict__ betas,
                                                                double* __restrict__ out) {
  __shared__ double sh[kThermoThreads];
  const int t = threadIdx.x;
  const double beta = betas[blockIdx.x];
  double bm = -CUDART_INF, am = -CUDART_INF;
  for (int m = t; m < j.np1; m += kThermoThreads)
    if (j.visited[m]) {
      const double E = static_cast<double>(4 * m - 2 * j.N);
      bm = fmax(bm, -j.W[m]);
      am = fmax(am, -j.W[m] - beta * E);
    }
  const double B = block_max(bm, sh);
  const double A = block_max(am, sh);
  double sg = 0.0, z = 0.0, e1 = 0.0;
  for (int m = t; m < j.np1; m += kThermoThreads)
    if (j.visited[m]) {
      const double E = static_cast<double>(4 * m - 2 * j.N);
      const double w = exp(-j.W[m] - beta * E - A);
      sg += exp(-j.W[m] - B);
      z += w;
      e1 += E * w;
    }
  const double SG = block_sum(sg, sh);
  const double Z = block_sum(z, sh);
  const double E1 = block_sum(e1, sh);
  const double Eav = E1 / Z;
  double v = 0.0;
  for (int m = t; m < j.np1; m += kThermoThreads)
    if (j.visited[m]) {
      const double E = static_cast<double>(4 * m - 2 * j.N);
      const double w = exp(-j.W[m] - beta * E - A);
      v += (E - Eav) * (E - Eav) * w;
    }
  const double V = block_sum(v, sh);
  if (t == 0) {
    const double lnZ = static_cast<double>(j.N) * log(2.0) + A + log(Z) - (B + log(SG));
    const double F = -lnZ / beta;
    double* o = out + 4 * blockIdx.x;
    o[0] = Eav;
    o[1] = beta * beta * (V / Z);
    o[2] = F;
    o[3] = beta * (Eav - F);
  }
}

// Joint thresholds for each listed chain's input level x: tj[i][m] = thr(W[m] - W[x]).
__global__ void tj_kernel(const DevJob j, const int32_t* __restrict__ list, const int n) {
  const long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<long long>(n) * j.np1) return;
  const int q = static_cast<int>(idx / j.np1), m = static_cast<int>(idx % j.np1);
  const int i = list ? list[q] : q;
  const int x = j.xused[i];
  if (x < 0) return;
  j.tj[static_cast<size_t>(i) * j.np1 + m] = threshold_det(__dsub_rn(j.W[m], j.W[x]));
}

// Speculated inputs: chain i is assumed to receive the last configuration of
// chain i-1 (chain 0 receives the carry from the previous round, or nothing
// in the job's first round).
__global__ void spec_inputs_kernel(const DevJob j) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // position in the joint
  if (q >= j.p) return;
  int x;
  if (q == 0)
    x = j.stats[kStatCarryValid] ? static_cast<int>(j.stats[kStatCarry]) : -1;
  else
    x = j.m[j.perm[q - 1]];
  j.xused[j.perm[q]] = x;
}

// Joint order (one block): identity, or -- energy-ordered joining -- the
// chains sorted by final level, equal levels in index order: a counting sort
// whose scatter walks the chains in index order a warp at a time (ranks among
// equal levels inside a warp from __match_any_sync).
__global__ void __launch_bounds__(1024) order_kernel(const DevJob j) {
  const int t = threadIdx.x, nt = blockDim.x;
  if (!j.ordered) {
    for (int q = t; q < j.p; q += nt) j.perm[q] = q;
    return;
  }
  __shared__ int s_part[1024];
  for (int v = t; v < j.np1; v += nt) j.lvcnt[v] = 0;
  __syncthreads();
  for (int c = t; c < j.p; c += nt) atomicAdd(&j.lvcnt[j.m[c]], 1);
  __syncthreads();
  // exclusive scan of the counts: contiguous ranges per thread
  const int per = (j.np1 + nt - 1) / nt;
  const int lo = min(j.np1, t * per), hi = min(j.np1, lo + per);
  int sum = 0;
  for (int v = lo; v < hi; ++v) sum += j.lvcnt[v];
  s_part[t] = sum;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    const int a = (t >= off) ? s_part[t - off] : 0;
    __syncthreads();
    s_part[t] += a;
    __syncthreads();
  }
  int run = s_part[t] - sum;
  for (int v = lo; v < hi; ++v) {
    const int c = j.lvcnt[v];
    j.lvcnt[v] = run;
    run += c;
  }
  __syncthreads();
  // stable scatter
  const int lane = t & 31, warp = t >> 5, nwarps = nt >> 5;
  for (int base = 0; base < j.p; base += nt) {
    const int c = base + t;
    const bool act = c < j.p;
    const unsigned amask = __ballot_sync(0xFFFFFFFFu, act);
    int v = -1;
    unsigned same = 0u;
    if (act) {
      v = j.m[c];
      same = __match_any_sync(amask, v);
    }
    for (int w = 0; w < nwarps; ++w) {
      if (warp == w && act) {
        const int rank = __popc(same & ((1u << lane) - 1u));
        j.perm[j.lvcnt[v] + rank] = c;
        __syncwarp(amask);
        if (rank == 0) j.lvcnt[v] += __popc(same);
      }
      __syncthreads();
    }
  }
}

// Segmented scan and histogram: kept length of chain i is M - k_i + 1 (0 if
// nothing is kept); offsets are the exclusive scan; h += hgen - dpre.
__global__ void __launch_bounds__(1024) finalize_kernel(const DevJob j, const int64_t M) {
  __shared__ long long s_tmp[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  for (int m = t; m < j.np1; m += nt) {
    j.h[m] += static_cast<long long>(j.hgen[m] - j.dpre[m]);
    j.hgen[m] = 0ull;
    j.dpre[m] = 0ull;
  }
  const int per = (j.p + nt - 1) / nt;
  const int lo = min(j.p, t * per), hi = min(j.p, lo + per);  // positions in the joint
  long long sum = 0, rej = 0;
  for (int q = lo; q < hi; ++q) {
    const int64_t k = j.k[j.perm[q]];
    sum += k > 0 ? (M - k + 1) : 0;
    rej += k > 0 ? 0 : 1;
  }
  s_tmp[t] = sum;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    const long long v = (t >= off) ? s_tmp[t - off] : 0;
    __syncthreads();
    s_tmp[t] += v;
    __syncthreads();
  }
  long long run = s_tmp[t] - sum;
  for (int q = lo; q < hi; ++q) {
    const int i = j.perm[q];
    j.offsets[i] = run;
    const int64_t k = j.k[i];
    run += k > 0 ? (M - k + 1) : 0;
  }
  if (t == nt - 1) {
    j.stats[kStatJoined] = s_tmp[t];
    j.stats[kStatJoinedTotal] += s_tmp[t];
  }
  __syncthreads();
  s_tmp[t] = rej;
  __syncthreads();
  if (t == 0) {
    long long r = 0;
    for (int q = 0; q < nt; ++q) r += s_tmp[q];
    j.stats[kStatRejected] = r;
  }
}

// Control experiment (no detailed balance at the joints): keep everything.
__global__ void naive_kernel(const DevJob j) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < j.p) {
    j.k[i] = 1;
    j.xused[i] = -1;
  }
  if (i == 0) {
    j.stats[kStatCarry] = j.m[j.perm[j.p - 1]];
    j.stats[kStatCarryValid] = 1;
    j.stats[kStatMismatch] = 0;
    j.stats[kStatPasses] = 0;
  }
}

__global__ void clear_stats_kernel(const DevJob j) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    j.stats[kStatSearched] = 0;
    j.stats[kStatMismatch] = 0;
    j.stats[kStatPasses] = 0;
    j.stats[kStatPending] = 0;
    j.stats[kStatQueuePrefix] = 0;
    j.stats[kStatPartial] = 0;
    j.stats[kStatWholeFill] = 0;
    j.stats[kStatScanned] = 0;
    j.stats[kStatFirstPending] = j.p;
  }
  // earliest accepted sample of each chain: none found yet
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < j.p; i += gridDim.x * blockDim.x) j.kmin[i] = kNoHit;
}

// One grid-wide resolution pass, part 1 (one block): with the current k's,
// the actual input of chain i is the last level of the nearest chain before
// it that kept samples (or the carry).  Chains whose k was computed for
// another input are queued in work[], with the new input in xused, and
// their joint thresholds are rebuilt by tj_list_kernel.
//
// defer (speculative passes ahead of the exact scan): the pass is left to
// the scan -- the pending count seen by the pass's kernels is 0 and the
// chains stay marked (k = -1), so the next mark lists them again (a chain
// with k < 0 is pending whatever its input) -- when more than p/16 chains
// are pending (rough weights: passes are unlikely to settle them) and the
// scan's serial cost, ~1.5 us per evaluated chain, is below that of two
// passes, ~70 ns per sample of a C-sweep segment replay: pending * 11 <
// C * N.  (Measured at 20 sweeps: joint L = 128 28 -> 18 ms, L = 96 15 ->
// 10 ms; L = 32 with 16384 chains, where the scan would be long, keeps the
// passes.)
__global__ void __launch_bounds__(1024) mark_kernel(const DevJob j, const int defer) {
  __shared__ int s_tmp[1024];
  __shared__ int s_count, s_first, s_new;
  block_last_accepted(j, s_tmp, j.lastacc);
  if (threadIdx.x == 0) {
    s_count = 0;
    s_first = j.p;
    s_new = 0;
  }
  __syncthreads();
  const int carry_in = j.stats[kStatCarryValid] ? static_cast<int>(j.stats[kStatCarry]) : -1;
  for (int q = threadIdx.x; q < j.p; q += blockDim.x) {   // positions in the joint
    const int last = j.lastacc[q];
    const int x = (last >= 0) ? j.m[j.perm[last]] : carry_in;
    const int i = j.perm[q];
    if (x != j.xused[i]) {
      j.xused[i] = x;
      j.k[i] = -1;
      j.kmin[i] = kNoHit;
      j.work[atomicAdd(&s_count, 1)] = i;
      atomicMin(&s_first, q);
      atomicAdd(&s_new, 1);
    } else if (j.k[i] < 0) {
      j.work[atomicAdd(&s_count, 1)] = i;   // marked earlier, not searched yet
      atomicMin(&s_first, q);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // (a recorded round's summary reads the record and the scan mostly
    // looks its answers up: whenever a sixteenth of the chains wait, it is
    // the shorter way)
    const bool deferred = defer && s_count > j.p / 16 &&
                          (j.rec != nullptr || static_cast<long long>(s_count) * 11 < static_cast<long long>(j.seg_len));
    j.stats[kStatPending] = deferred ? 0 : s_count;
    j.stats[kStatFirstPending] = s_first;
    if (s_new) {
      j.stats[kStatPasses] += 1;
      j.stats[kStatMismatch] += s_new;
    }
  }
}

// Summary replay, set-up: for the chains from the first pending one on, the
// per-level minimum of the joint uniforms (kept in tj, whose rows are
// rebuilt afterwards for the chains that still need a search) starts empty.
__global__ void summary_init_kernel(const DevJob j) {
  if (j.stats[kStatPending] == 0) return;
  const int f = static_cast<int>(j.stats[kStatFirstPending]);   // a position in the joint
  const long long n = static_cast<long long>(j.p - f) * j.np1;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < n;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = j.perm[f + static_cast<int>(idx / j.np1)];
    j.tj[static_cast<size_t>(i) * j.np1 + static_cast<size_t>(idx % j.np1)] = 0xFFFFFFFFu;
  }
  for (int q = f + blockIdx.x * blockDim.x + threadIdx.x; q < j.p; q += gridDim.x * blockDim.x) {
    const int i = j.perm[q];
    j.summ[i] = 0x7FFFFFFF;     // lowest level visited
    j.summ[j.p + i] = -1;       // highest level visited
    j.summ[2 * j.p + i] = 0;    // a level's minimum was 0xFFFFFFFF
  }
}

// Exact resolution of the joint (Sec. 2 step 4) in chain order, from the
// first chain whose speculated input was wrong: the input x of chain i is
// the last level of the nearest earlier chain that kept samples (else the
// carry).  Chain i keeps samples for input x iff some sample k passes
// u_k <= thr(W[m_k] - W[x]), i.e. iff some visited level m has
// min{u_k : m_k = m} <= thr(W[m] - W[x]) -- exact, from the summary replay.
// Where x is the input k_i was already found for, k_i decides.  Chains that
// keep samples under a new input are listed for one search pass (their x is
// now exact, so nothing cascades); the others get k_i = 0.  A chain whose
// answer the summary cannot give (a level whose every uniform was
// 0xFFFFFFFF, against a threshold of 0xFFFFFFFF) stops the scan; the chains
// from it on keep their speculated inputs for the ordinary passes.
//
// Most inputs the scan meets are the last level of one of the few chains
// just before (the rest of them kept nothing): cand_kernel settles, in
// parallel, chain q under the input of each of the kScanCand positions
// before it (position -1: the carry).  The serial rule then becomes a small
// state machine over positions -- state d = how many positions back the
// current input came from -- whose per-position transition functions are
// composed by a block-wide prefix scan, so the scan costs O(p / 1024) and
// not O(p); only an input from further back than kScanCand positions is
// evaluated one chain at a time.  The state machine is in mc_scan_fsm.cuh.

__device__ __forceinline__ uint8_t* scan_cand(const DevJob& j) {
  return reinterpret_cast<uint8_t*>(j.summ + 3 * static_cast<size_t>(j.p));   // [p][kScanCand]
}

// Whether the chain at joint position pos keeps samples for input level
// x >= 0, from its summary: 1 yes, 0 no, 2 undecidable (a level whose every
// uniform was 0xFFFFFFFF, against a threshold of 0xFFFFFFFF).  Warp-
// collective: the 32 lanes call it with the same arguments.
__device__ __forceinline__ int scan_decide(const DevJob& j, int pos, int x) {
  const int lane = threadIdx.x & 31;
  const int ch = j.perm[pos];
  const uint32_t* um = j.tj + static_cast<size_t>(ch) * j.np1;
  const double wx = j.W[x];
  const bool flag = j.summ[2 * j.p + ch] != 0;
  int hit = 0, amb = 0;
  for (int m = j.summ[ch] + lane; m <= j.summ[j.p + ch]; m += 32) {
    const uint32_t u = um[m];
    if (u != 0xFFFFFFFFu || flag) {
      const uint32_t thr = threshold_det(__dsub_rn(j.W[m], wx));
      if (u != 0xFFFFFFFFu) hit |= (u <= thr) ? 1 : 0;
      else amb |= (thr == 0xFFFFFFFFu) ? 1 : 0;
    }
  }
  hit = __any_sync(0xFFFFFFFFu, hit);
  amb = __any_sync(0xFFFFFFFFu, amb);
  return hit ? kAnsYes : (amb ? kAnsUndecided : kAnsNo);
}

// The answer codes of chain q under the inputs of the kScanCand positions
// before it (mc_scan_fsm.cuh).
__global__ void __launch_bounds__(256) cand_kernel(const DevJob j) {
  if (j.stats[kStatPending] == 0) return;
  const int f = static_cast<int>(j.stats[kStatFirstPending]);
  const int carry_in = j.stats[kStatCarryValid] ? static_cast<int>(j.stats[kStatCarry]) : -1;
  uint8_t* cand = scan_cand(j);
  const int lane = threadIdx.x & 31;
  const long long nwarps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  const long long n = static_cast<long long>(j.p - f) * kScanCand;
  for (long long w = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5; w < n; w += nwarps) {
    const int q = f + static_cast<int>(w / kScanCand), d = 1 + static_cast<int>(w % kScanCand);
    const int src = q - d;
    const int x = src >= 0 ? j.m[j.perm[src]] : (src == -1 ? carry_in : -1);
    int code = kAnsNone;
    if (x >= 0) {
      const int ch = j.perm[q];
      const int64_t kc = j.k[ch];
      code = (kc >= 0 && j.xused[ch] == x) ? (kc > 0 ? kAnsKnownYes : kAnsKnownNo) : scan_decide(j, q, x);
    }
    if (lane == 0) cand[static_cast<size_t>(q) * kScanCand + d - 1] = static_cast<uint8_t>(code);
  }
}

__device__ __forceinline__ unsigned long long cand_codes(const DevJob& j, int q) {
  const uint32_t* c32 = reinterpret_cast<const uint32_t*>(scan_cand(j));
  const size_t w = 2 * static_cast<size_t>(q);
  return c32[w] | (static_cast<unsigned long long>(c32[w + 1]) << 32);
}

__global__ void __launch_bounds__(1024) scan_kernel(const DevJob j) {
  if (j.stats[kStatPending] == 0) return;
  __shared__ Trans s_tr[1024];
  __shared__ int s_first, s_count, s_state, s_from, s_last, s_end;
  __shared__ unsigned long long s_scanned;
  const int t = threadIdx.x, nt = blockDim.x;
  const int f = static_cast<int>(j.stats[kStatFirstPending]);
  const int carry_in = j.stats[kStatCarryValid] ? static_cast<int>(j.stats[kStatCarry]) : -1;
  if (t == 0) {
    const int last = j.lastacc[f];   // position of the nearest chain before that kept samples (-1: none)
    s_state = (last < 0 && carry_in < 0) ? 0 : min(f - last, kFar);
    s_last = last;
    s_from = f;
    s_count = 0;
    s_end = -1;
    s_scanned = 0;
  }
  __syncthreads();
  unsigned long long scanned = 0;
  for (;;) {
    // a pass over positions [a, p) from state st0, each thread a range
    const int a = s_from, st0 = s_state;
    if (a >= j.p || s_end >= 0) break;
    const int len = j.p - a, per = (len + nt - 1) / nt;
    const int lo = min(j.p, a + t * per), hi = min(j.p, lo + per);
    Trans agg = tr_identity();
    for (int q = lo; q < hi; ++q) agg = tr_then(agg, tr_position(cand_codes(j, q)));
    s_tr[t] = agg;
    if (t == 0) s_first = j.p;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {   // inclusive prefix of the ranges' compositions
      const Trans prev = t >= off ? s_tr[t - off] : tr_identity();
      __syncthreads();
      s_tr[t] = tr_then(prev, s_tr[t]);
      __syncthreads();
    }
    const int s_in = tr_at(t > 0 ? s_tr[t - 1] : tr_identity(), st0);   // state entering this range
    // the first position entered in state kFar or kStop ends the pass
    int s = s_in;
    for (int q = lo; q < hi; ++q) {
      if (s >= kFar) {
        atomicMin(&s_first, q);
        break;
      }
      s = tr_at(tr_position(cand_codes(j, q)), s);
    }
    __syncthreads();
    const int stop_at = s_first;
    // the positions before it: inputs and outcomes, in parallel
    s = s_in;
    for (int q = lo; q < min(hi, stop_at); ++q) {
      const unsigned long long codes = cand_codes(j, q);
      const int ch = j.perm[q];
      if (s == 0) {   // no input yet: the chain is kept whole
        j.xused[ch] = -1;
        j.k[ch] = 1;
      } else {
        const int c = static_cast<int>((codes >> (8 * (s - 1))) & 0xFFu);
        if (c < kAnsKnownNo) {   // not known for this input
          const int src = q - s;
          j.xused[ch] = src >= 0 ? j.m[j.perm[src]] : carry_in;
          if (c == kAnsYes) {
            j.k[ch] = -1;   // to be searched under the exact input
            j.kmin[ch] = kNoHit;
            j.work[atomicAdd(&s_count, 1)] = ch;
          } else {
            j.k[ch] = 0;
          }
          ++scanned;
        }
      }
      s = tr_at(tr_position(codes), s);
    }
    if (stop_at >= j.p) break;   // uniform: every position is settled
    // at stop_at: kStop ends the scan; kFar (the input is the last level of
    // a chain more than kScanCand positions back) is carried one chain at a
    // time, by one warp, until a chain keeps samples
    if (t < 32) {
      const int owner = (stop_at - a) / per;   // the thread whose range holds stop_at
      int sst = tr_at(owner > 0 ? s_tr[owner - 1] : tr_identity(), st0);
      for (int q = a + owner * per; q < stop_at; ++q) sst = tr_at(tr_position(cand_codes(j, q)), sst);
      int end = -1, next_from = j.p;
      if (sst == kStop) {
        end = stop_at;
      } else {
        // the chain that kept samples last: kScanCand + 1 positions back if
        // the state became kFar in this pass, else the pass's own start
        const int last = stop_at > a ? stop_at - kFar : s_last;
        const int x = last >= 0 ? j.m[j.perm[last]] : carry_in;
        for (int q = stop_at; q < j.p; ++q) {
          const int ch = j.perm[q];
          const int64_t kc = j.k[ch];
          const int code = (kc >= 0 && j.xused[ch] == x) ? (kc > 0 ? kAnsKnownYes : kAnsKnownNo) : scan_decide(j, q, x);
          if (code == kAnsUndecided) {
            end = q;
            break;
          }
          if (t == 0 && code < kAnsKnownNo) {
            j.xused[ch] = x;
            ++scanned;
            if (code == kAnsYes) {
              j.k[ch] = -1;
              j.kmin[ch] = kNoHit;
              j.work[atomicAdd(&s_count, 1)] = ch;
            } else {
              j.k[ch] = 0;
            }
          }
          if (code == kAnsYes || code == kAnsKnownYes) {
            next_from = q + 1;
            break;
          }
        }
      }
      if (t == 0) {
        s_end = end;
        s_from = next_from;
        s_state = 1;
        s_last = next_from - 1;
      }
    }
    __syncthreads();
  }
  atomicAdd(&s_scanned, scanned);
  __syncthreads();
  // stopped early: chains still waiting for a search keep their inputs
  if (t == 0) {
    for (int q = s_end >= 0 ? s_end : j.p; q < j.p; ++q)
      if (j.k[j.perm[q]] < 0) j.work[s_count++] = j.perm[q];
    j.stats[kStatPending] = s_count;
    j.stats[kStatScanned] = static_cast<long long>(s_scanned);
  }
}

__global__ void tj_list_kernel(const DevJob j) {
  const long long total = j.stats[kStatPending] * static_cast<long long>(j.np1);
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = j.work[idx / j.np1], m = static_cast<int>(idx % j.np1);
    const int x = j.xused[i];
    j.tj[static_cast<size_t>(i) * j.np1 + m] = (x < 0) ? 0xFFFFFFFFu : threshold_det(__dsub_rn(j.W[m], j.W[x]));
  }
}

// Chains of the list (all, or work[]) that found no accepted sample in
// their first segment go to work2 -- only they need their later segments
// searched (one block).
__global__ void __launch_bounds__(1024) nohit_kernel(const DevJob j, const int list_mode) {
  __shared__ int s_count;
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  const int n = list_mode ? static_cast<int>(j.stats[kStatPending]) : j.p;
  const unsigned long long segN = static_cast<unsigned long long>(j.seg_len);
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int i = list_mode ? j.work[q] : q;
    if (j.kmin[i] > segN) j.work2[atomicAdd(&s_count, 1)] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) j.stats[kStatNoHit] = s_count;
}

// ------------------------------------------------------------------ rounds of any length
// Rounds that do not start or end on a sweep (Fig. 2's M_node = 100 < N):
// attempt t of a chain visits site t mod N and draws word t&3 of Philox
// block t>>2, with the thresholds and the acceptance rule of the sweep
// kernels, so the chains are the same whichever kernel runs them.  Meant for
// short rounds: one thread per chain works straight on its bit-packed
// lattice in global memory and counts every sample into hgen.
__device__ __forceinline__ int site_spin(const uint32_t* lat, int wd, int L, int x, int y) {
  x = (x + L) % L;
  y = (y + L) % L;
  return static_cast<int>((lat[y * wd + (x >> 5)] >> (x & 31)) & 1u);
}

// one attempt: returns the new level; flips the site in lat if accepted
__device__ __forceinline__ int attempt_one(const DevJob& j, uint32_t* lat, int m, uint64_t t, uint32_t chain,
                                           uint4& r, uint64_t& blk) {
  const int site = static_cast<int>(t % static_cast<uint64_t>(j.N));
  const int x = site % j.L, y = site / j.L;
  const int sv = site_spin(lat, j.wd, j.L, x, y);
  const int a = (site_spin(lat, j.wd, j.L, x - 1, y) == sv) + (site_spin(lat, j.wd, j.L, x + 1, y) == sv) +
                (site_spin(lat, j.wd, j.L, x, y - 1) == sv) + (site_spin(lat, j.wd, j.L, x, y + 1) == sv);
  if ((t >> 2) != blk) {
    blk = t >> 2;
    r = philox4x32_10(make_uint4(static_cast<uint32_t>(blk), static_cast<uint32_t>(blk >> 32), chain, kTagFlip),
                      j.key0, j.key1);
  }
  const uint32_t u = uint4_word(r, static_cast<uint32_t>(t & 3u));
  if (u <= j.T[a * j.np1 + m]) {
    lat[y * j.wd + (x >> 5)] ^= 1u << (x & 31);
    m += a - 2;
  }
  return m;
}

__global__ void attempts_kernel(const DevJob j, const uint64_t t0, const int64_t n, int32_t* __restrict__ rec) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= j.p) return;
  uint32_t* lat = j.spins + static_cast<size_t>(c) * j.L * j.wd;
  int m = j.m[c];
  uint4 r = make_uint4(0u, 0u, 0u, 0u);
  uint64_t blk = ~0ull;
  int32_t* lv = rec ? rec + static_cast<size_t>(c) * n : nullptr;
  for (int64_t k = 0; k < n; ++k) {
    m = attempt_one(j, lat, m, t0 + static_cast<uint64_t>(k), static_cast<uint32_t>(c), r, blk);
    atomicAdd(&j.hgen[m], 1ull);
    if (lv) lv[k] = m;
  }
  j.m[c] = m;
}

// The joint of such a round (Sec. 2 steps 3-5) from the recorded levels:
// the chains in joint order, one at a time (the input of each is the level
// passed on by those before it), the samples of a chain tested in parallel
// -- sample k passes iff its joint uniform Philox((k-1)>>2, r, chain, 1)
// word (k-1)&3 is at most thr(W[m_k] - W[x]) -- in blocks of the block's
// threads, stopping at the first block with a pass; k_i is the smallest
// passing k.  The samples before it (all M when none passes) go to dpre.
__global__ void __launch_bounds__(1024) partial_joint_kernel(const DevJob j, const int64_t M, const uint32_t r) {
  __shared__ unsigned long long s_k;
  __shared__ int s_carry, s_valid;
  const int t = threadIdx.x, nt = blockDim.x;
  if (t == 0) {
    s_valid = static_cast<int>(j.stats[kStatCarryValid]);
    s_carry = static_cast<int>(j.stats[kStatCarry]);
  }
  __syncthreads();
  long long searched = 0;
  for (int q = 0; q < j.p; ++q) {
    const int c = j.perm[q];
    const int valid = s_valid, carry = s_carry;
    const int32_t* lv = j.plv + static_cast<size_t>(c) * M;
    __syncthreads();   // everyone has read s_valid / s_carry of this chain
    if (t == 0) {
      s_k = kNoHit;
      j.xused[c] = valid ? carry : -1;
    }
    __syncthreads();
    int64_t kf = 1;   // nothing passed on yet: the chain is kept whole
    if (valid) {
      const double wx = j.W[carry];
      for (int64_t base = 0; base < M; base += nt) {
        const int64_t k0 = base + t;   // sample k0 + 1
        bool hit = false;
        if (k0 < M) {
          const uint4 v = philox4x32_10(make_uint4(static_cast<uint32_t>(k0 >> 2), r, static_cast<uint32_t>(c), kTagJoint),
                                        j.key0, j.key1);
          hit = uint4_word(v, static_cast<uint32_t>(k0 & 3)) <= threshold_det(__dsub_rn(j.W[lv[k0]], wx));
          ++searched;
        }
        if (hit) atomicMin(&s_k, static_cast<unsigned long long>(k0 + 1));
        if (__syncthreads_or(hit)) break;
      }
      kf = s_k == kNoHit ? 0 : static_cast<int64_t>(s_k);
    }
    const int64_t nd = kf > 0 ? kf - 1 : M;   // discarded samples
    for (int64_t k0 = t; k0 < nd; k0 += nt) atomicAdd(&j.dpre[lv[k0]], 1ull);
    if (t == 0) {
      j.k[c] = kf;
      if (kf > 0) {
        s_carry = j.m[c];
        s_valid = 1;
      }
    }
    __syncthreads();
  }
  if (searched) atomicAdd(reinterpret_cast<unsigned long long*>(&j.stats[kStatSearched]),
                          static_cast<unsigned long long>(searched));
  if (t == 0) {
    j.stats[kStatCarry] = s_carry;
    j.stats[kStatCarryValid] = s_valid;
    j.stats[kStatMismatch] = 0;
    j.stats[kStatPasses] = 0;
    j.stats[kStatScanned] = 0;
  }
}

__global__ void clear_searched_kernel(const DevJob j) {
  if (threadIdx.x == 0) j.stats[kStatSearched] = 0;
}

// The joint of such a round by the serial rule itself (Sec. 2 steps 3-5),
// one thread: each chain, in joint order, is regenerated from its round
// start until its first sample that passes the test against the level
// passed on; the samples before it go to dpre.
constexpr int kMaxLatWords = 128 * 4;
__global__ void serial_joint_kernel(const DevJob j, const uint64_t t0, const int64_t M, const uint32_t r) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int carry_valid = static_cast<int>(j.stats[kStatCarryValid]);
  int carry = static_cast<int>(j.stats[kStatCarry]);
  uint32_t lat[kMaxLatWords];
  long long searched = 0;
  for (int q = 0; q < j.p; ++q) {
    const int c = j.perm[q];
    int64_t kf = 0;
    j.xused[c] = carry_valid ? carry : -1;
    if (!carry_valid) {
      kf = 1;
    } else {
      const uint32_t* src = j.spins0 + static_cast<size_t>(c) * j.L * j.wd;
      for (int w = 0; w < j.L * j.wd; ++w) lat[w] = src[w];
      int m = j.m0[c];
      uint4 fr = make_uint4(0u, 0u, 0u, 0u), jr = fr;
      uint64_t blk = ~0ull;
      const double wx = j.W[carry];
      for (int64_t k = 1; k <= M; ++k) {
        m = attempt_one(j, lat, m, t0 + static_cast<uint64_t>(k - 1), static_cast<uint32_t>(c), fr, blk);
        const uint64_t qk = static_cast<uint64_t>(k - 1);
        if ((qk & 3u) == 0u || k == 1)
          jr = philox4x32_10(make_uint4(static_cast<uint32_t>(qk >> 2), r, static_cast<uint32_t>(c), kTagJoint),
                             j.key0, j.key1);
        ++searched;
        if (uint4_word(jr, static_cast<uint32_t>(qk & 3u)) <= threshold_det(__dsub_rn(j.W[m], wx))) {
          kf = k;
          break;
        }
        j.dpre[m] += 1ull;   // a discarded sample
      }
    }
    j.k[c] = kf;
    if (kf > 0) {
      carry = j.m[c];
      carry_valid = 1;
    }
  }
  j.stats[kStatCarry] = carry;
  j.stats[kStatCarryValid] = carry_valid;
  j.stats[kStatMismatch] = 0;
  j.stats[kStatPasses] = 0;
  j.stats[kStatScanned] = 0;
  j.stats[kStatSearched] = searched;
}

cudaError_t k_generate_attempts(const DevJob& j, uint64_t t0, int64_t n, bool record, cudaStream_t st) {
  attempts_kernel<<<blocks_for(j.p, 128), 128, 0, st>>>(j, t0, n, record ? j.plv : nullptr);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t k_join_attempts(const DevJob& j, uint64_t t0, int64_t M, uint32_t r, bool naive, bool recorded,
                            cudaStream_t st) {
  order_kernel<<<1, 1024, 0, st>>>(j);
  if (naive) {
    naive_kernel<<<blocks_for(j.p, 256), 256, 0, st>>>(j);
  } else if (recorded) {
    clear_searched_kernel<<<1, 32, 0, st>>>(j);
    partial_joint_kernel<<<1, 1024, 0, st>>>(j, M, r);
    launches_add(1);
  } else {
    serial_joint_kernel<<<1, 32, 0, st>>>(j, t0, M, r);
  }
  finalize_kernel<<<1, 1024, 0, st>>>(j, M);
  launches_add(3);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ host side
size_t gen_smem_bytes(int L, const LaunchShape& s, bool* table_in_smem) {
  const bool ts = table_fits(L, s, true);
  if (table_in_smem) *table_in_smem = ts;
  return plan_bytes(L, s, ts, true);
}

bool shape_supported(int L, const LaunchShape& s) {
  if (L < 4 || L > 128 || (L % 4) != 0) return false;
  if (s.cpw < 1 || s.cpw > 32 || s.wpb < 1 || s.wpb > 4) return false;
  if (s.placement == kPlaceReg && L > 32) return false;
  if (s.placement == kPlaceGlobal && L != 96 && L != 100 && L != 128) return false;
  if (s.placement != kPlaceReg && s.placement != kPlaceSmem && s.placement != kPlaceGlobal) return false;
  return plan_bytes(L, s, false, true) <= kMaxSmem;
}

LaunchShape default_shape(int L, int p, int num_sms) {
  LaunchShape s;
  // lattice rows in registers for L <= 32, except L = 24 and 32, whose
  // compile-time shared-memory bodies measured faster (L = 32, 16384 chains:
  // generation 6 % shorter, no rotation of 32 row registers per row)
  s.placement = (L <= 32 && L != 24 && L != 32) ? kPlaceReg : kPlaceSmem;
  s.wpb = 4;
  const int warps = std::max(1, num_sms) * 4;  // one warp per SM sub-partition
  s.cpw = std::min(32, std::max(1, (p + warps - 1) / warps));
  // lattices in global memory: at L = 96 so that the threshold table fits in
  // shared memory (generation 2.2x faster at 1024 and 2048 chains, 20
  // sweeps); at L = 100, 128 (table in global memory either way) only with
  // full warps, where they leave a block's shared memory to the histogram --
  // lane groups ran 6-9 % faster with the lattices in shared memory
  if (L == 96 || ((L == 100 || L == 128) && s.cpw > 8)) s.placement = kPlaceGlobal;
  while (s.wpb > 1 && !shape_supported(L, s)) s.wpb >>= 1;
  while (s.cpw > 1 && !shape_supported(L, s)) s.cpw >>= 1;
  return s;
}

// Densest shape for L and p: as many chains per warp as there are (up to 32),
// keeping the threshold table in shared memory if the default shape has it
// there.  The time of a round is set by the latency of one chain, which a
// fuller warp does not change (measured: within 5 % for L <= 64 and 128), so
// a job shaped this way takes the same time on far fewer warps -- the rest
// of the GPU stays free for other jobs (the server uses it).
LaunchShape dense_shape(int L, int p, int num_sms) {
  LaunchShape def = default_shape(L, p, num_sms);
  // full warps at L = 100, 128 keep their lattices in global memory: a block
  // of 128 chains then needs only the histogram's shared memory, so blocks
  // of other jobs fit beside it
  if (L == 100 || L == 128) def.placement = kPlaceGlobal;
  const bool ts = table_fits(L, def, true);
  for (int cpw = std::min(32, std::max(1, p)); cpw >= 1; --cpw)
    for (int w = 4; w >= 1; --w) {
      LaunchShape s{def.placement, cpw, w};
      if (w > 1 && (w - 1) * cpw >= p) continue;  // no empty warps
      if (shape_supported(L, s) && (!ts || table_fits(L, s, true))) return s;
    }
  return def;
}

// The joint's replay kernels take their own launch shape (their work items
// are (chain, segment) pairs, not chains): as many lanes a block as the
// lattices leave room for, preferring shapes whose threshold table (and the
// prefix pass's histogram) still fit in shared memory.  The prefix pass, which
// also needs the histogram there, narrows the warps further if it must
// (launch_join_t).  L = 128: 28 lanes x 4 warps instead of 32 x 2 -- the
// lattices, 2 KB a lane, fill shared memory either way, and four warps keep
// all four sub-partitions issuing.
static bool replay_fits(int L, const LaunchShape& s) {
  if (s.cpw < 1 || s.cpw > 32 || s.wpb < 1 || s.wpb > 4) return false;
  if (s.placement == kPlaceReg && L > 32) return false;
  return plan_bytes(L, s, false, false) <= kMaxSmem;
}

static LaunchShape join_shape(int L, const LaunchShape& gen_shape) {
  LaunchShape gen = gen_shape;
  if (gen.placement == kPlaceGlobal) gen.placement = kPlaceSmem;   // replays restore into shared memory
  LaunchShape best = gen;
  int best_lanes = 0;
  bool best_ts = false;
  for (int w = 4; w >= 1; --w) {
    int cpw = 32;
    while (cpw > 1 && !replay_fits(L, LaunchShape{gen.placement, cpw, w})) --cpw;
    const LaunchShape s{gen.placement, cpw, w};
    if (!replay_fits(L, s)) continue;
    int c2 = cpw;  // most chains per warp that leave the table and histogram in shared memory
    while (c2 >= 1 && !table_fits(L, LaunchShape{gen.placement, c2, w}, true)) --c2;
    if (c2 >= 16) {
      if (!best_ts || c2 * w > best_lanes) best = LaunchShape{gen.placement, c2, w}, best_lanes = c2 * w, best_ts = true;
    } else if (!best_ts && cpw * w > best_lanes) {
      best = s, best_lanes = cpw * w;
    }
  }
  return best;
}

cudaError_t join_prelude(const DevJob& j, cudaStream_t st) {
  order_kernel<<<1, 1024, 0, st>>>(j);
  spec_inputs_kernel<<<blocks_for(j.p, 256), 256, 0, st>>>(j);
  clear_stats_kernel<<<256, 256, 0, st>>>(j);
  tj_kernel<<<blocks_for(static_cast<long long>(j.p) * j.np1, 256), 256, 0, st>>>(j, nullptr, j.p);
  launches_add(4);
  return cudaGetLastError();
}

// k_i = the earliest accepted sample the search found (0: none).
__global__ void select_kernel(const DevJob j, const int listed, const int exact_first) {
  const int n = listed ? static_cast<int>(j.stats[kStatPending]) : j.p;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int i = listed ? j.work[q] : q;
  if (exact_first && rough_last_joint(j.stats[kStatRejected], j.p)) {
    j.k[i] = -1;   // not searched: every chain waits for the exact path
    return;
  }
  const unsigned long long k = j.kmin[i];
  j.k[i] = k == kNoHit ? 0 : static_cast<int64_t>(k);
}

// Work list of the prefix pass: for every chain, its whole segments before
// the one holding k_i (all segments if nothing is kept) and, if k_i is not
// the first sample of its segment, that segment as a partial item.  Whole
// segments are counted first, then placed at the front of the list.
__global__ void prefix_count_kernel(const DevJob j, const int64_t S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= j.p) return;
  const int64_t segN = j.seg_len;
  const int64_t k = j.k[i];
  const int whole = (k > 0) ? static_cast<int>((k - 1) / segN) : j.ck_K;
  atomicAdd(reinterpret_cast<unsigned long long*>(&j.stats[kStatQueuePrefix]), static_cast<unsigned long long>(whole));
  (void)S;
}

__global__ void prefix_fill_kernel(const DevJob j, const int64_t S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= j.p) return;
  const int64_t segN = j.seg_len;
  const int64_t k = j.k[i];
  const int whole = (k > 0) ? static_cast<int>((k - 1) / segN) : j.ck_K;
  unsigned long long* w = reinterpret_cast<unsigned long long*>(&j.stats[kStatWholeFill]);
  unsigned long long* pcount = reinterpret_cast<unsigned long long*>(&j.stats[kStatPartial]);
  if (whole > 0) {
    const unsigned long long pos = atomicAdd(w, static_cast<unsigned long long>(whole));
    for (int s = 0; s < whole; ++s) j.plist[pos + s] = make_int2(i, s);
  }
  if (k > 0 && (k - 1) % segN != 0) {
    const unsigned long long total_whole = static_cast<unsigned long long>(j.stats[kStatQueuePrefix]);
    const unsigned long long pos = total_whole + atomicAdd(pcount, 1ull);
    j.plist[pos] = make_int2(i, whole);
  }
  (void)S;
}

__global__ void prefix_total_kernel(const DevJob j) {
  if (threadIdx.x == 0) j.stats[kStatQueuePrefix] += j.stats[kStatPartial];
}

__global__ void reset_queue_kernel(const DevJob j) {
  if (threadIdx.x == 0) j.stats[kStatQueueSearch] = 0;
}

cudaError_t join_summary_init(const DevJob& j, cudaStream_t st) {
  summary_init_kernel<<<1024, 256, 0, st>>>(j);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t join_scan(const DevJob& j, cudaStream_t st) {
  // one warp per (chain, candidate input), grid-stride
  cand_kernel<<<std::min(1024u, blocks_for(static_cast<long long>(j.p) * kScanCand * 32, 256)), 256, 0, st>>>(j);
  scan_kernel<<<1, 1024, 0, st>>>(j);
  launches_add(2);
  return cudaGetLastError();
}

cudaError_t join_reset_queue(const DevJob& j, cudaStream_t st) {
  reset_queue_kernel<<<1, 32, 0, st>>>(j);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t join_prefix_list(const DevJob& j, cudaStream_t st) {
  prefix_count_kernel<<<blocks_for(j.p, 256), 256, 0, st>>>(j, 0);
  prefix_fill_kernel<<<blocks_for(j.p, 256), 256, 0, st>>>(j, 0);
  prefix_total_kernel<<<1, 32, 0, st>>>(j);
  launches_add(3);
  return cudaGetLastError();
}

cudaError_t join_select(const DevJob& j, bool listed, cudaStream_t st, bool exact_first) {
  select_kernel<<<blocks_for(j.p, 256), 256, 0, st>>>(j, listed ? 1 : 0, !listed && exact_first ? 1 : 0);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t join_mark(const DevJob& j, cudaStream_t st, bool thresholds, bool defer) {
  mark_kernel<<<1, 1024, 0, st>>>(j, defer ? 1 : 0);
  launches_add(1);
  return thresholds ? join_tj_list(j, st) : cudaGetLastError();
}

cudaError_t join_nohit(const DevJob& j, int list_mode, cudaStream_t st) {
  nohit_kernel<<<1, 1024, 0, st>>>(j, list_mode);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t join_tj_list(const DevJob& j, cudaStream_t st) {
  tj_list_kernel<<<256, 256, 0, st>>>(j);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t join_finalize(const DevJob& j, int64_t S, cudaStream_t st) {
  finalize_kernel<<<1, 1024, 0, st>>>(j, S * j.N);
  launches_add(1);
  return cudaGetLastError();
}

static cudaError_t dispatch(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace,
                            uint32_t r, cudaStream_t st) {
  if (s.placement == kPlaceReg) {
    if (j.L <= 16) return chain_kernels_reg_a(j, s, gen, t0, S, trace, r, st);
    if (j.L <= 28) return chain_kernels_reg_b(j, s, gen, t0, S, trace, r, st);
    return chain_kernels_reg_c(j, s, gen, t0, S, trace, r, st);
  }
  switch (j.L) {
    case 16:
    case 24: return chain_kernels_smem_L16_24(j, s, gen, t0, S, trace, r, st);
    case 32: return chain_kernels_smem_L32(j, s, gen, t0, S, trace, r, st);
    case 48: return chain_kernels_smem_L48(j, s, gen, t0, S, trace, r, st);
    case 64: return chain_kernels_smem_L64(j, s, gen, t0, S, trace, r, st);
    case 96: return chain_kernels_smem_L96(j, s, gen, t0, S, trace, r, st);
    case 100: return chain_kernels_smem_L100(j, s, gen, t0, S, trace, r, st);
    case 128: return chain_kernels_smem_L128(j, s, gen, t0, S, trace, r, st);
    default: break;
  }
  switch (j.wd) {
    case 1: return chain_kernels_smem_1(j, s, gen, t0, S, trace, r, st);
    case 2: return chain_kernels_smem_2(j, s, gen, t0, S, trace, r, st);
    case 3: return chain_kernels_smem_3(j, s, gen, t0, S, trace, r, st);
    case 4: return chain_kernels_smem_4(j, s, gen, t0, S, trace, r, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t k_generate(const DevJob& j, const LaunchShape& s, uint64_t t0, int64_t S, bool trace, cudaStream_t st) {
  if (j.rec) {   // a recorded round is never replayed: no checkpoints
    DevJob g = j;
    g.ckpt = nullptr;
    return dispatch(g, s, true, t0, S, trace, 0u, st);
  }
  return dispatch(j, s, true, t0, S, trace, 0u, st);
}

cudaError_t k_join(const DevJob& j, const LaunchShape& s, uint64_t t0, int64_t S, uint32_t r, bool naive,
                   cudaStream_t st) {
  if (naive) {
    order_kernel<<<1, 1024, 0, st>>>(j);
    naive_kernel<<<blocks_for(j.p, 256), 256, 0, st>>>(j);
    finalize_kernel<<<1, 1024, 0, st>>>(j, S * j.N);
    launches_add(3);
    return cudaGetLastError();
  }
  if (j.rec) return chain_kernels_record(j, t0, S, r, st);   // levels recorded: no replays
  return dispatch(j, join_shape(j.L, s), false, t0, S, false, r, st);
}

cudaError_t k_order(const DevJob& j, cudaStream_t st) {
  order_kernel<<<1, 1024, 0, st>>>(j);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t k_init_lattice(const DevJob& j, int start, cudaStream_t st) {
  const long long n = static_cast<long long>(j.p) * j.L * j.wd;
  init_lattice_kernel<<<blocks_for(n, 256), 256, 0, st>>>(j, start);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t k_levels(const DevJob& j, cudaStream_t st) {
  levels_kernel<<<blocks_for(j.p, 128), 128, 0, st>>>(j);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t k_build_table(const DevJob& j, cudaStream_t st) {
  table_kernel<<<blocks_for(5ll * j.np1, 256), 256, 0, st>>>(j);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t k_thermo(const DevJob& j, const double* betas, int n, double* out, cudaStream_t st) {
  thermo_kernel<<<n, kThermoThreads, 0, st>>>(j, betas, out);
  launches_add(1);
  return cudaGetLastError();
}

cudaError_t k_update_weights(const DevJob& j, cudaStream_t st) {
  weights_kernel<<<blocks_for(j.np1, 256), 256, 0, st>>>(j);
  launches_add(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return k_build_table(j, st);
}

}  // namespace mcgpu
