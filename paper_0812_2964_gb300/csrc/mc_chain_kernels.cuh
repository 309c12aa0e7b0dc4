// Templated chain kernels (generation, speculative joint search, resolution,
// prefix correction) and their launchers.  Included by the instantiation
// units mc_inst_*.cu, each of which compiles the kernels for a few lattice
// sizes so that the library builds in parallel.
#pragma once
#include <algorithm>
#include <type_traits>

#include "mc_chain.cuh"
#include "mc_internal.h"

namespace mcgpu {

inline unsigned blocks_for(long long n, int t) { return static_cast<unsigned>((n + t - 1) / t); }

// ------------------------------------------------------------------ runners
// A chain's lattice during a sweep, in registers (L <= 32, one word per row;
// rows rotate through the register array so that every index is static) or
// in shared memory (any L; per-thread column with a stride of the number of
// lanes that hold chains, so that a warp's accesses hit distinct banks).
template <int L>
struct RegRunner {
  static constexpr int WD = 1;
  uint32_t R[L];
  __device__ __forceinline__ void load(const uint32_t* __restrict__ g) {
#pragma unroll
    for (int y = 0; y < L; ++y) R[y] = g[y];
  }
  __device__ __forceinline__ void store(uint32_t* __restrict__ g) const {
#pragma unroll
    for (int y = 0; y < L; ++y) g[y] = R[y];
  }
  // word y of this chain at g[y * stride] (checkpoint layout [word][chain])
  __device__ __forceinline__ void save_strided(uint32_t* __restrict__ g, size_t stride) const {
#pragma unroll
    for (int y = 0; y < L; ++y) g[y * stride] = R[y];
  }
  __device__ __forceinline__ void load_strided(const uint32_t* __restrict__ g, size_t stride) {
#pragma unroll
    for (int y = 0; y < L; ++y) R[y] = g[y * stride];
  }
  template <bool EARLY, int GL = 1, class Hook>
  __device__ __forceinline__ void sweep(int& m, Prefetch& pf, const uint32_t* __restrict__ T, int np1,
                                        uint32_t chain, uint32_t k0, uint32_t k1, Hook& hk) {
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
      uint32_t cur[1] = {R[0]};
      const uint32_t up[1] = {R[L - 1]};
      const uint32_t dn[1] = {R[1]};
      sweep_row<1, GL>(cur, up, dn, L, m, T, np1, pf, chain, k0, k1, hk);
#pragma unroll
      for (int i = 0; i < L - 1; ++i) R[i] = R[i + 1];
      R[L - 1] = cur[0];
      if constexpr (EARLY) {
        if (hk.done) break;
      }
    }
  }
};

// SL > 0 fixes L at compile time (no per-site guards); SL == 0 reads L at run time.
template <int WD_, int SL = 0>
struct SmemRunner {
  static constexpr int WD = WD_;
  uint32_t* lat;  // this chain's column
  int stride, Lrt;
  __device__ __forceinline__ int len() const { return SL > 0 ? SL : Lrt; }
  __device__ __forceinline__ void load(const uint32_t* __restrict__ g) {
    const int L = len();
    for (int i = 0; i < L * WD; ++i) lat[i * stride] = g[i];
  }
  __device__ __forceinline__ void store(uint32_t* __restrict__ g) const {
    const int L = len();
    for (int i = 0; i < L * WD; ++i) g[i] = lat[i * stride];
  }
  __device__ __forceinline__ void save_strided(uint32_t* __restrict__ g, size_t gstride) const {
    const int L = len();
    for (int i = 0; i < L * WD; ++i) g[i * gstride] = lat[i * stride];
  }
  __device__ __forceinline__ void load_strided(const uint32_t* __restrict__ g, size_t gstride) {
    const int L = len();
    for (int i = 0; i < L * WD; ++i) lat[i * stride] = g[i * gstride];
  }
  template <bool EARLY, int GL = 1, class Hook>
  __device__ __forceinline__ void sweep(int& m, Prefetch& pf, const uint32_t* __restrict__ T, int np1,
                                        uint32_t chain, uint32_t k0, uint32_t k1, Hook& hk) {
    const int L = len();
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
      const int ym = (y == 0) ? L - 1 : y - 1, yp = (y + 1 == L) ? 0 : y + 1;
      uint32_t cur[WD], up[WD], dn[WD];
#pragma unroll
      for (int w = 0; w < WD; ++w) {
        cur[w] = lat[(y * WD + w) * stride];
        up[w] = lat[(ym * WD + w) * stride];
        dn[w] = lat[(yp * WD + w) * stride];
      }
      sweep_row<WD, GL>(cur, up, dn, L, m, T, np1, pf, chain, k0, k1, hk);
#pragma unroll
      for (int w = 0; w < WD; ++w) lat[(y * WD + w) * stride] = cur[w];
      if constexpr (EARLY) {
        if (hk.done) break;
      }
    }
  }
};

// Lattice in global memory (the job's spins, updated in place), rows
// streamed through registers: the row being swept, the one above (swept
// already in this sweep), the one below, the one after it (loaded two rows
// ahead, so that the load's latency hides behind two rows of sites) and row
// 0 as swept in this sweep (the last row's lower neighbour).  Shared memory
// is left to the threshold table and the histogram: at L = 96 both fit
// there, which lattices beside them would not allow; at L = 128 more chains
// share an SM.  The lanes of a lane group store the same words.  Generation
// only (the joint's replays restore checkpoints into shared memory).
template <int WD_, int SL>
struct GlobRunner {
  static_assert(SL >= 4, "compile-time L");
  static constexpr int WD = WD_;
  uint32_t* lat;  // this chain's L rows of WD words
  __device__ __forceinline__ void load(uint32_t* g) { lat = g; }
  __device__ __forceinline__ void store(uint32_t* g) const {
    if (g != lat)
      for (int i = 0; i < SL * WD; ++i) g[i] = lat[i];
  }
  __device__ __forceinline__ void save_strided(uint32_t* __restrict__ g, size_t gstride) const {
    for (int i = 0; i < SL * WD; ++i) g[i * gstride] = lat[i];
  }
  template <bool EARLY, int GL = 1, class Hook>
  __device__ __forceinline__ void sweep(int& m, Prefetch& pf, const uint32_t* __restrict__ T, int np1,
                                        uint32_t chain, uint32_t k0, uint32_t k1, Hook& hk) {
    constexpr int L = SL;
    uint32_t up[WD], cur[WD], dn[WD], nx[WD], r0[WD];
#pragma unroll
    for (int w = 0; w < WD; ++w) {
      up[w] = lat[(L - 1) * WD + w];
      cur[w] = lat[w];
      dn[w] = lat[WD + w];
      nx[w] = lat[2 * WD + w];
      r0[w] = 0u;
    }
#pragma unroll 1
    for (int y = 0; y < L; ++y) {
      sweep_row<WD, GL>(cur, up, dn, L, m, T, np1, pf, chain, k0, k1, hk);
#pragma unroll
      for (int w = 0; w < WD; ++w) {
        lat[y * WD + w] = cur[w];
        if (y == 0) r0[w] = cur[w];
        up[w] = cur[w];
        cur[w] = dn[w];
        dn[w] = nx[w];
      }
      // the row after next: not swept yet in this sweep, or row 0 as swept
      if (y + 3 < L) {
#pragma unroll
        for (int w = 0; w < WD; ++w) nx[w] = lat[(y + 3) * WD + w];
      } else if (y + 3 == L) {
#pragma unroll
        for (int w = 0; w < WD; ++w) nx[w] = r0[w];
      }
      if constexpr (EARLY) {
        if (hk.done) break;
      }
    }
  }
};

// Shared-memory plan of a block: [table (opt.)][histogram u32][lattices].
struct SmemPlan {
  int table_words, hist_words, lat_words;
};

__host__ __device__ inline SmemPlan smem_plan(int L, int placement, int cpw, int wpb, bool tsmem, bool hist) {
  const int np1 = L * L + 1, wd = (L + 31) / 32;
  SmemPlan s;
  s.table_words = tsmem ? ((5 * np1 + 3) & ~3) : 0;
  s.hist_words = hist ? ((np1 + 3) & ~3) : 0;
  s.lat_words = placement == kPlaceSmem ? cpw * wpb * L * wd : 0;
  return s;
}

struct BlockCtx {
  const uint32_t* T;
  uint32_t* hist;
  uint32_t* lat;
  int chain, lane, warp, slot, nslot;
  bool active;
  bool owner;  // the lane that writes the chain's results (first of its lane group)
};

// Lanes per chain gl (a power of two; 1 except in the generation kernel's
// lane-group variant): lane l of a warp works on the warp's chain l / gl.
template <bool TSMEM>
__device__ __forceinline__ BlockCtx block_setup(const DevJob& j, const SmemPlan& sp, int cpw, int first_chain,
                                                bool zero_hist, int gl = 1) {
  extern __shared__ __align__(16) uint32_t smem[];
  BlockCtx b;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (TSMEM)
    for (int i = tid; i < 5 * j.np1; i += nthr) smem[i] = j.T[i];
  b.T = TSMEM ? smem : j.T;
  b.hist = smem + sp.table_words;
  if (zero_hist)
    for (int i = tid; i < sp.hist_words; i += nthr) b.hist[i] = 0u;
  b.lat = smem + sp.table_words + sp.hist_words;
  b.lane = tid & 31;
  b.warp = tid >> 5;
  const int sub = b.lane / gl;
  b.slot = b.warp * cpw + sub;
  b.nslot = (nthr >> 5) * cpw;
  b.chain = first_chain + b.slot;
  b.active = sub < cpw && b.chain < j.p;
  b.owner = b.active && (b.lane % gl) == 0;
  return b;
}

// ------------------------------------------------------------------ generation
template <int L>
struct RunnerFactoryReg {
  __device__ __forceinline__ static RegRunner<L> make(const BlockCtx&, int) { return RegRunner<L>(); }
};
template <int WD, int SL>
struct RunnerFactoryGlob {
  __device__ __forceinline__ static GlobRunner<WD, SL> make(const BlockCtx&, int) { return GlobRunner<WD, SL>(); }
};
template <int WD, int SL>
struct RunnerFactorySmem {
  __device__ __forceinline__ static SmemRunner<WD, SL> make(const BlockCtx& b, int L) {
    SmemRunner<WD, SL> r;
    r.lat = b.lat + b.slot;
    r.stride = b.nslot;
    r.Lrt = L;
    return r;
  }
};

// The joint's kernels for a recorded round: levels come from the round
// record, so there is no lattice to replay and no threshold table (the
// launch shape's placement only sizes shared memory: none for lattices).
struct RecF {
  static constexpr int kPlacement = kPlaceReg;
};
template <class F>
struct IsRec : std::false_type {};
template <>
struct IsRec<RecF> : std::true_type {};
static_assert(kRecGroupStride == 4 * kRecTile, "record layout: generation and joint agree");

// Step 2: every chain performs S sweeps (M = S N attempts) under the current
// weight; per-level dwell counts accumulate in shared memory, then in the
// round histogram hgen.  trace[s][c] = energy after sweep s.
// (The body is a device function so that the batched launch can run it for
// one of several jobs per block.)
//
// GL > 1 (lattice in shared memory, few chains per warp): the GL lanes of a
// lane group share one chain -- same lattice column, same uniforms (split
// between them, see philox_fill) -- and only the group's first lane writes
// counts, checkpoints, trace and the final state.
template <class Factory, bool TSMEM, int GL = 1, bool REC = false>
__device__ __forceinline__ void gen_body(const DevJob& j, const int cpw, const uint64_t t0, const int64_t S,
                                         const int64_t flushF, const int do_trace, const int block) {
  const SmemPlan sp = smem_plan(j.L, Factory::kPlacement, cpw, blockDim.x >> 5, TSMEM, true);
  const int first = block * (blockDim.x >> 5) * cpw;
  BlockCtx b = block_setup<TSMEM>(j, sp, cpw, first, true, GL);
  auto run = Factory::make(b, j.L);
  __syncthreads();
  int m = 0;
  Prefetch pf;
  // (one lane a chain: every lane counts; a compile-time 1 keeps the
  // reduction's operand an immediate)
  GenHook<decltype(run)::WD == 1 ? 32 : 8, REC> hk;
  hk.init(b.hist, GL == 1 ? 1u : (b.owner ? 1u : 0u), j.np1);
  const bool writer = GL == 1 ? b.active : b.owner;
  if constexpr (REC) {
    // the chain's first group in the record; every lane of a group keeps a valid
    // address (pointer arithmetic on a null pointer would let the compiler
    // drop the writer test), only the writer stores
    hk.rec = j.rec + rec_index(b.active ? b.chain : 0, 0, S * j.N);
    hk.rec_on = writer;
  }
  if (b.active) {
    run.load(j.spins + static_cast<size_t>(b.chain) * j.L * j.wd);
    m = j.m[b.chain];
    prefetch_init<decltype(run)::WD, GL>(pf, j.L, t0, static_cast<uint32_t>(b.chain), j.key0, j.key1);
  }
  const size_t lw = static_cast<size_t>(j.L) * j.wd;
  // the lanes of the warp's working lane groups: they meet again after every
  // write that only a group's first lane makes, before the next shuffles
  unsigned amask = 0xFFFFFFFFu;
  if constexpr (GL > 1) amask = __ballot_sync(0xFFFFFFFFu, b.active);
  // countdowns to the next checkpoint and the next histogram flush (no
  // 64-bit division in the sweep loop)
  int ck_left = 0, seg = 0;
  int64_t fl_left = flushF;
  for (int64_t s = 0; s < S; ++s) {
    if (b.active) {
      if (j.ckpt && ck_left == 0 && writer) {
        // lattice and level at the start of segment s / C, for the joint's replays
        run.save_strided(j.ckpt + static_cast<size_t>(seg) * lw * j.p + b.chain, static_cast<size_t>(j.p));
        j.ckm[static_cast<size_t>(seg) * j.p + b.chain] = m;
      }
      if constexpr (GL > 1) __syncwarp(amask);
      run.template sweep<false, GL>(m, pf, b.T, j.np1, static_cast<uint32_t>(b.chain), j.key0, j.key1, hk);
      if (do_trace && writer) j.trace[s * j.p + b.chain] = 4 * m - 2 * j.N;
      if constexpr (GL > 1) __syncwarp(amask);
    }
    if (ck_left == 0) {
      ck_left = j.ck_C;
      ++seg;
    }
    --ck_left;
    if (flushF > 0 && --fl_left == 0 && s + 1 < S) {
      fl_left = flushF;
      if (b.active) hk.flush(m);
      asm volatile("" ::: "memory");
      __syncthreads();
      for (int i = threadIdx.x; i < j.np1; i += blockDim.x) {
        const uint32_t v = b.hist[i];
        if (v) {
          atomicAdd(&j.hgen[i], static_cast<unsigned long long>(v));
          b.hist[i] = 0u;
        }
      }
      __syncthreads();
    }
  }
  if (writer) {
    hk.flush(m);
    run.store(j.spins + static_cast<size_t>(b.chain) * j.L * j.wd);
    j.m[b.chain] = m;
  }
  asm volatile("" ::: "memory");
  __syncthreads();
  for (int i = threadIdx.x; i < j.np1; i += blockDim.x) {
    const uint32_t v = b.hist[i];
    if (v) atomicAdd(&j.hgen[i], static_cast<unsigned long long>(v));
  }
}

template <class Factory, bool TSMEM, int GL = 1, bool REC = false>
__global__ void __launch_bounds__(128) gen_kernel(const DevJob j, const int cpw, const uint64_t t0,
                                                  const int64_t S, const int64_t flushF, const int do_trace) {
  gen_body<Factory, TSMEM, GL, REC>(j, cpw, t0, S, flushF, do_trace, blockIdx.x);
}

// ------------------------------------------------------------------ joint: replays
// Replay chain i from its round-start configuration with the round's flip
// counters and run a hook over its samples.
template <class Factory, class Hook>
__device__ __forceinline__ void replay_chain(const DevJob& j, const BlockCtx& b, int i, uint64_t t0, int64_t S,
                                             Hook& hk) {
  auto run = Factory::make(b, j.L);
  run.load(j.spins0 + static_cast<size_t>(i) * j.L * j.wd);
  int m = j.m0[i];
  Prefetch pf;
  prefetch_init<decltype(run)::WD>(pf, j.L, t0, static_cast<uint32_t>(i), j.key0, j.key1);
  for (int64_t s = 0; s < S && !hk.done; ++s)
    run.template sweep<true>(m, pf, b.T, j.np1, static_cast<uint32_t>(i), j.key0, j.key1, hk);
}

// Replay one segment of chain i's round (sweeps [seg*C, min(seg*C + C, S)))
// from its checkpoint, with the round's flip counters, running hook hk on
// its samples (sample indices continue from the segment's start).
template <class Factory, class Hook>
__device__ __forceinline__ void replay_segment(const DevJob& j, const BlockCtx& b, int i, int seg, uint64_t t0,
                                               int64_t S, Hook& hk) {
  auto run = Factory::make(b, j.L);
  const size_t lw = static_cast<size_t>(j.L) * j.wd;
  run.load_strided(j.ckpt + static_cast<size_t>(seg) * lw * j.p + i, static_cast<size_t>(j.p));
  int m = j.ckm[static_cast<size_t>(seg) * j.p + i];
  const int64_t s0 = static_cast<int64_t>(seg) * j.ck_C;
  const int64_t s1 = min(S, s0 + j.ck_C);
  Prefetch pf;
  prefetch_init<decltype(run)::WD>(pf, j.L, t0 + static_cast<uint64_t>(s0) * j.N, static_cast<uint32_t>(i), j.key0,
                                   j.key1);
  for (int64_t s = s0; s < s1 && !hk.done; ++s) {
    run.template sweep<true>(m, pf, b.T, j.np1, static_cast<uint32_t>(i), j.key0, j.key1, hk);
    hk.poll();
  }
}

// The same samples as replay_segment, read from the round's record of
// levels (generation stored them, layout rec_index): a hook sees word(nb)
// before every 32 samples and sample(4 m, b) for each, in order; no
// Metropolis replay.  The joint uniforms of a hook depend only on the
// sample's index, so words need not follow lattice rows.  The next 32
// samples' groups are loaded while the current ones are tested, so a lane
// waits on memory once a segment rather than once a word.  (Segments start
// on multiples of 16 samples and hold multiples of 16.)
template <class Hook>
__device__ __forceinline__ void record_segment(const DevJob& j, int i, int seg, int64_t S, Hook& hk) {
  const int64_t M = S * j.N;
  const int64_t k0 = static_cast<int64_t>(seg) * j.seg_len;
  const int64_t k1 = min(M, k0 + j.seg_len);
  // group g (samples 4g .. 4g+3) of chain i is grp[g * kRecTile]
  const uint2* grp = reinterpret_cast<const uint2*>(j.rec + rec_index(i, 0, M));
  uint2 v[8], nv[8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
    v[q] = (k0 + 4 * q < k1) ? __ldg(grp + static_cast<size_t>((k0 >> 2) + q) * kRecTile) : make_uint2(0u, 0u);
  int words = 0;
  for (int64_t kb = k0; kb < k1 && !hk.done; kb += 32) {
    const int nb = static_cast<int>(min(static_cast<int64_t>(32), k1 - kb));
    const int64_t kn = kb + 32;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      nv[q] = (kn + 4 * q < k1) ? __ldg(grp + static_cast<size_t>((kn >> 2) + q) * kRecTile) : make_uint2(0u, 0u);
    hk.word(nb);
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      if (b < nb) {
        const uint32_t pair = (b & 2) ? v[b >> 2].y : v[b >> 2].x;
        const uint32_t lv = (b & 1) ? (pair >> 16) : (pair & 0xFFFFu);
        hk.sample(4 * static_cast<int>(lv), b);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = nv[q];
    if ((++words & 31) == 0) hk.poll();
  }
}

// Joint search (step 4) over segments [seg_lo, seg_hi): work item (chain,
// segment) finds the first sample inside the segment that passes the
// Metropolis test against the chain's input level and lowers the chain's
// kmin to it.  The chains are all of them (list_mode 0), work[] (1, a
// resolution pass) or work2[] (2, those without a hit in segment 0).
// Persistent: each warp takes the next cpw consecutive items (segment-major:
// one segment of consecutive chains) from a global counter, its lanes replay
// them side by side, and only then takes more, so a long replay holds up one
// warp, not a wave of blocks.  A segment is skipped, or its replay stopped
// at the next sweep, as soon as an earlier segment of its chain has found an
// accepted sample (kmin at or before the segment's start): so the items in
// flight are always early segments of the chains still without a hit, and
// as chains find theirs the rest of the GPU moves on to the others' later
// segments.  A block that starts after the queue ran dry leaves before any
// set-up.
template <class Factory, bool TSMEM>
__global__ void __launch_bounds__(128) search_kernel(const DevJob j, const int cpw, const uint64_t t0,
                                                     const int64_t S, const uint32_t r, const int list_mode,
                                                     const int seg_lo, const int seg_hi_in, const int exact_first) {
  if (exact_first && rough_last_joint(j.stats[kStatRejected], j.p)) return;   // (the first search only)
  const int nchains = list_mode == 0 ? j.p : static_cast<int>(j.stats[list_mode == 1 ? kStatPending : kStatNoHit]);
  const int seg_hi = min(seg_hi_in, j.ck_K);
  const long long items = static_cast<long long>(nchains) * max(0, seg_hi - seg_lo);
  if (items == 0) return;
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(&j.stats[kStatQueueSearch]);
  __shared__ int s_dry;
  if (threadIdx.x == 0) s_dry = static_cast<long long>(__ldcg(reinterpret_cast<const long long*>(queue))) >= items;
  __syncthreads();
  if (s_dry) return;
  const int32_t* list = list_mode == 1 ? j.work : j.work2;
  const SmemPlan sp = smem_plan(j.L, Factory::kPlacement, cpw, blockDim.x >> 5, TSMEM, false);
  BlockCtx b = block_setup<TSMEM>(j, sp, cpw, 0, false);
  __syncthreads();
  long long searched = 0;
  for (;;) {
    long long base = 0;
    if (b.lane == 0) base = static_cast<long long>(atomicAdd(queue, static_cast<unsigned long long>(cpw)));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= items) break;
    const long long item = base + b.lane;
    if (b.lane < cpw && item < items) {
      const int seg = seg_lo + static_cast<int>(item / nchains);
      const int q = static_cast<int>(item % nchains);
      const int i = list_mode ? list[q] : q;
      const unsigned long long seg_start = static_cast<unsigned long long>(seg) * j.seg_len;
      if (__ldcg(&j.kmin[i]) > seg_start) {   // no accepted sample before this segment yet
        const int x = j.xused[i];
        int64_t found;
        if (x < 0) {
          found = (seg == 0) ? 1 : 0;  // job's first joint: chain 0 is kept whole
        } else {
          SearchHook hk;
          hk.tj = j.tj + static_cast<size_t>(i) * j.np1;
          hk.k = static_cast<int64_t>(seg_start);
          hk.M = min(S * j.N, static_cast<int64_t>(seg_start) + j.seg_len);
          hk.found = 0;
          hk.chain = static_cast<uint32_t>(i);
          hk.r = r;
          hk.k0 = j.key0;
          hk.k1 = j.key1;
          hk.done = false;
          hk.kmin = &j.kmin[i];
          hk.stop = seg_start;
          const int64_t k_begin = hk.k;
          if constexpr (IsRec<Factory>::value) record_segment(j, i, seg, S, hk);
          else replay_segment<Factory>(j, b, i, seg, t0, S, hk);
          found = hk.found;
          searched += hk.k - k_begin;
        }
        if (found > 0) atomicMin(&j.kmin[i], static_cast<unsigned long long>(found));
      }
    }
    __syncwarp();
  }
  if (searched)
    atomicAdd(reinterpret_cast<unsigned long long*>(&j.stats[kStatSearched]), static_cast<unsigned long long>(searched));
}

// Summary replay for the exact scan: work items (chain, segment) for the
// chains from the first pending one on, all segments; persistent warps take
// cpw consecutive items at a time, as in search_kernel.  Nothing happens
// when no chain is pending.
template <class Factory, bool TSMEM>
__global__ void __launch_bounds__(128) summary_kernel(const DevJob j, const int cpw, const uint64_t t0,
                                                      const int64_t S, const uint32_t r) {
  if (j.stats[kStatPending] == 0) return;
  const int f = static_cast<int>(j.stats[kStatFirstPending]);
  const int nchains = j.p - f;
  const long long items = static_cast<long long>(nchains) * j.ck_K;
  const SmemPlan sp = smem_plan(j.L, Factory::kPlacement, cpw, blockDim.x >> 5, TSMEM, false);
  BlockCtx b = block_setup<TSMEM>(j, sp, cpw, 0, false);
  // a recorded round: every lane keeps a window of levels in shared memory
  constexpr int W = IsRec<Factory>::value ? 64 : 0;
  __shared__ uint32_t s_win[W > 0 ? W * kWinStride : 1];
  if constexpr (W > 0)
    for (int q = threadIdx.x; q < W * kWinStride; q += blockDim.x) s_win[q] = 0xFFFFFFFFu;
  __syncthreads();
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(&j.stats[kStatQueueSearch]);
  long long searched = 0;
  for (;;) {
    long long base = 0;
    if (b.lane == 0) base = static_cast<long long>(atomicAdd(queue, static_cast<unsigned long long>(cpw)));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= items) break;
    const long long item = base + b.lane;
    if (b.lane < cpw && item < items) {
      const int seg = static_cast<int>(item / nchains);
      const int i = j.perm[f + static_cast<int>(item % nchains)];
      SummaryHook<W> hk;
      if constexpr (W > 0) hk.win = s_win + threadIdx.x;
      hk.umin = j.tj + static_cast<size_t>(i) * j.np1;
      hk.k = static_cast<int64_t>(seg) * j.seg_len;
      hk.chain = static_cast<uint32_t>(i);
      hk.r = r;
      hk.k0 = j.key0;
      hk.k1 = j.key1;
      hk.cur = -1;
      hk.lo = 0x7FFFFFFF;
      hk.hi = -1;
      hk.run_min = 0xFFFFFFFFu;
      hk.flag = false;
      hk.done = false;
      const int64_t k_begin = hk.k;
      if constexpr (IsRec<Factory>::value) record_segment(j, i, seg, S, hk);
      else replay_segment<Factory>(j, b, i, seg, t0, S, hk);
      hk.flush();
      hk.drain();
      atomicMin(&j.summ[i], hk.lo);
      atomicMax(&j.summ[j.p + i], hk.hi);
      if (hk.flag) atomicOr(&j.summ[2 * j.p + i], 1);
      searched += hk.k - k_begin;
    }
    __syncwarp();
  }
  if (searched)
    atomicAdd(reinterpret_cast<unsigned long long*>(&j.stats[kStatSearched]), static_cast<unsigned long long>(searched));
}

// (k counts the samples of the words seen so far, as in SearchHook; done
// once a word reaches the cut)
struct PrefixHook {
  uint32_t* hist;
  int64_t k, cut;  // samples with index < cut are counted
  bool done;
  int64_t kw = 0;
  __device__ __forceinline__ void poll() {}
  __device__ __forceinline__ void word(int nb) {
    kw = k;
    k += nb;
    done = done || k >= cut;
  }
  __device__ __forceinline__ void sample(int m4, int b) {
    if (kw + b + 1 < cut) red_shared_add(hist, m4, 1u);
  }
};

// Discarded prefixes (samples before k_i; the whole chain if nothing is
// kept) counted into dpre.  Replays take the work list plist of (chain,
// segment) items; a recorded round takes every (segment, chain) pair,
// segment-major, and skips those that start at or after the chain's cut.
template <class Factory, bool TSMEM>
__global__ void __launch_bounds__(128) prefix_kernel(const DevJob j, const int cpw, const uint64_t t0,
                                                     const int64_t S) {
  const long long items =
      IsRec<Factory>::value ? static_cast<long long>(j.p) * j.ck_K : static_cast<long long>(j.stats[kStatQueuePrefix]);
  if (items == 0) return;
  const SmemPlan sp = smem_plan(j.L, Factory::kPlacement, cpw, blockDim.x >> 5, TSMEM, true);
  BlockCtx b = block_setup<TSMEM>(j, sp, cpw, 0, true);
  __shared__ long long s_base;
  __shared__ unsigned long long s_samples;
  if (threadIdx.x == 0) s_samples = 0ull;
  __syncthreads();
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(&j.stats[kStatQueueSearch]);
  const int slots = (blockDim.x >> 5) * cpw;
  const int64_t M = S * j.N;
  for (;;) {
    if (threadIdx.x == 0) s_base = static_cast<long long>(atomicAdd(queue, static_cast<unsigned long long>(slots)));
    __syncthreads();
    const long long base = s_base;
    if (base >= items) break;
    const long long item = base + b.slot;
    if (b.lane < cpw && item < items) {
      const int2 w = IsRec<Factory>::value ? make_int2(static_cast<int>(item % j.p), static_cast<int>(item / j.p))
                                           : j.plist[item];
      const int i = w.x, seg = w.y;
      const int64_t k = j.k[i];
      const int64_t cut = (k > 0) ? k : M + 1;
      const int64_t seg_first = static_cast<int64_t>(seg) * j.seg_len + 1;
      if (seg_first < cut) {
        PrefixHook hk{b.hist, seg_first - 1, cut, false};
        if constexpr (IsRec<Factory>::value) record_segment(j, i, seg, S, hk);
        else replay_segment<Factory>(j, b, i, seg, t0, S, hk);
        atomicAdd(&s_samples, static_cast<unsigned long long>(hk.k - (seg_first - 1)));
      }
    }
    asm volatile("" ::: "memory");
    __syncthreads();
    // a batch adds at most 128 * 2^24 = 2^31 samples: flush at 2^30
    if (s_samples >= (1ull << 30)) {
      for (int m = threadIdx.x; m < j.np1; m += blockDim.x) {
        const uint32_t v = b.hist[m];
        if (v) {
          atomicAdd(&j.dpre[m], static_cast<unsigned long long>(v));
          b.hist[m] = 0u;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_samples = 0ull;
    }
    __syncthreads();
  }
  asm volatile("" ::: "memory");
  __syncthreads();
  for (int m = threadIdx.x; m < j.np1; m += blockDim.x) {
    const uint32_t v = b.hist[m];
    if (v) atomicAdd(&j.dpre[m], static_cast<unsigned long long>(v));
  }
}

// Block-wide scan over positions of the joint: out[q] = the last position
// before q whose chain (perm[]) has k > 0 (or -1).  Each thread takes a
// contiguous range of positions; s_tmp holds blockDim.x ints.
__device__ __forceinline__ void block_last_accepted(const DevJob& j, int* s_tmp, int32_t* out) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int per = (j.p + nt - 1) / nt;
  const int lo = min(j.p, t * per), hi = min(j.p, lo + per);
  int last = -1;
  for (int i = lo; i < hi; ++i)
    if (j.k[j.perm[i]] > 0) last = i;
  s_tmp[t] = last;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    const int v = (t >= off) ? s_tmp[t - off] : -1;
    __syncthreads();
    s_tmp[t] = max(s_tmp[t], v);
    __syncthreads();
  }
  int run = (t > 0) ? s_tmp[t - 1] : -1;  // exclusive prefix
  for (int i = lo; i < hi; ++i) {
    out[i] = run;
    if (j.k[j.perm[i]] > 0) run = i;
  }
  __syncthreads();
}

// Resolution of the speculation, one block: the actual input of chain i is
// the last level of the nearest chain before it that kept samples (or the
// carry).  Chains whose k was computed for another input are searched again
// (their new thresholds first), in parallel, until no input changes; each
// pass settles at least the first such chain.  Also fixes the carry.
template <class Factory, bool TSMEM>
__global__ void __launch_bounds__(128) resolve_kernel(const DevJob j, const int cpw, const uint64_t t0,
                                                      const int64_t S, const uint32_t r) {
  const SmemPlan sp = smem_plan(j.L, Factory::kPlacement, cpw, blockDim.x >> 5, TSMEM, false);
  BlockCtx b = block_setup<TSMEM>(j, sp, cpw, 0, false);
  __shared__ int s_tmp[128];
  __shared__ int s_count;
  __syncthreads();
  const int carry_in = j.stats[kStatCarryValid] ? static_cast<int>(j.stats[kStatCarry]) : -1;
  long long searched = 0;
  int passes = 0, mism_total = 0;
  for (;;) {
    block_last_accepted(j, s_tmp, j.work);
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    // list of chains whose input changed (j.work reused: first the scan
    // result, then the list, written after the scan result was consumed)
    for (int q = threadIdx.x; q < j.p; q += blockDim.x) {   // positions in the joint
      const int last = j.work[q];
      const int x = (last >= 0) ? j.m[j.perm[last]] : carry_in;
      const int i = j.perm[q];
      if (x != j.xused[i]) {
        j.xused[i] = x;
        j.k[i] = -1;  // marked: to be searched again
        atomicAdd(&s_count, 1);
      } else if (j.k[i] < 0) {
        atomicAdd(&s_count, 1);  // marked earlier, not searched yet
      }
    }
    __syncthreads();
    const int count = s_count;
    if (count == 0 || passes > j.p) break;
    ++passes;
    mism_total += count;
    // compact the marked chains into work[]
    if (threadIdx.x == 0) {
      int n = 0;
      for (int i = 0; i < j.p; ++i)
        if (j.k[i] == -1) j.work[n++] = i;
    }
    __syncthreads();
    // thresholds of the new inputs
    for (long long idx = threadIdx.x; idx < static_cast<long long>(count) * j.np1; idx += blockDim.x) {
      const int i = j.work[idx / j.np1], mm = static_cast<int>(idx % j.np1);
      const int x = j.xused[i];
      j.tj[static_cast<size_t>(i) * j.np1 + mm] = (x < 0) ? 0xFFFFFFFFu : threshold_det(__dsub_rn(j.W[mm], j.W[x]));
    }
    __syncthreads();
    if (b.active) {
      for (int q = b.slot; q < count; q += b.nslot) {
        const int i = j.work[q];
        if (j.xused[i] < 0) {
          j.k[i] = 1;
          continue;
        }
        SearchHook hk;
        hk.tj = j.tj + static_cast<size_t>(i) * j.np1;
        hk.k = 0;
        hk.M = S * j.N;
        hk.found = 0;
        hk.chain = static_cast<uint32_t>(i);
        hk.r = r;
        hk.k0 = j.key0;
        hk.k1 = j.key1;
        hk.done = false;
        if constexpr (IsRec<Factory>::value) {
          for (int sg = 0; sg < j.ck_K && !hk.done; ++sg) record_segment(j, i, sg, S, hk);
        } else {
          replay_chain<Factory>(j, b, i, t0, S, hk);
        }
        j.k[i] = hk.found;
        searched += hk.k;
      }
    }
    __syncthreads();
  }
  // carry for the next round: the last level of the last chain (in joint
  // order) that kept samples
  if (threadIdx.x == 0) {
    int last = -1;
    for (int q = j.p - 1; q >= 0; --q)
      if (j.k[j.perm[q]] > 0) {
        last = j.perm[q];
        break;
      }
    if (last >= 0) {
      j.stats[kStatCarry] = j.m[last];
      j.stats[kStatCarryValid] = 1;
    }
    j.stats[kStatMismatch] += mism_total;
    j.stats[kStatPasses] += passes;
  }
  if (searched) atomicAdd(reinterpret_cast<unsigned long long*>(&j.stats[kStatSearched]),
                          static_cast<unsigned long long>(searched));
}

// ------------------------------------------------------------------ host-side launchers
template <int L>
struct RegF : RunnerFactoryReg<L> {
  static constexpr int kPlacement = kPlaceReg;
};
template <int WD, int SL = 0>
struct SmemF : RunnerFactorySmem<WD, SL> {
  static constexpr int kPlacement = kPlaceSmem;
};
template <int WD, int SL>
struct GlobF : RunnerFactoryGlob<WD, SL> {
  static constexpr int kPlacement = kPlaceGlobal;
};

constexpr size_t kMaxSmem = 227 * 1024;

// Blocks of a kernel that fit on the device at once (occupancy API).
template <class K>
inline long long resident_blocks(K kernel, int threads, size_t smem_bytes) {
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem_bytes) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return static_cast<long long>(sms) * per_sm;
}

inline bool table_fits(int L, const LaunchShape& s, bool hist) {
  const SmemPlan sp = smem_plan(L, s.placement, s.cpw, s.wpb, true, hist);
  return 4ull * (sp.table_words + sp.hist_words + sp.lat_words) <= kMaxSmem;
}

inline size_t plan_bytes(int L, const LaunchShape& s, bool tsmem, bool hist) {
  const SmemPlan sp = smem_plan(L, s.placement, s.cpw, s.wpb, tsmem, hist);
  return 4ull * (sp.table_words + sp.hist_words + sp.lat_words);
}

template <class F, bool TS>
inline cudaError_t launch_gen_t(const DevJob& j, const LaunchShape& s, uint64_t t0, int64_t S, bool trace,
                                cudaStream_t st) {
  const size_t bytes = plan_bytes(j.L, s, TS, true);
  // lattice in shared memory with at most 8 chains a warp: lane groups of 4
  // (groups of 8 for at most 4 chains measured slower at L = 48, 64 and 128)
  const bool rec = j.rec != nullptr;
  auto kern = rec ? gen_kernel<F, TS, 1, true> : gen_kernel<F, TS, 1, false>;
  if constexpr (F::kPlacement != kPlaceReg)
    if (s.cpw <= 8) kern = rec ? gen_kernel<F, TS, 4, true> : gen_kernel<F, TS, 4, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e != cudaSuccess) return e;
  const int per_block = s.cpw * s.wpb;
  const unsigned grid = blocks_for(j.p, per_block);
  // dwell counts are u32 in shared memory: flush before they can overflow
  // (up to 32 samples a chain wait one word to be counted)
  const long long per_sweep = static_cast<long long>(per_block) * j.N;
  const int64_t flushF = std::max<int64_t>(1, (0xFFFFFFFFll - 32ll * per_block) / per_sweep);
  kern<<<grid, 32 * s.wpb, bytes, st>>>(j, s.cpw, t0, S, S > flushF ? flushF : 0, trace ? 1 : 0);
  launches_add(1);
  return cudaGetLastError();
}

template <class F, bool TS>
inline cudaError_t launch_join_t(const DevJob& j, const LaunchShape& s, uint64_t t0, int64_t S, uint32_t r,
                                 cudaStream_t st) {
  const size_t bytes = plan_bytes(j.L, s, TS, false);
  // the prefix pass keeps a histogram beside the lattices: fewer chains a warp if need be
  LaunchShape sp = s;
  while (sp.cpw > 1 && plan_bytes(j.L, sp, TS, true) > kMaxSmem) --sp.cpw;
  const size_t pbytes = plan_bytes(j.L, sp, TS, true);
  const int per_block = s.cpw * s.wpb;
  const long long items = static_cast<long long>(j.p) * j.ck_K;
  cudaError_t e = join_prelude(j, st);
  if (e != cudaSuccess) return e;
  auto kq = search_kernel<F, TS>;
  if ((e = cudaFuncSetAttribute(kq, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes))) !=
      cudaSuccess)
    return e;
  // persistent grids: the blocks that are resident at once, no more than needed
  const unsigned grid_all = static_cast<unsigned>(
      std::min<long long>(blocks_for(items, per_block), resident_blocks(kq, 32 * s.wpb, bytes)));
  // a search over the chains of list_mode: their first segments, then the
  // later segments of those without a hit there
  const bool exact_scan = static_cast<long long>(j.p) * S * j.N <= j.scan_max_samples;
  // a recorded round may skip the speculative first search (rough_last_joint)
  const int exact_first = (IsRec<F>::value && exact_scan) ? 1 : 0;
  auto search = [&](int list_mode, int first) -> cudaError_t {
    cudaError_t e2 = join_reset_queue(j, st);
    if (e2 != cudaSuccess) return e2;
    kq<<<grid_all, 32 * s.wpb, bytes, st>>>(j, s.cpw, t0, S, r, list_mode, 0, 1, first);
    launches_add(1);
    if (j.ck_K > 1) {
      if ((e2 = join_nohit(j, list_mode, st)) != cudaSuccess) return e2;
      if ((e2 = join_reset_queue(j, st)) != cudaSuccess) return e2;
      kq<<<grid_all, 32 * s.wpb, bytes, st>>>(j, s.cpw, t0, S, r, 2, 1, j.ck_K, first);
      launches_add(1);
    }
    return cudaGetLastError();
  };
  // speculated inputs: every chain
  if ((e = search(0, exact_first)) != cudaSuccess) return e;
  if ((e = join_select(j, false, st, exact_first != 0)) != cudaSuccess) return e;
  // grid-wide speculative resolution passes
  auto pass = [&](int n, bool defer) -> cudaError_t {
    for (int q = 0; q < n; ++q) {
      cudaError_t e2 = join_mark(j, st, true, defer);
      if (e2 == cudaSuccess) e2 = search(1, 0);
      if (e2 == cudaSuccess) e2 = join_select(j, true, st);
      if (e2 != cudaSuccess) return e2;
    }
    return cudaSuccess;
  };
  if (exact_scan) {
    // a few speculative passes; if chains are still pending, the summary
    // replay and the exact scan settle every input, one search finds the
    // new k's, and the ordinary passes catch what the scan left
    if ((e = pass(j.passes_scan, true)) != cudaSuccess) return e;
    if ((e = join_mark(j, st, false)) != cudaSuccess) return e;
    if ((e = join_summary_init(j, st)) != cudaSuccess) return e;
    if ((e = join_reset_queue(j, st)) != cudaSuccess) return e;
    auto ks = summary_kernel<F, TS>;
    if ((e = cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes))) !=
        cudaSuccess)
      return e;
    const unsigned grid_sum = static_cast<unsigned>(
        std::min<long long>(blocks_for(items, per_block), resident_blocks(ks, 32 * s.wpb, bytes)));
    ks<<<grid_sum, 32 * s.wpb, bytes, st>>>(j, s.cpw, t0, S, r);
    launches_add(1);
    if ((e = join_scan(j, st)) != cudaSuccess) return e;
    if ((e = join_tj_list(j, st)) != cudaSuccess) return e;
    if ((e = search(1, 0)) != cudaSuccess) return e;
    if ((e = join_select(j, true, st)) != cudaSuccess) return e;
    if ((e = pass(j.passes_scan, false)) != cudaSuccess) return e;
  } else {
    if ((e = pass(j.passes_plain, false)) != cudaSuccess) return e;
  }
  auto kr = resolve_kernel<F, TS>;
  if ((e = cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes))) !=
      cudaSuccess)
    return e;
  kr<<<1, 32 * s.wpb, bytes, st>>>(j, s.cpw, t0, S, r);
  auto kp = prefix_kernel<F, TS>;
  if ((e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(pbytes))) !=
      cudaSuccess)
    return e;
  if constexpr (!IsRec<F>::value)
    if ((e = join_prefix_list(j, st)) != cudaSuccess) return e;
  if ((e = join_reset_queue(j, st)) != cudaSuccess) return e;
  const unsigned grid_pre = static_cast<unsigned>(
      std::min<long long>(blocks_for(items, sp.cpw * sp.wpb), resident_blocks(kp, 32 * sp.wpb, pbytes)));
  kp<<<grid_pre, 32 * sp.wpb, pbytes, st>>>(j, sp.cpw, t0, S);
  launches_add(2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return join_finalize(j, S, st);
}

// Whether a factory's lattice size is fixed at compile time with a
// threshold table that can never fit in shared memory (then only the
// global-table kernels are instantiated).
template <class F>
struct TableNeverFits : std::false_type {};
template <int WD, int SL>
struct TableNeverFits<SmemF<WD, SL>> : std::integral_constant<bool, (SL > 0 && 5ull * 4ull * (SL * SL + 1) > kMaxSmem)> {};
template <int WD, int SL>
struct TableNeverFits<GlobF<WD, SL>> : TableNeverFits<SmemF<WD, SL>> {};

template <class F>
struct IsGlob : std::false_type {};
template <int WD, int SL>
struct IsGlob<GlobF<WD, SL>> : std::true_type {};

template <class F>
inline cudaError_t dispatch_ts(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace,
                               uint32_t r, cudaStream_t st) {
  if constexpr (IsGlob<F>::value) {   // generation only
    if (!gen) return cudaErrorInvalidValue;
    if constexpr (TableNeverFits<F>::value) return launch_gen_t<F, false>(j, s, t0, S, trace, st);
    else return table_fits(j.L, s, true) ? launch_gen_t<F, true>(j, s, t0, S, trace, st)
                                         : launch_gen_t<F, false>(j, s, t0, S, trace, st);
  } else if constexpr (TableNeverFits<F>::value) {
    if (gen) return launch_gen_t<F, false>(j, s, t0, S, trace, st);
    return launch_join_t<F, false>(j, s, t0, S, r, st);
  } else {
    // the joint's prefix pass needs the histogram beside the table, like generation
    const bool ts = table_fits(j.L, s, true);
    if (gen) return ts ? launch_gen_t<F, true>(j, s, t0, S, trace, st) : launch_gen_t<F, false>(j, s, t0, S, trace, st);
    return ts ? launch_join_t<F, true>(j, s, t0, S, r, st) : launch_join_t<F, false>(j, s, t0, S, r, st);
  }
}

}  // namespace mcgpu
