// One chain's single-spin-flip Metropolis sweep on a bit-packed periodic
// L x L Ising lattice (Sec. 2 step 2 with the Hamiltonian of Sec. 4.1),
// shared by the generation kernels and by the joint's replay kernels so that
// a replay reproduces the generated chain exactly.
//
// Lattice layout: row y is WD = ceil(L/32) uint32 words; bit x%32 of word
// x/32 is site (x, y), 1 meaning spin +1.  Sites are visited in typewriter
// order (x fastest).  Attempt t of chain c (t counted from the start of the
// job) draws word t&3 of Philox4x32-10 at counter (t>>2 as 64 bits, c, 0).
// The sample after an attempt is the configuration that results from it.
//
// For site x the move changes the energy by dE = 4a - 8, where a in 0..4 is
// the number of neighbours aligned with the spin; the level index
// m = (E + 2N)/4 moves to m + a - 2.  The acceptance threshold is read from
// the planar table T[a * (N+1) + m].  Per row the neighbour agreements are
// computed bit-parallel: up/down/right (the right neighbour is not yet
// visited when a site is) are summed by a bit-sliced full adder; the left
// neighbour was visited one attempt earlier, so its agreement is the
// original one XOR that attempt's flip.  The last site of a row sees site 0
// of the row, already visited, in the same way.
#pragma once
#include "mc_device_math.cuh"

namespace mcgpu {

template <int WD>
struct RowInputs {
  uint32_t up[WD], dn[WD];
};

// Sweep one row in place.  blk is the Philox block index of the next
// attempt (the row starts on a block boundary since L % 4 == 0).
template <int WD, class Hook>
__device__ __forceinline__ void sweep_row(uint32_t (&cur)[WD], const uint32_t (&up)[WD],
                                          const uint32_t (&dn)[WD], const int L, int& m,
                                          const uint32_t* __restrict__ T, const int np1,
                                          uint64_t& blk, const uint32_t chain, const uint32_t k0,
                                          const uint32_t k1, Hook& hook) {
  const int lw = L - 32 * (WD - 1);  // sites in the last word of the row
  uint32_t s0[WD], s1[WD], el[WD], eu[WD], ed[WD], er[WD];
#pragma unroll
  for (int w = 0; w < WD; ++w) {
    const uint32_t c = cur[w];
    const uint32_t right = (w + 1 < WD) ? ((c >> 1) | (cur[w + 1] << 31))
                                        : ((c >> 1) | ((cur[0] & 1u) << (lw - 1)));
    const uint32_t left = (w > 0) ? ((c << 1) | (cur[w - 1] >> 31))
                                  : ((c << 1) | ((cur[WD - 1] >> (lw - 1)) & 1u));
    eu[w] = ~(c ^ up[w]);
    ed[w] = ~(c ^ dn[w]);
    er[w] = ~(c ^ right);
    el[w] = ~(c ^ left);
    s0[w] = eu[w] ^ ed[w] ^ er[w];                         // sum bit
    s1[w] = (eu[w] & ed[w]) | (er[w] & (eu[w] ^ ed[w]));  // carry bit
  }
  uint32_t f = 0u, f0 = 0u;  // flip of the previous site / of site 0
  uint4 rnd = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
  for (int w = 0; w < WD; ++w) {
    const int nb = (w + 1 < WD) ? 32 : lw;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      if (b < nb) {
        if ((b & 3) == 0) {
          rnd = philox4x32_10(make_uint4(static_cast<uint32_t>(blk), static_cast<uint32_t>(blk >> 32),
                                         chain, kTagFlip),
                              k0, k1);
          ++blk;
        }
        const uint32_t u = (b & 3) == 0 ? rnd.x : ((b & 3) == 1 ? rnd.y : ((b & 3) == 2 ? rnd.z : rnd.w));
        int a;
        if (w == WD - 1 && b == nb - 1) {
          a = static_cast<int>(((eu[w] >> b) & 1u) + ((ed[w] >> b) & 1u) + (((er[w] >> b) & 1u) ^ f0) +
                               (((el[w] >> b) & 1u) ^ f));
        } else {
          a = static_cast<int>(((s0[w] >> b) & 1u) + 2u * ((s1[w] >> b) & 1u) + (((el[w] >> b) & 1u) ^ f));
        }
        const uint32_t thr = T[a * np1 + m];
        const uint32_t acc = (u <= thr) ? 1u : 0u;
        const int mold = m;
        if (acc) {
          cur[w] ^= (1u << b);
          m += a - 2;
        }
        f = acc;
        if (w == 0 && b == 0) f0 = acc;
        hook.sample(mold, m);
      }
    }
  }
}

// ------------------------------------------------------------------ hooks
// Generation: dwell-time histogram in a warp-private u32 shared-memory
// array (one atomic per change of level, adding the run length).
struct GenHook {
  uint32_t* hist;
  uint32_t run;
  __device__ __forceinline__ void sample(int mold, int m) {
    if (m != mold) {
      atomicAdd(&hist[mold], run);
      run = 1u;
    } else {
      ++run;
    }
  }
  __device__ __forceinline__ void flush(int m) {
    if (run) atomicAdd(&hist[m], run);
    run = 0u;
  }
};

// Joint search (Sec. 2 step 4): for samples k = 1..M of the chain (the
// configuration after attempt k of the round) draw the joint uniform
// Philox((k-1)>>2, r, chain, 1) word (k-1)&3 and test it against the
// threshold of the move from the input level x to the sample's level.  The
// first k that passes is recorded; samples before it are the discarded
// prefix.  If ACCUM, the prefix's levels are added (dwell-time, 64-bit
// atomics) to a global histogram.
template <bool ACCUM>
struct SearchHook {
  const uint32_t* __restrict__ tj;  // thresholds for moves x -> m, indexed by m
  unsigned long long* D;
  int64_t k, M, found;
  uint32_t chain, r, k0, k1;
  uint4 jr;
  int cur_level;
  uint32_t run;
  bool done;
  __device__ __forceinline__ void sample(int /*mold*/, int m) {
    if (done) return;
    ++k;
    const uint64_t q = static_cast<uint64_t>(k - 1);
    if ((q & 3u) == 0u)
      jr = philox4x32_10(make_uint4(static_cast<uint32_t>(q >> 2), r, chain, kTagJoint), k0, k1);
    const uint32_t u = uint4_word(jr, static_cast<uint32_t>(q & 3u));
    if (u <= tj[m]) {
      found = k;
      done = true;
      if (ACCUM) flush();
      return;
    }
    if (ACCUM) {
      if (m != cur_level) {
        flush();
        cur_level = m;
      }
      ++run;
    }
    if (k == M) {
      found = 0;
      done = true;
      if (ACCUM) flush();
    }
  }
  __device__ __forceinline__ void flush() {
    if (run && cur_level >= 0) atomicAdd(&D[cur_level], static_cast<unsigned long long>(run));
    run = 0u;
  }
};

// Prefix correction: samples j in [lo, hi) (1-based) are added with the given
// sign (+1 or -1, two's complement in the unsigned accumulator).
struct CorrectHook {
  unsigned long long* D;
  int64_t k, lo, hi;
  unsigned long long sign;
  int cur_level;
  uint32_t run;
  bool done;
  __device__ __forceinline__ void sample(int /*mold*/, int m) {
    if (done) return;
    ++k;
    if (k >= hi) {
      flush();
      done = true;
      return;
    }
    if (k >= lo) {
      if (m != cur_level) {
        flush();
        cur_level = m;
      }
      ++run;
    }
  }
  __device__ __forceinline__ void flush() {
    if (run && cur_level >= 0)
      atomicAdd(&D[cur_level], sign * static_cast<unsigned long long>(run));
    run = 0u;
  }
};

}  // namespace mcgpu
