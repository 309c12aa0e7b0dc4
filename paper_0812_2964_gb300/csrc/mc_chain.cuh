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

// Uniforms of the next 32-site word, computed one word ahead so that the
// eight independent Philox blocks fill the latency gaps of the current
// word's serial Metropolis chain.  blk is the Philox block index of the
// first attempt after the prefetched word.
struct Prefetch {
  uint32_t U[32];
  uint64_t blk;
};

//
// GL > 1: a group of GL consecutive lanes (aligned) shares one chain and runs
// its sweep in lockstep on identical data; lane gi of the group computes
// Philox blocks gi, gi + GL, ... of the word and the group exchanges them by
// shuffles, so a warp with few chains spends 8 / GL Philox evaluations per
// word instead of 8 (the sweep's other work is the same for every lane).
template <int GL = 1>
__device__ __forceinline__ void philox_fill(uint32_t (&U)[32], const int n, const uint64_t blk, const uint32_t chain,
                                            const uint32_t k0, const uint32_t k1) {
  if constexpr (GL == 1) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (4 * q < n) {
        const uint64_t b = blk + static_cast<uint64_t>(q);
        const uint4 r =
            philox4x32_10(make_uint4(static_cast<uint32_t>(b), static_cast<uint32_t>(b >> 32), chain, kTagFlip), k0, k1);
        U[4 * q + 0] = r.x;
        U[4 * q + 1] = r.y;
        U[4 * q + 2] = r.z;
        U[4 * q + 3] = r.w;
      }
    }
  } else {
#ifdef __CUDACC__
    static_assert(GL == 2 || GL == 4 || GL == 8, "lane groups of 2, 4 or 8");
    constexpr int R = 8 / GL;
    const int lane = static_cast<int>(threadIdx.x & 31u);
    const int gi = lane & (GL - 1);
    const int gbase = lane - gi;
    const unsigned mask = ((1u << GL) - 1u) << gbase;
    uint4 r[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int q = gi + t * GL;
      r[t] = make_uint4(0u, 0u, 0u, 0u);
      if (4 * q < n) {
        const uint64_t b = blk + static_cast<uint64_t>(q);
        r[t] = philox4x32_10(make_uint4(static_cast<uint32_t>(b), static_cast<uint32_t>(b >> 32), chain, kTagFlip), k0,
                             k1);
      }
    }
#pragma unroll
    for (int t = 0; t < R; ++t)
#pragma unroll
      for (int sl = 0; sl < GL; ++sl) {
        const int q = sl + t * GL;
        U[4 * q + 0] = __shfl_sync(mask, r[t].x, gbase + sl);
        U[4 * q + 1] = __shfl_sync(mask, r[t].y, gbase + sl);
        U[4 * q + 2] = __shfl_sync(mask, r[t].z, gbase + sl);
        U[4 * q + 3] = __shfl_sync(mask, r[t].w, gbase + sl);
      }
#endif
  }
}

// Start a chain's attempt stream at attempt t0 (a multiple of 4).
template <int WD, int GL = 1>
__device__ __forceinline__ void prefetch_init(Prefetch& pf, const int L, const uint64_t t0, const uint32_t chain,
                                              const uint32_t k0, const uint32_t k1) {
  const int lw = L - 32 * (WD - 1);
  const int n0 = (WD == 1) ? lw : 32;
  philox_fill<GL>(pf.U, n0, t0 >> 2, chain, k0, k1);
  pf.blk = (t0 >> 2) + static_cast<uint64_t>(n0 / 4);
}

// Shared-memory reduction at a byte offset (no return value, no branch).
// (A host compiler -- used to check this logic on the CPU -- gets a plain add.)
__device__ __forceinline__ void red_shared_add(uint32_t* base, const int byte_off, const uint32_t v) {
#ifdef __CUDACC__
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(base)) + static_cast<uint32_t>(byte_off);
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v));
#else
  base[byte_off >> 2] += v;
#endif
}

// 8-byte global store of the round record, opaque to the compiler's memory
// ordering (no memory clobber): nothing in the sweep reads the record, and
// a plain store held back the threshold loads scheduled around it.
// (A host compiler gets a plain store.)
__device__ __forceinline__ void st_record(uint16_t* p, uint32_t a, uint32_t b) {
#ifdef __CUDACC__
  asm volatile("st.global.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(a), "r"(b));
#else
  p[0] = static_cast<uint16_t>(a);
  p[1] = static_cast<uint16_t>(a >> 16);
  p[2] = static_cast<uint16_t>(b);
  p[3] = static_cast<uint16_t>(b >> 16);
#endif
}

// Byte permute (PTX prmt, generic mode): selector nibble bit 3 set means
// "replicate the sign of the selected byte".
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t sel) {
#ifdef __CUDACC__
  uint32_t d;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(a), "r"(sel));
  return d;
#else
  uint32_t d = 0;
  for (int i = 0; i < 4; ++i) {
    const uint32_t s = (sel >> (4 * i)) & 0xFu;
    const uint32_t src = (s & 7u) < 4 ? ((a >> (8 * (s & 7u))) & 0xFFu) : 0u;
    const uint32_t v = (s & 8u) ? ((src & 0x80u) ? 0xFFu : 0u) : src;
    d |= v << (8 * i);
  }
  return d;
#endif
}

// Selector of byte k, sign-extended to 32 bits.
__device__ __forceinline__ constexpr uint32_t sign_sel(uint32_t k) {
  return k | ((k | 8u) << 4) | ((k | 8u) << 8) | ((k | 8u) << 12);
}

// Spread the 4 bits of n (0..15) into the low bits of 4 bytes.
__device__ __forceinline__ uint32_t spread4(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }

// Sweep one row in place.  The row starts on a Philox block boundary
// (L % 4 == 0); pf holds the uniforms of the row's first word.
//
// Per site b the move is to level m + a - 2 with a = as + (el ^ f): as counts
// the up/down/right neighbours aligned with the spin, el is 1 if the left
// neighbour was aligned before its own attempt, f is that attempt's flip.
// Per group of 4 sites the bytes A0 (4 a for f = 0) and D (4 a(f=1) - 4 a(f=0)
// = +-4, signed) are packed once; a site then needs one byte permute each.
// Levels are kept as byte offsets m4 = 4 m, so that table and histogram
// addresses are plain register + constant.  The thresholds of site b+1 under
// both flips of site b are loaded while site b is resolved, from the level
// before site b.  Accepted flips accumulate in a mask applied at the word's
// end; the left neighbour's flip is tracked in f.
template <int WD, int GL = 1, class Hook>
__device__ __forceinline__ void sweep_row(uint32_t (&cur)[WD], const uint32_t (&up)[WD],
                                          const uint32_t (&dn)[WD], const int L, int& m,
                                          const uint32_t* __restrict__ T, const int np1, Prefetch& pf,
                                          const uint32_t chain, const uint32_t k0, const uint32_t k1, Hook& hook) {
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
  int m4 = 4 * m;
  uint32_t f = 0u, f0 = 0u;  // flip of the previous site / of site 0
  const char* Tb = reinterpret_cast<const char*>(T);
#pragma unroll
  for (int w = 0; w < WD; ++w) {
    const int nb = (w + 1 < WD) ? 32 : lw;
    uint32_t u[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) u[i] = pf.U[i];
    const int nb_next = (w + 1 < WD) ? ((w + 2 < WD) ? 32 : lw) : ((WD == 1) ? lw : 32);
    philox_fill<GL>(pf.U, nb_next, pf.blk, chain, k0, k1);
    pf.blk += static_cast<uint64_t>(nb_next / 4);
    // packed per-site bytes
    uint32_t A0[8], D[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (4 * q < nb) {
        const uint32_t b0 = spread4((s0[w] >> (4 * q)) & 0xFu);
        const uint32_t b1 = spread4((s1[w] >> (4 * q)) & 0xFu);
        const uint32_t b2 = spread4((el[w] >> (4 * q)) & 0xFu);
        A0[q] = 4u * b0 + 8u * b1 + 4u * b2;     // 4 (s0 + 2 s1 + el), no carries
        D[q] = 0x04040404u + 0xF8u * b2;         // +4 (el = 0) or -4 (el = 1) as signed bytes
      }
    }
    uint32_t F = 0u;  // flips of this word
    hook.word(nb);    // per-word set-up of the hook (the joint's uniforms)
    uint32_t t0, t1;
    {
      // first site of the word: state before it is known, one load
      const int a4 = static_cast<int>(prmt(A0[0], 0x4440u)) + static_cast<int>(f) * static_cast<int>(prmt(D[0], 0x8880u));
      t0 = t1 = *reinterpret_cast<const uint32_t*>(Tb + (a4 * np1 + m4));
    }
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      if (b < nb) {
        const bool last = (w == WD - 1 && b == nb - 1);
        const uint32_t selz = 0x4440u | static_cast<uint32_t>(b & 3);
        const uint32_t sels = sign_sel(static_cast<uint32_t>(b & 3));
        int a0m, d4;
        if (last) {
          const uint32_t elb = (el[w] >> b) & 1u;
          a0m = 4 * static_cast<int>(((eu[w] >> b) & 1u) + ((ed[w] >> b) & 1u) + (((er[w] >> b) & 1u) ^ f0) + elb);
          d4 = elb ? -4 : 4;
        } else {
          a0m = static_cast<int>(prmt(A0[b >> 2], selz));
          d4 = static_cast<int>(prmt(D[b >> 2], sels));
        }
        const int a4 = a0m + static_cast<int>(f) * d4;   // 4 a for this site
        const int dl = a4 - 8;                            // level change (x4) if it flips
        const uint32_t thr = f ? t1 : t0;
        const uint32_t acc = (u[b] <= thr) ? 1u : 0u;
        if (b + 1 < nb) {
          const bool nlast = (w == WD - 1 && b + 1 == nb - 1);
          int na0, nd4;
          if (nlast) {
            const uint32_t ff0 = (w == 0 && b == 0) ? acc : f0;
            const uint32_t eln = (el[w] >> (b + 1)) & 1u;
            na0 = 4 * static_cast<int>(((eu[w] >> (b + 1)) & 1u) + ((ed[w] >> (b + 1)) & 1u) +
                                      (((er[w] >> (b + 1)) & 1u) ^ ff0) + eln);
            nd4 = eln ? -4 : 4;
          } else {
            na0 = static_cast<int>(prmt(A0[(b + 1) >> 2], 0x4440u | static_cast<uint32_t>((b + 1) & 3)));
            nd4 = static_cast<int>(prmt(D[(b + 1) >> 2], sign_sel(static_cast<uint32_t>((b + 1) & 3))));
          }
          // (offsets summed as 32-bit integers, one 64-bit address add each)
          const int off0 = na0 * np1 + m4;                 // site b not flipped
          const int off1 = off0 + nd4 * np1 + dl;          // site b flipped
          t0 = *reinterpret_cast<const uint32_t*>(Tb + off0);
          t1 = *reinterpret_cast<const uint32_t*>(Tb + off1);
        }
        if (acc) {   // (predicated: no multiply by the 0/1 outcome)
          F |= 1u << b;
          m4 += dl;
        }
        f = acc;
        if (w == 0 && b == 0) f0 = acc;
        hook.sample(m4, b);
      }
    }
    cur[w] ^= F;
  }
  m = m4 >> 2;
}

// ------------------------------------------------------------------ hooks
// A hook sees every sample: word(nb) before the nb sites of each lattice
// word, then sample(m4, b) after the attempt at site b of the word, with the
// sample's level as m4 = 4 m (a byte offset into u32 arrays); b is a
// compile-time constant once the site loop is unrolled.
//
// Generation: every sample adds 1 to its level's u32 counter in the block's
// shared-memory histogram (one reduction, no branch), D sites late: the
// sample at site b is counted while site b + D is attempted (D divides 32,
// so the slot b % D is a compile-time register), its level waiting in
// pend[b % D] meanwhile.  A reduction issued right after the level update
// sat on the chain's serial path -- the next site's threshold loads are
// shared-memory accesses of the same warp and stay behind it -- while one
// whose address is known sites early does not (measured at L = 32 with
// D = 32: 9 % off the generation time).  pend[] starts at a scratch counter
// past the last level; flush() counts what is pending.  D = 32 for one word
// a row; 8 where the row's words already fill the registers.
//
// REC: the round is recorded -- every sample's level is also stored, as a
// uint16, in the round record, four samples to one 8-byte store (rows and
// lattice words hold multiples of four sites, so site b of a word is sample
// b mod 4 of its group), for the joint to read instead of replaying.  A
// chain's consecutive groups of four lie kRecGroupStride entries apart (the
// 32 chains of a record tile interleaved group by group), so the lanes of a
// warp with consecutive chains store one contiguous run.
constexpr int kRecGroupStride = 4 * 32;
template <int D = 32, bool REC = false>
struct GenHook {
  uint32_t* hist;
  uint32_t inc;      // 1; 0 for the lanes of a lane group that only help (one count per chain)
  int scratch;       // byte offset of the scratch counter (4 (N+1))
  int pend[D];       // byte offsets (4 m) of the samples not counted yet
  uint16_t* rec;     // REC: the chain's next record entry (always a valid address)
  bool rec_on;       // REC: this lane writes the record (one lane per chain)
  uint32_t pk[2];    // REC: levels of the current group of four samples
  __device__ __forceinline__ void init(uint32_t* h, uint32_t i, int np1) {
    hist = h;
    inc = i;
    scratch = 4 * np1;
    rec = nullptr;
    rec_on = false;
    pk[0] = pk[1] = 0u;
#pragma unroll
    for (int b = 0; b < D; ++b) pend[b] = scratch;
  }
  __device__ __forceinline__ void word(int) {}
  __device__ __forceinline__ void sample(int m4, int b) {
    red_shared_add(hist, pend[b % D], inc);
    pend[b % D] = m4;
    if constexpr (REC) {
      const uint32_t lv = static_cast<uint32_t>(m4) >> 2;
      const int q = (b & 3) >> 1;   // (b is a compile-time constant: static indices)
      if (b & 1) pk[q] |= lv << 16;
      else pk[q] = lv;
      if ((b & 3) == 3) {
        if (rec_on) st_record(rec, pk[0], pk[1]);
        rec += kRecGroupStride;
      }
    }
  }
  __device__ __forceinline__ void flush(int) {
#pragma unroll
    for (int b = 0; b < D; ++b) {
      red_shared_add(hist, pend[b], inc);
      pend[b] = scratch;
    }
  }
};

// Joint uniforms of the next nb samples k+1..k+nb (k a multiple of 4, as
// every lattice word starts on a Philox block): Philox((k'-1)>>2, r, chain,
// 1) word (k'-1)&3 for sample k'.
__device__ __forceinline__ void joint_fill(uint32_t (&U)[32], const int nb, const int64_t k, const uint32_t r,
                                           const uint32_t chain, const uint32_t k0, const uint32_t k1) {
  const uint32_t blk = static_cast<uint32_t>(static_cast<uint64_t>(k) >> 2);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (4 * q < nb) {
      const uint4 v = philox4x32_10(make_uint4(blk + static_cast<uint32_t>(q), r, chain, kTagJoint), k0, k1);
      U[4 * q + 0] = v.x;
      U[4 * q + 1] = v.y;
      U[4 * q + 2] = v.z;
      U[4 * q + 3] = v.w;
    }
  }
}

// Joint search (Sec. 2 step 4): for samples k = 1..M of the chain (the
// configuration after attempt k of the round) draw the joint uniform
// Philox((k-1)>>2, r, chain, 1) word (k-1)&3 and test it against the
// threshold of the move from the input level x to the sample's level; the
// first k that passes is recorded.  The test does not steer control flow
// (the threshold load would then stall every sample): hits are folded into
// `found` branch-free and the replay loop looks at `done` once per row.
// poll() (once per sweep) ends the search early when another search has
// already found an accepted sample of the same chain at or before `stop`
// (the chain's earliest hit so far, *kmin; nullptr: never).
// (k counts the samples of the words seen so far; sample b of the current
// word is kw + b + 1, with no per-sample counter.)
struct SearchHook {
  const uint32_t* __restrict__ tj;  // thresholds for moves x -> m, indexed by m
  int64_t k, M, found;
  int64_t kw = 0;                   // samples before the current word
  uint32_t chain, r, k0, k1;
  uint32_t uj[32];
  bool done;
  const unsigned long long* kmin = nullptr;
  unsigned long long stop = 0;
  __device__ __forceinline__ void word(int nb) {
    joint_fill(uj, nb, k, r, chain, k0, k1);
    kw = k;
    k += nb;
  }
  __device__ __forceinline__ void sample(int m4, int b) {
    const int64_t kk = kw + b + 1;
    const bool hit = (uj[b] <= __ldg(&tj[m4 >> 2])) && !done && kk <= M;
    found = hit ? kk : found;
    done = done || hit;
  }
  __device__ __forceinline__ void poll() {
#ifdef __CUDACC__
    if (kmin && __ldcg(kmin) <= stop) done = true;
#endif
  }
};

// Summary replay (exact joint resolution, Sec. 2 step 4): over the samples
// of a segment, the smallest joint uniform seen at each level, folded into
// the chain's row with atomicMin once per run of equal levels; also the
// range of levels visited and whether some run's minimum was 0xFFFFFFFF.
// W > 0: the runs' minima first go to this lane's window of W levels in
// shared memory (column win, stride kWinStride; placed around the first
// level seen, every entry 0xFFFFFFFF on entry and again after drain()), and
// drain() folds the window into the row once a segment -- one global atomic
// per level visited instead of one per run (levels outside the window go to
// the row directly).
constexpr int kWinStride = 128;
template <int W = 0>
struct SummaryHook {
  uint32_t* umin;  // row of the chain, indexed by level
  int64_t k;
  uint32_t chain, r, k0, k1;
  uint32_t uj[32];
  int cur, lo, hi;
  uint32_t run_min;
  bool flag;
  bool done;       // never set: the whole segment is summarised
  uint32_t* win = nullptr;
  int base = kNoBase;
  static constexpr int kNoBase = -0x7FFFFFFF;
  __device__ __forceinline__ void put(int m, uint32_t v) {
    if constexpr (W > 0) {
      if (base == kNoBase) base = m - W / 2;
      const unsigned s = static_cast<unsigned>(m - base);
      if (s < static_cast<unsigned>(W)) {
        uint32_t* e = win + s * kWinStride;
        *e = min(*e, v);
        return;
      }
    }
    atomicMin(&umin[m], v);
  }
  __device__ __forceinline__ void drain() {
    if constexpr (W > 0) {
      if (base == kNoBase) return;
      for (int s = 0; s < W; ++s) {
        const uint32_t v = win[s * kWinStride];
        if (v != 0xFFFFFFFFu) {
          atomicMin(&umin[base + s], v);
          win[s * kWinStride] = 0xFFFFFFFFu;
        }
      }
      base = kNoBase;
    }
  }
  __device__ __forceinline__ void poll() {}
  __device__ __forceinline__ void word(int nb) {
    joint_fill(uj, nb, k, r, chain, k0, k1);
    k += nb;
  }
  __device__ __forceinline__ void sample(int m4, int b) {
    const int m = m4 >> 2;
    const uint32_t u = uj[b];
    if constexpr (W > 0) {
      // (branch-light: the range and the flag are kept per sample, the run
      // that ends here is one short conditional update of the window; only a
      // level outside the window takes the atomic)
      const bool put_run = m != cur && cur >= 0;
      base = (base == kNoBase) ? m - W / 2 : base;
      const unsigned s = static_cast<unsigned>(cur - base);
      if (put_run) {
        if (s < static_cast<unsigned>(W)) {
          uint32_t* e = win + s * kWinStride;
          *e = min(*e, run_min);
        } else {
          atomicMin(&umin[cur], run_min);
        }
      }
      flag = flag || (put_run && run_min == 0xFFFFFFFFu);
      lo = min(lo, m);
      hi = max(hi, m);
      run_min = (m != cur) ? u : min(run_min, u);
      cur = m;
    } else if (m != cur) {
      flush();
      cur = m;
      run_min = u;
    } else {
      run_min = min(run_min, u);
    }
  }
  __device__ __forceinline__ void flush() {
    if (cur >= 0) {
      put(cur, run_min);
      flag = flag || (run_min == 0xFFFFFFFFu);
      lo = min(lo, cur);
      hi = max(hi, cur);
    }
  }
};

}  // namespace mcgpu
