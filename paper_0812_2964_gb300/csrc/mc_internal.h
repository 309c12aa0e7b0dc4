// Internal declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace mcgpu {

// Lattice placement of a chain during a sweep.
enum Placement : int {
  kPlaceReg = 0,   // one chain per thread, rows in registers (L <= 32)
  kPlaceSmem = 1,  // one chain per thread, rows in shared memory (any L)
  kPlaceGlobal = 2,  // one chain per thread, lattice in global memory, rows streamed through
                     // registers (generation at L = 96, 100, 128; the joint's replays use 1)
};

struct LaunchShape {
  int placement;   // Placement
  int cpw;         // chains per warp (1..32; lanes >= cpw idle)
  int wpb;         // warps per block
};

// Device-resident state of one job (all pointers are device pointers).
struct DevJob {
  int L, N, np1, wd, p;
  uint32_t key0, key1;
  uint32_t* spins;     // [p][L][wd]
  uint32_t* spins0;    // round-start copy
  int32_t* m;          // [p] level now (after the round: level of sample M)
  int32_t* m0;         // [p] level at round start
  double* W;           // [np1]
  uint32_t* T;         // [5][np1] flip thresholds
  long long* h;        // [np1] histogram of the joined chain (this iteration)
  unsigned long long* hgen;  // [np1] all samples of the round
  unsigned long long* dpre;  // [np1] discarded prefixes of the round
  int64_t* k;          // [p] first kept sample (0 = none) after the joint
  int32_t* xused;      // [p] input level the current k was computed for (-1 = none)
  uint32_t* tj;        // [p][np1] joint thresholds for each chain's input
  int64_t* offsets;    // [p] position of each kept segment in the joined chain
  int32_t* work;       // [p] scratch list of chains
  int32_t* work2;      // [p] chains without a hit in their first segment
  int32_t* lastacc;    // [p] last chain before i that kept samples (-1: none)
  int32_t* trace;      // [S][p] energy after each sweep (nullable)
  uint32_t* ckpt;      // [kcap][L*wd][p] lattice at the start of each round segment
  int32_t* ckm;        // [kcap][p] level at the start of each round segment
  unsigned long long* kmin;  // [p] earliest accepted sample found so far for the chain's input (kNoHit: none)
  int2* plist;         // [p*kcap] (chain, segment) work list of the prefix pass
  int32_t* summ;       // [5][p] summary pass: lowest and highest level visited, flag; then
                       // [p][8] bytes: the exact scan's answers for candidate inputs
  uint8_t* visited;    // [np1] 1 once a weight update has seen h > 0 at the level
  int32_t* perm;       // [p] chain at each position of the joint (identity unless ordered)
  int32_t* lvcnt;      // [np1] scratch of the energy ordering
  int ordered;         // 1: chains joined by ascending final level (ties by index)
  // resolution policy of the joint (defaults kGridPassesScan, kGridPasses,
  // kScanMaxSamples; mc_set_join_policy changes them)
  int passes_scan, passes_plain;
  long long scan_max_samples;
  int ck_C;            // sweeps per checkpoint segment in the current round
  int ck_K;            // segments of the joint in the current round
  int64_t seg_len;     // samples per segment of the joint: ck_C * N for replays from
                       // checkpoints, shorter for a recorded round (nothing to restore)
  int kcap;            // segment capacity
  long long* stats;    // [kStatCount] small device counters
  int32_t* plv;        // [p][M] level after each attempt of a round that is not whole sweeps (nullable)
  uint16_t* rec;       // level after each attempt of the current whole-sweep round, when the
                       // round is small enough to record (nullable; layout: rec_index): the
                       // joint reads it instead of replaying the chains
};

// Round record layout: chains in tiles of 32; inside a tile, each group of
// four consecutive samples of the 32 chains lies side by side, so that a warp
// of consecutive chains stores (generation) or loads (joint, all chains at
// the same sample) 256 contiguous bytes per group.  Sample k (0-based) of
// chain c of a round of M samples (M a multiple of 4) is the uint16 at
// rec_index(c, k, M); the buffer holds ceil(p / 32) * 32 * M entries.
constexpr int kRecTile = 32;
__host__ __device__ inline size_t rec_index(int c, int64_t k, int64_t M) {
  return ((static_cast<size_t>(c / kRecTile) * static_cast<size_t>(M / 4) + static_cast<size_t>(k >> 2)) *
              kRecTile +
          static_cast<size_t>(c % kRecTile)) *
             4 +
         static_cast<size_t>(k & 3);
}
inline long long rec_entries(int p, int64_t M) {
  return static_cast<long long>((p + kRecTile - 1) / kRecTile) * kRecTile * M;
}

// whole-sweep rounds of at most this many samples (p * M) record every
// sample's level (2 bytes each, at most 16 GiB) for the joint: reading the
// record beats replaying from checkpoints by more than the record costs
// generation (weight iterations measured on GB300, record against replay:
// 20 sweeps and 2048 chains, L = 16 15 % shorter, 32 20 %, 48 14 %, 64 20 %,
// 96 19 %, 128 34 %; L = 32, 16384 chains 15 %; L = 64, 4096 chains, 100
// sweeps 29 %; L = 96, 200 sweeps 32 %; L = 128, 1024 chains, 400 sweeps
// 13 %)
constexpr long long kRecordMax = 1ll << 33;
inline long long default_record_max(int /*L*/) { return kRecordMax; }

// rounds that are not whole sweeps record every sample's level (for their
// parallel joint) when p * M is at most this many entries
constexpr long long kPartialLevelsMax = 1ll << 26;

// kmin[] value of a chain with no accepted sample found (yet)
constexpr unsigned long long kNoHit = 0x7FFFFFFFFFFFFFFFull;

// Whether the job's previous joint rejected so many chains that this one
// skips its speculative first search (where the caller allows it): with more
// than p/16 of them, the speculated inputs fail for as many chains and the
// joint takes the exact path anyway, and the speculative search would have
// read every rejecting chain whole
__host__ __device__ inline bool rough_last_joint(long long rejected, int p) { return rejected > p / 16; }

enum StatIndex : int {
  kStatCarry = 0,        // level passed on to the next round's chain 0
  kStatCarryValid = 1,
  kStatJoined = 2,       // samples kept in the last joint
  kStatMismatch = 3,     // searches repeated because the speculated input was wrong
  kStatPasses = 4,       // resolution passes that had work (last joint)
  kStatRejected = 5,     // chains with no kept sample (last joint)
  kStatSearched = 6,     // samples replayed by the last joint's searches
  kStatJoinedTotal = 7,  // samples kept by all joints of the job
  kStatPending = 8,      // chains queued for the current resolution pass
  kStatWholeFill = 9,    // running position while the prefix work list is filled
  kStatQueueSearch = 11, // next work item of the running persistent pass
  kStatQueuePrefix = 10, // work items of the prefix pass
  kStatPartial = 12,     // partial-segment items of the prefix pass (listed after the whole ones)
  kStatFirstPending = 13,// lowest chain queued by the last mark pass (p if none)
  kStatScanned = 14,     // chains whose input the exact scan settled (last joint)
  kStatNoHit = 15,       // chains listed in work2
  kStatCount = 16
};

// ---- kernels (mc_kernels.cu) ----
cudaError_t k_init_lattice(const DevJob& j, int start, cudaStream_t st);
// the joint order (perm) for the job's current levels and j.ordered
cudaError_t k_order(const DevJob& j, cudaStream_t st);
cudaError_t k_levels(const DevJob& j, cudaStream_t st);
cudaError_t k_build_table(const DevJob& j, cudaStream_t st);
cudaError_t k_update_weights(const DevJob& j, cudaStream_t st);
// rounds that are not whole sweeps: n attempts per chain from attempt t0
// (levels recorded in j.plv when `record`), and their joint by the serial
// rule (M attempts per chain): over the recorded levels, one chain at a time
// with its samples tested in parallel, else by replay in one thread
cudaError_t k_generate_attempts(const DevJob& j, uint64_t t0, int64_t n, bool record, cudaStream_t st);
cudaError_t k_join_attempts(const DevJob& j, uint64_t t0, int64_t M, uint32_t r, bool naive, bool recorded,
                            cudaStream_t st);
// E, C, F, S at n inverse temperatures (device arrays betas[n], out[n][4])
cudaError_t k_thermo(const DevJob& j, const double* betas, int n, double* out, cudaStream_t st);
cudaError_t k_generate(const DevJob& j, const LaunchShape& s, uint64_t t0, int64_t S,
                       bool trace, cudaStream_t st);
cudaError_t k_join(const DevJob& j, const LaunchShape& s, uint64_t t0, int64_t S, uint32_t r,
                   bool naive, cudaStream_t st);

// pieces of the joint shared by all lattice sizes
// grid-wide speculative resolution passes: before the exact scan (when the
// round is short enough for the summary replay), and without it
constexpr int kGridPassesScan = 2;
constexpr int kGridPasses = 10;
// rounds with at most this many samples (all chains) take the summary replay
// and the exact scan when speculation has not settled after kGridPassesScan
constexpr long long kScanMaxSamples = 20000000000ll;
cudaError_t join_prelude(const DevJob& j, cudaStream_t st);
cudaError_t join_mark(const DevJob& j, cudaStream_t st, bool thresholds = true, bool defer = false);
cudaError_t join_tj_list(const DevJob& j, cudaStream_t st);
// list (in work2) the chains of list_mode (0 all, 1 work) with no hit in segment 0
cudaError_t join_nohit(const DevJob& j, int list_mode, cudaStream_t st);
// exact_first: a recorded round whose exact path is enabled -- when the job's
// previous joint rejected more than p/16 chains, the speculative first
// search is skipped (select marks every chain unsearched) and the joint goes
// straight to the summary and the exact scan
cudaError_t join_select(const DevJob& j, bool listed, cudaStream_t st, bool exact_first = false);
cudaError_t join_prefix_list(const DevJob& j, cudaStream_t st);
cudaError_t join_reset_queue(const DevJob& j, cudaStream_t st);
cudaError_t join_finalize(const DevJob& j, int64_t S, cudaStream_t st);
cudaError_t join_summary_init(const DevJob& j, cudaStream_t st);
cudaError_t join_scan(const DevJob& j, cudaStream_t st);

// per-unit launchers of the templated chain kernels (mc_inst_*.cu)
#define MC_CHAIN_UNIT(name)                                                                              \
  cudaError_t name(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace, \
                   uint32_t r, cudaStream_t st)
MC_CHAIN_UNIT(chain_kernels_reg_a);
MC_CHAIN_UNIT(chain_kernels_reg_b);
MC_CHAIN_UNIT(chain_kernels_reg_c);
MC_CHAIN_UNIT(chain_kernels_smem_1);
MC_CHAIN_UNIT(chain_kernels_smem_2);
MC_CHAIN_UNIT(chain_kernels_smem_3);
MC_CHAIN_UNIT(chain_kernels_smem_4);
MC_CHAIN_UNIT(chain_kernels_smem_L16_24);
MC_CHAIN_UNIT(chain_kernels_smem_L32);
MC_CHAIN_UNIT(chain_kernels_smem_L48);
MC_CHAIN_UNIT(chain_kernels_smem_L64);
MC_CHAIN_UNIT(chain_kernels_smem_L96);
MC_CHAIN_UNIT(chain_kernels_smem_L100);
MC_CHAIN_UNIT(chain_kernels_smem_L128);
#undef MC_CHAIN_UNIT
// the joint of a recorded round (any L): kernels without lattices or table
cudaError_t chain_kernels_record(const DevJob& j, uint64_t t0, int64_t S, uint32_t r, cudaStream_t st);

// launch shape chosen by default for (L, p)
LaunchShape default_shape(int L, int p, int num_sms);
// fullest warps with the same table placement (what concurrent jobs want)
LaunchShape dense_shape(int L, int p, int num_sms);
bool shape_supported(int L, const LaunchShape& s);
size_t gen_smem_bytes(int L, const LaunchShape& s, bool* table_in_smem);

// message returned by mc_last_error() on this thread
void set_last_error(const char* msg);

// total kernel launches issued by this library (for accounting)
uint64_t launches_add(uint64_t n);

}  // namespace mcgpu
