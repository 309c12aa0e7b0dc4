// The joint's kernels for a recorded round (search, summary, resolution,
// prefix correction reading the round record instead of replaying
// lattices): one instantiation serves every L, since nothing in them
// depends on the lattice size at compile time.
#include "mc_chain_kernels.cuh"

namespace mcgpu {

// Samples per segment of a recorded round's joint.  A segment is one lane's
// work item; with nothing to restore at its start it can be much shorter
// than a replay segment, so that even the first pass (segment 0 of every
// chain) and a few thousand chains keep the whole GPU busy.
constexpr int64_t kRecordSegment = 2048;

cudaError_t chain_kernels_record(const DevJob& j, uint64_t t0, int64_t S, uint32_t r, cudaStream_t st) {
  DevJob jr = j;
  jr.seg_len = std::min<int64_t>(j.seg_len, kRecordSegment);
  jr.ck_K = static_cast<int>((S * j.N + jr.seg_len - 1) / jr.seg_len);
  // full warps, four a block; shared memory holds only the prefix pass's histogram
  const LaunchShape s{kPlaceReg, 32, 4};
  return launch_join_t<RecF, false>(jr, s, t0, S, r, st);
}

}  // namespace mcgpu
