// Instantiation unit: 3 word(s) per row, L = 96 fixed at compile time; lattice in shared
// memory, or (generation) in global memory with rows in registers.
#include "mc_chain_kernels.cuh"

namespace mcgpu {

cudaError_t chain_kernels_smem_L96(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace,
                   uint32_t r, cudaStream_t st) {
  if (s.placement == kPlaceGlobal) return dispatch_ts<GlobF<3, 96>>(j, s, gen, t0, S, trace, r, st);
  return dispatch_ts<SmemF<3, 96>>(j, s, gen, t0, S, trace, r, st);
}

}  // namespace mcgpu
