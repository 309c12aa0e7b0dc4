// Instantiation unit: lattice in shared memory, 2 word(s) per row, L = 64 fixed at compile time.
#include "mc_chain_kernels.cuh"

namespace mcgpu {

cudaError_t chain_kernels_smem_L64(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace,
                   uint32_t r, cudaStream_t st) {
  return dispatch_ts<SmemF<2, 64>>(j, s, gen, t0, S, trace, r, st);
}

}  // namespace mcgpu
