// Instantiation unit: lattice in shared memory, 1 word per row, L = 32 fixed at compile time.
#include "mc_chain_kernels.cuh"

namespace mcgpu {

cudaError_t chain_kernels_smem_L32(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace,
                   uint32_t r, cudaStream_t st) {
  return dispatch_ts<SmemF<1, 32>>(j, s, gen, t0, S, trace, r, st);
}

}  // namespace mcgpu
