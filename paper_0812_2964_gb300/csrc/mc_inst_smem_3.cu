// Instantiation unit: lattice in shared memory, 3 word(s) per row, L read at run time.
#include "mc_chain_kernels.cuh"

namespace mcgpu {

cudaError_t chain_kernels_smem_3(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace,
                   uint32_t r, cudaStream_t st) {
  return dispatch_ts<SmemF<3>>(j, s, gen, t0, S, trace, r, st);
}

}  // namespace mcgpu
