// Instantiation unit: lattice in shared memory, 1 word per row, L = 16 and 24 fixed at compile time.
#include "mc_chain_kernels.cuh"

namespace mcgpu {

cudaError_t chain_kernels_smem_L16_24(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S,
                                      bool trace, uint32_t r, cudaStream_t st) {
  switch (j.L) {
    case 16: return dispatch_ts<SmemF<1, 16>>(j, s, gen, t0, S, trace, r, st);
    case 24: return dispatch_ts<SmemF<1, 24>>(j, s, gen, t0, S, trace, r, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mcgpu
