// Instantiation unit: lattice in registers, L = 32.
#include "mc_chain_kernels.cuh"

namespace mcgpu {

cudaError_t chain_kernels_reg_c(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace,
                   uint32_t r, cudaStream_t st) {
  switch (j.L) {
    case 32: return dispatch_ts<RegF<32>>(j, s, gen, t0, S, trace, r, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mcgpu
