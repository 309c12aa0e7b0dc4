// Instantiation unit: lattice in registers, L = 20, 24, 28.
#include "mc_chain_kernels.cuh"

namespace mcgpu {

cudaError_t chain_kernels_reg_b(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace,
                   uint32_t r, cudaStream_t st) {
  switch (j.L) {
    case 20: return dispatch_ts<RegF<20>>(j, s, gen, t0, S, trace, r, st);
    case 24: return dispatch_ts<RegF<24>>(j, s, gen, t0, S, trace, r, st);
    case 28: return dispatch_ts<RegF<28>>(j, s, gen, t0, S, trace, r, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mcgpu
