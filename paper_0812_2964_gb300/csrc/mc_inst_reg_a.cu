// Instantiation unit: lattice in registers, L = 4, 8, 12, 16.
#include "mc_chain_kernels.cuh"

namespace mcgpu {

cudaError_t chain_kernels_reg_a(const DevJob& j, const LaunchShape& s, bool gen, uint64_t t0, int64_t S, bool trace,
                   uint32_t r, cudaStream_t st) {
  switch (j.L) {
    case 4: return dispatch_ts<RegF<4>>(j, s, gen, t0, S, trace, r, st);
    case 8: return dispatch_ts<RegF<8>>(j, s, gen, t0, S, trace, r, st);
    case 12: return dispatch_ts<RegF<12>>(j, s, gen, t0, S, trace, r, st);
    case 16: return dispatch_ts<RegF<16>>(j, s, gen, t0, S, trace, r, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mcgpu
