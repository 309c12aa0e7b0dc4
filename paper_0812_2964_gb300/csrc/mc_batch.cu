// Batched generation: one launch runs the round (Sec. 2 step 2) of several
// independent jobs with different lattice sizes.  Blocks are assigned to
// jobs by contiguous ranges; each block runs the generation body compiled
// for its job's L and placement (lattice rows in registers for L <= 32, in
// shared memory with compile-time L for 24, 32, 48 and 64, with lane groups
// of 4 where a warp holds at most 8 chains).  Every job's chains are exactly
// those of its own launch, so results are identical to one launch per job.
#include "mc_batch.h"
#include "mc_chain_kernels.cuh"

namespace mcgpu {

__global__ void __launch_bounds__(128) gen_batched_kernel(const BatchParams P) {
  int i = 0;
  while (i + 1 < P.n && static_cast<int>(blockIdx.x) >= P.items[i + 1].first_block) ++i;
  const BatchItem& it = P.items[i];
  const int block = static_cast<int>(blockIdx.x) - it.first_block;
  const bool sm = it.placement == kPlaceSmem;
  switch (it.j.L) {
    case 8: gen_body<RegF<8>, true>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block); break;
    case 16: gen_body<RegF<16>, true>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block); break;
    case 24:
      if (sm) gen_body<SmemF<1, 24>, true>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block);
      else gen_body<RegF<24>, true>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block);
      break;
    case 32:
      if (sm) gen_body<SmemF<1, 32>, true>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block);
      else gen_body<RegF<32>, true>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block);
      break;
    case 48:
      if (it.gl == 4) gen_body<SmemF<2, 48>, true, 4>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block);
      else gen_body<SmemF<2, 48>, true>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block);
      break;
    case 64:
      if (it.gl == 4) gen_body<SmemF<2, 64>, true, 4>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block);
      else gen_body<SmemF<2, 64>, true>(it.j, it.cpw, it.t0, it.S, it.flushF, it.trace, block);
      break;
    default: break;
  }
}

bool batch_supported(int L, const LaunchShape& s) {
  const bool reg = (L == 8 || L == 16 || L == 24 || L == 32) && s.placement == kPlaceReg;
  const bool sm = (L == 24 || L == 32 || L == 48 || L == 64) && s.placement == kPlaceSmem;
  return (reg || sm) && s.wpb == kBatchWarps && shape_supported(L, s) && table_fits(L, s, true);
}

long long batch_resident_blocks(size_t smem_bytes) {
  if (cudaFuncSetAttribute(gen_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem_bytes)) != cudaSuccess)
    return 0;
  return resident_blocks(gen_batched_kernel, 32 * kBatchWarps, smem_bytes);
}

cudaError_t batch_item(const DevJob& j, const LaunchShape& s, uint64_t t0, int64_t S, bool trace, BatchItem* out,
                       size_t* smem_bytes, int* blocks) {
  out->j = j;
  out->cpw = s.cpw;
  out->placement = s.placement;
  out->gl = (s.placement == kPlaceSmem && s.cpw <= 8 && j.L > 32) ? 4 : 1;
  out->t0 = t0;
  out->S = S;
  out->trace = trace ? 1 : 0;
  const int per_block = s.cpw * s.wpb;
  const long long per_sweep = static_cast<long long>(per_block) * j.N;
  const int64_t flushF = std::max<int64_t>(1, (0xFFFFFFFFll - 32ll * per_block) / per_sweep);
  out->flushF = S > flushF ? flushF : 0;
  *smem_bytes = plan_bytes(j.L, s, true, true);
  *blocks = static_cast<int>(blocks_for(j.p, per_block));
  return cudaSuccess;
}

cudaError_t k_generate_batched(BatchParams& P, size_t smem_bytes, int total_blocks, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(gen_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem_bytes));
  if (e != cudaSuccess) return e;
  gen_batched_kernel<<<total_blocks, 32 * kBatchWarps, smem_bytes, st>>>(P);
  launches_add(1);
  return cudaGetLastError();
}

}  // namespace mcgpu
