// Batched generation launch (several jobs, one grid).
#pragma once
#include "mc_internal.h"

namespace mcgpu {

constexpr int kMaxBatch = 8;   // jobs per fused launch (kernel parameter space)
constexpr int kBatchWarps = 4;  // warps per block in the fused launch

struct BatchItem {
  DevJob j;
  int cpw;
  int placement;    // kPlaceReg or kPlaceSmem
  int gl;           // lanes per chain (4: lane groups, lattice in shared memory and cpw <= 8)
  int first_block;  // first block of this job in the fused grid
  int trace;
  uint64_t t0;
  int64_t S;
  int64_t flushF;
};

struct BatchParams {
  BatchItem items[kMaxBatch];
  int n;
};

// Whether a job of lattice size L with this shape can join a fused launch.
bool batch_supported(int L, const LaunchShape& s);
// Fill one item; returns its dynamic shared memory and block count.
cudaError_t batch_item(const DevJob& j, const LaunchShape& s, uint64_t t0, int64_t S, bool trace, BatchItem* out,
                       size_t* smem_bytes, int* blocks);
cudaError_t k_generate_batched(BatchParams& P, size_t smem_bytes, int total_blocks, cudaStream_t st);
// blocks of the fused kernel that fit on the device at once with this much
// dynamic shared memory per block
long long batch_resident_blocks(size_t smem_bytes);

}  // namespace mcgpu
