// Inner-loop exit test of Sec. 4: partial sums of |a - b|^2 and |b|^2 in FP64.
// Internal to the library (sr_api.cu <-> sr_inner.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace srk {

// partials[2 blk + 0] = sum (a - b)^2, partials[2 blk + 1] = sum b^2 over the
// block's share of the n elements; nblocks CTAs
cudaError_t launch_change_partials(const float* a, const float* b, size_t n, double* partials,
                                   int nblocks, cudaStream_t s);

}  // namespace srk
