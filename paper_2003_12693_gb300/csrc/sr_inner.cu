// Partial sums for the inner-loop exit of Sec. 4: the loop over s stops once
// ||phi^{k+1,s+1} - phi^{k+1,s}|| / (||phi^{k+1,s}|| + 1e-6) <= Tol.  Each CTA
// accumulates its grid-stride share in FP64 (float4 loads) and writes two
// partial sums; the library's FP64 reduction kernel adds them.
#include "sr_inner.h"

namespace srk {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_change_partials(const float* __restrict__ a,
                                                              const float* __restrict__ b,
                                                              size_t n, double* __restrict__ part) {
  double num = 0.0, den = 0.0;
  const size_t n4 = n / 4;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 x = a4[i], y = b4[i];
    const double d0 = (double)x.x - y.x, d1 = (double)x.y - y.y, d2 = (double)x.z - y.z,
                 d3 = (double)x.w - y.w;
    num += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
    den += (double)y.x * y.x + (double)y.y * y.y + (double)y.z * y.z + (double)y.w * y.w;
  }
  for (size_t i = 4 * n4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const double d = (double)a[i] - b[i];
    num += d * d;
    den += (double)b[i] * b[i];
  }
  __shared__ double red[2][kThreads];
  red[0][threadIdx.x] = num;
  red[1][threadIdx.x] = den;
  __syncthreads();
  for (int k = kThreads / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      red[0][threadIdx.x] += red[0][threadIdx.x + k];
      red[1][threadIdx.x] += red[1][threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = red[0][0];
    part[2 * blockIdx.x + 1] = red[1][0];
  }
}

}  // namespace

cudaError_t launch_change_partials(const float* a, const float* b, size_t n, double* partials,
                                   int nblocks, cudaStream_t s) {
  k_change_partials<<<nblocks, kThreads, 0, s>>>(a, b, n, partials);
  return cudaGetLastError();
}

}  // namespace srk
