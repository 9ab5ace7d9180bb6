// The iterated solution of the w sub-problem, Eqs. (38)-(40).
//
// From w^{k+1,0} = w^k, each sweep forms
//   v^{k+1,r}(x) = sum_{p,q} k(p) k(q) h_eps(phi^{k+1}(y)) w^{k+1,r}(y),  y = x + (p, q)
// (Eq. (38), window terms outside the image dropped), then Eq. (39) and the
// projection (40).  The denominator gamma g delta_eps + mu of Eq. (39) is a
// positive scalar at each pixel, so the projection removes it:
//   w^{k+1,r+1} = B / |B|,  B = grad phi^{k+1} + b^k + (2 beta / mu) h_eps(phi^{k+1}) v^{k+1,r},
// with the zero vector kept at zero.  After the last sweep, Eq. (23) gives
// b^{k+1} = b^k + grad phi^{k+1} - w^{k+1}; b is carried as e = b - w.
//
// One CTA per 32 x 32 tile: h w over the tile and its halo in shared memory,
// the separable window sum as a vertical then a horizontal pass, then the
// per-pixel update (forward differences, periodic, Eq. (35)).
#include <cuda_runtime.h>

#include "sr_wfix.h"

namespace srk {
namespace {

constexpr int kWT = 32;          // tile side
constexpr int kWThreads = 256;

// H_eps of Eq. (5)
__device__ __forceinline__ float heaviside(float x, const Model& m) {
  if (x > m.eps) return 1.f;
  if (x < -m.eps) return 0.f;
  const float z = x * m.inv_eps;
  return 0.5f * (1.f + z + sinpif(z) * 0.31830988618379067f);
}

// h_eps of Eq. (11): the narrow band of half width l around the contour
__device__ __forceinline__ float band_of(float x, const Model& m) {
  return heaviside(x + m.band_l, m) * (1.f - heaviside(x - m.band_l, m));
}

__global__ void __launch_bounds__(kWThreads) k_wfix_sweep(WFixArgs a) {
  extern __shared__ float sm[];
  const int R = a.mod.R, S = kWT + 2 * R;
  const int M = a.geo.M, N = a.geo.N;
  float* u1 = sm;
  float* u2 = u1 + S * S;
  float* t1 = u2 + S * S;      // vertical sums: kWT rows x S columns
  float* t2 = t1 + kWT * S;
  const int i0 = blockIdx.y * kWT, j0 = blockIdx.x * kWT;

  for (int idx = threadIdx.x; idx < S * S; idx += kWThreads) {
    const int r = idx / S, c = idx % S;
    const int i = i0 - R + r, j = j0 - R + c;
    float v1 = 0.f, v2 = 0.f;
    if (i >= 0 && i < M && j >= 0 && j < N) {
      const size_t o = (size_t)i * N + j;
      const float h = band_of(a.phi1[o], a.mod);
      v1 = h * a.cw1[o];
      v2 = h * a.cw2[o];
    }
    u1[idx] = v1;
    u2[idx] = v2;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kWT * S; idx += kWThreads) {
    const int r = idx / S, c = idx % S;
    float s1 = 0.f, s2 = 0.f;
    for (int p = -R; p <= R; ++p) {
      const float k = a.mod.kw[p + R];
      s1 = fmaf(k, u1[(r + R + p) * S + c], s1);
      s2 = fmaf(k, u2[(r + R + p) * S + c], s2);
    }
    t1[idx] = s1;
    t2[idx] = s2;
  }
  __syncthreads();

  double num = 0.0, den = 0.0;
  for (int idx = threadIdx.x; idx < kWT * kWT; idx += kWThreads) {
    const int r = idx / kWT, c = idx % kWT;
    const int i = i0 + r, j = j0 + c;
    if (i >= M || j >= N) continue;
    float v1 = 0.f, v2 = 0.f;
    for (int q = -R; q <= R; ++q) {
      const float k = a.mod.kw[q + R];
      v1 = fmaf(k, t1[r * S + c + R + q], v1);
      v2 = fmaf(k, t2[r * S + c + R + q], v2);
    }
    const size_t o = (size_t)i * N + j;
    const float phi = a.phi1[o];
    const float d1 = a.phi1[(size_t)((i + 1) % M) * N + j] - phi;
    const float d2 = a.phi1[(size_t)i * N + (j + 1) % N] - phi;
    const float bk1 = a.ek1[o] + a.wk1[o], bk2 = a.ek2[o] + a.wk2[o];
    const float ch = a.mod.beta2_mu * band_of(phi, a.mod);
    const float B1 = d1 + bk1 + ch * v1, B2 = d2 + bk2 + ch * v2;
    const float n = sqrtf(B1 * B1 + B2 * B2);
    const float w1 = n > 0.f ? B1 / n : 0.f;
    const float w2 = n > 0.f ? B2 / n : 0.f;
    a.nw1[o] = w1;
    a.nw2[o] = w2;
    if (a.e1o) {
      a.e1o[o] = (bk1 + d1 - w1) - w1;
      a.e2o[o] = (bk2 + d2 - w2) - w2;
    }
    if (a.phi_old) {
      const double po = a.phi_old[o];
      num += ((double)phi - po) * ((double)phi - po);
      den += po * po;
    }
  }
  if (a.phi_old) {
    __shared__ double red[2][kWThreads];
    red[0][threadIdx.x] = num;
    red[1][threadIdx.x] = den;
    __syncthreads();
    for (int k = kWThreads / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) {
        red[0][threadIdx.x] += red[0][threadIdx.x + k];
        red[1][threadIdx.x] += red[1][threadIdx.x + k];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double* pt = a.partials + 2 * (blockIdx.y * gridDim.x + blockIdx.x);
      pt[0] = red[0][0];
      pt[1] = red[1][0];
    }
  }
}

}  // namespace

cudaError_t launch_wfix_sweep(const WFixArgs& a, cudaStream_t s) {
  const int R = a.mod.R, S = kWT + 2 * R;
  const size_t smem = sizeof(float) * (2 * S * S + 2 * kWT * S);
  const dim3 grid((a.geo.N + kWT - 1) / kWT, (a.geo.M + kWT - 1) / kWT);
  k_wfix_sweep<<<grid, kWThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace srk
