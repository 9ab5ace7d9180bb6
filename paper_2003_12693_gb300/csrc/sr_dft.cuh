// Small complex DFTs held in registers, used by the FFT passes of the phi
// solve (Eqs. (31)-(33)).  Every dftN<INV> takes x[0..N) in natural order and
// leaves its DFT in natural order: X[k] = sum_n x[n] exp(-+2 pi i n k / N),
// the minus sign forward (INV = false), plus for the inverse (unnormalised).
#pragma once

#include <cuda_runtime.h>

namespace srk {
namespace cdft {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <bool INV>
__device__ __forceinline__ float2 mul_w(float2 a, float cr, float ci) {
  const float s = INV ? ci : -ci;
  return make_float2(a.x * cr - a.y * s, a.x * s + a.y * cr);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2* x) {
  const float2 a = x[0], b = x[1];
  x[0] = cadd(a, b);
  x[1] = csub(a, b);
}
template <bool INV>
__device__ __forceinline__ void dft4(float2* x) {
  const float2 a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
  const float2 a2 = cadd(x[1], x[3]), a3 = mul_mi<INV>(csub(x[1], x[3]));
  x[0] = cadd(a0, a2);
  x[2] = csub(a0, a2);
  x[1] = cadd(a1, a3);
  x[3] = csub(a1, a3);
}
template <bool INV>
__device__ __forceinline__ void dft8(float2* x) {
  float2 e[4] = {x[0], x[2], x[4], x[6]};
  float2 o[4] = {x[1], x[3], x[5], x[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  const float c = 0.70710678118654752440f;
  o[1] = mul_w<INV>(o[1], c, c);
  o[2] = mul_mi<INV>(o[2]);
  o[3] = mul_w<INV>(o[3], -c, c);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    x[m] = cadd(e[m], o[m]);
    x[m + 4] = csub(e[m], o[m]);
  }
}
template <bool INV>
__device__ __forceinline__ void dft16(float2* x) {
  float2 e[8], o[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    e[m] = x[2 * m];
    o[m] = x[2 * m + 1];
  }
  dft8<INV>(e);
  dft8<INV>(o);
  const float C1 = 0.92387953251128675613f, S1 = 0.38268343236508977173f;
  const float c = 0.70710678118654752440f;
  o[1] = mul_w<INV>(o[1], C1, S1);
  o[2] = mul_w<INV>(o[2], c, c);
  o[3] = mul_w<INV>(o[3], S1, C1);
  o[4] = mul_mi<INV>(o[4]);
  o[5] = mul_w<INV>(o[5], -S1, C1);
  o[6] = mul_w<INV>(o[6], -c, c);
  o[7] = mul_w<INV>(o[7], -C1, S1);
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    x[m] = cadd(e[m], o[m]);
    x[m + 8] = csub(e[m], o[m]);
  }
}
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* x) {
  if constexpr (R == 16) dft16<INV>(x);
  else if constexpr (R == 8) dft8<INV>(x);
  else if constexpr (R == 4) dft4<INV>(x);
  else dft2<INV>(x);
}

}  // namespace cdft
}  // namespace srk
