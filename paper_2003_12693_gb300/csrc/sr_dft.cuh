// Small complex DFTs held in registers, and the register-resident Stockham
// stages built from them, used by the FFT passes of the phi solve (Eqs.
// (31)-(33)) in 2-D and in 3-D.  Every dftN<INV> takes x[0..N) in natural order and
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

// padded shared-memory position of sequence index a (1 pad per 16 values)
__device__ __forceinline__ int pad(int a) { return a + (a >> 4); }

// Twiddles of the Stockham stages, laid out per stage as [t - 1][k]
// (t = 1..R-1, k = 0..Ns-1, value exp(-2 pi i k t / (Ns R))), so that the
// threads of a warp, which hold consecutive k, read consecutive entries.
// Stage s >= 1 has Ns = E^s; only the last stage may have a radix below E.
template <int LOGL, int LOGE>
struct TwPlan {
  static constexpr int NST = (LOGL + LOGE - 1) / LOGE;
  __host__ __device__ static constexpr int log_r(int s) {
    return s < LOGL / LOGE ? LOGE : LOGL % LOGE;
  }
  __host__ __device__ static constexpr int offset(int s) {
    int o = 0;
    for (int q = 1; q < s; ++q) o += ((1 << log_r(q)) - 1) << (LOGE * q);
    return o;
  }
  static constexpr int TOTAL = offset(NST);
};

// Copy a stage-twiddle table into shared memory (the caller synchronises).
template <int N>
__device__ __forceinline__ void stage_table(float2* dst, const float2* __restrict__ src) {
  for (int q = threadIdx.x; q < N; q += blockDim.x) dst[q] = __ldg(src + q);
}

// Element a of the thread's sequence lives at smem[pad(a) * STRIDE] (STRIDE =
// 1 for rows, CB for interleaved columns; `base` already includes the
// sequence offset).  The thread holds E = 2^LOGE values x[m] = seq[u + (L/E) m];
// stages use radix E, the last one radix 2^(LOGL mod LOGE) if that is not 1.
// stw is the stage-twiddle table: in shared memory, or with TWG in global
// memory read through the read-only cache (the row passes: every CTA reads
// the same table, so it stays in L1 and no per-CTA copy is needed).
// With WS the exchanges synchronise the warp only: every sequence is held by
// lanes of one warp (L / E threads dividing 32), so no other warp reads its
// exchange area, and warps without a sequence need not take part.
template <int LOGL, int LOGE, int S, bool INV, int STRIDE, bool DB = false, bool TWG = false,
          bool WS = false>
__device__ __forceinline__ void stages(float2 (&x)[1 << LOGE], float2* base, int u,
                                       const float2* stw, float2* base2 = nullptr) {
  using TP = TwPlan<LOGL, LOGE>;
  constexpr int E = 1 << LOGE;
  constexpr int NST = TP::NST;
  if constexpr (S < NST) {
    constexpr int LOGR = TP::log_r(S);
    constexpr int R = 1 << LOGR, NB = E / R;
    constexpr int LOGNS = LOGE * S;
    constexpr int LOGTP = LOGL - LOGE;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = u + (b << LOGTP);
      float2 v[R];
#pragma unroll
      for (int t = 0; t < R; ++t) v[t] = x[b + t * NB];
      if constexpr (LOGNS > 0) {
        const int k = j & ((1 << LOGNS) - 1);
        constexpr int OFF = TP::offset(S);
#pragma unroll
        for (int t = 1; t < R; ++t) {
          const int ti = OFF + ((t - 1) << LOGNS) + k;
          float2 w = TWG ? __ldg(stw + ti) : stw[ti];
          if (INV) w.y = -w.y;
          v[t] = cmul(v[t], w);
        }
      }
      dft<R, INV>(v);
#pragma unroll
      for (int t = 0; t < R; ++t) x[b + t * NB] = v[t];
    }
    if constexpr (S + 1 < NST) {
      // with DB the exchanges alternate between two buffers: a buffer is
      // written again only after the barrier of the exchange in between, so
      // the barrier after the read-back is not needed
      float2* buf = (DB && (S & 1)) ? base2 : base;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int j = u + (b << LOGTP);
        const int k = j & ((1 << LOGNS) - 1);
        const int o = ((j >> LOGNS) << (LOGNS + LOGR)) + k;
#pragma unroll
        for (int t = 0; t < R; ++t) buf[pad(o + (t << LOGNS)) * STRIDE] = x[b + t * NB];
      }
      if constexpr (WS) {
        static_assert((1 << LOGTP) <= 32, "a warp-synchronous sequence fits one warp");
        __syncwarp();
      } else {
        __syncthreads();
      }
#pragma unroll
      for (int m = 0; m < E; ++m) x[m] = buf[pad(u + (m << LOGTP)) * STRIDE];
      if constexpr (!DB) {
        if constexpr (WS) __syncwarp();
        else __syncthreads();
      }
      stages<LOGL, LOGE, S + 1, INV, STRIDE, DB, TWG, WS>(x, base, u, stw, base2);
    }
  }
}

}  // namespace cdft
}  // namespace srk
