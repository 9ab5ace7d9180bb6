// AOS solve of the phi sub-problem: the alternative to the FFT solve that the
// paper mentions at the end of Sec. 4, in the additive form of Eqs. (19)-(20):
//     phi = 1/2 [ (I - k A_1)^{-1} F + (I - k A_2)^{-1} F ],   k = 2 tau mu,
// with A_1, A_2 the periodic second differences down the columns (axis 0) and
// along the rows (axis 1).  The right-hand side of Eq. (37) is
// F = (I - tau mu (A_1 + A_2)) psi + G, G the increment right-hand side of
// k_prep, and since (I - k A)^{-1} psi = psi + (I - k A)^{-1} (k A psi),
//     phi = psi + 1/2 [ (I - k A_1)^{-1} x_1 + (I - k A_2)^{-1} x_2 ],
//     x_1 = G + tau mu (A_1 - A_2) psi,   x_2 = G - tau mu (A_1 - A_2) psi
// (the recursions then work on increments, as the FFT solve does).
//
// Each line solve (1 + 2k) y_i - k (y_{i-1} + y_{i+1}) = x_i (cyclic) has the
// same constant coefficients everywhere, so it factors once:
//     y = (r / k) (1 - r S)^{-1} (1 - r S^{-1})^{-1} x,
// r in (0, 1) the root of k r^2 - (1 + 2k) r + k = 0: a forward recursion
// u_i = x_i + r u_{i-1} and a backward one v_i = u_i + r v_{i+1}.  Recursions
// start R places early with a zero state; r^R < 2^-27 (R from the host).
//
//   k_aos_cols<R>: one thread per column and run of kRecRows rows (lanes on
//                  adjacent columns: coalesced), writes T1 = (I - k A_1)^{-1} x_1
//                  and the row pass's input x_2
//   k_aos_rows:    one warp per row, lanes on 32 adjacent columns; the
//                  recursions run as warp scans over blocks of 32 with the
//                  block's carry; the forward states are kept in shared
//                  memory for the backward sweep; writes phi
#include <cmath>

#include "sr_internal.h"

namespace srk {

template <int R>
__global__ void __launch_bounds__(32 * kRecChunks) k_aos_cols(const AosArgs a) {
  constexpr int TR = kRecRows;
  const int M = a.geo.M, N = a.geo.N;
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int i0 = (blockIdx.y * kRecChunks + threadIdx.y) * TR;
  pdl_wait();
  pdl_trigger();
  if (j >= N || i0 >= M) return;
  const float r = a.r, tm = a.tm, s = a.s;
  const int jl = j == 0 ? N - 1 : j - 1, jr = j == N - 1 ? 0 : j + 1;
  auto wrap = [M](int i) {
    while (i < 0) i += M;
    while (i >= M) i -= M;
    return i;
  };
  // tau mu (A_1 - A_2) psi = tau mu (psi_up + psi_down - psi_left - psi_right)
  auto stencil = [&](int i) {
    if (!a.psi) return 0.f;
    const size_t ro = (size_t)i * N;
    const float up = a.psi[(size_t)wrap(i - 1) * N + j], dn = a.psi[(size_t)wrap(i + 1) * N + j];
    return tm * ((up + dn) - (a.psi[ro + jl] + a.psi[ro + jr]));
  };
  // x_1 = G + tau mu (A_1 - A_2) psi
  auto input = [&](int i) { return a.G[(size_t)i * N + j] + stencil(i); };
  // the row pass's input x_2 = G - tau mu (A_1 - A_2) psi for this run of rows:
  // the row pass may overwrite psi in place, so it must not read psi's
  // neighbouring rows itself
#pragma unroll 4
  for (int q = 0; q < TR; ++q)
    if (i0 + q < M) a.X2[(size_t)(i0 + q) * N + j] = a.G[(size_t)(i0 + q) * N + j] - stencil(i0 + q);
  float u = 0.f;
#pragma unroll 4
  for (int q = 0; q < R; ++q) u = fmaf(r, u, input(wrap(i0 - R + q)));
  float b[TR + R];
#pragma unroll
  for (int q = 0; q < TR + R; ++q) b[q] = input(wrap(i0 + q));
#pragma unroll
  for (int q = 0; q < TR + R; ++q) {
    u = fmaf(r, u, b[q]);
    b[q] = u;
  }
  float v = 0.f;
#pragma unroll
  for (int q = TR + R - 1; q >= TR; --q) v = fmaf(r, v, b[q]);
#pragma unroll
  for (int q = TR - 1; q >= 0; --q) {
    v = fmaf(r, v, b[q]);
    b[q] = s * v;
  }
#pragma unroll
  for (int q = 0; q < TR; ++q)
    if (i0 + q < M) a.T1[(size_t)(i0 + q) * N + j] = b[q];
}

// inclusive scan of x_l <- x_l + r x_{l-1} over the 32 lanes (FWD) or of
// x_l <- x_l + r x_{l+1} (backward), then the carry c from the previous block
// enters as r^(distance) c; returns the lane's value; pw[m] = r^m
template <bool FWD>
__device__ __forceinline__ float warp_recursion(float x, float carry, const AosArgs& a, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float t = FWD ? __shfl_up_sync(0xffffffffu, x, d) : __shfl_down_sync(0xffffffffu, x, d);
    const bool take = FWD ? lane >= d : lane + d < 32;
    if (take) x = fmaf(a.pw[d], t, x);
  }
  const int dist = FWD ? lane + 1 : 32 - lane;
  return fmaf(a.pw[dist], carry, x);
}

__global__ void __launch_bounds__(32 * kAosRowWarps) k_aos_rows(const AosArgs a) {
  extern __shared__ float srow[];  // kAosRowWarps rows of N floats
  const int M = a.geo.M, N = a.geo.N;
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
  const int i = blockIdx.x * kAosRowWarps + wv;
  pdl_wait();
  pdl_trigger();
  if (i >= M) return;
  float* ub = srow + (size_t)wv * N;
  const size_t ro = (size_t)i * N;
  // x_2, formed by the column pass
  auto input = [&](int j) { return a.X2[ro + j]; };
  const int nb = (N + 31) / 32;
  const int wb = a.warm_blocks;  // blocks of warm-up (>= R places), may exceed nb
  // forward u_j = x_j + r u_{j-1}: warm-up over the wb blocks before block 0
  // (cyclically), then the row.  Lanes 0..cnt-1 of a block hold its values
  // (cnt < 32 only in a last, partial block), the rest zero; the carry into
  // the next block is the state at the last real value.
  float carry = 0.f;
  for (int q = -wb; q < nb; ++q) {
    const int blk = ((q % nb) + nb) % nb;
    const int base = blk * 32, cnt = min(32, N - base);
    const int j = base + lane;
    const float x = lane < cnt ? input(j) : 0.f;
    const float u = warp_recursion<true>(x, carry, a, lane);
    carry = __shfl_sync(0xffffffffu, u, cnt - 1);
    if (q >= 0 && lane < cnt) ub[j] = u;
  }
  __syncwarp();
  // backward v_j = u_j + r v_{j+1}: warm-up over the wb blocks after the last
  // one (blocks wb-1, ..., 0 cyclically), then the row from its end.  A block's
  // values sit in lanes 32-cnt..31 so that the carry enters at its last value.
  carry = 0.f;
  for (int q = -wb; q < nb; ++q) {
    const int blk = q < 0 ? (-q - 1) % nb : nb - 1 - q;
    const int base = blk * 32, cnt = min(32, N - base);
    const int off = 32 - cnt;
    const int j = base + lane - off;
    const bool real = lane >= off;
    const float v = warp_recursion<false>(real ? ub[j] : 0.f, carry, a, lane);
    carry = __shfl_sync(0xffffffffu, v, off);
    if (q >= 0 && real) {
      const size_t o = ro + j;
      const float p = a.psi ? a.psi[o] : 0.f;
      a.phi[o] = p + 0.5f * (a.T1[o] + a.s * v);
    }
  }
}

int aos_radius(double r) {
  if (!(r >= 0.0) || r >= 1.0) return 0;
  const double need = r <= 0.0 ? 1.0 : std::ceil(-27.0 * std::log(2.0) / std::log(r));
  const int buckets[] = {8, 12, 16, 20, 24, 32, 40, 48, 64, 96, 128};
  for (int R : buckets)
    if (R >= need) return R;
  return 0;
}

size_t aos_rows_smem(int N) { return (size_t)kAosRowWarps * N * sizeof(float); }

cudaError_t launch_aos(const AosArgs& a, cudaStream_t s, bool set_attr) {
  if (set_attr)
    return cudaFuncSetAttribute(k_aos_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)aos_rows_smem(4096));
  const dim3 cb(32, kRecChunks);
  const dim3 cg((a.geo.N + 31) / 32, (a.geo.M + kRecRows * kRecChunks - 1) / (kRecRows * kRecChunks));
  cudaError_t e = cudaErrorInvalidValue;
  switch (a.R) {
#define SR_AOS(r) \
  case r: e = launch_k(k_aos_cols<r>, cg, cb, 0, s, a); break;
    SR_AOS(8) SR_AOS(12) SR_AOS(16) SR_AOS(20) SR_AOS(24) SR_AOS(32) SR_AOS(40) SR_AOS(48)
    SR_AOS(64) SR_AOS(96) SR_AOS(128)
#undef SR_AOS
  }
  if (e != cudaSuccess) return e;
  return launch_k(k_aos_rows, dim3((a.geo.M + kAosRowWarps - 1) / kAosRowWarps),
                  dim3(32 * kAosRowWarps), aos_rows_smem(a.geo.N), s, a);
}

}  // namespace srk
