// Column pass of the phi solve (Eqs. (30)-(33)) without a column FFT.
//
// After the row transforms, column k of the half spectrum holds one row
// frequency.  What the column FFT, the division by the symbol of Eq. (32) and
// the inverse column FFT do to it is the periodic tridiagonal solve
//     c_k y_i - tau mu (y_{i-1} + y_{i+1}) = x_i / N,   i mod M,
//     c_k = 1 + 2 tau mu + tau mu 4 sin^2(pi k / N),
// because tau mu 4 sin^2(pi l / M) is the symbol of tau mu (2 - S - S^-1) along
// the column (S the cyclic shift).  Its coefficients do not depend on i, so
// the operator factors once and for all: with r_k in (0, 1) the root of
// tau mu r^2 - c_k r + tau mu = 0,
//     c_k - tau mu (S + S^-1) = (tau mu / r_k) (1 - r_k S^-1) (1 - r_k S),
// hence y = s_k (1 - r_k S)^-1 (1 - r_k S^-1)^-1 x with s_k = r_k / (tau mu N):
// a forward recursion u_i = x_i + r_k u_{i-1} followed by a backward one
// v_i = u_i + r_k v_{i+1}, y_i = s_k v_i.  (This is the paper's remark that
// with constant coefficients the factorisation is computed once; here the
// factors are scalar.)
//
// Each thread takes one column and a run of kRecRows rows.  Both recursions
// start R rows outside the run with a zero state; the influence of the
// missing state decays as r_k^R, and R (a template bucket chosen by the host)
// makes r_0^R, the slowest decay, smaller than 2^-27.  Indices wrap modulo M,
// so the periodic solve is reproduced for any M, including M < R.  Threads
// read rows other threads write, so the result goes to a second buffer.
//
// Column 0 packs the real DC and Nyquist columns of the row transforms as
// X_0 + i X_{N/2}; its real and imaginary parts take their own r and s.
#include <cmath>

#include "sr_internal.h"

namespace srk {

// MIRROR: the column is read as its even extension of length 2M (rows
// 0..M-1, then M-1..0), whose periodic solve is the solve with reflective
// ends (the Neumann reading of Eq. (27)); only rows 0..M-1 are written.
template <int R, bool MIRROR>
__global__ void __launch_bounds__(32 * kRecChunks) k_colsolve_rec(const ColArgs a) {
  constexpr int TR = kRecRows;
  const int L = a.geo.L, M = a.geo.M;
  const int Mv = MIRROR ? 2 * M : M;  // length of the periodic sequence
  auto at = [M](int n) { return (MIRROR && n >= M) ? 2 * M - 1 - n : n; };
  const int k = blockIdx.x * 32 + threadIdx.x;
  const int i0 = (blockIdx.y * kRecChunks + threadIdx.y) * TR;
  pdl_wait();
  pdl_trigger();
  if (k >= L || i0 >= M) return;
  const float4 p = __ldg(a.rec + k);
  const float rr = p.x, sr = p.y, ri = p.z, si = p.w;
  const float2* __restrict__ src = a.X + k;
  float2* __restrict__ dst = a.Xout + k;
  int row = i0 - R;
  while (row < 0) row += Mv;
  // forward recursion: R rows of warm-up, then the run and the R rows after it
  float ux = 0.f, uy = 0.f;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const float2 x = src[(size_t)at(row) * L];
    ux = fmaf(rr, ux, x.x);
    uy = fmaf(ri, uy, x.y);
    row = row + 1 == Mv ? 0 : row + 1;
  }
  float2 b[TR + R];
#pragma unroll
  for (int j = 0; j < TR + R; ++j) {
    b[j] = src[(size_t)at(row) * L];
    row = row + 1 == Mv ? 0 : row + 1;
  }
#pragma unroll
  for (int j = 0; j < TR + R; ++j) {
    ux = fmaf(rr, ux, b[j].x);
    uy = fmaf(ri, uy, b[j].y);
    b[j] = make_float2(ux, uy);
  }
  // backward recursion: R rows of warm-up after the run, then the run
  float vx = 0.f, vy = 0.f;
#pragma unroll
  for (int j = TR + R - 1; j >= TR; --j) {
    vx = fmaf(rr, vx, b[j].x);
    vy = fmaf(ri, vy, b[j].y);
  }
#pragma unroll
  for (int j = TR - 1; j >= 0; --j) {
    vx = fmaf(rr, vx, b[j].x);
    vy = fmaf(ri, vy, b[j].y);
    b[j] = make_float2(sr * vx, si * vy);
  }
#pragma unroll
  for (int j = 0; j < TR; ++j)
    if (i0 + j < M) dst[(size_t)(i0 + j) * L] = b[j];
}

namespace {
constexpr int kRecBuckets[] = {8, 12, 16, 20, 24, 32, 40, 48, 64};
}

int colsolve_rec_radius(double r_max) {
  if (!(r_max >= 0.0) || r_max >= 1.0) return 0;
  // smallest R with r_max^R <= 2^-27
  const double need = r_max <= 0.0 ? 1.0 : std::ceil(-27.0 * std::log(2.0) / std::log(r_max));
  for (int R : kRecBuckets)
    if (R >= need) return R;
  return 0;
}

cudaError_t launch_colsolve_rec(const ColArgs& a, cudaStream_t s) {
  const dim3 block(32, kRecChunks);
  const dim3 grid((a.geo.L + 31) / 32, (a.geo.M + kRecRows * kRecChunks - 1) / (kRecRows * kRecChunks));
  switch (a.rec_R) {
#define SR_REC(r)                                                                \
  case r:                                                                        \
    return a.mirror ? launch_k(k_colsolve_rec<r, true>, grid, block, 0, s, a)    \
                    : launch_k(k_colsolve_rec<r, false>, grid, block, 0, s, a);
    SR_REC(8) SR_REC(12) SR_REC(16) SR_REC(20) SR_REC(24) SR_REC(32) SR_REC(40) SR_REC(48)
    SR_REC(64)
#undef SR_REC
  }
  return cudaErrorInvalidValue;
}

__global__ void k_mirror_rows(const float* __restrict__ in, float* __restrict__ out, Geo geo) {
  const int i = blockIdx.y, N = geo.N;
  pdl_wait();
  pdl_trigger();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 2 * N; j += gridDim.x * blockDim.x)
    out[(size_t)i * 2 * N + j] = in[(size_t)i * N + (j < N ? j : 2 * N - 1 - j)];
}

__global__ void k_add_half(const float* __restrict__ psi, const float* __restrict__ T,
                           float* __restrict__ out, Geo geo) {
  const int i = blockIdx.y, N = geo.N;
  pdl_wait();
  pdl_trigger();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    const size_t o = (size_t)i * N + j;
    out[o] = (psi ? psi[o] : 0.f) + T[(size_t)i * 2 * N + j];
  }
}

cudaError_t launch_mirror_rows(const float* in, float* out, const Geo& geo, cudaStream_t s) {
  const int bx = (2 * geo.N + 255) / 256;
  return launch_k(k_mirror_rows, dim3(bx, geo.M), dim3(256), 0, s, in, out, geo);
}

cudaError_t launch_add_half(const float* psi, const float* T, float* out, const Geo& geo,
                            cudaStream_t s) {
  const int bx = (geo.N + 255) / 256;
  return launch_k(k_add_half, dim3(bx, geo.M), dim3(256), 0, s, psi, T, out, geo);
}

}  // namespace srk
