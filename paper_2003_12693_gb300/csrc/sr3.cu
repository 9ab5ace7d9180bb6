// The Split Bregman SR iteration on volumes (the 3-D use of Fig. 6): Alg. 1
// with a third axis everywhere, under the 2-D readings -- periodic forward
// differences (Eq. (35)) and backward divergence (Eq. (36)); the window sum
// of Eq. (38) over the cube |p|, |q|, |r| <= R with the separable weight
// exp(-(p^2 + q^2 + r^2) / d^2), terms outside the volume dropped; Eq. (37)
// with the 3-D Laplacian; Eqs. (41), (42), (40), (23) on 3-vectors.
//
// Volumes are Z x M x N float32, row-major (z slowest).  The solve
// (1 - tau mu Lap) delta = G (increment form, phi = psi + delta) transforms
// the two inner axes with complex FFTs (register Stockham stages of
// sr_dft.cuh; N and M powers of two in [16, 1024]) and solves along z, for
// each pair of frequencies (l, k), the periodic tridiagonal system
//     c y_z - tau mu (y_{z-1} + y_{z+1}) = x_z,
//     c = 1 + 2 tau mu + tau mu (4 sin^2(pi k / N) + 4 sin^2(pi l / M)),
// by its factorisation into a forward and a backward first-order recursion
// (the same as the 2-D column pass, k_colsolve_rec); Z is any size.
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "sr.h"
#include "sr3.h"
#include "sr_dft.cuh"
#include "sr_internal.h"

namespace srk {
namespace vol {

using namespace srk::cdft;

struct Vol {
  int Z, M, N;
};

struct Model3 {
  float alpha, beta, gamma, mu, tau, eps, l;
  int R;
  float kw[2 * kMaxR + 1];
};

// Eqs. (5), (6), (11), (28), (29), written out in FP32
__device__ __forceinline__ float H_(float x, float e) {
  if (x > e) return 1.f;
  if (x < -e) return 0.f;
  return 0.5f * (1.f + x / e + sinpif(x / e) * 0.31830988618379067f);
}
__device__ __forceinline__ float D_(float x, float e) {
  return fabsf(x) <= e ? 0.5f / e * (1.f + cospif(x / e)) : 0.f;
}
__device__ __forceinline__ float Dp_(float x, float e) {
  return fabsf(x) <= e ? -1.5707963267948966f / (e * e) * sinpif(x / e) : 0.f;
}
__device__ __forceinline__ float h_(float x, const Model3& m) {
  return H_(x + m.l, m.eps) * (1.f - H_(x - m.l, m.eps));
}
__device__ __forceinline__ float hp_(float x, const Model3& m) {
  return D_(x + m.l, m.eps) * (1.f - H_(x - m.l, m.eps)) - H_(x + m.l, m.eps) * D_(x - m.l, m.eps);
}

__device__ __forceinline__ size_t at(const Vol& v, int z, int i, int j) {
  return ((size_t)z * v.M + i) * v.N + j;
}

#define SR3_LOOP(v)                                                            \
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x,               \
              n_ = (size_t)(v).Z * (v).M * (v).N;                              \
       q < n_; q += (size_t)gridDim.x * blockDim.x)

__device__ __forceinline__ void coords(const Vol& v, size_t q, int& z, int& i, int& j) {
  j = (int)(q % v.N);
  const size_t r = q / v.N;
  i = (int)(r % v.M);
  z = (int)(r / v.M);
}

// u_c = h(phi) w_c
__global__ void k3_band_u(const float* __restrict__ phi, const float* __restrict__ w1,
                          const float* __restrict__ w2, const float* __restrict__ w3,
                          float* __restrict__ u1, float* __restrict__ u2, float* __restrict__ u3,
                          Vol v, Model3 m) {
  SR3_LOOP(v) {
    const float h = h_(phi[q], m);
    u1[q] = h * w1[q];
    u2[q] = h * w2[q];
    u3[q] = h * w3[q];
  }
}

// one axis of the separable window sum, terms outside the volume dropped
template <int AXIS>
__global__ void k3_conv(const float* __restrict__ a1, const float* __restrict__ a2,
                        const float* __restrict__ a3, float* __restrict__ o1,
                        float* __restrict__ o2, float* __restrict__ o3, Vol v, Model3 m) {
  const int len = AXIS == 0 ? v.Z : AXIS == 1 ? v.M : v.N;
  const size_t step = AXIS == 0 ? (size_t)v.M * v.N : AXIS == 1 ? (size_t)v.N : 1;
  SR3_LOOP(v) {
    int z, i, j;
    coords(v, q, z, i, j);
    const int pos = AXIS == 0 ? z : AXIS == 1 ? i : j;
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int t = -m.R; t <= m.R; ++t) {
      const int p = pos + t;
      if (p < 0 || p >= len) continue;
      const size_t o = q + (ptrdiff_t)t * (ptrdiff_t)step;
      const float k = m.kw[t + m.R];
      s1 = fmaf(k, a1[o], s1);
      s2 = fmaf(k, a2[o], s2);
      s3 = fmaf(k, a3[o], s3);
    }
    o1[q] = s1;
    o2[q] = s2;
    o3[q] = s3;
  }
}

// G = tau [ -gamma g |w| delta'(psi) + alpha g delta(psi) + 2 beta h'(psi) (w . v)
//           + mu (div(b - w) + Lap psi) ]   (Eq. (37), increment form)
__global__ void k3_rhs(const float* __restrict__ psi, const float* __restrict__ g,
                       const float* __restrict__ w1, const float* __restrict__ w2,
                       const float* __restrict__ w3, const float* __restrict__ b1,
                       const float* __restrict__ b2, const float* __restrict__ b3,
                       const float* __restrict__ v1, const float* __restrict__ v2,
                       const float* __restrict__ v3, float* __restrict__ G, Vol v, Model3 m) {
  SR3_LOOP(v) {
    int z, i, j;
    coords(v, q, z, i, j);
    const size_t zm = at(v, z == 0 ? v.Z - 1 : z - 1, i, j), zp = at(v, z == v.Z - 1 ? 0 : z + 1, i, j);
    const size_t im = at(v, z, i == 0 ? v.M - 1 : i - 1, j), ip = at(v, z, i == v.M - 1 ? 0 : i + 1, j);
    const size_t jm = at(v, z, i, j == 0 ? v.N - 1 : j - 1), jp = at(v, z, i, j == v.N - 1 ? 0 : j + 1);
    const float x = psi[q];
    const float lap = (psi[zm] + psi[zp]) + (psi[im] + psi[ip]) + (psi[jm] + psi[jp]) - 6.f * x;
    const float dv = ((b1[q] - w1[q]) - (b1[zm] - w1[zm])) + ((b2[q] - w2[q]) - (b2[im] - w2[im])) +
                     ((b3[q] - w3[q]) - (b3[jm] - w3[jm]));
    float f = m.mu * (dv + lap);
    const float wn = sqrtf(w1[q] * w1[q] + w2[q] * w2[q] + w3[q] * w3[q]);
    const float gg = g[q];
    f += -m.gamma * gg * wn * Dp_(x, m.eps) + m.alpha * gg * D_(x, m.eps) +
         2.f * m.beta * hp_(x, m) * (w1[q] * v1[q] + w2[q] * v2[q] + w3[q] * v3[q]);
    G[q] = m.tau * f;
  }
}

__global__ void k3_to_complex(const float* __restrict__ G, float2* __restrict__ C, Vol v) {
  SR3_LOOP(v) C[q] = make_float2(G[q], 0.f);
}

__global__ void k3_add_real(const float* __restrict__ psi, const float2* __restrict__ C,
                            float* __restrict__ out, Vol v) {
  SR3_LOOP(v) out[q] = (psi ? psi[q] : 0.f) + C[q].x;
}

// Complex FFT of length L = 2^LOGL along lines: line n starts at
// (n / pdiv) * outer + (n % pdiv) * inner, its elements es apart.  CB lines per
// CTA; UFAST puts a line's threads next to each other (lines of contiguous
// elements), else the CB lines' threads interleave (lines side by side).
template <int LOGL, int CB, bool INV, bool UFAST>
__global__ void __launch_bounds__(CB*(1 << (LOGL - 4)))
    k3_lines(float2* __restrict__ D, int nlines, int pdiv, long long outer, long long inner,
             long long es, const float2* __restrict__ tws) {
  constexpr int E = 16, L = 1 << LOGL, TP = L / E;
  extern __shared__ __align__(16) float2 sm3[];
  float2* stw = sm3 + CB * (L + L / 16);
  stage_table<TwPlan<LOGL, 4>::TOTAL>(stw, tws);
  __syncthreads();
  const int tid = threadIdx.x;
  const int c = UFAST ? tid / TP : tid % CB, u = UFAST ? tid % TP : tid / CB;
  const int line = blockIdx.x * CB + c;
  const bool live = line < nlines;
  const long long base = live ? (long long)(line / pdiv) * outer + (long long)(line % pdiv) * inner : 0;
  float2 x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = live ? D[base + (long long)(u + m * TP) * es] : make_float2(0.f, 0.f);
  // exchange layout: a line's values contiguous (UFAST) or the CB lines'
  // values interleaved, so that a warp's accesses hit distinct banks
  if constexpr (UFAST)
    stages<LOGL, 4, 0, INV, 1>(x, sm3 + c * (L + L / 16), u, stw);
  else
    stages<LOGL, 4, 0, INV, CB>(x, sm3 + c, u, stw);
  if (live) {
#pragma unroll
    for (int m = 0; m < E; ++m) D[base + (long long)(u + m * TP) * es] = x[m];
  }
}

// recursion along z for every (l, k): threads on adjacent (l, k) (coalesced),
// each a run of kRecRows planes, warm-up R planes on both sides (mod Z)
template <int R>
__global__ void __launch_bounds__(32 * kRecChunks)
    k3_zrec(const float2* __restrict__ C, float2* __restrict__ Co, Vol v, float a, float inv_mn) {
  constexpr int TR = kRecRows;
  const int MN = v.M * v.N;
  const int col = blockIdx.x * 32 + threadIdx.x;
  const int z0 = (blockIdx.y * kRecChunks + threadIdx.y) * TR;
  if (col >= MN || z0 >= v.Z) return;
  const int l = col / v.N, k = col - l * v.N;
  const float sk = sinpif((float)k / (float)v.N), sl = sinpif((float)l / (float)v.M);
  const float c = 1.f + 2.f * a + a * 4.f * (sk * sk + sl * sl);
  const float r = 2.f * a / (c + sqrtf(c * c - 4.f * a * a));
  const float s = r / a * inv_mn;
  const float2* src = C + col;
  int zz = z0 - R;
  while (zz < 0) zz += v.Z;
  float ux = 0.f, uy = 0.f;
#pragma unroll 4
  for (int t = 0; t < R; ++t) {
    const float2 x = src[(size_t)zz * MN];
    ux = fmaf(r, ux, x.x);
    uy = fmaf(r, uy, x.y);
    zz = zz + 1 == v.Z ? 0 : zz + 1;
  }
  float2 b[TR + R];
#pragma unroll
  for (int t = 0; t < TR + R; ++t) {
    b[t] = src[(size_t)zz * MN];
    zz = zz + 1 == v.Z ? 0 : zz + 1;
  }
#pragma unroll
  for (int t = 0; t < TR + R; ++t) {
    ux = fmaf(r, ux, b[t].x);
    uy = fmaf(r, uy, b[t].y);
    b[t] = make_float2(ux, uy);
  }
  float vx = 0.f, vy = 0.f;
#pragma unroll
  for (int t = TR + R - 1; t >= TR; --t) {
    vx = fmaf(r, vx, b[t].x);
    vy = fmaf(r, vy, b[t].y);
  }
#pragma unroll
  for (int t = TR - 1; t >= 0; --t) {
    vx = fmaf(r, vx, b[t].x);
    vy = fmaf(r, vy, b[t].y);
    b[t] = make_float2(s * vx, s * vy);
  }
#pragma unroll
  for (int t = 0; t < TR; ++t)
    if (z0 + t < v.Z) Co[(size_t)(z0 + t) * MN + col] = b[t];
}

// Eqs. (41), (42), (40), (23) on 3-vectors: B = grad phi + b + (2 beta / mu) h v,
// t = (gamma / mu) g delta(phi); w = B / |B| if |B| > t else 0; b' = b + grad phi - w
__global__ void k3_wb(const float* __restrict__ phi, const float* __restrict__ g,
                      const float* __restrict__ b1, const float* __restrict__ b2,
                      const float* __restrict__ b3, const float* __restrict__ v1,
                      const float* __restrict__ v2, const float* __restrict__ v3,
                      float* __restrict__ w1o, float* __restrict__ w2o, float* __restrict__ w3o,
                      float* __restrict__ b1o, float* __restrict__ b2o, float* __restrict__ b3o,
                      Vol v, Model3 m) {
  SR3_LOOP(v) {
    int z, i, j;
    coords(v, q, z, i, j);
    const float x = phi[q];
    const float d1 = phi[at(v, z == v.Z - 1 ? 0 : z + 1, i, j)] - x;
    const float d2 = phi[at(v, z, i == v.M - 1 ? 0 : i + 1, j)] - x;
    const float d3 = phi[at(v, z, i, j == v.N - 1 ? 0 : j + 1)] - x;
    const float hb = h_(x, m) * (2.f * m.beta / m.mu);
    const float B1 = d1 + b1[q] + hb * v1[q], B2 = d2 + b2[q] + hb * v2[q], B3 = d3 + b3[q] + hb * v3[q];
    const float t = m.gamma / m.mu * g[q] * D_(x, m.eps);
    const float nB = sqrtf(B1 * B1 + B2 * B2 + B3 * B3);
    float W1 = 0.f, W2 = 0.f, W3 = 0.f;
    if (nB > t && nB > 0.f) {
      W1 = B1 / nB;
      W2 = B2 / nB;
      W3 = B3 / nB;
    }
    const float c1 = b1[q] + d1 - W1, c2 = b2[q] + d2 - W2, c3 = b3[q] + d3 - W3;
    w1o[q] = W1;
    w2o[q] = W2;
    w3o[q] = W3;
    b1o[q] = c1;
    b2o[q] = c2;
    b3o[q] = c3;
  }
}

// Alg. 1 initialisation: w = grad phi (forward, periodic), b = 0
__global__ void k3_init(const float* __restrict__ phi, float* __restrict__ w1,
                        float* __restrict__ w2, float* __restrict__ w3, float* __restrict__ b1,
                        float* __restrict__ b2, float* __restrict__ b3, Vol v) {
  SR3_LOOP(v) {
    int z, i, j;
    coords(v, q, z, i, j);
    const float x = phi[q];
    w1[q] = phi[at(v, z == v.Z - 1 ? 0 : z + 1, i, j)] - x;
    w2[q] = phi[at(v, z, i == v.M - 1 ? 0 : i + 1, j)] - x;
    w3[q] = phi[at(v, z, i, j == v.N - 1 ? 0 : j + 1)] - x;
    b1[q] = b2[q] = b3[q] = 0.f;
  }
}

}  // namespace vol
}  // namespace srk

using namespace srk::vol;

struct sr3_ctx {
  Vol v{};
  Model3 m{};
  sr_params prm{};
  cudaStream_t stream = nullptr;
  int nsm = 0;
  int zrec_R = 0;
  float* phi = nullptr;
  float* psi = nullptr;
  float* w[3] = {nullptr, nullptr, nullptr};
  float* b[3] = {nullptr, nullptr, nullptr};
  float* wn[3] = {nullptr, nullptr, nullptr};  // w^{k+1}, b^{k+1} before the swap
  float* bn[3] = {nullptr, nullptr, nullptr};
  float* g = nullptr;
  float* G = nullptr;
  float* u[3] = {nullptr, nullptr, nullptr};
  float* t[3] = {nullptr, nullptr, nullptr};
  float* vs[3] = {nullptr, nullptr, nullptr};
  float2* C = nullptr;
  float2* C2 = nullptr;
  float2* twsN = nullptr;
  float2* twsM = nullptr;
  long long launches = 0;
};

namespace {

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

dim3 grid_for(const sr3_ctx* c) {
  const size_t n = (size_t)c->v.Z * c->v.M * c->v.N;
  const size_t blocks = (n + 255) / 256;
  const size_t cap = (size_t)c->nsm * 8;
  return dim3((unsigned)(blocks < cap ? blocks : cap));
}

#define SR3_CUDA(call)                                             \
  do {                                                             \
    const cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess)                                         \
      return e_ == cudaErrorMemoryAllocation ? SR_ENOMEM : SR_ECUDA; \
  } while (0)

template <int LOGL, bool INV>
cudaError_t lines_go(sr3_ctx* c, float2* D, int nlines, int pdiv, long long outer, long long inner,
                     long long es, bool ufast, const float2* tws) {
  constexpr int L = 1 << LOGL, TP = L / 16;
  const size_t table = (size_t)TwPlan<LOGL, 4>::TOTAL * sizeof(float2);
  if (ufast) {
    constexpr int CB = (4096 >> LOGL) > 1 ? (4096 >> LOGL) : 1;
    const size_t smem = (size_t)CB * (L + L / 16) * sizeof(float2) + table;
    cudaError_t e = cudaFuncSetAttribute(k3_lines<LOGL, CB, INV, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k3_lines<LOGL, CB, INV, true><<<(nlines + CB - 1) / CB, CB * TP, smem, c->stream>>>(
        D, nlines, pdiv, outer, inner, es, tws);
  } else {
    constexpr int CB = 8;
    const size_t smem = (size_t)CB * (L + L / 16) * sizeof(float2) + table;
    cudaError_t e = cudaFuncSetAttribute(k3_lines<LOGL, CB, INV, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k3_lines<LOGL, CB, INV, false><<<(nlines + CB - 1) / CB, CB * TP, smem, c->stream>>>(
        D, nlines, pdiv, outer, inner, es, tws);
  }
  c->launches += 1;
  return cudaGetLastError();
}

template <bool INV>
cudaError_t lines(sr3_ctx* c, float2* D, int len, int nlines, int pdiv, long long outer,
                  long long inner, long long es, bool ufast, const float2* tws) {
  switch (len) {
#define SR3_L(lg) \
  case (1 << lg): return lines_go<lg, INV>(c, D, nlines, pdiv, outer, inner, es, ufast, tws);
    SR3_L(4) SR3_L(5) SR3_L(6) SR3_L(7) SR3_L(8) SR3_L(9) SR3_L(10)
#undef SR3_L
  }
  return cudaErrorInvalidValue;
}

cudaError_t zrec(sr3_ctx* c, const float2* C, float2* Co) {
  const int MN = c->v.M * c->v.N;
  const dim3 block(32, srk::kRecChunks);
  const dim3 grid((MN + 31) / 32, (c->v.Z + srk::kRecRows * srk::kRecChunks - 1) /
                                      (srk::kRecRows * srk::kRecChunks));
  const float a = c->prm.tau * c->prm.mu;
  const float inv_mn = 1.f / ((float)c->v.M * (float)c->v.N);
  switch (c->zrec_R) {
#define SR3_R(r) \
  case r: k3_zrec<r><<<grid, block, 0, c->stream>>>(C, Co, c->v, a, inv_mn); break;
    SR3_R(8) SR3_R(12) SR3_R(16) SR3_R(20) SR3_R(24) SR3_R(32) SR3_R(40) SR3_R(48) SR3_R(64)
#undef SR3_R
    default: return cudaErrorInvalidValue;
  }
  c->launches += 1;
  return cudaGetLastError();
}

// (1 - tau mu Lap) delta = G: out = psi + delta (psi may be null)
sr_status solve(sr3_ctx* c, const float* G, const float* psi, float* out) {
  const Vol& v = c->v;
  const dim3 gr = grid_for(c);
  k3_to_complex<<<gr, 256, 0, c->stream>>>(G, c->C, v);
  SR3_CUDA(cudaGetLastError());
  const long long MN = (long long)v.M * v.N;
  // rows (axis N): lines z*M + i, contiguous
  SR3_CUDA(lines<false>(c, c->C, v.N, v.Z * v.M, 1, v.N, 0, 1, true, c->twsN));
  // columns (axis M): lines (z, j), elements N apart
  SR3_CUDA(lines<false>(c, c->C, v.M, v.Z * v.N, v.N, MN, 1, v.N, false, c->twsM));
  SR3_CUDA(zrec(c, c->C, c->C2));
  SR3_CUDA(lines<true>(c, c->C2, v.M, v.Z * v.N, v.N, MN, 1, v.N, false, c->twsM));
  SR3_CUDA(lines<true>(c, c->C2, v.N, v.Z * v.M, 1, v.N, 0, 1, true, c->twsN));
  k3_add_real<<<gr, 256, 0, c->stream>>>(psi, c->C2, out, v);
  SR3_CUDA(cudaGetLastError());
  c->launches += 2;
  return SR_OK;
}

// v = window sum of h(phi) w over the cube (Eq. (38)), into c->vs
sr_status window(sr3_ctx* c, const float* phi, float* const w[3]) {
  const dim3 gr = grid_for(c);
  k3_band_u<<<gr, 256, 0, c->stream>>>(phi, w[0], w[1], w[2], c->u[0], c->u[1], c->u[2], c->v, c->m);
  k3_conv<2><<<gr, 256, 0, c->stream>>>(c->u[0], c->u[1], c->u[2], c->t[0], c->t[1], c->t[2], c->v, c->m);
  k3_conv<1><<<gr, 256, 0, c->stream>>>(c->t[0], c->t[1], c->t[2], c->u[0], c->u[1], c->u[2], c->v, c->m);
  k3_conv<0><<<gr, 256, 0, c->stream>>>(c->u[0], c->u[1], c->u[2], c->vs[0], c->vs[1], c->vs[2], c->v, c->m);
  c->launches += 4;
  SR3_CUDA(cudaGetLastError());
  return SR_OK;
}

sr_status phi_step(sr3_ctx* c, const float* psi_in, float* const w[3], float* const b[3],
                   float* psi_out) {
  sr_status st = window(c, psi_in, w);
  if (st != SR_OK) return st;
  k3_rhs<<<grid_for(c), 256, 0, c->stream>>>(psi_in, c->g, w[0], w[1], w[2], b[0], b[1], b[2],
                                             c->vs[0], c->vs[1], c->vs[2], c->G, c->v, c->m);
  SR3_CUDA(cudaGetLastError());
  c->launches += 1;
  return solve(c, c->G, psi_in, psi_out);
}

sr_status wb_update(sr3_ctx* c, const float* phi1, float* const w[3], float* const b[3],
                    float* const wo[3], float* const bo[3]) {
  sr_status st = window(c, phi1, w);
  if (st != SR_OK) return st;
  k3_wb<<<grid_for(c), 256, 0, c->stream>>>(phi1, c->g, b[0], b[1], b[2], c->vs[0], c->vs[1],
                                            c->vs[2], wo[0], wo[1], wo[2], bo[0], bo[1], bo[2],
                                            c->v, c->m);
  SR3_CUDA(cudaGetLastError());
  c->launches += 1;
  return SR_OK;
}

}  // namespace

extern "C" {

sr_status sr3_create(int Z, int M, int N, const sr_params* p, void* cuda_stream, sr3_ctx** out) {
  if (!out || !p) return SR_EINVAL;
  *out = nullptr;
  if (Z < 1 || M < 1 || N < 1) return SR_EINVAL;
  const float vals[] = {p->alpha, p->beta, p->gamma, p->mu, p->tau, p->eps, p->band_l, p->d};
  for (float x : vals)
    if (!std::isfinite(x)) return SR_EINVAL;
  if (p->mu <= 0.f || p->tau <= 0.f || p->eps <= 0.f || p->band_l < 0.f || p->inner_S < 1)
    return SR_EINVAL;
  if (p->win_radius < 0 || p->win_radius > srk::kMaxR || (p->win_radius > 0 && p->d <= 0.f))
    return SR_EINVAL;
  if (!pow2(M) || !pow2(N) || M < 16 || N < 16 || M > 1024 || N > 1024 || Z > 4096)
    return SR_EUNSUPPORTED;
  const double a = (double)p->tau * (double)p->mu;
  const double c0 = 1.0 + 2.0 * a;
  const int R = srk::colsolve_rec_radius(2.0 * a / (c0 + std::sqrt(c0 * c0 - 4.0 * a * a)));
  if (R <= 0) return SR_EUNSUPPORTED;
  sr3_ctx* c = new (std::nothrow) sr3_ctx();
  if (!c) return SR_ENOMEM;
  c->v = Vol{Z, M, N};
  c->prm = *p;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  c->zrec_R = R;
  Model3& m = c->m;
  m.alpha = p->alpha;
  m.beta = p->beta;
  m.gamma = p->gamma;
  m.mu = p->mu;
  m.tau = p->tau;
  m.eps = p->eps;
  m.l = p->band_l;
  m.R = p->win_radius;
  for (int t = -m.R; t <= m.R; ++t)
    m.kw[t + m.R] = (float)std::exp(-(double)(t * t) / ((double)p->d * (double)p->d));
  auto bail = [&](sr_status s) {
    sr3_destroy(c);
    return s;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return bail(SR_ECUDA);
  const size_t n = (size_t)Z * M * N;
  std::vector<float**> planes = {&c->phi, &c->psi, &c->g, &c->G};
  for (int k = 0; k < 3; ++k)
    for (float** pl : {&c->w[k], &c->b[k], &c->wn[k], &c->bn[k], &c->u[k], &c->t[k], &c->vs[k]})
      planes.push_back(pl);
  for (float** pl : planes)
    if (cudaMalloc((void**)pl, n * sizeof(float)) != cudaSuccess) return bail(SR_ENOMEM);
  if (cudaMalloc((void**)&c->C, n * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->C2, n * sizeof(float2)) != cudaSuccess)
    return bail(SR_ENOMEM);
  const std::vector<float2> tN = srk::stage_twiddle_table(N, 4), tM = srk::stage_twiddle_table(M, 4);
  if (cudaMalloc((void**)&c->twsN, tN.size() * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&c->twsM, tM.size() * sizeof(float2)) != cudaSuccess)
    return bail(SR_ENOMEM);
  if (cudaMemcpy(c->twsN, tN.data(), tN.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->twsM, tM.data(), tM.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(SR_ECUDA);
  // g = 1 until sr3_set_g
  std::vector<float> ones(n, 1.f);
  if (cudaMemcpy(c->g, ones.data(), n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(SR_ECUDA);
  *out = c;
  return SR_OK;
}

void sr3_destroy(sr3_ctx* c) {
  if (!c) return;
  std::vector<void*> bufs = {c->phi, c->psi, c->g, c->G, c->C, c->C2, c->twsN, c->twsM};
  for (int k = 0; k < 3; ++k)
    for (void* p : {(void*)c->w[k], (void*)c->b[k], (void*)c->wn[k], (void*)c->bn[k],
                    (void*)c->u[k], (void*)c->t[k], (void*)c->vs[k]})
      bufs.push_back(p);
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete c;
}

static sr_status copy_in(sr3_ctx* c, float* dst, const float* src) {
  if (!src) return SR_EINVAL;
  const size_t n = (size_t)c->v.Z * c->v.M * c->v.N;
  SR3_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  return SR_OK;
}

sr_status sr3_set_g(sr3_ctx* c, const float* g) {
  if (!c) return SR_EINVAL;
  return copy_in(c, c->g, g);
}

sr_status sr3_set_phi(sr3_ctx* c, const float* phi0) {
  if (!c) return SR_EINVAL;
  sr_status st = copy_in(c, c->phi, phi0);
  if (st != SR_OK) return st;
  k3_init<<<grid_for(c), 256, 0, c->stream>>>(c->phi, c->w[0], c->w[1], c->w[2], c->b[0], c->b[1],
                                              c->b[2], c->v);
  c->launches += 1;
  SR3_CUDA(cudaGetLastError());
  return SR_OK;
}

sr_status sr3_set_state(sr3_ctx* c, const float* phi, const float* const w[3], const float* const b[3]) {
  if (!c || !w || !b) return SR_EINVAL;
  sr_status st = copy_in(c, c->phi, phi);
  for (int k = 0; k < 3 && st == SR_OK; ++k) {
    st = copy_in(c, c->w[k], w[k]);
    if (st == SR_OK) st = copy_in(c, c->b[k], b[k]);
  }
  return st;
}

sr_status sr3_get_state(sr3_ctx* c, float* phi, float* const w[3], float* const b[3]) {
  if (!c || !phi || !w || !b) return SR_EINVAL;
  const size_t bytes = (size_t)c->v.Z * c->v.M * c->v.N * sizeof(float);
  SR3_CUDA(cudaMemcpyAsync(phi, c->phi, bytes, cudaMemcpyDeviceToDevice, c->stream));
  for (int k = 0; k < 3; ++k) {
    if (!w[k] || !b[k]) return SR_EINVAL;
    SR3_CUDA(cudaMemcpyAsync(w[k], c->w[k], bytes, cudaMemcpyDeviceToDevice, c->stream));
    SR3_CUDA(cudaMemcpyAsync(b[k], c->b[k], bytes, cudaMemcpyDeviceToDevice, c->stream));
  }
  return SR_OK;
}

sr_status sr3_fft_solve(sr3_ctx* c, const float* rhs, float* out) {
  if (!c || !rhs || !out) return SR_EINVAL;
  return solve(c, rhs, nullptr, out);
}

sr_status sr3_window_sum(sr3_ctx* c, const float* phi, const float* const w[3], float* const v[3]) {
  if (!c || !phi || !w || !v) return SR_EINVAL;
  float* ww[3] = {const_cast<float*>(w[0]), const_cast<float*>(w[1]), const_cast<float*>(w[2])};
  sr_status st = window(c, phi, ww);
  if (st != SR_OK) return st;
  const size_t bytes = (size_t)c->v.Z * c->v.M * c->v.N * sizeof(float);
  for (int k = 0; k < 3; ++k)
    SR3_CUDA(cudaMemcpyAsync(v[k], c->vs[k], bytes, cudaMemcpyDeviceToDevice, c->stream));
  return SR_OK;
}

sr_status sr3_phi_step(sr3_ctx* c, const float* psi_in, const float* const w[3],
                       const float* const b[3], float* psi_out) {
  if (!c || !psi_in || !w || !b || !psi_out) return SR_EINVAL;
  float* ww[3] = {const_cast<float*>(w[0]), const_cast<float*>(w[1]), const_cast<float*>(w[2])};
  float* bb[3] = {const_cast<float*>(b[0]), const_cast<float*>(b[1]), const_cast<float*>(b[2])};
  return phi_step(c, psi_in, ww, bb, psi_out);
}

sr_status sr3_w_b_update(sr3_ctx* c, const float* phi1, const float* const w[3],
                         const float* const b[3], float* const wo[3], float* const bo[3]) {
  if (!c || !phi1 || !w || !b || !wo || !bo) return SR_EINVAL;
  float* ww[3] = {const_cast<float*>(w[0]), const_cast<float*>(w[1]), const_cast<float*>(w[2])};
  float* bb[3] = {const_cast<float*>(b[0]), const_cast<float*>(b[1]), const_cast<float*>(b[2])};
  return wb_update(c, phi1, ww, bb, wo, bo);
}

sr_status sr3_iterate(sr3_ctx* c, int max_outer) {
  if (!c || max_outer < 0) return SR_EINVAL;
  const size_t bytes = (size_t)c->v.Z * c->v.M * c->v.N * sizeof(float);
  for (int k = 0; k < max_outer; ++k) {
    const float* in = c->phi;
    for (int s = 0; s < c->prm.inner_S; ++s) {
      sr_status st = phi_step(c, in, c->w, c->b, c->psi);
      if (st != SR_OK) return st;
      in = c->psi;
    }
    sr_status st = wb_update(c, c->psi, c->w, c->b, c->wn, c->bn);
    if (st != SR_OK) return st;
    for (int q = 0; q < 3; ++q) {
      std::swap(c->w[q], c->wn[q]);
      std::swap(c->b[q], c->bn[q]);
    }
    SR3_CUDA(cudaMemcpyAsync(c->phi, c->psi, bytes, cudaMemcpyDeviceToDevice, c->stream));
  }
  return SR_OK;
}

long long sr3_kernel_launches(const sr3_ctx* c) { return c ? c->launches : -1; }

}  // extern "C"
