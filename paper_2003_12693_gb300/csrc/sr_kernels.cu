// sm_103a kernels of the Split Bregman self-repelling snake.
//
// One outer iteration of Alg. 1 is, per inner step s (Eq. (37)):
//   k_prep     repulsion window sum (Sec. 4) and the right-hand side, 2-D tiles
//   k_rowfwd   row R2C FFT of the right-hand side
//   k_colsolve column FFT, divide by the symbol of Eq. (32), inverse column FFT
//   k_rowinv   row C2R FFT and phi update
// (k_rowfwd can also build the right-hand side itself from row blocks; the
// allocation-free single step uses that form.)
// and after the inner loop:
//   k_wb_update repulsion window sum of Eq. (41), soft threshold (42),
//               projection (40), Bregman update (23)
//
// The phi solve uses the increment form of Eq. (30): with L = 1 - tau mu Lap,
//   L^{-1} F = psi + L^{-1} (F - L psi) = psi + L^{-1} [tau (force + mu Lap psi)],
// which is the same solution in exact arithmetic but rounds relative to the
// increment instead of |psi| (|phi| reaches 10^3 on large images).
//
// All kernels are memory-bound stencils, window sums and FFT passes: FP32
// CUDA-core arithmetic, shared-memory staging, coalesced global access.
#include <math.h>

#include <algorithm>

#include "sr_internal.h"
#include "sr_tma.cuh"

// every supported repulsion window half width R
#define SR_FOR_R(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

namespace srk {

// ---------------------------------------------------------------------------
// Complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// a * (-i) for the forward transform, a * (+i) for the inverse
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a * (c_re + sgn c_im i) with the sign chosen by the direction
template <bool INV>
__device__ __forceinline__ float2 mul_w(float2 a, float cr, float ci) {
  const float s = INV ? ci : -ci;
  return make_float2(a.x * cr - a.y * s, a.x * s + a.y * cr);
}

// ---------------------------------------------------------------------------
// Small DFTs in registers, natural-order output.  Forward: exp(-2 pi i tm/r).
// ---------------------------------------------------------------------------
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
  // W16^m = cos(pi m / 8) -+ i sin(pi m / 8)
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

// ---------------------------------------------------------------------------
// Stockham autosort FFT in shared memory.  A CTA transforms several
// sequences at once; each thread holds kE complex values per stage (kE / R
// butterflies).  Stage (R, Ns): butterfly j reads x[j + t L/R], multiplies by
// W_{Ns R}^{(j mod Ns) t}, applies the R-point DFT and writes
// y[(j div Ns) Ns R + (j mod Ns) + t Ns].  All reads of a stage finish before
// any write (barrier), so one buffer suffices.
// ---------------------------------------------------------------------------
struct RowLay {  // sequences stored one after another, 1 pad per 16 values
  int S;
  __device__ __forceinline__ int transform(int g, int logLr) const { return g >> logLr; }
  __device__ __forceinline__ int index(int g, int logLr) const { return g & ((1 << logLr) - 1); }
  __device__ __forceinline__ int addr(int c, int a) const { return c * S + a + (a >> 4); }
};

struct ColLay {  // kColCB sequences interleaved: value a of sequence c at a*CB + c
  __device__ __forceinline__ int transform(int g, int) const { return g % kColCB; }
  __device__ __forceinline__ int index(int g, int) const { return g / kColCB; }
  __device__ __forceinline__ int addr(int c, int a) const { return a * kColCB + c; }
};

template <int R>
struct Log2 {
  static constexpr int v = R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1;
};

template <int R, bool INV, class Lay>
__device__ __forceinline__ void fft_stage(float2* buf, const Lay& lay, const Fft& f, int logNs) {
  constexpr int NB = kE / R;
  constexpr int logR = Log2<R>::v;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int logLr = f.logL - logR;
  const int Lr = 1 << logLr;
  const int Ns = 1 << logNs;
  float2 v[NB][R];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int gi = tid + b * NT;
    const int c = lay.transform(gi, logLr), j = lay.index(gi, logLr);
#pragma unroll
    for (int t = 0; t < R; ++t) v[b][t] = buf[lay.addr(c, j + t * Lr)];
  }
  __syncthreads();
  const int tshift = f.logL - logNs - logR;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int gi = tid + b * NT;
    const int c = lay.transform(gi, logLr), j = lay.index(gi, logLr);
    const int k = j & (Ns - 1);
    if (logNs > 0) {
#pragma unroll
      for (int t = 1; t < R; ++t) {
        float2 w = __ldg(&f.tw[(k * t) << tshift]);
        if (INV) w.y = -w.y;
        v[b][t] = cmul(v[b][t], w);
      }
    }
    dft<R, INV>(v[b]);
    const int base = ((j >> logNs) << (logNs + logR)) + k;
#pragma unroll
    for (int t = 0; t < R; ++t) buf[lay.addr(c, base + (t << logNs))] = v[b][t];
  }
  __syncthreads();
}

template <bool INV, class Lay>
__device__ void fft_run(float2* buf, const Lay& lay, const Fft& f) {
  int logNs = 0;
  for (int s = 0; s < f.n16; ++s) {
    fft_stage<16, INV>(buf, lay, f, logNs);
    logNs += 4;
  }
  if (f.tail == 8) fft_stage<8, INV>(buf, lay, f, logNs);
  else if (f.tail == 4) fft_stage<4, INV>(buf, lay, f, logNs);
  else if (f.tail == 2) fft_stage<2, INV>(buf, lay, f, logNs);
}

// ---------------------------------------------------------------------------
// Regularised functions, Eqs. (5), (6), (11), (28), (29), in FP32
// ---------------------------------------------------------------------------
__device__ __forceinline__ float heps(float x, float eps) {
  if (x > eps) return 1.f;
  if (x < -eps) return 0.f;
  const float y = x / eps;
  return 0.5f * (1.f + y + sinpif(y) * 0.318309886183790671538f);
}
__device__ __forceinline__ float deps(float x, float eps) {
  if (fabsf(x) > eps) return 0.f;
  return (1.f + cospif(x / eps)) * (0.5f / eps);
}
__device__ __forceinline__ float dpeps(float x, float eps) {
  if (fabsf(x) > eps) return 0.f;
  return -(1.57079632679489661923f / (eps * eps)) * sinpif(x / eps);
}
__device__ __forceinline__ float band_h(float x, const Model& m) {
  if (fabsf(x) >= m.band_l + m.eps) return 0.f;
  return heps(x + m.band_l, m.eps) * (1.f - heps(x - m.band_l, m.eps));
}
__device__ __forceinline__ float band_hp(float x, const Model& m) {
  if (fabsf(x) >= m.band_l + m.eps) return 0.f;
  return deps(x + m.band_l, m.eps) * (1.f - heps(x - m.band_l, m.eps)) -
         heps(x + m.band_l, m.eps) * deps(x - m.band_l, m.eps);
}

// ---------------------------------------------------------------------------
// Row pass, forward.  CTA = T rows.  RHS mode: for each column chunk, stage
// u = h(psi) w on the chunk plus an R halo (zero outside the image), sum the
// window separably (rows, then columns), then form the increment right-hand
// side G = tau (force + mu Lap psi) of one inner step.  LOAD mode: G is read.
// G of the T rows goes to shared memory as z[n] = G[2n] + i G[2n+1]; a length
// L = N/2 complex FFT and the even/odd split give the N/2+1 values of the
// real row transform, stored packed: X[0] = X_0 + i X_{N/2}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rhs_increment(const RowFwdArgs& a, int i, int j, float v1,
                                               float v2) {
  const int M = a.geo.M, N = a.geo.N;
  const Model& m = a.mod;
  const size_t o = (size_t)i * N + j;
  const size_t up = (size_t)(i == 0 ? M - 1 : i - 1) * N + j;
  const size_t dn = (size_t)(i == M - 1 ? 0 : i + 1) * N + j;
  const size_t lf = (size_t)i * N + (j == 0 ? N - 1 : j - 1);
  const size_t rt = (size_t)i * N + (j == N - 1 ? 0 : j + 1);
  const float x = a.psi[o];
  const float lap = (a.psi[up] + a.psi[dn]) + (a.psi[lf] + a.psi[rt]) - 4.f * x;
  const float W1 = a.w1[o], W2 = a.w2[o];
  const float dv = ((a.b1[o] - W1) - (a.b1[up] - a.w1[up])) +
                   ((a.b2[o] - W2) - (a.b2[lf] - a.w2[lf]));
  float force = m.mu * (dv + lap);
  if (fabsf(x) < m.band_l + m.eps) {
    const float gg = a.g[o];
    const float wn = sqrtf(W1 * W1 + W2 * W2);
    force += -m.gamma * gg * wn * dpeps(x, m.eps) + m.alpha * gg * deps(x, m.eps) +
             2.f * m.beta * band_hp(x, m) * (W1 * v1 + W2 * v2);
  }
  return m.tau * force;
}

template <int MODE>
__global__ void __launch_bounds__(512) k_rowfwd(const RowFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = a.geo.M, N = a.geo.N, L = a.geo.L, T = a.T;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int S = L + (L >> 4);
  float2* Z = reinterpret_cast<float2*>(smem_raw);
  float* Zf = reinterpret_cast<float*>(smem_raw);
  const int r0 = blockIdx.x * T;

  if (MODE == kRowLOAD) {
    for (int idx = tid; idx < T * N; idx += NT) {
      const int t = idx >> a.geo.logN, j = idx & (N - 1);
      const int i = r0 + t;
      const float G = i < M ? a.src[(size_t)i * N + j] : 0.f;
      const int cz = j >> 1;
      Zf[2 * (t * S + cz + (cz >> 4)) + (j & 1)] = G;
    }
  } else {
    const int R = a.mod.R;
    const int CW = a.CW, CWH = CW + 2 * R, TH = T + 2 * R;
    float* U1 = reinterpret_cast<float*>(Z + T * S);
    float* U2 = U1 + TH * CWH;
    float* V1 = U2 + TH * CWH;
    float* V2 = V1 + T * CWH;
    for (int c0 = 0; c0 < N; c0 += CW) {
      for (int idx = tid; idx < TH * CWH; idx += NT) {
        const int rr = idx / CWH, cc = idx - rr * CWH;
        const int i = r0 - R + rr, j = c0 - R + cc;
        float u1 = 0.f, u2 = 0.f;
        if (i >= 0 && i < M && j >= 0 && j < N) {
          const size_t o = (size_t)i * N + j;
          const float h = band_h(a.psi[o], a.mod);
          if (h != 0.f) {
            u1 = h * a.w1[o];
            u2 = h * a.w2[o];
          }
        }
        U1[idx] = u1;
        U2[idx] = u2;
      }
      __syncthreads();
      for (int idx = tid; idx < T * CWH; idx += NT) {
        const int t = idx / CWH, cc = idx - t * CWH;
        float s1 = 0.f, s2 = 0.f;
        for (int p = 0; p <= 2 * R; ++p) {
          const float kw = a.mod.kw[p];
          s1 = fmaf(kw, U1[(t + p) * CWH + cc], s1);
          s2 = fmaf(kw, U2[(t + p) * CWH + cc], s2);
        }
        V1[idx] = s1;
        V2[idx] = s2;
      }
      __syncthreads();
      for (int idx = tid; idx < T * CW; idx += NT) {
        const int t = idx / CW, c = idx - t * CW;
        const int i = r0 + t, j = c0 + c;
        float G = 0.f;
        if (i < M) {
          float v1 = 0.f, v2 = 0.f;
          for (int q = 0; q <= 2 * R; ++q) {
            const float kw = a.mod.kw[q];
            v1 = fmaf(kw, V1[t * CWH + c + q], v1);
            v2 = fmaf(kw, V2[t * CWH + c + q], v2);
          }
          G = rhs_increment(a, i, j, v1, v2);
        }
        const int cz = j >> 1;
        Zf[2 * (t * S + cz + (cz >> 4)) + (j & 1)] = G;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  fft_run<false>(Z, RowLay{S}, a.fft);

  const int half = L / 2;
  for (int idx = tid; idx < T * (half + 1); idx += NT) {
    const int t = idx / (half + 1), k = idx - t * (half + 1);
    const int i = r0 + t;
    if (i >= M) continue;
    const float2 Zk = Z[t * S + k + (k >> 4)];
    float2* Xrow = a.X + (size_t)i * L;
    if (k == 0) {
      Xrow[0] = make_float2(Zk.x + Zk.y, Zk.x - Zk.y);
      continue;
    }
    const int km = L - k;
    const float2 Zm = Z[t * S + km + (km >> 4)];
    // E = (Z_k + conj Z_{L-k}) / 2, O = -i (Z_k - conj Z_{L-k}) / 2
    const float2 E = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    const float2 D = make_float2(0.5f * (Zk.x - Zm.x), 0.5f * (Zk.y + Zm.y));
    const float2 O = make_float2(D.y, -D.x);
    Xrow[k] = cadd(E, cmul(__ldg(&a.twN[k]), O));
    if (km != k) Xrow[km] = cadd(cconj(E), cmul(__ldg(&a.twN[km]), cconj(O)));
  }
}

// ---------------------------------------------------------------------------
// Column pass: kColCB columns of X per CTA, all M rows, in shared memory.
// Forward column FFT, multiply by 1 / (M N lambda), inverse column FFT, with
// lambda(l, k) = 1 + tau mu (4 sin^2(pi l/M) + 4 sin^2(pi k/N)) (Eq. (32)).
// Column 0 packs the DC and Nyquist columns of the row transforms; both are
// transforms of real sequences, split here with the conjugate pair (l, M-l)
// so that each gets its own symbol.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_colsolve(const ColArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Z = reinterpret_cast<float2*>(smem_raw);
  const int M = a.geo.M, L = a.geo.L;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int c0 = blockIdx.x * kColCB;
  const float inv_mn = 1.f / ((float)M * (float)a.geo.N);
  for (int idx = tid; idx < M * kColCB; idx += NT) {
    const int r = idx / kColCB, c = idx - r * kColCB;
    Z[idx] = a.X[(size_t)r * L + c0 + c];
  }
  __syncthreads();
  fft_run<false>(Z, ColLay{}, a.fft);
  for (int idx = tid; idx < M * kColCB; idx += NT) {
    const int l = idx / kColCB, c = idx - l * kColCB;
    const int k = c0 + c;
    if (k == 0) continue;
    const float s = inv_mn / (1.f + a.aM[l] + a.aN[k]);
    Z[idx] = make_float2(Z[idx].x * s, Z[idx].y * s);
  }
  if (c0 == 0) {
    const float aNy = a.aN[L];
    for (int l = tid; l <= M / 2; l += NT) {
      const int lm = (M - l) & (M - 1);
      const float2 Cl = Z[l * kColCB], Cm = Z[lm * kColCB];
      const float sA = inv_mn / (1.f + a.aM[l] + a.aN[0]);
      const float sB = inv_mn / (1.f + a.aM[l] + aNy);
      // A = (C_l + conj C_{M-l}) / 2, B = (C_l - conj C_{M-l}) / (2i)
      const float2 A = make_float2(0.5f * (Cl.x + Cm.x) * sA, 0.5f * (Cl.y - Cm.y) * sA);
      const float2 D = make_float2(0.5f * (Cl.x - Cm.x), 0.5f * (Cl.y + Cm.y));
      const float2 B = make_float2(D.y * sB, -D.x * sB);
      Z[l * kColCB] = make_float2(A.x - B.y, A.y + B.x);
      if (lm != l) Z[lm * kColCB] = make_float2(A.x + B.y, B.x - A.y);
    }
  }
  __syncthreads();
  fft_run<true>(Z, ColLay{}, a.fft);
  for (int idx = tid; idx < M * kColCB; idx += NT) {
    const int r = idx / kColCB, c = idx - r * kColCB;
    a.X[(size_t)r * L + c0 + c] = Z[idx];
  }
}

// ---------------------------------------------------------------------------
// Row pass, inverse: rebuild the length-L complex sequence whose inverse FFT
// interleaves the even and odd samples of the real row, transform, unpack.
// ADD mode: out = psi_in + x (the increment form), STORE mode: out = x.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(512) k_rowinv(const RowInvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Z = reinterpret_cast<float2*>(smem_raw);
  const int M = a.geo.M, N = a.geo.N, L = a.geo.L, T = a.T;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int S = L + (L >> 4);
  const int r0 = blockIdx.x * T;
  const int half = L / 2;
  for (int idx = tid; idx < T * (half + 1); idx += NT) {
    const int t = idx / (half + 1), k = idx - t * (half + 1);
    const int i = r0 + t;
    const int km = (L - k) & (L - 1);
    if (i >= M) {
      Z[t * S + k + (k >> 4)] = make_float2(0.f, 0.f);
      Z[t * S + km + (km >> 4)] = make_float2(0.f, 0.f);
      continue;
    }
    const float2* Xrow = a.X + (size_t)i * L;
    if (k == 0) {
      const float2 Y = Xrow[0];  // (X_0, X_{N/2})
      Z[t * S] = make_float2(Y.x + Y.y, Y.x - Y.y);
      continue;
    }
    const float2 Xk = Xrow[k], Xm = Xrow[km];
    // Xe = X_k + conj X_{L-k},  Xo = (X_k - conj X_{L-k}) exp(+2 pi i k / N)
    const float2 Xe = make_float2(Xk.x + Xm.x, Xk.y - Xm.y);
    const float2 D = make_float2(Xk.x - Xm.x, Xk.y + Xm.y);
    const float2 Xo = cmul(D, cconj(__ldg(&a.twN[k])));
    Z[t * S + k + (k >> 4)] = make_float2(Xe.x - Xo.y, Xe.y + Xo.x);
    if (km != k) {
      const float2 Xe2 = cconj(Xe);
      const float2 D2 = make_float2(-D.x, D.y);
      const float2 Xo2 = cmul(D2, cconj(__ldg(&a.twN[km])));
      Z[t * S + km + (km >> 4)] = make_float2(Xe2.x - Xo2.y, Xe2.y + Xo2.x);
    }
  }
  __syncthreads();
  fft_run<true>(Z, RowLay{S}, a.fft);
  for (int idx = tid; idx < T * L; idx += NT) {
    const int t = idx / L, n = idx - t * L;
    const int i = r0 + t;
    if (i >= M) continue;
    const float2 z = Z[t * S + n + (n >> 4)];
    const size_t o = (size_t)i * N + 2 * n;
    float2 r = z;
    if (MODE == kInvADD) {
      const float2 p = *reinterpret_cast<const float2*>(a.psi_in + o);
      r = make_float2(p.x + z.x, p.y + z.y);
    }
    *reinterpret_cast<float2*>(a.out + o) = r;
  }
}

// ---------------------------------------------------------------------------
// 2-D tile helpers for the window sum: u = h(phi) w on the tile plus an R
// halo (zero outside the image), rows then columns.
// ---------------------------------------------------------------------------
struct TileSmem {
  float U1[(kTileY + 2 * kMaxR) * (kTileX + 2 * kMaxR)];
  float U2[(kTileY + 2 * kMaxR) * (kTileX + 2 * kMaxR)];
  float V1[kTileY * (kTileX + 2 * kMaxR)];
  float V2[kTileY * (kTileX + 2 * kMaxR)];
};

// After the call, (v1, v2) hold the window sum at this thread's pixel.
template <class UFn>
__device__ __forceinline__ void tile_window_sum(TileSmem& sm, const Geo& geo, const Model& m,
                                                int i0, int j0, UFn ufn, float& v1, float& v2) {
  const int R = m.R;
  const int TW = kTileX + 2 * R, TH = kTileY + 2 * R;
  const int tid = threadIdx.y * kTileX + threadIdx.x;
  const int NT = kTileX * kTileY;
  for (int idx = tid; idx < TH * TW; idx += NT) {
    const int rr = idx / TW, cc = idx - rr * TW;
    const int i = i0 - R + rr, j = j0 - R + cc;
    float u1 = 0.f, u2 = 0.f;
    if (i >= 0 && i < geo.M && j >= 0 && j < geo.N) ufn(i, j, u1, u2);
    sm.U1[idx] = u1;
    sm.U2[idx] = u2;
  }
  __syncthreads();
  for (int idx = tid; idx < kTileY * TW; idx += NT) {
    const int t = idx / TW, cc = idx - t * TW;
    float s1 = 0.f, s2 = 0.f;
    for (int p = 0; p <= 2 * R; ++p) {
      const float kw = m.kw[p];
      s1 = fmaf(kw, sm.U1[(t + p) * TW + cc], s1);
      s2 = fmaf(kw, sm.U2[(t + p) * TW + cc], s2);
    }
    sm.V1[idx] = s1;
    sm.V2[idx] = s2;
  }
  __syncthreads();
  float a1 = 0.f, a2 = 0.f;
  for (int q = 0; q <= 2 * R; ++q) {
    const float kw = m.kw[q];
    a1 = fmaf(kw, sm.V1[threadIdx.y * TW + threadIdx.x + q], a1);
    a2 = fmaf(kw, sm.V2[threadIdx.y * TW + threadIdx.x + q], a2);
  }
  v1 = a1;
  v2 = a2;
}

// Fixed-order block reduction of NC doubles; thread 0 writes out[0..NC).
template <int NC>
__device__ __forceinline__ void block_sum_store(double (&val)[NC], double* out) {
  __shared__ double red[NC][32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double v = val[c];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[c][warp] = v;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[c][w];
      out[c] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// 32 x 32 output tiles, block (8, 32): a thread owns four consecutive pixels
// of one row, so every global access is a float4.  The tile is staged with a
// halo of HY = max(R, 1) rows and HX >= max(R, 1) columns, HX a multiple of 4
// so that staged float4s stay aligned; the kernels are templated on R so the
// staging and window loops unroll.
//
// u = h(psi) w vanishes outside the narrow band |psi| < l + eps (Eq. (11)), so
// a tile whose halo holds no band pixel has v = 0 exactly: psi is staged
// first, the block tests for band pixels, and w is staged and summed over the
// window only when the test succeeds.  Neighbours of the periodic stencils
// that fall outside the image are read from global memory with the wrap.
// ---------------------------------------------------------------------------
constexpr int kT = 32;
constexpr int kTBX = 8, kTBY = 32;      // block shape
constexpr int kTN = kTBX * kTBY;        // threads per tile CTA

template <int R>
struct Tile {
  static constexpr int HY = R > 1 ? R : 1;
  static constexpr int HX = R > 4 ? 8 : 4;
  static constexpr int SH = kT + 2 * HY;   // staged rows
  static constexpr int SW = kT + 2 * HX;   // staged columns
  static constexpr int SW4 = SW / 4;
  static constexpr int N4 = SH * SW4;      // staged float4 per plane
  static constexpr int IT = (N4 + kTN - 1) / kTN;
  static constexpr int NP = SH * SW;       // floats per staged plane
  static constexpr int FLOATS = 5 * NP + 2 * kT * SW;
};

__host__ __device__ constexpr int tile32_floats(int R) {
  return 5 * (kT + 2 * (R > 1 ? R : 1)) * (kT + 2 * (R > 4 ? 8 : 4)) +
         2 * kT * (kT + 2 * (R > 4 ? 8 : 4));
}

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ bool in_band(float x, const Model& m) { return fabsf(x) < m.band_l + m.eps; }

// Stage one plane (zero outside the image); returns whether a staged value
// lies in the narrow band when BAND is set.
template <int R, bool BAND>
__device__ __forceinline__ int stage4(float* dst, const float* __restrict__ src, const Geo& geo,
                                      int i0, int j0, const Model& m) {
  using TL = Tile<R>;
  const int tid = threadIdx.y * kTBX + threadIdx.x;
  float4 val[TL::IT];
#pragma unroll
  for (int k = 0; k < TL::IT; ++k) {
    const int idx = tid + k * kTN;
    const int r = idx / TL::SW4, c4 = idx - r * TL::SW4;
    const int i = i0 - TL::HY + r, j = j0 - TL::HX + 4 * c4;
    val[k] = (idx < TL::N4 && i >= 0 && i < geo.M && j >= 0 && j < geo.N)
                 ? ld4(src + (size_t)i * geo.N + j)
                 : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  int any = 0;
#pragma unroll
  for (int k = 0; k < TL::IT; ++k) {
    const int idx = tid + k * kTN;
    if (idx < TL::N4) {
      st4(dst + 4 * idx, val[k]);
      if (BAND)
        any |= in_band(val[k].x, m) | in_band(val[k].y, m) | in_band(val[k].z, m) |
               in_band(val[k].w, m);
    }
  }
  return any;
}

// With psi and w in shared memory ([SH][SW] planes, zero outside the image):
// form u = h(psi) w and return the window sums of the thread's four pixels.
template <int R>
__device__ __forceinline__ void window_sum(const float* t_psi, const float* t_w1,
                                           const float* t_w2, float* t_u1, float* t_u2,
                                           float* t_V1, float* t_V2, const Model& m,
                                           float (&v1)[4], float (&v2)[4]) {
  using TL = Tile<R>;
  const int tid = threadIdx.y * kTBX + threadIdx.x;
  for (int idx = tid; idx < TL::NP; idx += kTN) {
    const float x = t_psi[idx];
    const float hh = in_band(x, m) ? band_h(x, m) : 0.f;
    t_u1[idx] = hh * t_w1[idx];  // w = 0 outside the image
    t_u2[idx] = hh * t_w2[idx];
  }
  __syncthreads();
  // sum down the columns: a task is 4 rows x 4 columns, sliding over 4 + 2R rows
  constexpr int NTASK = (kT / 4) * TL::SW4;
  if (tid < NTASK) {
    const int r0 = (tid / TL::SW4) * 4, c = 4 * (tid % TL::SW4);
    float4 a1[4], a2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) a1[q] = a2[q] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int t = 0; t < 4 + 2 * R; ++t) {
      const int row = r0 + TL::HY - R + t;
      const float4 x1 = *reinterpret_cast<const float4*>(t_u1 + row * TL::SW + c);
      const float4 x2 = *reinterpret_cast<const float4*>(t_u2 + row * TL::SW + c);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int p = t - q;  // output row r0 + q takes input rows r0 + q - R .. r0 + q + R
        if (p >= 0 && p <= 2 * R) {
          const float kw = m.kw[p];
          a1[q].x = fmaf(kw, x1.x, a1[q].x);
          a1[q].y = fmaf(kw, x1.y, a1[q].y);
          a1[q].z = fmaf(kw, x1.z, a1[q].z);
          a1[q].w = fmaf(kw, x1.w, a1[q].w);
          a2[q].x = fmaf(kw, x2.x, a2[q].x);
          a2[q].y = fmaf(kw, x2.y, a2[q].y);
          a2[q].z = fmaf(kw, x2.z, a2[q].z);
          a2[q].w = fmaf(kw, x2.w, a2[q].w);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      st4(t_V1 + (r0 + q) * TL::SW + c, a1[q]);
      st4(t_V2 + (r0 + q) * TL::SW + c, a2[q]);
    }
  }
  __syncthreads();
  // across the row: outputs c .. c+3 take inputs c - R .. c + 3 + R
  const int r = threadIdx.y, c = 4 * threadIdx.x + TL::HX;
#pragma unroll
  for (int q = 0; q < 4; ++q) v1[q] = v2[q] = 0.f;
#pragma unroll
  for (int t = 0; t < 4 + 2 * R; ++t) {
    const float x1 = t_V1[r * TL::SW + c - R + t];
    const float x2 = t_V2[r * TL::SW + c - R + t];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = t - q;
      if (p >= 0 && p <= 2 * R) {
        v1[q] = fmaf(m.kw[p], x1, v1[q]);
        v2[q] = fmaf(m.kw[p], x2, v2[q]);
      }
    }
  }
}

// With psi staged: stage w, then the window sums of the thread's four pixels
// (zero for tiles without band pixels).
template <int R>
__device__ __forceinline__ void tile_window(float* sm, const Geo& geo, const Model& m,
                                            const float* __restrict__ w1,
                                            const float* __restrict__ w2, int i0, int j0,
                                            bool band, float (&v1)[4], float (&v2)[4]) {
  using TL = Tile<R>;
#pragma unroll
  for (int q = 0; q < 4; ++q) v1[q] = v2[q] = 0.f;
  if (!band) return;  // uniform across the block
  float* t_w1 = sm + 3 * TL::NP;
  float* t_w2 = sm + 4 * TL::NP;
  stage4<R, false>(t_w1, w1, geo, i0, j0, m);
  stage4<R, false>(t_w2, w2, geo, i0, j0, m);
  __syncthreads();
  float* t_V1 = sm + 5 * TL::NP;
  window_sum<R>(sm, t_w1, t_w2, sm + TL::NP, sm + 2 * TL::NP, t_V1, t_V1 + kT * TL::SW, m, v1,
                v2);
}

size_t tile32_smem(int R) { return (size_t)tile32_floats(R) * sizeof(float); }

// G = tau [ mu (div e + Lap psi) - gamma g |w| delta'(psi) + alpha g delta(psi)
//           + 2 beta h'(psi) (w . v) ] at one pixel (the band terms only where
// |psi| < l + eps; e = b - w, div the backward divergence).
__device__ __forceinline__ float rhs_point(const Model& m, float x, float up, float dn, float lf,
                                           float rt, float e1, float e1u, float e2, float e2l,
                                           float w1, float w2, float g, float v1, float v2) {
  const float lap = (up + dn) + (lf + rt) - 4.f * x;
  const float dv = (e1 - e1u) + (e2 - e2l);
  float force = m.mu * (dv + lap);
  if (in_band(x, m)) {
    const float wn = sqrtf(w1 * w1 + w2 * w2);
    force += -m.gamma * g * wn * dpeps(x, m.eps) + m.alpha * g * deps(x, m.eps) +
             2.f * m.beta * band_hp(x, m) * (w1 * v1 + w2 * v2);
  }
  return m.tau * force;
}

// Eqs. (41), (42), (40), (23) at one pixel: B = grad phi + b + (2 beta/mu) h v,
// t = (gamma/mu) g delta(phi); w = B/|B| if |B| > t else 0; b' = b + grad phi - w;
// returns w' and e' = b' - w'.
__device__ __forceinline__ void wb_point(const Model& m, float x, float d1, float d2, float b1,
                                         float b2, float g, float v1, float v2, float& wo1,
                                         float& wo2, float& eo1, float& eo2) {
  float Bv1 = d1 + b1;
  float Bv2 = d2 + b2;
  float thr = 0.f;
  if (in_band(x, m)) {
    const float h = band_h(x, m);
    Bv1 = fmaf(m.beta2_mu * h, v1, Bv1);
    Bv2 = fmaf(m.beta2_mu * h, v2, Bv2);
    thr = m.gamma_mu * g * deps(x, m.eps);
  }
  const float nB = sqrtf(Bv1 * Bv1 + Bv2 * Bv2);
  float W1 = 0.f, W2 = 0.f;
  if (nB > thr) {
    W1 = Bv1 / nB;
    W2 = Bv2 / nB;
  }
  wo1 = W1;
  wo2 = W2;
  eo1 = ((b1 + d1) - W1) - W1;
  eo2 = ((b2 + d2) - W2) - W2;
}

// Increment right-hand side of one inner step, Eq. (37) in the form
// G = tau [ -gamma g |w| delta'(psi) + alpha g delta(psi) + 2 beta h'(psi) (w . v)
//           + mu (div(b - w) + Lap psi) ], so that phi^{k+1,s+1} = psi + L^{-1} G.
template <int R>
__global__ void __launch_bounds__(kTN, 4) k_prep(const PrepArgs a) {
  using TL = Tile<R>;
  extern __shared__ __align__(16) float smem_f[];
  const int i0 = blockIdx.y * kT, j0 = blockIdx.x * kT;
  const int M = a.geo.M, N = a.geo.N;
  const Model& m = a.mod;
  const int any = stage4<R, true>(smem_f, a.psi, a.geo, i0, j0, m);
  const bool band = __syncthreads_or(any) != 0;
  float v1[4], v2[4];
  tile_window<R>(smem_f, a.geo, m, a.w1, a.w2, i0, j0, band, v1, v2);
  const int i = i0 + threadIdx.y, j = j0 + 4 * threadIdx.x;
  if (i >= M || j >= N) return;
  const size_t o = (size_t)i * N + j;
  const size_t ou = (size_t)(i > 0 ? i - 1 : M - 1) * N + j;
  const size_t ol = (size_t)i * N + (j > 0 ? j - 1 : N - 1);
  const float4 E1 = ld4(a.e1 + o), E2 = ld4(a.e2 + o), E1u = ld4(a.e1 + ou);
  const float e2l = __ldg(a.e2 + ol);
  const float* t_psi = smem_f;
  const int q = (threadIdx.y + TL::HY) * TL::SW + 4 * threadIdx.x + TL::HX;
  const float4 X = *reinterpret_cast<const float4*>(t_psi + q);
  const float4 UP = i > 0 ? *reinterpret_cast<const float4*>(t_psi + q - TL::SW) : ld4(a.psi + ou);
  const float4 DN = i < M - 1 ? *reinterpret_cast<const float4*>(t_psi + q + TL::SW)
                              : ld4(a.psi + j);
  const float LF = j > 0 ? t_psi[q - 1] : __ldg(a.psi + ol);
  const float RT = j + 4 < N ? t_psi[q + 4] : __ldg(a.psi + (size_t)i * N);
  float4 W1 = make_float4(0.f, 0.f, 0.f, 0.f), W2 = W1, G4 = W1;
  if (band) {  // w and g enter only through the narrow-band terms
    W1 = ld4(a.w1 + o);
    W2 = ld4(a.w2 + o);
    G4 = ld4(a.g + o);
  }
  const float x[4] = {X.x, X.y, X.z, X.w};
  const float up[4] = {UP.x, UP.y, UP.z, UP.w}, dn[4] = {DN.x, DN.y, DN.z, DN.w};
  const float lf[4] = {LF, X.x, X.y, X.z}, rt[4] = {X.y, X.z, X.w, RT};
  const float e1[4] = {E1.x, E1.y, E1.z, E1.w}, e2[4] = {E2.x, E2.y, E2.z, E2.w};
  const float e1u[4] = {E1u.x, E1u.y, E1u.z, E1u.w}, e2l4[4] = {e2l, E2.x, E2.y, E2.z};
  const float w1[4] = {W1.x, W1.y, W1.z, W1.w}, w2[4] = {W2.x, W2.y, W2.z, W2.w};
  const float gg[4] = {G4.x, G4.y, G4.z, G4.w};
  float out[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) out[t] = rhs_point(m, x[t], up[t], dn[t], lf[t], rt[t], e1[t], e1u[t],
                                                 e2[t], e2l4[t], w1[t], w2[t], gg[t], v1[t], v2[t]);
  st4(a.G + o, make_float4(out[0], out[1], out[2], out[3]));
}

// w and b update (Eqs. (41), (42), (40), (23)) with the window sum fused in.
// Soft threshold then projection: w = B/|B| if |B| > t, else 0.
template <int R>
__global__ void __launch_bounds__(kTN, 4) k_wb_update(const WBArgs a) {
  using TL = Tile<R>;
  extern __shared__ __align__(16) float smem_f[];
  const int i0 = blockIdx.y * kT, j0 = blockIdx.x * kT;
  const int M = a.geo.M, N = a.geo.N;
  const Model& m = a.mod;
  const int any = stage4<R, true>(smem_f, a.phi1, a.geo, i0, j0, m);
  const bool band = __syncthreads_or(any) != 0;
  float v1[4], v2[4];
  tile_window<R>(smem_f, a.geo, m, a.w1, a.w2, i0, j0, band, v1, v2);
  const int i = i0 + threadIdx.y, j = j0 + 4 * threadIdx.x;
  double part[2] = {0.0, 0.0};
  if (i < M && j < N) {
    const size_t o = (size_t)i * N + j;
    const float4 E1 = ld4(a.e1 + o), E2 = ld4(a.e2 + o), W1 = ld4(a.w1 + o), W2 = ld4(a.w2 + o);
    const float4 G4 = band ? ld4(a.g + o) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float* t_psi = smem_f;
    const int q = (threadIdx.y + TL::HY) * TL::SW + 4 * threadIdx.x + TL::HX;
    const float4 X = *reinterpret_cast<const float4*>(t_psi + q);
    const float4 DN = i < M - 1 ? *reinterpret_cast<const float4*>(t_psi + q + TL::SW)
                                : ld4(a.phi1 + j);
    const float RT = j + 4 < N ? t_psi[q + 4] : __ldg(a.phi1 + (size_t)i * N);
    const float x[4] = {X.x, X.y, X.z, X.w};
    const float dn[4] = {DN.x, DN.y, DN.z, DN.w}, rt[4] = {X.y, X.z, X.w, RT};
    const float b1[4] = {E1.x + W1.x, E1.y + W1.y, E1.z + W1.z, E1.w + W1.w};
    const float b2[4] = {E2.x + W2.x, E2.y + W2.y, E2.z + W2.z, E2.w + W2.w};
    const float gg[4] = {G4.x, G4.y, G4.z, G4.w};
    float wo1[4], wo2[4], eo1[4], eo2[4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
      wb_point(m, x[t], dn[t] - x[t], rt[t] - x[t], b1[t], b2[t], gg[t], v1[t], v2[t], wo1[t],
               wo2[t], eo1[t], eo2[t]);
    st4(a.w1o + o, make_float4(wo1[0], wo1[1], wo1[2], wo1[3]));
    st4(a.w2o + o, make_float4(wo2[0], wo2[1], wo2[2], wo2[3]));
    st4(a.e1o + o, make_float4(eo1[0], eo1[1], eo1[2], eo1[3]));
    st4(a.e2o + o, make_float4(eo2[0], eo2[1], eo2[2], eo2[3]));
    if (a.phi_old) {
      const float4 P = ld4(a.phi_old + o);
      const float po[4] = {P.x, P.y, P.z, P.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const double df = (double)x[t] - (double)po[t];
        part[0] += df * df;
        part[1] += (double)po[t] * (double)po[t];
      }
    }
  }
  if (a.phi_old) block_sum_store<2>(part, a.partials + 2 * (blockIdx.y * gridDim.x + blockIdx.x));
}

// ---------------------------------------------------------------------------
// TMA versions of the two tile kernels.  One thread issues 2-D box loads of
// every plane the tile needs (zero fill outside the image gives the window
// sum's dropped terms); they complete on an mbarrier, and the block then
// works from shared memory only.  Boxes: psi, w1, w2 with the (HX, HY) halo;
// b1 with the row above (33 x 32), b2 with four columns to the left
// (32 x 36), g and the old phi 32 x 32.  k_wb_tma loads w only for tiles with
// narrow-band pixels (second phase).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int a32(int n) { return (n + 31) / 32 * 32; }

template <int R>
struct TileT {
  using TL = Tile<R>;
  static constexpr int PSI = 0;
  static constexpr int W1 = PSI + a32(TL::NP);
  static constexpr int W2 = W1 + a32(TL::NP);
  static constexpr int B1 = W2 + a32(TL::NP);    // 33 rows x 32
  static constexpr int B2 = B1 + a32(33 * 32);    // 32 rows x 36
  static constexpr int GG = B2 + a32(32 * 36);    // 32 x 32
  static constexpr int PO = GG + a32(32 * 32);    // 32 x 32 (old phi)
  static constexpr int U1 = PO + a32(32 * 32);
  static constexpr int U2 = U1 + a32(TL::NP);
  static constexpr int V1 = U2 + a32(TL::NP);
  static constexpr int V2 = V1 + a32(kT * TL::SW);
  static constexpr int BAR = V2 + a32(kT * TL::SW);
  static constexpr int FLOATS = BAR + 8;  // two mbarriers
};

__device__ __forceinline__ float* align128(unsigned char* p) {
  return reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(p) + 127) & ~static_cast<uintptr_t>(127));
}

template <int R>
__global__ void __launch_bounds__(kTN, 3) k_prep_tma(const PrepArgs a, const __grid_constant__ PrepMaps tm) {
  using TL = Tile<R>;
  using TT = TileT<R>;
  extern __shared__ __align__(16) unsigned char smem_tt[];
  float* sm = align128(smem_tt);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TT::BAR);
  const int tid = threadIdx.y * kTBX + threadIdx.x;
  const int i0 = blockIdx.y * kT, j0 = blockIdx.x * kT;
  const int M = a.geo.M, N = a.geo.N;
  const Model& m = a.mod;
  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0) {
    constexpr uint32_t bytes = 4u * (TL::NP + 33 * 32 + 32 * 36);
    tma::mbar_expect_tx(&bar[0], bytes);
    tma::load_2d(sm + TT::PSI, &tm.psi, j0 - TL::HX, i0 - TL::HY, &bar[0]);
    tma::load_2d(sm + TT::B1, &tm.e1, j0, i0 - 1, &bar[0]);
    tma::load_2d(sm + TT::B2, &tm.e2, j0 - 4, i0, &bar[0]);
  }
  bool ok = tma::mbar_wait(&bar[0], 0);
  if (!__syncthreads_and(ok)) {
    if (tid == 0) tma::on_timeout(&bar[0], 0, a.err);
    return;
  }
  const float* t_psi = sm + TT::PSI;
  int any = 0;
  for (int idx = tid; idx < TL::NP; idx += kTN) any |= in_band(t_psi[idx], m);
  const bool band = __syncthreads_or(any) != 0;
  float v1[4] = {0.f, 0.f, 0.f, 0.f}, v2[4] = {0.f, 0.f, 0.f, 0.f};
  if (band) {
    if (tid == 0) {
      tma::mbar_expect_tx(&bar[1], 4u * (2 * TL::NP + 32 * 32));
      tma::load_2d(sm + TT::W1, &tm.w1, j0 - TL::HX, i0 - TL::HY, &bar[1]);
      tma::load_2d(sm + TT::W2, &tm.w2, j0 - TL::HX, i0 - TL::HY, &bar[1]);
      tma::load_2d(sm + TT::GG, &tm.g, j0, i0, &bar[1]);
    }
    ok = tma::mbar_wait(&bar[1], 0);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) tma::on_timeout(&bar[1], 0, a.err);
      return;
    }
    window_sum<R>(t_psi, sm + TT::W1, sm + TT::W2, sm + TT::U1, sm + TT::U2, sm + TT::V1,
                  sm + TT::V2, m, v1, v2);
  }
  const int ty = threadIdx.y, tx = threadIdx.x;
  const int i = i0 + ty, j = j0 + 4 * tx;
  if (i >= M || j >= N) return;
  const int q = (ty + TL::HY) * TL::SW + 4 * tx + TL::HX;
  auto f4 = [&](int off) { return *reinterpret_cast<const float4*>(sm + off); };
  const float4 X = f4(TT::PSI + q);
  const float4 UP = i > 0 ? f4(TT::PSI + q - TL::SW) : ld4(a.psi + (size_t)(M - 1) * N + j);
  const float4 DN = i < M - 1 ? f4(TT::PSI + q + TL::SW) : ld4(a.psi + j);
  const float LF = j > 0 ? sm[TT::PSI + q - 1] : __ldg(a.psi + (size_t)i * N + N - 1);
  const float RT = j + 4 < N ? sm[TT::PSI + q + 4] : __ldg(a.psi + (size_t)i * N);
  const float4 E1 = f4(TT::B1 + (ty + 1) * 32 + 4 * tx);
  const float4 E1u = i > 0 ? f4(TT::B1 + ty * 32 + 4 * tx) : ld4(a.e1 + (size_t)(M - 1) * N + j);
  const float4 E2 = f4(TT::B2 + ty * 36 + 4 + 4 * tx);
  const float e2l = j > 0 ? sm[TT::B2 + ty * 36 + 3 + 4 * tx] : __ldg(a.e2 + (size_t)i * N + N - 1);
  float4 W1 = make_float4(0.f, 0.f, 0.f, 0.f), W2 = W1, G4 = W1;
  if (band) {
    W1 = f4(TT::W1 + q);
    W2 = f4(TT::W2 + q);
    G4 = f4(TT::GG + ty * 32 + 4 * tx);
  }
  const float x[4] = {X.x, X.y, X.z, X.w};
  const float up[4] = {UP.x, UP.y, UP.z, UP.w}, dn[4] = {DN.x, DN.y, DN.z, DN.w};
  const float lf[4] = {LF, X.x, X.y, X.z}, rt[4] = {X.y, X.z, X.w, RT};
  const float e1[4] = {E1.x, E1.y, E1.z, E1.w}, e2[4] = {E2.x, E2.y, E2.z, E2.w};
  const float e1u[4] = {E1u.x, E1u.y, E1u.z, E1u.w}, e2l4[4] = {e2l, E2.x, E2.y, E2.z};
  const float w1[4] = {W1.x, W1.y, W1.z, W1.w}, w2[4] = {W2.x, W2.y, W2.z, W2.w};
  const float gg[4] = {G4.x, G4.y, G4.z, G4.w};
  float out[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) out[t] = rhs_point(m, x[t], up[t], dn[t], lf[t], rt[t], e1[t], e1u[t],
                                                 e2[t], e2l4[t], w1[t], w2[t], gg[t], v1[t], v2[t]);
  st4(a.G + (size_t)i * N + j, make_float4(out[0], out[1], out[2], out[3]));
}

template <int R>
__global__ void __launch_bounds__(kTN, 3) k_wb_tma(const WBArgs a, const __grid_constant__ WBMaps tm) {
  using TL = Tile<R>;
  using TT = TileT<R>;
  extern __shared__ __align__(16) unsigned char smem_tt[];
  float* sm = align128(smem_tt);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TT::BAR);
  const int tid = threadIdx.y * kTBX + threadIdx.x;
  const int i0 = blockIdx.y * kT, j0 = blockIdx.x * kT;
  const int M = a.geo.M, N = a.geo.N;
  const Model& m = a.mod;
  const bool chk = a.phi_old != nullptr;
  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bytes = 4u * (TL::NP + 4 * 32 * 32 + (chk ? 32 * 32 : 0));
    tma::mbar_expect_tx(&bar[0], bytes);
    tma::load_2d(sm + TT::PSI, &tm.psi, j0 - TL::HX, i0 - TL::HY, &bar[0]);
    tma::load_2d(sm + TT::B1, &tm.e1, j0, i0, &bar[0]);
    tma::load_2d(sm + TT::B2, &tm.e2, j0, i0, &bar[0]);
    tma::load_2d(sm + TT::U1, &tm.w1c, j0, i0, &bar[0]);
    tma::load_2d(sm + TT::U2, &tm.w2c, j0, i0, &bar[0]);
    if (chk) tma::load_2d(sm + TT::PO, &tm.phi_old, j0, i0, &bar[0]);
  }
  bool ok = tma::mbar_wait(&bar[0], 0);
  if (!__syncthreads_and(ok)) {
    if (tid == 0) tma::on_timeout(&bar[0], 0, a.err);
    return;
  }
  const float* t_psi = sm + TT::PSI;
  int any = 0;
  for (int idx = tid; idx < TL::NP; idx += kTN) any |= in_band(t_psi[idx], m);
  const bool band = __syncthreads_or(any) != 0;
  const int ty = threadIdx.y, tx = threadIdx.x;
  const int c32 = ty * 32 + 4 * tx;
  // w^k of the thread's pixels before the window sum reuses U1/U2
  auto f4 = [&](int off) { return *reinterpret_cast<const float4*>(sm + off); };
  const float4 W1 = f4(TT::U1 + c32), W2 = f4(TT::U2 + c32);
  float v1[4] = {0.f, 0.f, 0.f, 0.f}, v2[4] = {0.f, 0.f, 0.f, 0.f};
  if (band) {
    __syncthreads();  // every thread holds its w before U1/U2 are overwritten
    if (tid == 0) {
      tma::mbar_expect_tx(&bar[1], 4u * (2 * TL::NP + 32 * 32));
      tma::load_2d(sm + TT::W1, &tm.w1, j0 - TL::HX, i0 - TL::HY, &bar[1]);
      tma::load_2d(sm + TT::W2, &tm.w2, j0 - TL::HX, i0 - TL::HY, &bar[1]);
      tma::load_2d(sm + TT::GG, &tm.g, j0, i0, &bar[1]);
    }
    ok = tma::mbar_wait(&bar[1], 0);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) tma::on_timeout(&bar[1], 0, a.err);
      return;
    }
    window_sum<R>(t_psi, sm + TT::W1, sm + TT::W2, sm + TT::U1, sm + TT::U2, sm + TT::V1,
                  sm + TT::V2, m, v1, v2);
  }
  const int i = i0 + ty, j = j0 + 4 * tx;
  double part[2] = {0.0, 0.0};
  if (i < M && j < N) {
    const size_t o = (size_t)i * N + j;
    const int q = (ty + TL::HY) * TL::SW + 4 * tx + TL::HX;
    const float4 X = f4(TT::PSI + q);
    const float4 DN = i < M - 1 ? f4(TT::PSI + q + TL::SW) : ld4(a.phi1 + j);
    const float RT = j + 4 < N ? sm[TT::PSI + q + 4] : __ldg(a.phi1 + (size_t)i * N);
    const float4 E1 = f4(TT::B1 + c32), E2 = f4(TT::B2 + c32);
    const float4 G4 = band ? f4(TT::GG + c32) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float x[4] = {X.x, X.y, X.z, X.w};
    const float dn[4] = {DN.x, DN.y, DN.z, DN.w}, rt[4] = {X.y, X.z, X.w, RT};
    const float b1[4] = {E1.x + W1.x, E1.y + W1.y, E1.z + W1.z, E1.w + W1.w};
    const float b2[4] = {E2.x + W2.x, E2.y + W2.y, E2.z + W2.z, E2.w + W2.w};
    const float gg[4] = {G4.x, G4.y, G4.z, G4.w};
    float wo1[4], wo2[4], eo1[4], eo2[4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
      wb_point(m, x[t], dn[t] - x[t], rt[t] - x[t], b1[t], b2[t], gg[t], v1[t], v2[t], wo1[t],
               wo2[t], eo1[t], eo2[t]);
    st4(a.w1o + o, make_float4(wo1[0], wo1[1], wo1[2], wo1[3]));
    st4(a.w2o + o, make_float4(wo2[0], wo2[1], wo2[2], wo2[3]));
    st4(a.e1o + o, make_float4(eo1[0], eo1[1], eo1[2], eo1[3]));
    st4(a.e2o + o, make_float4(eo2[0], eo2[1], eo2[2], eo2[3]));
    if (chk) {
      const float4 P = f4(TT::PO + c32);
      const float po[4] = {P.x, P.y, P.z, P.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const double df = (double)x[t] - (double)po[t];
        part[0] += df * df;
        part[1] += (double)po[t] * (double)po[t];
      }
    }
  }
  if (chk) block_sum_store<2>(part, a.partials + 2 * (blockIdx.y * gridDim.x + blockIdx.x));
}

__global__ void __launch_bounds__(kTileX* kTileY) k_repulsion(const RepArgs a) {
  __shared__ TileSmem sm;
  const int i0 = blockIdx.y * kTileY, j0 = blockIdx.x * kTileX;
  const int N = a.geo.N;
  float v1, v2;
  tile_window_sum(sm, a.geo, a.mod, i0, j0,
                  [&](int i, int j, float& u1, float& u2) {
                    const size_t o = (size_t)i * N + j;
                    const float h = band_h(a.phi[o], a.mod);
                    if (h != 0.f) {
                      u1 = h * a.w1[o];
                      u2 = h * a.w2[o];
                    }
                  },
                  v1, v2);
  const int i = i0 + threadIdx.y, j = j0 + threadIdx.x;
  if (i < a.geo.M && j < N) {
    a.v1[(size_t)i * N + j] = v1;
    a.v2[(size_t)i * N + j] = v2;
  }
}

// Discrete energy: per-pixel terms in FP32, accumulated in FP64.
__global__ void __launch_bounds__(kTileX* kTileY) k_energy(const EnergyArgs a) {
  __shared__ TileSmem sm;
  const int i0 = blockIdx.y * kTileY, j0 = blockIdx.x * kTileX;
  const int M = a.geo.M, N = a.geo.N;
  const Model& m = a.mod;
  auto grad = [&](int i, int j, float& d1, float& d2) {
    const float x = a.phi[(size_t)i * N + j];
    d1 = a.phi[(size_t)(i == M - 1 ? 0 : i + 1) * N + j] - x;
    d2 = a.phi[(size_t)i * N + (j == N - 1 ? 0 : j + 1)] - x;
  };
  float v1, v2;
  tile_window_sum(sm, a.geo, m, i0, j0,
                  [&](int i, int j, float& u1, float& u2) {
                    const float h = band_h(a.phi[(size_t)i * N + j], m);
                    if (h != 0.f) {
                      float d1, d2;
                      grad(i, j, d1, d2);
                      u1 = h * d1;
                      u2 = h * d2;
                    }
                  },
                  v1, v2);
  const int i = i0 + threadIdx.y, j = j0 + threadIdx.x;
  double part[3] = {0.0, 0.0, 0.0};
  if (i < M && j < N) {
    const size_t o = (size_t)i * N + j;
    const float x = a.phi[o];
    float d1, d2;
    grad(i, j, d1, d2);
    const double gg = a.g[o];
    part[0] = gg * (double)sqrtf(d1 * d1 + d2 * d2) * (double)deps(x, m.eps);
    part[1] = gg * (1.0 - (double)heps(x, m.eps));
    part[2] = -(double)band_h(x, m) * ((double)d1 * v1 + (double)d2 * v2);
  }
  block_sum_store<3>(part, a.partials + 3 * (blockIdx.y * gridDim.x + blockIdx.x));
}

// Sum the per-CTA partials in a fixed order (one CTA, deterministic).
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ partials, int nblocks,
                                                int ncomp, double* __restrict__ out) {
  __shared__ double red[4][256];
  for (int c = 0; c < ncomp; ++c) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(size_t)b * ncomp + c];
    red[c][threadIdx.x] = s;
  }
  __syncthreads();
  for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
      for (int c = 0; c < ncomp; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < ncomp; ++c) out[c] = red[c][0];
}

// Alg. 1 initialisation: w = grad phi (forward, periodic), b = 0, i.e. e = -w.
__global__ void k_init_wb(const float* __restrict__ phi, float* __restrict__ w1,
                          float* __restrict__ w2, float* __restrict__ e1, float* __restrict__ e2,
                          Geo geo) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= geo.N) return;
  const size_t o = (size_t)i * geo.N + j;
  const float x = phi[o];
  const float d1 = phi[(size_t)(i == geo.M - 1 ? 0 : i + 1) * geo.N + j] - x;
  const float d2 = phi[(size_t)i * geo.N + (j == geo.N - 1 ? 0 : j + 1)] - x;
  w1[o] = d1;
  w2[o] = d2;
  e1[o] = -d1;
  e2[o] = -d2;
}

__global__ void k_axpb(const float* __restrict__ a, const float* __restrict__ b, float sign,
                       float* __restrict__ out, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x)
    out[q] = a[q] + sign * b[q];
}

__global__ void k_mask(const float* __restrict__ phi, unsigned char* __restrict__ mask, int ld,
                       Geo geo) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= geo.N) return;
  mask[(size_t)i * ld + j] = phi[(size_t)i * geo.N + j] < 0.f ? 1 : 0;
}

// Edge detector, Eq. (1): blur along rows (index i), then columns, replicated
// border; central differences inside, one-sided on the border.
__global__ void k_blur_i(const EdgeArgs a, const float* __restrict__ f, int ld,
                         float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= a.geo.N) return;
  float s = 0.f;
  for (int t = -a.r; t <= a.r; ++t) {
    const int ii = min(max(i + t, 0), a.geo.M - 1);
    s = fmaf(a.k[t + a.r], f[(size_t)ii * ld + j], s);
  }
  out[(size_t)i * a.geo.N + j] = s;
}

__global__ void k_blur_j(const EdgeArgs a, const float* __restrict__ in, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= a.geo.N) return;
  float s = 0.f;
  for (int t = -a.r; t <= a.r; ++t) {
    const int jj = min(max(j + t, 0), a.geo.N - 1);
    s = fmaf(a.k[t + a.r], in[(size_t)i * a.geo.N + jj], s);
  }
  out[(size_t)i * a.geo.N + j] = s;
}

__global__ void k_edge_g(const EdgeArgs a, const float* __restrict__ b, float* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  const int M = a.geo.M, N = a.geo.N;
  if (j >= N) return;
  auto B = [&](int ii, int jj) { return b[(size_t)ii * N + jj]; };
  float gi, gj;
  if (M == 1) gi = 0.f;
  else if (i == 0) gi = B(1, j) - B(0, j);
  else if (i == M - 1) gi = B(M - 1, j) - B(M - 2, j);
  else gi = 0.5f * (B(i + 1, j) - B(i - 1, j));
  if (N == 1) gj = 0.f;
  else if (j == 0) gj = B(i, 1) - B(i, 0);
  else if (j == N - 1) gj = B(i, N - 1) - B(i, N - 2);
  else gj = 0.5f * (B(i, j + 1) - B(i, j - 1));
  const float m2 = gi * gi + gj * gj;
  const float mag = a.s_pow == 2 ? m2 : sqrtf(m2);
  g[(size_t)i * N + j] = 1.f / (1.f + a.rho * mag);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
size_t rowfwd_smem(int T, int L, int R, int CW, int mode) {
  const size_t S = (size_t)L + (L >> 4);
  size_t bytes = (size_t)T * S * sizeof(float2);
  if (mode == kRowRHS) {
    const size_t CWH = (size_t)CW + 2 * R, TH = (size_t)T + 2 * R;
    bytes += (2 * TH * CWH + 2 * (size_t)T * CWH) * sizeof(float);
  }
  return bytes;
}
size_t colsolve_smem(int M) { return (size_t)M * kColCB * sizeof(float2); }
size_t rowinv_smem(int T, int L) { return (size_t)T * (L + (L >> 4)) * sizeof(float2); }
size_t tile_smem(int) { return sizeof(TileSmem); }

int tile_blocks(const Geo& geo) {
  return ((geo.N + kTileX - 1) / kTileX) * ((geo.M + kTileY - 1) / kTileY);
}

// Allow each kernel the largest dynamic shared memory the device grants on
// top of its own static shared memory.
template <class K>
static cudaError_t allow_big_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

cudaError_t configure_kernels() {
  cudaError_t e;
  if ((e = allow_big_smem(k_rowfwd<kRowRHS>))) return e;
  if ((e = allow_big_smem(k_rowfwd<kRowLOAD>))) return e;
  if ((e = allow_big_smem(k_colsolve))) return e;
  if ((e = allow_big_smem(k_rowinv<kInvADD>))) return e;
  if ((e = allow_big_smem(k_rowinv<kInvSTORE>))) return e;
#define SR_CASE(r)                                                   \
  if ((e = allow_big_smem(k_prep<r>)) != cudaSuccess) return e;      \
  if ((e = allow_big_smem(k_wb_update<r>)) != cudaSuccess) return e; \
  if ((e = allow_big_smem(k_prep_tma<r>)) != cudaSuccess) return e;  \
  if ((e = allow_big_smem(k_wb_tma<r>)) != cudaSuccess) return e;
  SR_FOR_R(SR_CASE)
#undef SR_CASE
  return cudaSuccess;
}

cudaError_t launch_rowfwd(const RowFwdArgs& a, int mode, int nthreads, cudaStream_t s) {
  const int grid = (a.geo.M + a.T - 1) / a.T;
  const size_t sm = rowfwd_smem(a.T, a.geo.L, a.mod.R, a.CW, mode);
  if (mode == kRowRHS) k_rowfwd<kRowRHS><<<grid, nthreads, sm, s>>>(a);
  else k_rowfwd<kRowLOAD><<<grid, nthreads, sm, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_colsolve(const ColArgs& a, cudaStream_t s) {
  const int grid = a.geo.L / kColCB;
  const int nthreads = a.geo.M * kColCB / kE;
  k_colsolve<<<grid, nthreads, colsolve_smem(a.geo.M), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rowinv(const RowInvArgs& a, int mode, int nthreads, cudaStream_t s) {
  const int grid = (a.geo.M + a.T - 1) / a.T;
  const size_t sm = rowinv_smem(a.T, a.geo.L);
  if (mode == kInvADD) k_rowinv<kInvADD><<<grid, nthreads, sm, s>>>(a);
  else k_rowinv<kInvSTORE><<<grid, nthreads, sm, s>>>(a);
  return cudaGetLastError();
}

static dim3 tile_grid(const Geo& geo) {
  return dim3((geo.N + kTileX - 1) / kTileX, (geo.M + kTileY - 1) / kTileY);
}

static dim3 tile32_grid(const Geo& geo) { return dim3((geo.N + kT - 1) / kT, (geo.M + kT - 1) / kT); }

int tile32_blocks(const Geo& geo) { return ((geo.N + kT - 1) / kT) * ((geo.M + kT - 1) / kT); }

cudaError_t launch_wb_update(const WBArgs& a, cudaStream_t s) {
  const dim3 g = tile32_grid(a.geo), b(kTBX, kTBY);
  const size_t sm = tile32_smem(a.mod.R);
  switch (a.mod.R) {
#define SR_CASE(r) \
  case r: k_wb_update<r><<<g, b, sm, s>>>(a); break;
    SR_FOR_R(SR_CASE)
#undef SR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t tile_tma_smem(int R) {
  switch (R) {
#define SR_CASE(r) \
  case r: return (size_t)TileT<r>::FLOATS * sizeof(float) + 128;
    SR_FOR_R(SR_CASE)
#undef SR_CASE
  }
  return 0;
}

int tile_halo_x(int R) { return R > 4 ? 8 : 4; }
int tile_halo_y(int R) { return R > 1 ? R : 1; }

cudaError_t launch_prep_tma(const PrepArgs& a, const PrepMaps& tm, cudaStream_t s) {
  const dim3 g = tile32_grid(a.geo), b(kTBX, kTBY);
  const size_t sm = tile_tma_smem(a.mod.R);
  switch (a.mod.R) {
#define SR_CASE(r) \
  case r: k_prep_tma<r><<<g, b, sm, s>>>(a, tm); break;
    SR_FOR_R(SR_CASE)
#undef SR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_wb_tma(const WBArgs& a, const WBMaps& tm, cudaStream_t s) {
  const dim3 g = tile32_grid(a.geo), b(kTBX, kTBY);
  const size_t sm = tile_tma_smem(a.mod.R);
  switch (a.mod.R) {
#define SR_CASE(r) \
  case r: k_wb_tma<r><<<g, b, sm, s>>>(a, tm); break;
    SR_FOR_R(SR_CASE)
#undef SR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s) {
  const dim3 g = tile32_grid(a.geo), b(kTBX, kTBY);
  const size_t sm = tile32_smem(a.mod.R);
  switch (a.mod.R) {
#define SR_CASE(r) \
  case r: k_prep<r><<<g, b, sm, s>>>(a); break;
    SR_FOR_R(SR_CASE)
#undef SR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_repulsion(const RepArgs& a, cudaStream_t s) {
  k_repulsion<<<tile_grid(a.geo), dim3(kTileX, kTileY), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_energy(const EnergyArgs& a, cudaStream_t s) {
  k_energy<<<tile_grid(a.geo), dim3(kTileX, kTileY), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double* partials, int nblocks, int ncomp, double* out,
                          cudaStream_t s) {
  k_reduce<<<1, 256, 0, s>>>(partials, nblocks, ncomp, out);
  return cudaGetLastError();
}

static dim3 row_grid(const Geo& geo) { return dim3((geo.N + 127) / 128, geo.M); }

cudaError_t launch_init_wb(const float* phi, float* w1, float* w2, float* e1, float* e2, Geo geo,
                           cudaStream_t s) {
  k_init_wb<<<row_grid(geo), 128, 0, s>>>(phi, w1, w2, e1, e2, geo);
  return cudaGetLastError();
}

cudaError_t launch_axpb(const float* a, const float* b, float sign, float* out, size_t n,
                        cudaStream_t s) {
  const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
  k_axpb<<<grid, 256, 0, s>>>(a, b, sign, out, n);
  return cudaGetLastError();
}

cudaError_t launch_mask(const float* phi, unsigned char* mask, int ld, Geo geo, cudaStream_t s) {
  k_mask<<<row_grid(geo), 128, 0, s>>>(phi, mask, ld, geo);
  return cudaGetLastError();
}

cudaError_t launch_edge(const EdgeArgs& a, const float* f, int ld, float* tmp1, float* tmp2,
                        float* g, cudaStream_t s) {
  k_blur_i<<<row_grid(a.geo), 128, 0, s>>>(a, f, ld, tmp1);
  k_blur_j<<<row_grid(a.geo), 128, 0, s>>>(a, tmp1, tmp2);
  k_edge_g<<<row_grid(a.geo), 128, 0, s>>>(a, tmp2, g);
  return cudaGetLastError();
}

}  // namespace srk
