// Mixed-radix FFT passes of the phi solve (Eqs. (31)-(33)) for image sides
// that are not powers of two (the register-resident passes of sr_fft.cu need
// 2^k).  Same three passes and data layout: the forward row pass builds the
// packed half spectrum X[M][L] of the real rows (L = W/2, X[0] = X_0 + i X_{W/2}),
// the column pass transforms each column, divides by the symbol lambda and
// transforms back, the inverse row pass rebuilds the real rows.
//
// The transforms are Stockham autosort stages held in shared memory (two
// buffers, ping-pong): stage s of radix R with Ns = product of the earlier
// radices reads x[j + t n/R], t < R, multiplies by w^{t k} with
// w = exp(-2 pi i / (Ns R)) and k = j mod Ns, applies the length-R DFT and
// writes y[(j / Ns) Ns R + k + t Ns].  Radices 2, 4, 8, 16, 3 and 5 have
// dedicated butterflies; any other prime up to kGenMaxRadix goes through a
// direct length-R DFT with a table of its roots.
#include "sr_internal.h"

namespace srk {
namespace fftgen {

constexpr int kGenThreads = 128;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 mul_mi(float2 a, bool inv) {  // a * (-i), or a * i when inv
  return inv ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
__device__ __forceinline__ float2 mul_w(float2 a, float cr, float ci, bool inv) {
  const float s = inv ? ci : -ci;  // a * exp(-+ i theta), cos theta = cr, sin theta = ci
  return make_float2(a.x * cr - a.y * s, a.x * s + a.y * cr);
}

__device__ __forceinline__ void dft2(float2* x) {
  const float2 a = x[0], b = x[1];
  x[0] = cadd(a, b);
  x[1] = csub(a, b);
}
__device__ __forceinline__ void dft4(float2* x, bool inv) {
  const float2 a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
  const float2 a2 = cadd(x[1], x[3]), a3 = mul_mi(csub(x[1], x[3]), inv);
  x[0] = cadd(a0, a2);
  x[2] = csub(a0, a2);
  x[1] = cadd(a1, a3);
  x[3] = csub(a1, a3);
}
__device__ __forceinline__ void dft8(float2* x, bool inv) {
  float2 e[4] = {x[0], x[2], x[4], x[6]};
  float2 o[4] = {x[1], x[3], x[5], x[7]};
  dft4(e, inv);
  dft4(o, inv);
  const float c = 0.70710678118654752440f;
  o[1] = mul_w(o[1], c, c, inv);
  o[2] = mul_mi(o[2], inv);
  o[3] = mul_w(o[3], -c, c, inv);
  for (int m = 0; m < 4; ++m) {
    x[m] = cadd(e[m], o[m]);
    x[m + 4] = csub(e[m], o[m]);
  }
}
__device__ __forceinline__ void dft16(float2* x, bool inv) {
  float2 e[8], o[8];
  for (int m = 0; m < 8; ++m) {
    e[m] = x[2 * m];
    o[m] = x[2 * m + 1];
  }
  dft8(e, inv);
  dft8(o, inv);
  const float C1 = 0.92387953251128675613f, S1 = 0.38268343236508977173f;
  const float c = 0.70710678118654752440f;
  o[1] = mul_w(o[1], C1, S1, inv);
  o[2] = mul_w(o[2], c, c, inv);
  o[3] = mul_w(o[3], S1, C1, inv);
  o[4] = mul_mi(o[4], inv);
  o[5] = mul_w(o[5], -S1, C1, inv);
  o[6] = mul_w(o[6], -c, c, inv);
  o[7] = mul_w(o[7], -C1, S1, inv);
  for (int m = 0; m < 8; ++m) {
    x[m] = cadd(e[m], o[m]);
    x[m + 8] = csub(e[m], o[m]);
  }
}
// length 3: y0 = a + b + c, y1,2 = a - (b + c)/2 -+ i (sqrt 3 / 2)(b - c) (forward)
__device__ __forceinline__ void dft3(float2* x, bool inv) {
  const float s3 = inv ? -0.86602540378443864676f : 0.86602540378443864676f;
  const float2 a = x[0], b = x[1], c = x[2];
  const float2 t = cadd(b, c);
  const float2 m = make_float2(a.x - 0.5f * t.x, a.y - 0.5f * t.y);
  const float2 d = csub(b, c);
  x[0] = cadd(a, t);
  x[1] = make_float2(m.x + s3 * d.y, m.y - s3 * d.x);
  x[2] = make_float2(m.x - s3 * d.y, m.y + s3 * d.x);
}
// length 5 from the symmetric and antisymmetric sums of the pairs (1, 4), (2, 3)
__device__ __forceinline__ void dft5(float2* x, bool inv) {
  const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
  const float s1 = inv ? -0.95105651629515357212f : 0.95105651629515357212f;
  const float s2 = inv ? -0.58778525229247312917f : 0.58778525229247312917f;
  const float2 a = x[0];
  const float2 p1 = cadd(x[1], x[4]), m1 = csub(x[1], x[4]);
  const float2 p2 = cadd(x[2], x[3]), m2 = csub(x[2], x[3]);
  x[0] = cadd(a, cadd(p1, p2));
  const float2 r1 = make_float2(a.x + c1 * p1.x + c2 * p2.x, a.y + c1 * p1.y + c2 * p2.y);
  const float2 r2 = make_float2(a.x + c2 * p1.x + c1 * p2.x, a.y + c2 * p1.y + c1 * p2.y);
  // the forward transform multiplies the antisymmetric parts by -i
  const float2 i1 = make_float2(s1 * m1.y + s2 * m2.y, -(s1 * m1.x + s2 * m2.x));
  const float2 i2 = make_float2(s2 * m1.y - s1 * m2.y, -(s2 * m1.x - s1 * m2.x));
  x[1] = cadd(r1, i1);
  x[4] = csub(r1, i1);
  x[2] = cadd(r2, i2);
  x[3] = csub(r2, i2);
}

template <int R>
__host__ __device__ constexpr bool dedicated() {
  return R == 2 || R == 3 || R == 4 || R == 5 || R == 8 || R == 16;
}

template <int R>
__device__ __forceinline__ void dft_fixed(float2 (&x)[R], bool inv) {
  if constexpr (R == 2) dft2(x);
  else if constexpr (R == 3) dft3(x, inv);
  else if constexpr (R == 4) dft4(x, inv);
  else if constexpr (R == 5) dft5(x, inv);
  else if constexpr (R == 8) dft8(x, inv);
  else if constexpr (R == 16) dft16(x, inv);
}

// One Stockham stage of radix R over nseq sequences of length n (a -> b).
// Primes without a dedicated butterfly take the direct DFT y_q = sum_t x_t
// root[(t q) mod R], root[e] = exp(-2 pi i e / R) (conjugated when inv),
// each y_q written as soon as it is summed.
// x / d for x < 2^20 from magic = ceil(2^32 / d) (host-computed): exact, since
// x (magic d - 2^32) < 2^32 there.  d = 1 is passed as magic 0.
__device__ __forceinline__ int divm(int x, unsigned magic) {
  return magic ? (int)__umulhi((unsigned)x, magic) : x;
}

template <int R>
__device__ __forceinline__ void stage_r(const float2* a, float2* b, int nseq, int n, int Ns,
                                        unsigned mag_m, unsigned mag_ns, const float2* tw,
                                        const float2* root, bool inv) {
  const int m = n / R;
  for (int idx = threadIdx.x; idx < nseq * m; idx += blockDim.x) {
    const int q = divm(idx, mag_m), j = idx - q * m;
    const int jn = divm(j, mag_ns), k = j - jn * Ns;
    const float2* in = a + (size_t)q * n;
    float2* out = b + (size_t)q * n;
    float2 v[R];
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = in[j + t * m];
    if (Ns > 1) {
#pragma unroll
      for (int t = 1; t < R; ++t) {
        float2 w = __ldg(tw + (t - 1) * Ns + k);
        if (inv) w.y = -w.y;
        v[t] = cmul(v[t], w);
      }
    }
    const int o = jn * Ns * R + k;
    if constexpr (dedicated<R>()) {
      dft_fixed<R>(v, inv);
#pragma unroll
      for (int t = 0; t < R; ++t) out[o + t * Ns] = v[t];
    } else {
#pragma unroll 1
      for (int y = 0; y < R; ++y) {
        float2 acc = v[0];
        int e = 0;  // (t y) mod R
#pragma unroll
        for (int t = 1; t < R; ++t) {
          e += y;
          if (e >= R) e -= R;
          float2 w = __ldg(root + e);
          if (inv) w.y = -w.y;
          acc.x += v[t].x * w.x - v[t].y * w.y;
          acc.y += v[t].x * w.y + v[t].y * w.x;
        }
        out[o + y * Ns] = acc;
      }
    }
  }
}

// The transforms of nseq sequences of length P.n stored one after another in
// a; b is the second buffer.  Every thread of the block takes part; returns
// the buffer that holds the result (synchronised).
__device__ float2* stockham(float2* a, float2* b, int nseq, const GenPlan& P, bool inv) {
  const int n = P.n;
  for (int s = 0; s < P.nst; ++s) {
    const int Ns = P.ns[s];
    const float2* tw = P.tw + P.twoff[s];
    const float2* root = P.roots + P.rootoff[s];
    switch (P.radix[s]) {
#define SR_RADIX(r) \
  case r: stage_r<r>(a, b, nseq, n, Ns, P.mag_m[s], P.mag_ns[s], tw, root, inv); break;
      SR_RADIX(2) SR_RADIX(3) SR_RADIX(4) SR_RADIX(5) SR_RADIX(7) SR_RADIX(8) SR_RADIX(11)
      SR_RADIX(13) SR_RADIX(16) SR_RADIX(17) SR_RADIX(19) SR_RADIX(23) SR_RADIX(29) SR_RADIX(31)
#undef SR_RADIX
      default: break;  // the host builds plans from these radices only
    }
    __syncthreads();
    float2* tmp = a;
    a = b;
    b = tmp;
  }
  return a;
}

// ---------------------------------------------------------------------------
// rows, forward: z[n] = G[2n] + i G[2n+1], FFT_L, even/odd split -> X
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_rowfft_gen(const RowFwdArgs a, const GenPlan P) {
  extern __shared__ __align__(16) float2 gsm[];
  pdl_wait();
  pdl_trigger();
  const int L = a.geo.L, N = a.geo.N;
  const int r0 = blockIdx.x * a.T;
  const int nrow = min(a.T, a.geo.M - r0);
  float2* A = gsm;
  float2* B = gsm + (size_t)a.T * L;
  for (int idx = threadIdx.x; idx < nrow * L; idx += blockDim.x) {
    const int q = idx / L, t = idx - q * L;
    A[idx] = __ldg(reinterpret_cast<const float2*>(a.src + (size_t)(r0 + q) * N) + t);
  }
  __syncthreads();
  const float2* Z = stockham(A, B, nrow, P, false);
  for (int idx = threadIdx.x; idx < nrow * L; idx += blockDim.x) {
    const int q = idx / L, k = idx - q * L;
    const float2 Zk = Z[(size_t)q * L + k];
    float2* Xrow = a.X + (size_t)(r0 + q) * L;
    if (k == 0) {
      Xrow[0] = make_float2(Zk.x + Zk.y, Zk.x - Zk.y);
      continue;
    }
    const float2 Zm = Z[(size_t)q * L + (L - k)];
    const float2 Ev = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    const float2 D = make_float2(0.5f * (Zk.x - Zm.x), 0.5f * (Zk.y + Zm.y));
    const float2 O = make_float2(D.y, -D.x);
    Xrow[k] = cadd(Ev, cmul(__ldg(&a.twN[k]), O));
  }
}

// ---------------------------------------------------------------------------
// columns: CB columns of X per CTA, forward FFT_M, / (M N lambda), inverse
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_colsolve_gen(const ColArgs a, const GenPlan P, int CB) {
  extern __shared__ __align__(16) float2 gsm[];
  pdl_wait();
  pdl_trigger();
  const int M = a.geo.M, L = a.geo.L;
  const int c0 = blockIdx.x * CB;
  const int ncol = min(CB, L - c0);
  float2* A = gsm;
  float2* B = gsm + (size_t)CB * M;
  for (int idx = threadIdx.x; idx < ncol * M; idx += blockDim.x) {
    const int l = idx / ncol, c = idx - l * ncol;  // consecutive threads: consecutive columns
    A[(size_t)c * M + l] = a.X[(size_t)l * L + c0 + c];
  }
  __syncthreads();
  float2* F = stockham(A, B, ncol, P, false);
  float2* other = F == A ? B : A;
  const float inv_mn = 1.f / ((float)M * (float)a.geo.N);
  for (int idx = threadIdx.x; idx < ncol * M; idx += blockDim.x) {
    const int c = idx / M, l = idx - c * M;
    const int k = c0 + c;
    const float2 Cl = F[(size_t)c * M + l];
    float2 r;
    if (k == 0) {
      // column 0 packs the DC and Nyquist columns of the row transforms:
      // split them with the conjugate pair (l, M - l), each gets its symbol
      const float2 Cm = F[(size_t)c * M + (l == 0 ? 0 : M - l)];
      const float sA = inv_mn / (1.f + __ldg(a.aM + l) + __ldg(a.aN));
      const float sB = inv_mn / (1.f + __ldg(a.aM + l) + __ldg(a.aN + L));
      const float2 Av = make_float2(0.5f * (Cl.x + Cm.x) * sA, 0.5f * (Cl.y - Cm.y) * sA);
      const float2 D = make_float2(0.5f * (Cl.x - Cm.x), 0.5f * (Cl.y + Cm.y));
      const float2 Bv = make_float2(D.y * sB, -D.x * sB);
      r = make_float2(Av.x - Bv.y, Av.y + Bv.x);
    } else {
      const float sc = inv_mn / (1.f + __ldg(a.aM + l) + __ldg(a.aN + k));
      r = make_float2(Cl.x * sc, Cl.y * sc);
    }
    other[(size_t)c * M + l] = r;  // out of place: column 0 reads F at M - l
  }
  __syncthreads();
  const float2* Y = stockham(other, F, ncol, P, true);
  for (int idx = threadIdx.x; idx < ncol * M; idx += blockDim.x) {
    const int l = idx / ncol, c = idx - l * ncol;
    a.X[(size_t)l * L + c0 + c] = Y[(size_t)c * M + l];
  }
}

// ---------------------------------------------------------------------------
// rows, inverse: rebuild the length-L sequence, inverse FFT_L, interleave,
// add psi (ADD) or store
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_rowifft_gen(const RowInvArgs a, const GenPlan P, int add) {
  extern __shared__ __align__(16) float2 gsm[];
  pdl_wait();
  pdl_trigger();
  const int L = a.geo.L, N = a.geo.N;
  const int r0 = blockIdx.x * a.T;
  const int nrow = min(a.T, a.geo.M - r0);
  float2* A = gsm;
  float2* B = gsm + (size_t)a.T * L;
  for (int idx = threadIdx.x; idx < nrow * L; idx += blockDim.x) {
    const int q = idx / L, k = idx - q * L;
    const float2* Xrow = a.X + (size_t)(r0 + q) * L;
    const float2 xk = __ldg(Xrow + k);
    if (k == 0) {
      A[idx] = make_float2(xk.x + xk.y, xk.x - xk.y);  // (X_0 + X_{N/2}, X_0 - X_{N/2})
      continue;
    }
    const float2 xm = __ldg(Xrow + (L - k));
    // Xe = X_k + conj X_{L-k},  Xo = (X_k - conj X_{L-k}) exp(+2 pi i k / N)
    const float2 Xe = make_float2(xk.x + xm.x, xk.y - xm.y);
    const float2 D = make_float2(xk.x - xm.x, xk.y + xm.y);
    const float2 Xo = cmul(D, cconj(__ldg(&a.twN[k])));
    A[idx] = make_float2(Xe.x - Xo.y, Xe.y + Xo.x);
  }
  __syncthreads();
  const float2* Z = stockham(A, B, nrow, P, true);
  for (int idx = threadIdx.x; idx < nrow * L; idx += blockDim.x) {
    const int q = idx / L, t = idx - q * L;
    float2 r = Z[idx];
    float2* orow = reinterpret_cast<float2*>(a.out + (size_t)(r0 + q) * N);
    if (add) {
      const float2 p = __ldg(reinterpret_cast<const float2*>(a.psi_in + (size_t)(r0 + q) * N) + t);
      r = make_float2(p.x + r.x, p.y + r.y);
    }
    orow[t] = r;
  }
}

}  // namespace fftgen

using fftgen::kGenThreads;

// sequences per CTA for `count` sequences of length n: the two buffers stay
// within kGenSmemFloat2 values and hold at most 16 sequences.  Alone, an image
// spreads over a few hundred CTAs (about count / 256 sequences each); in a
// batched group the other images fill the GPU, so the CTAs are filled up.
int gen_rows_per_cta(int n, int count, bool batched) {
  const int fit = n >= kGenSmemFloat2 / 2 ? 1 : kGenSmemFloat2 / 2 / n;
  int t = batched ? 16 : count / 256;
  if (t < 1) t = 1;
  if (t > 16) t = 16;
  return t < fit ? t : fit;
}

// threads per CTA: 256 for the filled CTAs of a group, 128 alone
static int gen_threads(bool batched) { return batched ? 256 : kGenThreads; }

size_t gen_smem(int nseq, int n) { return 2 * (size_t)nseq * n * sizeof(float2); }

cudaError_t configure_fftgen() {
  cudaError_t e = cudaSuccess;
  const int bytes = (int)(kGenSmemFloat2 * sizeof(float2));
  for (auto k : {(const void*)fftgen::k_rowfft_gen, (const void*)fftgen::k_colsolve_gen,
                 (const void*)fftgen::k_rowifft_gen}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return e;
}

cudaError_t launch_rowfft_gen(const RowFwdArgs& a, const GenPlan& P, bool batched,
                              cudaStream_t s) {
  const int grid = (a.geo.M + a.T - 1) / a.T;
  return launch_k(fftgen::k_rowfft_gen, dim3(grid), dim3(gen_threads(batched)),
                  gen_smem(a.T, a.geo.L), s, a, P);
}

cudaError_t launch_colsolve_gen(const ColArgs& a, const GenPlan& P, bool batched,
                                cudaStream_t s) {
  const int CB = gen_rows_per_cta(a.geo.M, a.geo.L, batched);
  const int grid = (a.geo.L + CB - 1) / CB;
  return launch_k(fftgen::k_colsolve_gen, dim3(grid), dim3(gen_threads(batched)),
                  gen_smem(CB, a.geo.M), s, a, P, CB);
}

cudaError_t launch_rowifft_gen(const RowInvArgs& a, const GenPlan& P, bool add, bool batched,
                               cudaStream_t s) {
  const int grid = (a.geo.M + a.T - 1) / a.T;
  return launch_k(fftgen::k_rowifft_gen, dim3(grid), dim3(gen_threads(batched)),
                  gen_smem(a.T, a.geo.L), s, a, P, add ? 1 : 0);
}

}  // namespace srk
