// Register-resident Stockham FFT passes of the phi solve (Eqs. (31)-(33)).
//
// A thread owns 16 values x[m] = seq[u + (L/16) m] of one sequence.  In every
// Stockham stage (radix R, Ns = product of the earlier radices) the inputs of
// the thread's 16/R butterflies are exactly those 16 values, so the
// butterflies run in registers; only the outputs move, through shared memory,
// to the positions the next stage reads.  The outputs of the last stage land
// back in the thread's own positions (natural order).  So the first stage
// reads global memory directly, the last stage writes it directly, and a
// length-L transform needs ceil(log16 L) - 1 shared-memory exchanges.
//
//   k_rowfft<LOGL>    rows: z[n] = G[2n] + i G[2n+1] -> FFT_L -> even/odd split
//                     -> packed half spectrum X[0] = X_0 + i X_{N/2}, X[k]
//   k_colsolve2<..>   columns: FFT_M, multiply by 1/(M N lambda), inverse FFT_M
//   k_rowifft<LOGL>   rows: rebuild the length-L sequence, inverse FFT_L,
//                     interleave, add psi (increment form) or store
#include <cmath>
#include <vector>

#include "sr_dft.cuh"
#include "sr_internal.h"
#include "sr_tma.cuh"

namespace srk {
namespace fft2 {

using namespace srk::cdft;

// ---------------------------------------------------------------------------
// rows, forward: packed half spectrum of the real rows of src
// ---------------------------------------------------------------------------
template <int LOGL, int LOGE>
__global__ void __launch_bounds__(512) k_rowfft(const RowFwdArgs a) {
  constexpr int E = 1 << LOGE;
  constexpr int L = 1 << LOGL, LOGTP = LOGL - LOGE, TP = 1 << LOGTP;
  constexpr int S = L + L / 16;
  extern __shared__ __align__(16) float2 smem2[];
  const int tid = threadIdx.x;
  const int t = tid >> LOGTP, u = tid & (TP - 1);
  const int i = blockIdx.x * a.T + t;
  const bool live = i < a.geo.M;
  float2* base = smem2 + t * S;
  const float2* stw = LOGE == 4 ? a.fft.tws16 : a.fft.tws8;
  pdl_wait();
  pdl_trigger();
  float2 x[E];
  const float2* row = reinterpret_cast<const float2*>(a.src + (size_t)(live ? i : 0) * a.geo.N);
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = live ? __ldg(row + u + (m << LOGTP)) : make_float2(0.f, 0.f);
  stages<LOGL, LOGE, 0, false, 1, false, true>(x, base, u, stw);
  // even/odd split needs Z_{L-k}: exchange through shared memory
#pragma unroll
  for (int m = 0; m < E; ++m) base[pad(u + (m << LOGTP))] = x[m];
  __syncthreads();
  if (!live) return;
  float2* Xrow = a.X + (size_t)i * L;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = u + (m << LOGTP);
    const float2 Zk = x[m];
    if (k == 0) {
      Xrow[0] = make_float2(Zk.x + Zk.y, Zk.x - Zk.y);
      continue;
    }
    const float2 Zm = base[pad(L - k)];
    const float2 E = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    const float2 D = make_float2(0.5f * (Zk.x - Zm.x), 0.5f * (Zk.y + Zm.y));
    const float2 O = make_float2(D.y, -D.x);
    Xrow[k] = cadd(E, cmul(__ldg(&a.twN[k]), O));
  }
}

// ---------------------------------------------------------------------------
// rows, inverse: out = psi_in + x (ADD) or out = x (STORE)
// ---------------------------------------------------------------------------
template <int LOGL, int LOGE, bool ADD>
__global__ void __launch_bounds__(512) k_rowifft(const RowInvArgs a) {
  constexpr int E = 1 << LOGE;
  constexpr int L = 1 << LOGL, LOGTP = LOGL - LOGE, TP = 1 << LOGTP;
  constexpr int S = L + L / 16;
  extern __shared__ __align__(16) float2 smem2[];
  const int tid = threadIdx.x;
  const int t = tid >> LOGTP, u = tid & (TP - 1);
  const int i = blockIdx.x * a.T + t;
  const bool live = i < a.geo.M;
  const int ii = live ? i : 0;
  float2* base = smem2 + t * S;
  const float2* stw = LOGE == 4 ? a.fft.tws16 : a.fft.tws8;
  pdl_wait();
  pdl_trigger();
  float2 p[E];
  if (ADD) {
    const float2* prow = reinterpret_cast<const float2*>(a.psi_in + (size_t)ii * a.geo.N);
#pragma unroll
    for (int m = 0; m < E; ++m) p[m] = __ldg(prow + u + (m << LOGTP));
  }
  const float2* Xrow = a.X + (size_t)ii * L;
  float2 xk[E], xm[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = u + (m << LOGTP);
    xk[m] = __ldg(Xrow + k);
    xm[m] = __ldg(Xrow + ((L - k) & (L - 1)));
  }
  float2 x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = u + (m << LOGTP);
    if (k == 0) {
      x[m] = make_float2(xk[m].x + xk[m].y, xk[m].x - xk[m].y);  // (X_0 + X_{N/2}, X_0 - X_{N/2})
      continue;
    }
    // Xe = X_k + conj X_{L-k},  Xo = (X_k - conj X_{L-k}) exp(+2 pi i k / N)
    const float2 Xe = make_float2(xk[m].x + xm[m].x, xk[m].y - xm[m].y);
    const float2 D = make_float2(xk[m].x - xm[m].x, xk[m].y + xm[m].y);
    const float2 Xo = cmul(D, cconj(__ldg(&a.twN[k])));
    x[m] = make_float2(Xe.x - Xo.y, Xe.y + Xo.x);
  }
  stages<LOGL, LOGE, 0, true, 1, false, true>(x, base, u, stw);
  if (!live) return;
  float2* orow = reinterpret_cast<float2*>(a.out + (size_t)i * a.geo.N);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    float2 r = x[m];
    if (ADD) r = make_float2(p[m].x + r.x, p[m].y + r.y);
    orow[u + (m << LOGTP)] = r;
  }
}

// ---------------------------------------------------------------------------
// columns: CB adjacent columns of X per CTA, thread (u, c) with c fastest
// ---------------------------------------------------------------------------
template <int LOGM, int CB, int LOGE>
__host__ __device__ constexpr int col_threads() { return CB * (1 << LOGM) / (1 << LOGE); }
template <int LOGM, int CB, int LOGE>
__host__ __device__ constexpr int col_min_blocks() {
  return (LOGE == 3 && col_threads<LOGM, CB, LOGE>() <= 512) ? 3
         : (col_threads<LOGM, CB, LOGE>() <= 256)            ? 2
                                                              : 1;
}

template <int LOGM, int CB, int LOGE, bool DB, int MINB>
__global__ void __launch_bounds__(col_threads<LOGM, CB, LOGE>(), MINB)
    k_colsolve2(const ColArgs a) {
  constexpr int E = 1 << LOGE;
  constexpr int M = 1 << LOGM, LOGTP = LOGM - LOGE;
  extern __shared__ __align__(16) float2 smem2[];
  const int tid = threadIdx.x;
  const int c = tid % CB, u = tid / CB;
  const int L = a.geo.L;
  const int c0 = blockIdx.x * CB;
  const int k = c0 + c;
  float2* base = smem2 + c;
  float2* base2 = DB ? base + CB * (M + M / 16) : nullptr;
  float2* stw = smem2 + (DB ? 2 : 1) * CB * (M + M / 16);
  float* sM = reinterpret_cast<float*>(stw + TwPlan<LOGM, LOGE>::TOTAL);
  // the symbol (constant tables) is fetched before the data, so that the
  // scaling between the two transforms waits on shared memory only
  const float ak = a.aN[k];
  const float a0 = a.aN[0], aNy = a.aN[L];
  for (int q = threadIdx.x; q < M; q += blockDim.x) sM[q] = __ldg(a.aM + q);
  stage_table<TwPlan<LOGM, LOGE>::TOTAL>(stw, LOGE == 4 ? a.fft.tws16 : a.fft.tws8);
  pdl_wait();
  pdl_trigger();
  float2 x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = a.X[(size_t)(u + (m << LOGTP)) * L + k];
  if constexpr (TwPlan<LOGM, LOGE>::NST == 1) __syncthreads();  // no exchange barrier before use
  stages<LOGM, LOGE, 0, false, CB, DB>(x, base, u, stw, base2);
  const float inv_mn = 1.f / ((float)M * (float)a.geo.N);
  if (c0 == 0) {
    // column 0 packs the DC and Nyquist columns of the row transforms: split
    // them with the conjugate pair (l, M - l) so each gets its own symbol
    if (c == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) base[pad(u + (m << LOGTP)) * CB] = x[m];
    }
    __syncthreads();
    if (c == 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int l = u + (m << LOGTP);
        const float2 Cl = x[m], Cm = base[pad((M - l) & (M - 1)) * CB];
        const float sA = inv_mn / (1.f + sM[l] + a0);
        const float sB = inv_mn / (1.f + sM[l] + aNy);
        const float2 A = make_float2(0.5f * (Cl.x + Cm.x) * sA, 0.5f * (Cl.y - Cm.y) * sA);
        const float2 D = make_float2(0.5f * (Cl.x - Cm.x), 0.5f * (Cl.y + Cm.y));
        const float2 B = make_float2(D.y * sB, -D.x * sB);
        x[m] = make_float2(A.x - B.y, A.y + B.x);
      }
    }
    __syncthreads();
  }
  if (k != 0) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float sc = __fdividef(inv_mn, 1.f + sM[u + (m << LOGTP)] + ak);  // lambda >= 1
      x[m] = make_float2(x[m].x * sc, x[m].y * sc);
    }
  }
  stages<LOGM, LOGE, 0, true, CB, DB>(x, base, u, stw, base2);
#pragma unroll
  for (int m = 0; m < E; ++m) a.X[(size_t)(u + (m << LOGTP)) * L + k] = x[m];
}

// ---------------------------------------------------------------------------
// columns, persistent with TMA: each CTA walks over column blocks; the block
// it works on was brought into shared memory by a 2-D TMA load (boxes of
// CB columns x up to 256 rows) while the previous block was computed, and
// goes back by TMA store.  The shared buffer of a block doubles as the
// exchange buffer of its FFT stages once the values are in registers.
// ---------------------------------------------------------------------------
// float2 per TMA column buffer: room for the padded exchange layout, rounded
// up to 128 bytes so the second buffer and every box stay 128-byte aligned
template <int LOGM, int CB>
__host__ __device__ constexpr int col_tma_buf() {
  return ((((1 << LOGM) + (1 << LOGM) / 16) * CB + 15) / 16) * 16;
}
template <int LOGM, int CB>
__host__ __device__ constexpr size_t col_tma_smem() {
  return 2 * (size_t)col_tma_buf<LOGM, CB>() * sizeof(float2) +
         (size_t)TwPlan<LOGM, 4>::TOTAL * sizeof(float2) + (size_t)(1 << LOGM) * sizeof(float) + 128 +
         3 * sizeof(uint64_t);
}

template <int LOGM, int CB, int LOGE>
__global__ void __launch_bounds__(col_threads<LOGM, CB, LOGE>(), 1)
    k_colsolve_tma(const ColArgs a, const __grid_constant__ CUtensorMap tmX) {
  pdl_wait();
  pdl_trigger();
  constexpr int E = 1 << LOGE, M = 1 << LOGM, LOGTP = LOGM - LOGE;
  constexpr int BOXR = M < 256 ? M : 256;
  constexpr int NBOX = M / BOXR;
  constexpr int BUF = col_tma_buf<LOGM, CB>();
  constexpr uint32_t BYTES = (uint32_t)M * CB * sizeof(float2);
  // dynamic shared memory: [up to 128 B of alignment][buffer 0][buffer 1][tables]
  // [3 mbarriers: the two buffers' and one that nothing arrives on, waited on
  // only when a failure-path test asks for a stall]
  extern __shared__ __align__(16) unsigned char smem_tma[];
  float2* smem2 = reinterpret_cast<float2*>(
      (reinterpret_cast<uintptr_t>(smem_tma) + 127) & ~static_cast<uintptr_t>(127));
  float2* stw = smem2 + 2 * BUF;
  float* s_aM = reinterpret_cast<float*>(stw + TwPlan<LOGM, LOGE>::TOTAL);
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_aM + M);
  stage_table<TwPlan<LOGM, LOGE>::TOTAL>(stw, a.fft.tws16);
  for (int q = threadIdx.x; q < M; q += blockDim.x) s_aM[q] = __ldg(a.aM + q);
  const int tid = threadIdx.x;
  const int c = tid % CB, u = tid / CB;
  const int L = a.geo.L, nb = L / CB;
  const float inv_mn = 1.f / ((float)M * (float)a.geo.N);
  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::mbar_init(&bar[2], 1);
    tma::mbar_init_fence();
  }
  __syncthreads();
  int blk = blockIdx.x;
  if (tid == 0 && blk < nb) {
    tma::mbar_expect_tx(&bar[0], BYTES);
#pragma unroll
    for (int q = 0; q < NBOX; ++q)
      tma::load_2d(smem2 + q * BOXR * CB, &tmX, 2 * CB * blk, q * BOXR, &bar[0]);
  }
  for (int it = 0; blk < nb; blk += gridDim.x, ++it) {
    const int b = it & 1;
    const uint32_t par = (it >> 1) & 1;
    float2* B = smem2 + b * BUF;
    const int nxt = blk + gridDim.x;
    if (tid == 0 && nxt < nb) {
      tma::store_wait_read();  // the other buffer's stores have read it
      float2* Bn = smem2 + (1 - b) * BUF;
      tma::mbar_expect_tx(&bar[1 - b], BYTES);
#pragma unroll
      for (int q = 0; q < NBOX; ++q)
        tma::load_2d(Bn + q * BOXR * CB, &tmX, 2 * CB * nxt, q * BOXR, &bar[1 - b]);
    }
    const bool ok = (a.stall_cycles > 0 && it == 0) ? tma::mbar_wait(&bar[2], 0, a.stall_cycles)
                                                    : tma::mbar_wait(&bar[b], par);
    if (!__syncthreads_and(ok)) {
      // drain this CTA's transfers before it exits: the load being waited
      // for, the prefetch of the next block, the stores of earlier blocks
      if (tid == 0) {
        tma::on_timeout(&bar[b], par, a.err);
        if (nxt < nb) tma::mbar_wait(&bar[1 - b], ((it + 1) >> 1) & 1);
        tma::store_wait_all();
      }
      return;
    }
    const int k = blk * CB + c;
    float2 x[E];
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = B[(u + (m << LOGTP)) * CB + c];
    __syncthreads();  // B is now the exchange buffer
    float2* base = B + c;
    stages<LOGM, LOGE, 0, false, CB>(x, base, u, stw);
    if (blk == 0) {
      if (c == 0) {
#pragma unroll
        for (int m = 0; m < E; ++m) base[pad(u + (m << LOGTP)) * CB] = x[m];
      }
      __syncthreads();
      if (c == 0) {
        const float aNy = a.aN[L];
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int l = u + (m << LOGTP);
          const float2 Cl = x[m], Cm = base[pad((M - l) & (M - 1)) * CB];
          const float sA = inv_mn / (1.f + s_aM[l] + a.aN[0]);
          const float sB = inv_mn / (1.f + s_aM[l] + aNy);
          const float2 A = make_float2(0.5f * (Cl.x + Cm.x) * sA, 0.5f * (Cl.y - Cm.y) * sA);
          const float2 D = make_float2(0.5f * (Cl.x - Cm.x), 0.5f * (Cl.y + Cm.y));
          const float2 Bq = make_float2(D.y * sB, -D.x * sB);
          x[m] = make_float2(A.x - Bq.y, A.y + Bq.x);
        }
      }
      __syncthreads();
    }
    if (k != 0) {
      const float ak = a.aN[k];
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float sc = inv_mn / (1.f + s_aM[u + (m << LOGTP)] + ak);
        x[m] = make_float2(x[m].x * sc, x[m].y * sc);
      }
    }
    stages<LOGM, LOGE, 0, true, CB>(x, base, u, stw);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) B[(u + (m << LOGTP)) * CB + c] = x[m];
    tma::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
#pragma unroll
      for (int q = 0; q < NBOX; ++q) tma::store_2d(&tmX, B + q * BOXR * CB, 2 * CB * blk, q * BOXR);
      tma::store_commit();
    }
  }
  if (tid == 0) tma::store_wait_all();
}

}  // namespace fft2

// ---------------------------------------------------------------------------
// Host dispatch.  With set_attr the call only raises the kernel's dynamic
// shared-memory limit (done once per context, outside any graph capture).
// The schedule (values per thread E for rows and columns, columns per CTA)
// is chosen by the context's autotuner.
// ---------------------------------------------------------------------------
using namespace fft2;

template <class K>
static cudaError_t set_smem(K kernel, size_t smem) {
  // The attribute belongs to the kernel, not to a context: contexts of other
  // sizes launch the same instantiation with other shared-memory sizes, so
  // raise it to the device maximum once instead of to this context's size.
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int limit = optin - (int)fa.sharedSizeBytes;
  if ((int)smem > limit) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
}

template <int LOGL, int LOGE>
static cudaError_t rowfft_go(const RowFwdArgs& a, int nthreads, size_t smem, cudaStream_t s,
                             bool set_attr) {
  if (set_attr) return set_smem(k_rowfft<LOGL, LOGE>, smem);
  return launch_k(k_rowfft<LOGL, LOGE>, dim3((a.geo.M + a.T - 1) / a.T), dim3(nthreads), smem, s, a);
}

template <int LOGL, int LOGE>
static cudaError_t rowifft_go(const RowInvArgs& a, bool add, int nthreads, size_t smem,
                              cudaStream_t s, bool set_attr) {
  if (set_attr) {
    cudaError_t e = set_smem(k_rowifft<LOGL, LOGE, true>, smem);
    return e != cudaSuccess ? e : set_smem(k_rowifft<LOGL, LOGE, false>, smem);
  }
  const int grid = (a.geo.M + a.T - 1) / a.T;
  if (add) return launch_k(k_rowifft<LOGL, LOGE, true>, dim3(grid), dim3(nthreads), smem, s, a);
  return launch_k(k_rowifft<LOGL, LOGE, false>, dim3(grid), dim3(nthreads), smem, s, a);
}

template <int LOGM, int CB, int LOGE, bool DB = false, int MINB = col_min_blocks<LOGM, CB, LOGE>()>
static cudaError_t col_go(const ColArgs& a, cudaStream_t s, bool set_attr) {
  constexpr int M = 1 << LOGM;
  const size_t smem = ((size_t)(DB ? 2 : 1) * CB * (M + M / 16) + TwPlan<LOGM, LOGE>::TOTAL) *
                          sizeof(float2) +
                      (size_t)M * sizeof(float);
  if (set_attr) return set_smem(k_colsolve2<LOGM, CB, LOGE, DB, MINB>, smem);
  return launch_k(k_colsolve2<LOGM, CB, LOGE, DB, MINB>, dim3(a.geo.L / CB),
                  dim3(CB * M / (1 << LOGE)), smem, s, a);
}

static int ilog2_host(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

std::vector<float2> twiddle_table(int n, int len) {
  // exp(-2 pi i q / len), q in [0, n), computed in double and rounded once
  std::vector<float2> t(n);
  for (int q = 0; q < n; ++q) {
    const double a = -2.0 * M_PI * (double)q / (double)len;
    t[q] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  return t;
}

// Stage twiddles of the register FFT for a length-len transform with 2^logE
// values per thread: stage q >= 1 has Ns = 2^(logE q) and radix 2^logE (the
// last stage 2^(log2(len) mod logE) if that is not 1); its entries
// exp(-2 pi i k t / (Ns R)) are stored at [t - 1][k].
std::vector<float2> stage_twiddle_table(int len, int logE) {
  const int logL = ilog2_host(len);
  const int nst = (logL + logE - 1) / logE;
  std::vector<float2> v;
  for (int q = 1; q < nst; ++q) {
    const int logR = q < logL / logE ? logE : logL % logE;
    const int R = 1 << logR, Ns = 1 << (logE * q);
    for (int t = 1; t < R; ++t)
      for (int k = 0; k < Ns; ++k) {
        const double ang = -2.0 * M_PI * (double)k * (double)t / ((double)Ns * (double)R);
        v.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
      }
  }
  if (v.empty()) v.push_back(make_float2(1.f, 0.f));  // keep the allocation non-empty
  return v;
}

bool fft2_supported(const Geo& geo) { return geo.L >= 16 && geo.L <= 2048 && geo.M >= 16 && geo.M <= 4096; }

template <int LOGL>
static int tw_total(int logE) { return logE == 3 ? TwPlan<LOGL, 3>::TOTAL : TwPlan<LOGL, 4>::TOTAL; }

int stage_twiddles(int L, int logE) {
  switch (L) {
    case 16: return tw_total<4>(logE);
    case 32: return tw_total<5>(logE);
    case 64: return tw_total<6>(logE);
    case 128: return tw_total<7>(logE);
    case 256: return tw_total<8>(logE);
    case 512: return tw_total<9>(logE);
    case 1024: return tw_total<10>(logE);
    case 2048: return tw_total<11>(logE);
    case 4096: return tw_total<12>(logE);
  }
  return 0;
}

size_t rowfft2_smem(int T, int L, int) { return (size_t)T * (L + L / 16) * sizeof(float2); }

#define SR_ROW_SWITCH(CALL)                         \
  switch (a.geo.L) {                                \
    case 16: CALL(4) case 32: CALL(5)               \
    case 64: CALL(6) case 128: CALL(7)              \
    case 256: CALL(8) case 512: CALL(9)             \
    case 1024: CALL(10) case 2048: CALL(11)         \
  }

cudaError_t launch_rowfft2(const RowFwdArgs& a, int logE, int nthreads, cudaStream_t s,
                           bool set_attr) {
  const size_t sm = rowfft2_smem(a.T, a.geo.L, logE);
#define SR_CALL(l)                                                                   \
  return logE == 3 ? rowfft_go<l, 3>(a, nthreads, sm, s, set_attr)                  \
                   : rowfft_go<l, 4>(a, nthreads, sm, s, set_attr);
  SR_ROW_SWITCH(SR_CALL)
#undef SR_CALL
  return cudaErrorInvalidValue;
}

cudaError_t launch_rowifft2(const RowInvArgs& a, bool add, int logE, int nthreads, cudaStream_t s,
                            bool set_attr) {
  const size_t sm = rowfft2_smem(a.T, a.geo.L, logE);
#define SR_CALL(l)                                                                   \
  return logE == 3 ? rowifft_go<l, 3>(a, add, nthreads, sm, s, set_attr)            \
                   : rowifft_go<l, 4>(a, add, nthreads, sm, s, set_attr);
  SR_ROW_SWITCH(SR_CALL)
#undef SR_CALL
  return cudaErrorInvalidValue;
}

// column schedules: 0 = (CB 4, E 16), 1 = (CB 2, E 8), 2 = (CB 4, E 8),
// 4 = (CB 2, E 16), 5 = (CB 4, E 16) with double-buffered exchanges,
// 6 = (CB 4, E 16) with registers capped for two CTAs per SM
cudaError_t launch_colsolve2(const ColArgs& a, int sched, cudaStream_t s, bool set_attr) {
#define SR_COL(lm)                                                                  \
  case (1 << lm):                                                                   \
    if (sched == 1) return col_go<lm, 2, 3>(a, s, set_attr);                        \
    if (sched == 2) return col_go<lm, 4, 3>(a, s, set_attr);                        \
    if (sched == 4) return col_go<lm, 2, 4>(a, s, set_attr);                        \
    if (sched == 5)                                                                 \
      return (lm == 12) ? col_go<lm, 2, 4, true>(a, s, set_attr)                    \
                        : col_go<lm, 4, 4, true>(a, s, set_attr);                   \
    if (sched == 6)                                                                 \
      return (lm == 12) ? col_go<lm, 2, 4, false, 2>(a, s, set_attr)                \
                        : col_go<lm, 4, 4, false, 2>(a, s, set_attr);               \
    return (lm == 12) ? col_go<lm, 2, 4>(a, s, set_attr) : col_go<lm, 4, 4>(a, s, set_attr);
  switch (a.geo.M) {
    SR_COL(4) SR_COL(5) SR_COL(6) SR_COL(7) SR_COL(8) SR_COL(9) SR_COL(10) SR_COL(11) SR_COL(12)
  }
#undef SR_COL
  return cudaErrorInvalidValue;
}

template <int LOGM, int CB, int LOGE>
static cudaError_t col_tma_go(const ColArgs& a, const CUtensorMap& tm, int grid, cudaStream_t s,
                              bool set_attr) {
  const size_t smem = col_tma_smem<LOGM, CB>();
  if (set_attr) return set_smem(k_colsolve_tma<LOGM, CB, LOGE>, smem);
  return launch_k(k_colsolve_tma<LOGM, CB, LOGE>, dim3(grid), dim3(col_threads<LOGM, CB, LOGE>()),
                  smem, s, a, tm);
}

// schedule 3: persistent TMA columns (4 columns x 16 values; 2 columns at H = 4096)
cudaError_t launch_colsolve_tma(const ColArgs& a, const CUtensorMap& tm, int grid, cudaStream_t s,
                                bool set_attr) {
#define SR_COL(lm)                                                                  \
  case (1 << lm):                                                                   \
    return (lm == 12) ? col_tma_go<lm, 2, 4>(a, tm, grid, s, set_attr)              \
                      : col_tma_go<lm, 4, 4>(a, tm, grid, s, set_attr);
  switch (a.geo.M) {
    SR_COL(4) SR_COL(5) SR_COL(6) SR_COL(7) SR_COL(8) SR_COL(9) SR_COL(10) SR_COL(11) SR_COL(12)
  }
#undef SR_COL
  return cudaErrorInvalidValue;
}

int colsolve_tma_cb(int M) { return M == 4096 ? 2 : 4; }

template <int LOGM, int CB, int LOGE>
static cudaError_t col_tma_occ(int* blocks) {
  const size_t smem = col_tma_smem<LOGM, CB>();
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_colsolve_tma<LOGM, CB, LOGE>,
                                                       col_threads<LOGM, CB, LOGE>(), smem);
}

cudaError_t colsolve_tma_occupancy(int M, int* blocks_per_sm) {
#define SR_COL(lm) \
  case (1 << lm):  \
    return (lm == 12) ? col_tma_occ<lm, 2, 4>(blocks_per_sm) : col_tma_occ<lm, 4, 4>(blocks_per_sm);
  switch (M) {
    SR_COL(4) SR_COL(5) SR_COL(6) SR_COL(7) SR_COL(8) SR_COL(9) SR_COL(10) SR_COL(11) SR_COL(12)
  }
#undef SR_COL
  return cudaErrorInvalidValue;
}

int colsolve2_threads(int M, int sched) {
  if (sched == 3) return colsolve_tma_cb(M) * M / 16;
  if (sched == 1) return 2 * M / 8;
  if (sched == 2) return 4 * M / 8;
  if (sched == 4) return 2 * M / 16;
  return M == 4096 ? 2 * M / 16 : 4 * M / 16;
}

}  // namespace srk
