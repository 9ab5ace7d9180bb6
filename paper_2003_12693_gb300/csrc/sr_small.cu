// The whole solve of one inner step (Eqs. (31)-(33)) in one CTA, for images
// whose rows fit one pass of the CTA's threads at 16 values each (M * N/32
// <= kSmallThreads): the row R2C transforms, the column solve by the factored
// recursions of sr_colrec.cu, and the row C2R transforms with psi += result,
// without the two kernel boundaries and the global round trips of the half
// spectrum that the three-pass solve has.  Small images are bound by
// launches, not bytes.
//
// Shared memory holds two buffers of (rows per pass) x (L + L/16) complex
// values (the padded exchange layout of the register Stockham stages): A
// takes the row exchanges, then the recursions' output; B the packed half
// spectrum, then the inverse row exchanges.
#include "sr_dft.cuh"
#include "sr_internal.h"

namespace srk {
namespace small {

using namespace srk::cdft;

template <int LOGL, int R>
__global__ void __launch_bounds__(kSmallThreads) k_solve_small(const SmallArgs a) {
  constexpr int E = 16, L = 1 << LOGL, LOGTP = LOGL - 4, TP = 1 << LOGTP;
  constexpr int RS = L + L / 16;          // padded row stride (float2)
  constexpr int RPP = kSmallThreads / TP; // rows per pass of the row transforms
  extern __shared__ __align__(16) float2 sms[];
  const int M = a.geo.M, N = a.geo.N;
  float2* A = sms;
  float2* B = sms + (size_t)RPP * RS;
  const int tid = threadIdx.x;
  const int t = tid >> LOGTP, u = tid & (TP - 1);
  pdl_wait();
  pdl_trigger();

  // 1. row R2C: z[n] = G[2n] + i G[2n+1], FFT_L, even/odd split; the packed
  //    half spectrum goes to B as M unpadded rows of L.  All rows in one pass
  //    (M <= rows per pass); thread slot t takes row t and its own exchange
  //    region A + t RS, so that the idle slots of a short image stay apart.
  {
    const int i = t;
    const bool live = i < M;
    float2* base = A + (size_t)t * RS;
    float2 x[E];
    const float2* row = reinterpret_cast<const float2*>(a.G + (size_t)(live ? i : 0) * N);
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = live ? row[u + (m << LOGTP)] : make_float2(0.f, 0.f);
    stages<LOGL, 4, 0, false, 1, false, true>(x, base, u, a.tws16);
#pragma unroll
    for (int m = 0; m < E; ++m) base[pad(u + (m << LOGTP))] = x[m];
    __syncthreads();
    if (live) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = u + (m << LOGTP);
        const float2 Zk = x[m];
        float2 o;
        if (k == 0) {
          o = make_float2(Zk.x + Zk.y, Zk.x - Zk.y);
        } else {
          const float2 Zm = base[pad(L - k)];
          const float2 Ev = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
          const float2 D = make_float2(0.5f * (Zk.x - Zm.x), 0.5f * (Zk.y + Zm.y));
          const float2 O = make_float2(D.y, -D.x);
          o = cadd(Ev, cmul(__ldg(&a.twN[k]), O));
        }
        B[(size_t)i * L + k] = o;
      }
    }
  }
  __syncthreads();

  // 2. column solve: per column k the forward and backward recursions of
  //    sr_colrec.cu (warm-up R rows, modulo M), B -> A (unpadded, M x L);
  //    threads on adjacent columns read adjacent words.  Chunks of 16 rows:
  //    at these sizes more, shorter chains fill the CTA better than the
  //    longer chunks that amortise the warm-up on large images.
  {
    constexpr int TR = 16;
    const int nchunk = (M + TR - 1) / TR;
    for (int q = tid; q < L * nchunk; q += kSmallThreads) {
      const int k = q % L, i0 = (q / L) * TR;
      const float4 p = __ldg(a.rec + k);
      const float rr = p.x, sr = p.y, ri = p.z, si = p.w;
      int row = i0 - R;
      while (row < 0) row += M;
      float ux = 0.f, uy = 0.f;
      for (int j = 0; j < R; ++j) {
        const float2 v = B[(size_t)row * L + k];
        ux = fmaf(rr, ux, v.x);
        uy = fmaf(ri, uy, v.y);
        row = row + 1 == M ? 0 : row + 1;
      }
      float2 buf[TR + R];
#pragma unroll
      for (int j = 0; j < TR + R; ++j) {
        const float2 v = B[(size_t)row * L + k];
        ux = fmaf(rr, ux, v.x);
        uy = fmaf(ri, uy, v.y);
        buf[j] = make_float2(ux, uy);
        row = row + 1 == M ? 0 : row + 1;
      }
      float vx = 0.f, vy = 0.f;
#pragma unroll
      for (int j = TR + R - 1; j >= TR; --j) {
        vx = fmaf(rr, vx, buf[j].x);
        vy = fmaf(ri, vy, buf[j].y);
      }
#pragma unroll
      for (int j = TR - 1; j >= 0; --j) {
        vx = fmaf(rr, vx, buf[j].x);
        vy = fmaf(ri, vy, buf[j].y);
        if (i0 + j < M) A[(size_t)(i0 + j) * L + k] = make_float2(sr * vx, si * vy);
      }
    }
  }
  __syncthreads();

  // 3. row C2R from A, inverse FFT_L with B as the exchange buffer (slot t,
  //    as in step 1), out = psi_in + x (or x without psi_in)
  {
    const int i = t;
    const bool live = i < M;
    const float2* Xrow = A + (size_t)(live ? i : 0) * L;
    float2 x[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = u + (m << LOGTP);
      const float2 xk = Xrow[k], xm = Xrow[(L - k) & (L - 1)];
      if (k == 0) {
        x[m] = make_float2(xk.x + xk.y, xk.x - xk.y);
        continue;
      }
      const float2 Xe = make_float2(xk.x + xm.x, xk.y - xm.y);
      const float2 D = make_float2(xk.x - xm.x, xk.y + xm.y);
      const float2 Xo = cmul(D, cconj(__ldg(&a.twN[k])));
      x[m] = make_float2(Xe.x - Xo.y, Xe.y + Xo.x);
    }
    stages<LOGL, 4, 0, true, 1, false, true>(x, B + (size_t)t * RS, u, a.tws16);
    if (live) {
      float2* orow = reinterpret_cast<float2*>(a.out + (size_t)i * N);
      const float2* prow = reinterpret_cast<const float2*>(a.psi_in + (size_t)i * N);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        float2 r = x[m];
        if (a.psi_in) {
          const float2 pv = prow[u + (m << LOGTP)];
          r = make_float2(pv.x + r.x, pv.y + r.y);
        }
        orow[u + (m << LOGTP)] = r;
      }
    }
  }
}

}  // namespace small

using namespace small;

bool solve_small_supported(const Geo& geo, int rec_R) {
  const int L = geo.L;
  if (geo.M < 16 || L < 16 || L > 512 || (L & (L - 1)) || (geo.M & (geo.M - 1))) return false;
  // one pass of the row transforms: M rows of L / 16 threads each
  if ((long long)geo.M * (L / 16) > kSmallThreads) return false;
  if (rec_R != 8 && rec_R != 12 && rec_R != 16 && rec_R != 20 && rec_R != 24 && rec_R != 32)
    return false;
  return solve_small_smem(geo) <= 227 * 1024;
}

size_t solve_small_smem(const Geo& geo) {
  // two buffers of (rows per pass) x (L + L/16) complex values
  const size_t RS = (size_t)geo.L + geo.L / 16;
  const size_t rpp = (size_t)kSmallThreads * 16 / geo.L;
  return 2 * rpp * RS * sizeof(float2);
}

template <int LOGL, int R>
static cudaError_t small_go(const SmallArgs& a, cudaStream_t s, bool set_attr) {
  const size_t smem = solve_small_smem(a.geo);
  if (set_attr)
    return cudaFuncSetAttribute(k_solve_small<LOGL, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  return launch_k(k_solve_small<LOGL, R>, dim3(1), dim3(kSmallThreads), smem, s, a);
}

template <int LOGL>
static cudaError_t small_r(const SmallArgs& a, cudaStream_t s, bool set_attr) {
  switch (a.rec_R) {
    case 8: return small_go<LOGL, 8>(a, s, set_attr);
    case 12: return small_go<LOGL, 12>(a, s, set_attr);
    case 16: return small_go<LOGL, 16>(a, s, set_attr);
    case 20: return small_go<LOGL, 20>(a, s, set_attr);
    case 24: return small_go<LOGL, 24>(a, s, set_attr);
    case 32: return small_go<LOGL, 32>(a, s, set_attr);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_solve_small(const SmallArgs& a, cudaStream_t s, bool set_attr) {
  if (!solve_small_supported(a.geo, a.rec_R)) return cudaErrorInvalidValue;
  switch (a.geo.L) {
    case 16: return small_r<4>(a, s, set_attr);
    case 32: return small_r<5>(a, s, set_attr);
    case 64: return small_r<6>(a, s, set_attr);
    case 128: return small_r<7>(a, s, set_attr);
    case 256: return small_r<8>(a, s, set_attr);
    case 512: return small_r<9>(a, s, set_attr);
  }
  return cudaErrorInvalidValue;
}

}  // namespace srk
