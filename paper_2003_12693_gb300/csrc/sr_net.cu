// Learned warm start: a 6-layer 3x3 convolutional encoder-decoder that
// proposes phi0, trained and run by the kernels of this file (the network and
// its loss are defined in include/sr_net.h).
//
// Convolutions are implicit GEMMs on the tensor cores: bf16 operands staged
// in shared memory by cp.async (zero fill supplies the padding), fragments
// loaded with ldmatrix, mma.sync m16n8k16 with fp32 accumulators.
//   forward        Y[p, o]  = sum_{tap, c} X[p + s(tap), c] W[o, tap, c]
//   input gradient dX[p, c] = sum_{tap, o} dY[p + s(tap), o] W[o, 8 - tap, c]
//                  (the forward kernel with the flipped, transposed weights)
//   weight grad.   dW[o, tap, c] = sum_p dY[p, o] X[p + s(tap), c]
//                  (a GEMM whose reduction runs over the pixels; the operands
//                  are read transposed by ldmatrix.trans, partial sums of
//                  pixel slabs meet in fp32 atomics)
// where s(tap) is the (ky - 1, kx - 1) shift of tap = 3 ky + kx and pixels
// shifted outside the image read zero.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sr_net.h"

namespace {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 16-byte global -> shared copy; src_bytes 0 writes zeros (padding, tails)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(unsigned (&r)[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned (&r)[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_u32(p)));
}

// D = A B + D, A 16x16 (row), B 16x8 (col), bf16 in, fp32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4],
                                         const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ---------------------------------------------------------------------------
// Convolution (forward and input gradient)
// ---------------------------------------------------------------------------
struct ConvArgs {
  const bf16* x;      // [B, H, W, Cin]
  const bf16* w;      // [Cout, 9, Cin]
  const float* bias;  // [Cout] or null
  const bf16* ref;    // MASK: [B, H, W, Cout]
  void* y;            // bf16 [B, H, W, Cout] or float [B, H, W] (OUT1)
  int B, H, W, Cin, Cout;
  int mode;
  float out_scale;
  int taps;           // 9: 3x3 window; 1: a 1x1 product (the input holds the taps)
};

constexpr int kConvBM = 128;   // pixels per CTA
constexpr int kConvThreads = 256;
constexpr int kConvStages = 3;

// BN output channels per CTA, KC input channels per pipeline stage, warps
// arranged WM (pixels) x WN (channels).
template <int BN, int KC, int WM, int WN>
__global__ void __launch_bounds__(kConvThreads, 4) k_conv3x3(ConvArgs a) {
  constexpr int BM = kConvBM, NT = kConvThreads, ST = kConvStages;
  constexpr int LDS = KC + 8;       // shared row stride: conflict-free ldmatrix
  constexpr int VPR = KC / 8;       // 16-byte vectors per row
  constexpr int RSTEP = NT / VPR;   // rows between one thread's A loads
  constexpr int AV = BM / RSTEP;    // A vectors per thread
  constexpr int BVEC = BN * VPR;    // B vectors per stage
  constexpr int TM = BM / WM, TN = BN / WN;
  constexpr int MT = TM / 16, NTL = TN / 8;
  static_assert(WM * WN * 32 == NT, "warp layout");
  static_assert(BM % RSTEP == 0 && MT >= 1 && NTL >= 1, "tile shape");
  __shared__ __align__(16) bf16 As[ST][BM * LDS];
  __shared__ __align__(16) bf16 Bs[ST][BN * LDS];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % WM, wn = warp / WM;
  const long long HW = (long long)a.H * a.W;
  const long long Mtot = HW * a.B;
  const long long m0 = (long long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;

  // the pixel rows this thread stages, decoded once
  int ry[AV], rx[AV];
  long long rp[AV];
  bool rok[AV];
#pragma unroll
  for (int i = 0; i < AV; ++i) {
    const long long p = m0 + tid / VPR + i * RSTEP;
    rok[i] = p < Mtot;
    const long long pp = rok[i] ? p : 0;
    const long long rem = pp % HW;
    ry[i] = (int)(rem / a.W);
    rx[i] = (int)(rem - (long long)ry[i] * a.W);
    rp[i] = pp;
  }
  const int av = tid % VPR;
  const int cchunks = a.Cin / KC;
  const int NK = a.taps * cchunks;

  auto load = [&](int kc, int st) {
    const int tap = kc / cchunks;
    const int c0 = (kc - tap * cchunks) * KC;
    const int dy = a.taps == 9 ? tap / 3 - 1 : 0, dx = a.taps == 9 ? tap % 3 - 1 : 0;
#pragma unroll
    for (int i = 0; i < AV; ++i) {
      const int r = tid / VPR + i * RSTEP;
      const int ys = ry[i] + dy, xs = rx[i] + dx;
      const bool ok = rok[i] && ys >= 0 && ys < a.H && xs >= 0 && xs < a.W;
      const bf16* src = ok ? a.x + (rp[i] + (long long)dy * a.W + dx) * a.Cin + c0 + av * 8 : a.x;
      cp_async16(&As[st][r * LDS + av * 8], src, ok ? 16 : 0);
    }
#pragma unroll
    for (int idx = tid; idx < BVEC; idx += NT) {
      const int n = idx / VPR, v = idx % VPR;
      const bf16* src = a.w + ((long long)(n0 + n) * a.taps + tap) * a.Cin + c0 + v * 8;
      cp_async16(&Bs[st][n * LDS + v * 8], src, 16);
    }
  };

  float acc[MT][NTL][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NTL; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

#pragma unroll
  for (int s = 0; s < ST - 1; ++s) {
    if (s < NK) load(s, s);
    cp_async_commit();
  }
  for (int kc = 0; kc < NK; ++kc) {
    cp_async_wait<ST - 2>();
    __syncthreads();
    const int nk = kc + ST - 1;
    if (nk < NK) load(nk, nk % ST);
    cp_async_commit();
    const bf16* as = As[kc % ST];
    const bf16* bs = Bs[kc % ST];
#pragma unroll
    for (int ks = 0; ks < KC / 16; ++ks) {
      unsigned af[MT][4], bfr[NTL][2];
#pragma unroll
      for (int i = 0; i < MT; ++i)
        ldsm_x4(af[i], as + (wm * TM + i * 16 + (lane & 15)) * LDS + ks * 16 + (lane >> 4) * 8);
#pragma unroll
      for (int j = 0; j < NTL; ++j)
        ldsm_x2(bfr[j], bs + (wn * TN + j * 8 + (lane & 7)) * LDS + ks * 16 + ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NTL; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
  }
  cp_async_wait<0>();

  // epilogue: rows g, g + 8 of each m-tile, channels 2t, 2t + 1 of each n-tile
#pragma unroll
  for (int i = 0; i < MT; ++i) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long p = m0 + wm * TM + i * 16 + (lane >> 2) + h * 8;
      if (p >= Mtot) continue;
#pragma unroll
      for (int j = 0; j < NTL; ++j) {
        const int n = n0 + wn * TN + j * 8 + (lane & 3) * 2;
        float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if (a.mode == SR_CONV_OUT1) {
          if (n == 0) static_cast<float*>(a.y)[p] = a.out_scale * (v0 + a.bias[0]);
          continue;
        }
        if (a.bias != nullptr && a.mode != SR_CONV_MASK) {
          v0 += a.bias[n];
          v1 += a.bias[n + 1];
        }
        if (a.mode == SR_CONV_RELU) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        } else if (a.mode == SR_CONV_MASK) {
          const __nv_bfloat162 r =
              *reinterpret_cast<const __nv_bfloat162*>(a.ref + p * a.Cout + n);
          if (!(__bfloat162float(r.x) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(r.y) > 0.f)) v1 = 0.f;
        }
        *reinterpret_cast<__nv_bfloat162*>(static_cast<bf16*>(a.y) + p * a.Cout + n) =
            __floats2bfloat162_rn(v0, v1);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Weight gradient
// ---------------------------------------------------------------------------
struct WgradArgs {
  const bf16* dy;  // [B, H, W, Cout]
  const bf16* x;   // [B, H, W, Cin]
  float* dw;       // [cout_real, 9, cin_real], accumulated
  int B, H, W, Cin, Cout, cin_real, cout_real;
  long long pix_per_cta;  // multiple of kWgKP
  int taps;               // 9, or 1 for a 1x1 product
};

constexpr int kWgKP = 64;        // pixels per pipeline stage
constexpr int kWgStages = 3;
constexpr int kWgThreads = 256;

template <int BCO, int BCI>
constexpr size_t wgrad_smem() {
  return (size_t)kWgStages * kWgKP * ((BCO + 8) + (BCI + 8)) * sizeof(bf16);
}

// CTA tile: BCO output channels x BCI input channels of one tap, summed over
// a slab of pixels.  Warps WM (co) x WN (ci) x WK (pixel k-steps), WK partial
// sums reduced in shared memory at the end.
template <int BCO, int BCI, int WM, int WN, int WK>
__global__ void __launch_bounds__(kWgThreads) k_conv_wgrad(WgradArgs a) {
  constexpr int KP = kWgKP, ST = kWgStages, NT = kWgThreads;
  constexpr int LDD = BCO + 8, LDX = BCI + 8;
  constexpr int VD = BCO / 8, VX = BCI / 8;
  constexpr int TMo = BCO / WM, TNi = BCI / WN;
  constexpr int MT = TMo / 16, NTL = TNi / 8;
  constexpr int KSTEPS = KP / 16;
  static_assert(WM * WN * WK * 32 == NT, "warp layout");
  static_assert(KSTEPS % WK == 0 && MT >= 1 && NTL >= 1, "tile shape");
  extern __shared__ __align__(16) unsigned char wg_smem[];
  bf16* Ds = reinterpret_cast<bf16*>(wg_smem);
  bf16* Xs = Ds + ST * KP * LDD;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % WM, wn = (warp / WM) % WN, wk = warp / (WM * WN);
  const int nco = a.Cout / BCO, nci = a.Cin / BCI;
  int by = blockIdx.y;
  const int cob = by % nco;
  by /= nco;
  const int cib = by % nci;
  const int tap = by / nci;
  const int co0 = cob * BCO, ci0 = cib * BCI;
  const int dy = a.taps == 9 ? tap / 3 - 1 : 0, dx = a.taps == 9 ? tap % 3 - 1 : 0;
  const long long HW = (long long)a.H * a.W;
  const long long Mtot = HW * a.B;
  const long long pb = (long long)blockIdx.x * a.pix_per_cta;
  const long long pe = min(Mtot, pb + a.pix_per_cta);
  const int nch = (int)((pe - pb + KP - 1) / KP);

  auto load = [&](int ch, int st) {
    const long long pc = pb + (long long)ch * KP;
    for (int idx = tid; idx < KP * VD; idx += NT) {
      const int r = idx / VD, v = idx % VD;
      const long long p = pc + r;
      const bool ok = p < pe;
      const bf16* src = ok ? a.dy + p * a.Cout + co0 + v * 8 : a.dy;
      cp_async16(Ds + (st * KP + r) * LDD + v * 8, src, ok ? 16 : 0);
    }
    for (int idx = tid; idx < KP * VX; idx += NT) {
      const int r = idx / VX, v = idx % VX;
      const long long p = pc + r;
      bool ok = p < pe;
      if (ok) {
        const long long rem = p % HW;
        const int yy = (int)(rem / a.W) + dy, xx = (int)(rem % a.W) + dx;
        ok = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
      }
      const bf16* src = ok ? a.x + (p + (long long)dy * a.W + dx) * a.Cin + ci0 + v * 8 : a.x;
      cp_async16(Xs + (st * KP + r) * LDX + v * 8, src, ok ? 16 : 0);
    }
  };

  float acc[MT][NTL][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NTL; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

#pragma unroll
  for (int s = 0; s < ST - 1; ++s) {
    if (s < nch) load(s, s);
    cp_async_commit();
  }
  for (int ch = 0; ch < nch; ++ch) {
    cp_async_wait<ST - 2>();
    __syncthreads();
    const int nx = ch + ST - 1;
    if (nx < nch) load(nx, nx % ST);
    cp_async_commit();
    const bf16* ds = Ds + (ch % ST) * KP * LDD;
    const bf16* xs = Xs + (ch % ST) * KP * LDX;
#pragma unroll
    for (int kk = 0; kk < KSTEPS / WK; ++kk) {
      const int ks = kk * WK + wk;
      unsigned af[MT][4], bfr[NTL][2];
#pragma unroll
      for (int i = 0; i < MT; ++i)
        ldsm_x4_t(af[i], ds + (ks * 16 + (lane & 7) + (lane >> 4) * 8) * LDD + wm * TMo + i * 16 +
                             ((lane >> 3) & 1) * 8);
      if constexpr (NTL % 2 == 0) {
#pragma unroll
        for (int j = 0; j < NTL; j += 2) {
          unsigned r4[4];
          ldsm_x4_t(r4, xs + (ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * LDX + wn * TNi +
                            j * 8 + (lane >> 4) * 8);
          bfr[j][0] = r4[0];
          bfr[j][1] = r4[1];
          bfr[j + 1][0] = r4[2];
          bfr[j + 1][1] = r4[3];
        }
      } else {
#pragma unroll
        for (int j = 0; j < NTL; ++j)
          ldsm_x2_t(bfr[j], xs + (ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * LDX + wn * TNi +
                                j * 8);
      }
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NTL; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
  }
  cp_async_wait<0>();

  if constexpr (WK > 1) {
    // reduce the WK partial tiles through shared memory (pipeline buffers)
    __syncthreads();
    float* red = reinterpret_cast<float*>(wg_smem);
    constexpr int PER = MT * NTL * 4;
    const int slot = (wm + WM * wn) * 32 + lane;   // same for the WK warps of one tile
    if (wk > 0) {
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NTL; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e)
            red[((wk - 1) * (WM * WN * 32) + slot) * PER + (i * NTL + j) * 4 + e] = acc[i][j][e];
    }
    __syncthreads();
    if (wk > 0) return;
#pragma unroll
    for (int q = 0; q < WK - 1; ++q)
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NTL; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e)
            acc[i][j][e] += red[(q * (WM * WN * 32) + slot) * PER + (i * NTL + j) * 4 + e];
  }
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NTL; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int co = co0 + wm * TMo + i * 16 + (lane >> 2) + (e >> 1) * 8;
        const int ci = ci0 + wn * TNi + j * 8 + (lane & 3) * 2 + (e & 1);
        if (co < a.cout_real && ci < a.cin_real)
          atomicAdd(a.dw + ((long long)co * a.taps + tap) * a.cin_real + ci, acc[i][j][e]);
      }
}

// db[c] += sum_p dy[p, c] for c < c_real; 8 channels (16 bytes) per thread,
// C / 8 threads per pixel row (C a multiple of 8 dividing 256 * 8)
__global__ void __launch_bounds__(256) k_bias_grad(const bf16* __restrict__ dy, long long Mtot,
                                                   int C, int c_real, long long pix_per_cta,
                                                   float* __restrict__ db) {
  __shared__ float red[256][9];
  const int CV = C / 8;
  const int v = threadIdx.x % CV, row = threadIdx.x / CV, rows = 256 / CV;
  const long long pb = (long long)blockIdx.x * pix_per_cta;
  const long long pe = min(Mtot, pb + pix_per_cta);
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (row < rows) {
    for (long long p = pb + row; p < pe; p += rows) {
      const uint4 u = *reinterpret_cast<const uint4*>(dy + p * C + v * 8);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(h[k]);
        s[2 * k] += f.x;
        s[2 * k + 1] += f.y;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) red[threadIdx.x][k] = s[k];
  __syncthreads();
  if (threadIdx.x < C) {
    const int c = threadIdx.x, cv = c / 8, ck = c % 8;
    float t = 0.f;
    for (int r = 0; r < rows; ++r) t += red[r * CV + cv][ck];
    if (c < c_real) atomicAdd(db + c, t);
  }
}

// ---------------------------------------------------------------------------
// Pooling, upsampling and their adjoints (8 channels = 16 bytes per thread)
// ---------------------------------------------------------------------------
struct V8 {
  float v[8];
};
__device__ __forceinline__ V8 load8(const bf16* p) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
  V8 r;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = __bfloat1622float2(h[k]);
    r.v[2 * k] = f.x;
    r.v[2 * k + 1] = f.y;
  }
  return r;
}
__device__ __forceinline__ void store8(bf16* p, const V8& r) {
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(r.v[2 * k], r.v[2 * k + 1]);
  *reinterpret_cast<uint4*>(p) = u;
}

// y [B, H/2, W/2, C] = 2x2 mean of x [B, H, W, C]
__global__ void k_pool2(const bf16* __restrict__ x, bf16* __restrict__ y, int B, int H, int W,
                        int C) {
  const int Ho = H / 2, Wo = W / 2, CV = C / 8;
  const long long n = (long long)B * Ho * Wo * CV;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(idx % CV);
    long long q = idx / CV;
    const int ox = (int)(q % Wo);
    q /= Wo;
    const int oy = (int)(q % Ho);
    const long long b = q / Ho;
    const bf16* s = x + (((b * H + 2 * oy) * W + 2 * ox) * C + v * 8);
    const V8 a0 = load8(s), a1 = load8(s + C), a2 = load8(s + (long long)W * C),
             a3 = load8(s + (long long)W * C + C);
    V8 r;
#pragma unroll
    for (int k = 0; k < 8; ++k) r.v[k] = 0.25f * ((a0.v[k] + a1.v[k]) + (a2.v[k] + a3.v[k]));
    store8(y + (((b * Ho + oy) * Wo + ox) * C + v * 8), r);
  }
}

// y [B, 2h, 2w, C] = x [B, h, w, C] repeated 2x2
__global__ void k_up2(const bf16* __restrict__ x, bf16* __restrict__ y, int B, int h, int w,
                      int C) {
  const int H = 2 * h, W = 2 * w, CV = C / 8;
  const long long n = (long long)B * H * W * CV;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(idx % CV);
    long long q = idx / CV;
    const int xx = (int)(q % W);
    q /= W;
    const int yy = (int)(q % H);
    const long long b = q / H;
    *reinterpret_cast<uint4*>(y + idx * 8) = *reinterpret_cast<const uint4*>(
        x + (((b * h + yy / 2) * w + xx / 2) * C + v * 8));
  }
}

// dz [B, H, W, C] = (a > 0) * dp[y/2, x/2] / 4: adjoint of the 2x2 mean, ReLU mask
__global__ void k_pool2_adj_mask(const bf16* __restrict__ dp, const bf16* __restrict__ a,
                                 bf16* __restrict__ dz, int B, int H, int W, int C) {
  const int CV = C / 8, Ho = H / 2, Wo = W / 2;
  const long long n = (long long)B * H * W * CV;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(idx % CV);
    long long q = idx / CV;
    const int xx = (int)(q % W);
    q /= W;
    const int yy = (int)(q % H);
    const long long b = q / H;
    const V8 g = load8(dp + (((b * Ho + yy / 2) * Wo + xx / 2) * C + v * 8));
    const V8 m = load8(a + idx * 8);
    V8 r;
#pragma unroll
    for (int k = 0; k < 8; ++k) r.v[k] = m.v[k] > 0.f ? 0.25f * g.v[k] : 0.f;
    store8(dz + idx * 8, r);
  }
}

// dz [B, h, w, C] = (a > 0) * sum of the 2x2 copies in du [B, 2h, 2w, C]
__global__ void k_up2_adj_mask(const bf16* __restrict__ du, const bf16* __restrict__ a,
                               bf16* __restrict__ dz, int B, int h, int w, int C) {
  const int CV = C / 8, W = 2 * w;
  const long long n = (long long)B * h * w * CV;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(idx % CV);
    long long q = idx / CV;
    const int xx = (int)(q % w);
    q /= w;
    const int yy = (int)(q % h);
    const long long b = q / h;
    const bf16* s = du + (((b * 2 * h + 2 * yy) * W + 2 * xx) * C + v * 8);
    const V8 a0 = load8(s), a1 = load8(s + C), a2 = load8(s + (long long)W * C),
             a3 = load8(s + (long long)W * C + C);
    const V8 m = load8(a + idx * 8);
    V8 r;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      r.v[k] = m.v[k] > 0.f ? (a0.v[k] + a1.v[k]) + (a2.v[k] + a3.v[k]) : 0.f;
    store8(dz + idx * 8, r);
  }
}

// The first layer has one input channel, so its 3x3 window is packed into
// the channels instead: x0[p, t] = f[p + s(t)] for the nine taps t (zero
// outside the image), channels 9..15 zero, and the layer becomes a 1x1
// product with K = 16 instead of a 3x3 one with K = 9 x 16.
__global__ void k_pack_input(const float* __restrict__ f, bf16* __restrict__ x0, int B, int H,
                             int W) {
  const long long P = (long long)B * H * W;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    const long long HW = (long long)H * W;
    const int rem = (int)(p % HW);
    const int y = rem / W, x = rem % W;
    uint4 u[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
    unsigned short* h = reinterpret_cast<unsigned short*>(u);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int ys = y + t / 3 - 1, xs = x + t % 3 - 1;
      const float v = (ys >= 0 && ys < H && xs >= 0 && xs < W) ? f[p + (ys - y) * W + (xs - x)] : 0.f;
      const bf16 b = __float2bfloat16_rn(v);
      h[t] = *reinterpret_cast<const unsigned short*>(&b);
    }
    uint4* d = reinterpret_cast<uint4*>(x0 + p * 16);
    d[0] = u[0];
    d[1] = u[1];
  }
}

// t = clip(phi*, -c, c) / c, r = y - t; dout[p] = r / n (fp32);
// loss += sum r^2 / (2 n) in fp64; db_last += sum r / n (the last layer's bias)
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ y,
                                              const float* __restrict__ phi, long long n,
                                              float clip, float* __restrict__ dout,
                                              double* __restrict__ loss,
                                              float* __restrict__ db_last) {
  __shared__ double red[2][256];
  double s2 = 0.0, s1 = 0.0;
  const float inv_n = (float)(1.0 / (double)n);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const float t = fminf(fmaxf(phi[p], -clip), clip) / clip;
    const float r = y[p] - t;
    s2 += (double)r * (double)r;
    const float d = r * inv_n;
    s1 += (double)d;
    dout[p] = d;
  }
  red[0][threadIdx.x] = s2;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      red[0][threadIdx.x] += red[0][threadIdx.x + k];
      red[1][threadIdx.x] += red[1][threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (loss != nullptr) atomicAdd(loss, 0.5 * red[0][0] / (double)n);
    atomicAdd(db_last, (float)red[1][0]);
  }
}

// ---------------------------------------------------------------------------
// The last layer (32 -> 1 channel, on the 2x upsampled a5) by direct kernels:
// a single output channel leaves nothing for a tensor-core tile to share, and
// the upsampling is folded into the indexing (u5[y, x] = a5[y / 2, x / 2]).
// w6 is the layer's float weights [9][32] (tap-major), read from the
// parameter vector.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load32(const bf16* p, float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const V8 r = load8(p + q * 8);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[q * 8 + k] = r.v[k];
  }
}

// y[p] = scale * (b6 + sum_{tap, c} u5[p + s(tap), c] w6[tap, c]).  With u5
// constant on 2 x 2 blocks, the four outputs p = 2q + (i, j) of a half-
// resolution pixel q read only the 2 x 2 neighbours q + (i - 1 + ar, j - 1 + br),
// ar, br in {0, 1}, with the taps that land on the same neighbour summed:
// wc[i][j][ar][br][c] = sum of w6[dy, dx, c] over floor((i + dy) / 2) = i - 1 + ar
// and floor((j + dx) / 2) = j - 1 + br.  One thread per q; neighbours outside
// the half-resolution image are the zero padding of the full-resolution one.
__global__ void __launch_bounds__(256) k_out_fwd(const bf16* __restrict__ a5,
                                                 const float* __restrict__ w6,
                                                 const float* __restrict__ b6,
                                                 float* __restrict__ y, int B, int H, int W,
                                                 float scale) {
  __shared__ float wc[2][2][2][2][32];
  for (int idx = threadIdx.x; idx < 512; idx += blockDim.x) {
    const int c = idx % 32, br = (idx / 32) % 2, ar = (idx / 64) % 2, j = (idx / 128) % 2,
              i = idx / 256;
    float acc = 0.f;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        if ((i + dy + 2) / 2 - 1 == i - 1 + ar && (j + dx + 2) / 2 - 1 == j - 1 + br)
          acc += w6[((dy + 1) * 3 + dx + 1) * 32 + c];
    wc[i][j][ar][br][c] = acc;
  }
  __syncthreads();
  const int h = H / 2, w = W / 2;
  const long long Q = (long long)B * h * w;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Q;
       q += (long long)gridDim.x * blockDim.x) {
    const long long hw = (long long)h * w;
    const long long b = q / hw;
    const int rem = (int)(q - b * hw);
    const int qy = rem / w, qx = rem % w;
#pragma unroll 1
    for (int ij = 0; ij < 4; ++ij) {
      const int i = ij >> 1, j = ij & 1;
      {
        float acc = 0.f;
#pragma unroll
        for (int ar = 0; ar < 2; ++ar) {
#pragma unroll
          for (int br = 0; br < 2; ++br) {
            const int ny = qy + i - 1 + ar, nx = qx + j - 1 + br;
            if (ny < 0 || ny >= h || nx < 0 || nx >= w) continue;
            const bf16* src = a5 + ((b * h + ny) * w + nx) * 32;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const V8 v = load8(src + g * 8);
#pragma unroll
              for (int k = 0; k < 8; ++k) acc = fmaf(v.v[k], wc[i][j][ar][br][g * 8 + k], acc);
            }
          }
        }
        y[(b * H + 2 * qy + i) * W + 2 * qx + j] = scale * (acc + b6[0]);
      }
    }
  }
}

// dz5[q, c] = (a5[q, c] > 0) * sum over the four copies p of q in u5 of
// sum_tap dout[p - s(tap)] w6[tap, c]: the last layer's input gradient, the
// upsampling's adjoint and a5's ReLU mask in one pass over half-resolution q
__global__ void __launch_bounds__(256) k_out_dgrad(const float* __restrict__ dout,
                                                   const float* __restrict__ w6,
                                                   const bf16* __restrict__ a5,
                                                   bf16* __restrict__ dz5, int B, int H, int W) {
  __shared__ float ws[288];
  for (int i = threadIdx.x; i < 288; i += blockDim.x) ws[i] = w6[i];
  __syncthreads();
  const int h = H / 2, w = W / 2;
  const long long Q = (long long)B * h * w;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Q;
       q += (long long)gridDim.x * blockDim.x) {
    const long long hw = (long long)h * w;
    const long long b = q / hw;
    const int rem = (int)(q - b * hw);
    const int qy = rem / w, qx = rem % w;
    // the 4 x 4 block of dout around the four copies, rows 2qy-1 .. 2qy+2
    float D[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int yy = 2 * qy - 1 + r, xx = 2 * qx - 1 + c;
        D[r][c] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? dout[(b * H + yy) * W + xx] : 0.f;
      }
    // E[tap] = sum over the copies (i, j) of dout[(2qy + i, 2qx + j) - s(tap)]
    float E[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int dy = t / 3 - 1, dx = t % 3 - 1;
      E[t] = (D[1 - dy][1 - dx] + D[1 - dy][2 - dx]) + (D[2 - dy][1 - dx] + D[2 - dy][2 - dx]);
    }
    float m[32];
    load32(a5 + q * 32, m);
    V8 out[4];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int t = 0; t < 9; ++t) acc = fmaf(E[t], ws[t * 32 + c], acc);
      out[c / 8].v[c % 8] = m[c] > 0.f ? acc : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) store8(dz5 + q * 32 + k * 8, out[k]);
  }
}

// dw6[tap, c] += sum_p dout[p] u5[p + s(tap), c].  Grouped by the half-
// resolution pixel q that p + s(tap) falls in: dw6[tap, c] = sum_q a5[q, c]
// D_tap[q], D_tap[q] = sum over (i, j) in {0, 1}^2 of dout[2q + (i, j) - s(tap)]
// (zero outside the image).  One warp per tap, a slab of half-resolution
// pixels per CTA, lane l takes pixels l, l + 32, ...
__global__ void __launch_bounds__(288) k_out_wgrad(const float* __restrict__ dout,
                                                   const bf16* __restrict__ a5,
                                                   float* __restrict__ dw6, int B, int H, int W,
                                                   long long pix_per_cta) {
  __shared__ float red[9][32][33];
  const int t = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int dy = t / 3 - 1, dx = t % 3 - 1;
  const int h = H / 2, w = W / 2;
  const long long hw = (long long)h * w, Q = hw * B;
  const long long pb = (long long)blockIdx.x * pix_per_cta;
  const long long pe = min(Q, pb + pix_per_cta);
  float acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = 0.f;
  for (long long q = pb + lane; q < pe; q += 32) {
    const long long b = q / hw;
    const int rem = (int)(q - b * hw);
    const int qy = rem / w, qx = rem % w;
    float D = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int yy = 2 * qy + i - dy, xx = 2 * qx + j - dx;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) D += dout[(b * H + yy) * W + xx];
      }
    float v[32];
    load32(a5 + q * 32, v);
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = fmaf(D, v[c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) red[t][lane][c] = acc[c];
  __syncthreads();
  float sum = 0.f;
  for (int l = 0; l < 32; ++l) sum += red[t][l][lane];
  atomicAdd(dw6 + t * 32 + lane, sum);
}

// Per-layer weight repacking: forward [CoutP, 9, CinP] and flipped
// transposed [CinP, 9, CoutP] (wb[c, tap, o] = w[o, 8 - tap, c]), zero padded.
struct PackLayer {
  int cin, cout, cinp, coutp;
  long long off;     // offset of W in the flat parameter vector
  bf16* wf;
  bf16* wb;          // null: no input-gradient copy
  int taps_packed;   // 1: one input channel, wf [coutp][1][cinp] holds the 9 taps
};
struct PackArgs {
  PackLayer l[SR_NET_LAYERS];
  const float* theta;
};

__global__ void k_pack_weights(PackArgs a) {
  const PackLayer L = a.l[blockIdx.y];
  if (L.wf == nullptr) return;
  if (L.taps_packed) {
    const int n = L.coutp * L.cinp;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
      const int t = idx % L.cinp, o = idx / L.cinp;
      const float v = (o < L.cout && t < 9) ? a.theta[L.off + (long long)o * 9 + t] : 0.f;
      L.wf[idx] = __float2bfloat16_rn(v);
    }
    return;
  }
  const int n = L.coutp * 9 * L.cinp;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int c = idx % L.cinp;
    const int tap = (idx / L.cinp) % 9;
    const int o = idx / (9 * L.cinp);
    const float v =
        (o < L.cout && c < L.cin) ? a.theta[L.off + ((long long)o * 9 + tap) * L.cin + c] : 0.f;
    const bf16 b = __float2bfloat16_rn(v);
    L.wf[idx] = b;
    if (L.wb) L.wb[((long long)c * 9 + (8 - tap)) * L.coutp + o] = b;
  }
}

// wt [cin, 9, cout] = w [cout, 8 - tap, cin]: the input-gradient weights of a
// forward layer given in bf16
__global__ void k_flip_transpose(const bf16* __restrict__ w, bf16* __restrict__ wt, int cout,
                                 int cin) {
  const long long n = (long long)cout * 9 * cin;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx % cin);
    const int tap = (int)((idx / cin) % 9);
    const long long o = idx / (9LL * cin);
    wt[((long long)c * 9 + (8 - tap)) * cout + o] = w[idx];
  }
}

// Adam with bias correction; bc1 = 1 - beta1^t, bc2 = 1 - beta2^t, computed
// on the host from the same float beta values the moments use
constexpr float kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdamEps = 1e-8f;
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, long long n, float lr, float bc1, float bc2) {
  const float b1 = kAdamB1, b2 = kAdamB2, eps = kAdamEps;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// ---------------------------------------------------------------------------
// Host side: launch selection
// ---------------------------------------------------------------------------
thread_local std::string g_err;

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

int ew_grid(long long n) {
  const long long b = (n + 255) / 256;
  return (int)std::max(1LL, std::min(b, (long long)num_sms() * 16));
}

bool conv_shape_ok(int cin, int cout) {
  return cin > 0 && cin % 16 == 0 && (cout == 16 || cout == 32 || (cout > 0 && cout % 64 == 0));
}

template <int BN, int KC, int WM, int WN>
cudaError_t conv_go(const ConvArgs& a, cudaStream_t s) {
  const long long M = (long long)a.B * a.H * a.W;
  dim3 grid((unsigned)((M + kConvBM - 1) / kConvBM), a.Cout / BN);
  k_conv3x3<BN, KC, WM, WN><<<grid, kConvThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s) {
  const bool k32 = a.Cin % 32 == 0;
  if (a.Cout == 16) return k32 ? conv_go<16, 32, 8, 1>(a, s) : conv_go<16, 16, 8, 1>(a, s);
  if (a.Cout == 32) return k32 ? conv_go<32, 32, 4, 2>(a, s) : conv_go<32, 16, 4, 2>(a, s);
  return k32 ? conv_go<64, 32, 4, 2>(a, s) : conv_go<64, 16, 4, 2>(a, s);
}

template <int BCO, int BCI, int WM, int WN, int WK>
cudaError_t wgrad_go(const WgradArgs& a0, cudaStream_t s) {
  WgradArgs a = a0;
  constexpr size_t smem = wgrad_smem<BCO, BCI>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad<BCO, BCI, WM, WN, WK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long M = (long long)a.B * a.H * a.W;
  const int tiles = a.taps * (a.Cout / BCO) * (a.Cin / BCI);
  // about six CTAs per SM in total (the partial tiles meet in fp32 atomics),
  // slabs a multiple of the stage size
  long long slabs = std::max(1LL, (long long)(6 * num_sms() + tiles - 1) / tiles);
  long long per = (M + slabs - 1) / slabs;
  per = std::max((long long)kWgKP, (per + kWgKP - 1) / kWgKP * kWgKP);
  slabs = (M + per - 1) / per;
  a.pix_per_cta = per;
  dim3 grid((unsigned)slabs, tiles);
  k_conv_wgrad<BCO, BCI, WM, WN, WK><<<grid, kWgThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const WgradArgs& a, cudaStream_t s) {
  // (Cout, Cin) of the layers: (32, 16), (64, 32), (128, 64), (64, 128), (32, 64), (16, 32)
  if (a.Cin == 16) {
    if (a.Cout == 16) return wgrad_go<16, 16, 1, 2, 4>(a, s);
    if (a.Cout == 32) return wgrad_go<32, 16, 2, 1, 4>(a, s);
    return wgrad_go<64, 16, 4, 1, 2>(a, s);
  }
  if (a.Cin == 32) {
    if (a.Cout == 16) return wgrad_go<16, 32, 1, 2, 4>(a, s);
    if (a.Cout == 32) return wgrad_go<32, 32, 2, 1, 4>(a, s);
    return wgrad_go<64, 32, 4, 1, 2>(a, s);
  }
  if (a.Cout == 16) return wgrad_go<16, 64, 1, 2, 4>(a, s);
  if (a.Cout == 32) return wgrad_go<32, 64, 2, 2, 2>(a, s);
  return wgrad_go<64, 64, 4, 2, 1>(a, s);
}

bool wgrad_shape_ok(int cin, int cout) {
  return cin > 0 && cout > 0 && cin % 16 == 0 && cout % 16 == 0 && (cin <= 32 || cin % 64 == 0) &&
         (cout <= 32 || cout % 64 == 0);
}

cudaError_t launch_bias_grad(const bf16* dy, long long M, int C, int c_real, float* db,
                             cudaStream_t s) {
  const long long blocks = std::min<long long>(2 * num_sms(), std::max(1LL, M / 256));
  const long long per = (M + blocks - 1) / blocks;
  k_bias_grad<<<(unsigned)((M + per - 1) / per), 256, 0, s>>>(dy, M, C, c_real, per, db);
  return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// The network object
// ---------------------------------------------------------------------------
static const int kLayerCin[SR_NET_LAYERS] = {1, 32, 64, 128, 64, 32};
static const int kLayerCout[SR_NET_LAYERS] = {32, 64, 128, 64, 32, 1};

struct sr_net {
  int H, W, maxB, device;
  float clip;
  cudaStream_t stream;
  long long P;  // parameters
  float *theta, *grad, *m, *v;
  long long woff[SR_NET_LAYERS], boff[SR_NET_LAYERS];
  int cinp[SR_NET_LAYERS], coutp[SR_NET_LAYERS];
  // bf16 weights of the tensor-core layers: wf forward [coutp][taps][cinp],
  // wb input gradient [cinp][9][coutp]; layer 1 has no wb (no input gradient
  // is needed) and a tap-packed wf; layer 6 runs on the float weights
  bf16 *wf[SR_NET_LAYERS], *wb[SR_NET_LAYERS];
  bool packed;
  long long step;
  // activations (NHWC bf16) and gradients
  bf16 *x0, *a1, *p1, *a2, *p2, *a3, *a4, *u4, *a5;
  bf16 *dz5, *du4, *dz4, *dz3, *dp2, *dz2, *dp1, *dz1;
  float *y, *dout;
  long long launches;
  std::string err;
  std::vector<void*> allocs;
};

static sr_status net_fail(sr_net* n, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (n) n->err = m;
  g_err = m;
  return SR_ECUDA;
}

#define NET_CK(n, call, what)                      \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return net_fail(n, e_, what); \
  } while (0)

#define NET_TRY(x)                 \
  do {                             \
    sr_status s_ = (x);            \
    if (s_ != SR_OK) return s_;    \
  } while (0)

static sr_status net_alloc(sr_net* n, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    net_fail(n, e, "cudaMalloc");
    return SR_ENOMEM;
  }
  n->allocs.push_back(*p);
  return SR_OK;
}

static sr_status net_conv(sr_net* n, const bf16* x, int B, int H, int W, int cin, const bf16* w,
                          const float* bias, int cout, int mode, const bf16* ref, void* y,
                          int taps = 9) {
  ConvArgs a{x, w, bias, ref, y, B, H, W, cin, cout, mode, 1.f, taps};
  NET_CK(n, launch_conv(a, n->stream), "conv3x3");
  ++n->launches;
  return SR_OK;
}

// weight and bias gradients of tensor-core layer k (0-based)
static sr_status net_wgrad(sr_net* n, int k, const bf16* dy, const bf16* x, int B, int H, int W) {
  const bool packed = k == 0;   // tap-packed first layer: a 1x1 product over 9 "channels"
  WgradArgs a{dy, x, n->grad + n->woff[k], B, H, W, n->cinp[k], n->coutp[k],
              packed ? 9 : kLayerCin[k], kLayerCout[k], 0, packed ? 1 : 9};
  NET_CK(n, launch_wgrad(a, n->stream), "conv3x3 weight gradient");
  NET_CK(n, launch_bias_grad(dy, (long long)B * H * W, n->coutp[k], kLayerCout[k],
                             n->grad + n->boff[k], n->stream),
         "bias gradient");
  n->launches += 2;
  return SR_OK;
}

static sr_status net_pack(sr_net* n) {
  if (n->packed) return SR_OK;
  PackArgs a;
  int maxn = 0;
  for (int k = 0; k < SR_NET_LAYERS; ++k) {
    a.l[k] = PackLayer{kLayerCin[k], kLayerCout[k], n->cinp[k], n->coutp[k], n->woff[k],
                       n->wf[k], n->wb[k], k == 0 ? 1 : 0};
    maxn = std::max(maxn, n->coutp[k] * 9 * n->cinp[k]);
  }
  a.theta = n->theta;
  k_pack_weights<<<dim3((maxn + 255) / 256, SR_NET_LAYERS), 256, 0, n->stream>>>(a);
  NET_CK(n, cudaGetLastError(), "pack weights");
  ++n->launches;
  n->packed = true;
  return SR_OK;
}

static sr_status net_forward(sr_net* n, const float* f, int B, float out_scale, float* yout) {
  const int H = n->H, W = n->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
  cudaStream_t s = n->stream;
  NET_TRY(net_pack(n));
  const long long P0 = (long long)B * H * W;
  k_pack_input<<<ew_grid(P0), 256, 0, s>>>(f, n->x0, B, H, W);
  NET_CK(n, cudaGetLastError(), "pack input");
  ++n->launches;
  const float* th = n->theta;
  NET_TRY(net_conv(n, n->x0, B, H, W, 16, n->wf[0], th + n->boff[0], 32, SR_CONV_RELU, nullptr,
                   n->a1, 1));
  k_pool2<<<ew_grid((long long)B * H2 * W2 * 4), 256, 0, s>>>(n->a1, n->p1, B, H, W, 32);
  NET_TRY(net_conv(n, n->p1, B, H2, W2, 32, n->wf[1], th + n->boff[1], 64, SR_CONV_RELU, nullptr,
                   n->a2));
  k_pool2<<<ew_grid((long long)B * H4 * W4 * 8), 256, 0, s>>>(n->a2, n->p2, B, H2, W2, 64);
  NET_TRY(net_conv(n, n->p2, B, H4, W4, 64, n->wf[2], th + n->boff[2], 128, SR_CONV_RELU,
                   nullptr, n->a3));
  NET_TRY(net_conv(n, n->a3, B, H4, W4, 128, n->wf[3], th + n->boff[3], 64, SR_CONV_RELU,
                   nullptr, n->a4));
  k_up2<<<ew_grid((long long)B * H2 * W2 * 8), 256, 0, s>>>(n->a4, n->u4, B, H4, W4, 64);
  NET_TRY(net_conv(n, n->u4, B, H2, W2, 64, n->wf[4], th + n->boff[4], 32, SR_CONV_RELU, nullptr,
                   n->a5));
  k_out_fwd<<<ew_grid((long long)B * H2 * W2), 256, 0, s>>>(n->a5, th + n->woff[5],
                                                             th + n->boff[5], yout, B, H, W,
                                                             out_scale);
  NET_CK(n, cudaGetLastError(), "pool / upsample / output layer");
  n->launches += 4;
  return SR_OK;
}

static sr_status net_backward(sr_net* n, const float* phi_star, int B, double* loss) {
  const int H = n->H, W = n->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
  cudaStream_t s = n->stream;
  const long long P0 = (long long)B * H * W;
  NET_CK(n, cudaMemsetAsync(n->grad, 0, sizeof(float) * n->P, s), "zero gradient");
  if (loss) NET_CK(n, cudaMemsetAsync(loss, 0, sizeof(double), s), "zero loss");
  k_loss<<<ew_grid(P0), 256, 0, s>>>(n->y, phi_star, P0, n->clip, n->dout, loss,
                                     n->grad + n->boff[5]);
  NET_CK(n, cudaGetLastError(), "loss");
  // layer 6: y = conv(up2(a5)); weight gradient, then input gradient through
  // the upsampling and a5's ReLU
  {
    const long long Q = (long long)B * H2 * W2;
    const long long blocks = std::min<long long>(4 * num_sms(), std::max(1LL, Q / 256));
    const long long per = (Q + blocks - 1) / blocks;
    k_out_wgrad<<<(unsigned)((Q + per - 1) / per), 288, 0, s>>>(n->dout, n->a5,
                                                                n->grad + n->woff[5], B, H, W,
                                                                per);
  }
  k_out_dgrad<<<ew_grid((long long)B * H2 * W2), 256, 0, s>>>(n->dout, n->theta + n->woff[5],
                                                              n->a5, n->dz5, B, H, W);
  NET_CK(n, cudaGetLastError(), "output layer gradients");
  n->launches += 3;
  // layer 5: a5 = relu(conv(u4))
  NET_TRY(net_wgrad(n, 4, n->dz5, n->u4, B, H2, W2));
  NET_TRY(net_conv(n, n->dz5, B, H2, W2, 32, n->wb[4], nullptr, 64, SR_CONV_PLAIN, nullptr,
                   n->du4));
  k_up2_adj_mask<<<ew_grid((long long)B * H4 * W4 * 8), 256, 0, s>>>(n->du4, n->a4, n->dz4, B,
                                                                     H4, W4, 64);
  // layer 4: a4 = relu(conv(a3)); its input gradient carries a3's ReLU mask
  NET_TRY(net_wgrad(n, 3, n->dz4, n->a3, B, H4, W4));
  NET_TRY(net_conv(n, n->dz4, B, H4, W4, 64, n->wb[3], nullptr, 128, SR_CONV_MASK, n->a3,
                   n->dz3));
  // layer 3: a3 = relu(conv(p2))
  NET_TRY(net_wgrad(n, 2, n->dz3, n->p2, B, H4, W4));
  NET_TRY(net_conv(n, n->dz3, B, H4, W4, 128, n->wb[2], nullptr, 64, SR_CONV_PLAIN, nullptr,
                   n->dp2));
  k_pool2_adj_mask<<<ew_grid((long long)B * H2 * W2 * 8), 256, 0, s>>>(n->dp2, n->a2, n->dz2, B,
                                                                       H2, W2, 64);
  // layer 2: a2 = relu(conv(p1))
  NET_TRY(net_wgrad(n, 1, n->dz2, n->p1, B, H2, W2));
  NET_TRY(net_conv(n, n->dz2, B, H2, W2, 64, n->wb[1], nullptr, 32, SR_CONV_PLAIN, nullptr,
                   n->dp1));
  k_pool2_adj_mask<<<ew_grid((long long)B * H * W * 4), 256, 0, s>>>(n->dp1, n->a1, n->dz1, B, H,
                                                                     W, 32);
  // layer 1: a1 = relu(x0 . w1), tap-packed
  NET_TRY(net_wgrad(n, 0, n->dz1, n->x0, B, H, W));
  NET_CK(n, cudaGetLastError(), "adjoint kernels");
  n->launches += 3;
  return SR_OK;
}

extern "C" {

sr_status sr_net_layer_shape(int k, int* cin, int* cout) {
  if (k < 0 || k >= SR_NET_LAYERS || !cin || !cout) return SR_EINVAL;
  *cin = kLayerCin[k];
  *cout = kLayerCout[k];
  return SR_OK;
}

long long sr_net_param_count(void) {
  long long n = 0;
  for (int k = 0; k < SR_NET_LAYERS; ++k) n += (long long)kLayerCout[k] * (9 * kLayerCin[k] + 1);
  return n;
}

void sr_net_destroy(sr_net* n) {
  if (!n) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(n->device);
  for (void* p : n->allocs) cudaFree(p);
  cudaSetDevice(cur);
  delete n;
}

sr_status sr_net_create(int H, int W, int max_batch, float phi_clip, void* cuda_stream,
                        sr_net** out) {
  if (!out) return SR_EINVAL;
  *out = nullptr;
  if (H < 8 || W < 8 || H > 4096 || W > 4096 || H % 4 || W % 4 || max_batch < 1 ||
      !(phi_clip > 0.f) || !std::isfinite(phi_clip)) {
    g_err = "sr_net_create: H, W must be multiples of 4 in [8, 4096], max_batch >= 1, clip > 0";
    return SR_EINVAL;
  }
  sr_net* n = new sr_net();
  n->H = H;
  n->W = W;
  n->maxB = max_batch;
  n->clip = phi_clip;
  n->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&n->device);
  n->P = sr_net_param_count();
  long long off = 0;
  for (int k = 0; k < SR_NET_LAYERS; ++k) {
    n->woff[k] = off;
    off += (long long)kLayerCout[k] * 9 * kLayerCin[k];
    n->boff[k] = off;
    off += kLayerCout[k];
    n->cinp[k] = std::max(16, kLayerCin[k]);
    n->coutp[k] = std::max(16, kLayerCout[k]);
  }
  sr_status st = SR_OK;
  auto A = [&](void** p, size_t bytes) {
    if (st == SR_OK) st = net_alloc(n, p, bytes);
  };
  A((void**)&n->theta, sizeof(float) * n->P);
  A((void**)&n->grad, sizeof(float) * n->P);
  A((void**)&n->m, sizeof(float) * n->P);
  A((void**)&n->v, sizeof(float) * n->P);
  for (int k = 0; k < SR_NET_LAYERS - 1; ++k) {
    const size_t nw = (size_t)n->coutp[k] * 9 * n->cinp[k];
    A((void**)&n->wf[k], sizeof(bf16) * nw);
    if (k > 0) A((void**)&n->wb[k], sizeof(bf16) * nw);
  }
  const size_t P0 = (size_t)max_batch * H * W, P1 = P0 / 4, P2 = P0 / 16;
  const size_t b = sizeof(bf16);
  A((void**)&n->x0, b * P0 * 16);
  A((void**)&n->a1, b * P0 * 32);
  A((void**)&n->p1, b * P1 * 32);
  A((void**)&n->a2, b * P1 * 64);
  A((void**)&n->p2, b * P2 * 64);
  A((void**)&n->a3, b * P2 * 128);
  A((void**)&n->a4, b * P2 * 64);
  A((void**)&n->u4, b * P1 * 64);
  A((void**)&n->a5, b * P1 * 32);
  A((void**)&n->dout, sizeof(float) * P0);
  A((void**)&n->dz5, b * P1 * 32);
  A((void**)&n->du4, b * P1 * 64);
  A((void**)&n->dz4, b * P2 * 64);
  A((void**)&n->dz3, b * P2 * 128);
  A((void**)&n->dp2, b * P2 * 64);
  A((void**)&n->dz2, b * P1 * 64);
  A((void**)&n->dp1, b * P1 * 32);
  A((void**)&n->dz1, b * P0 * 32);
  A((void**)&n->y, sizeof(float) * P0);
  if (st != SR_OK) {
    g_err = n->err;
    sr_net_destroy(n);
    return st;
  }
  cudaError_t e = cudaMemsetAsync(n->theta, 0, sizeof(float) * n->P, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, sizeof(float) * n->P, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, sizeof(float) * n->P, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->grad, 0, sizeof(float) * n->P, n->stream);
  if (e != cudaSuccess) {
    net_fail(n, e, "cudaMemsetAsync");
    sr_net_destroy(n);
    return SR_ECUDA;
  }
  *out = n;
  return SR_OK;
}

const char* sr_net_last_error(const sr_net* n) { return n ? n->err.c_str() : g_err.c_str(); }

sr_status sr_net_set_params(sr_net* n, const float* theta) {
  if (!n || !theta) return SR_EINVAL;
  NET_CK(n, cudaMemcpyAsync(n->theta, theta, sizeof(float) * n->P, cudaMemcpyDeviceToDevice,
                            n->stream),
         "set params");
  NET_CK(n, cudaMemsetAsync(n->m, 0, sizeof(float) * n->P, n->stream), "reset Adam");
  NET_CK(n, cudaMemsetAsync(n->v, 0, sizeof(float) * n->P, n->stream), "reset Adam");
  n->step = 0;
  n->packed = false;
  return SR_OK;
}

sr_status sr_net_get_params(sr_net* n, float* theta) {
  if (!n || !theta) return SR_EINVAL;
  NET_CK(n, cudaMemcpyAsync(theta, n->theta, sizeof(float) * n->P, cudaMemcpyDeviceToDevice,
                            n->stream),
         "get params");
  return SR_OK;
}

sr_status sr_net_get_grads(sr_net* n, float* grad) {
  if (!n || !grad) return SR_EINVAL;
  NET_CK(n, cudaMemcpyAsync(grad, n->grad, sizeof(float) * n->P, cudaMemcpyDeviceToDevice,
                            n->stream),
         "get grads");
  return SR_OK;
}

sr_status sr_net_forward(sr_net* n, const float* f, int B, float* phi0) {
  if (!n || !f || !phi0 || B < 1 || B > n->maxB) return SR_EINVAL;
  return net_forward(n, f, B, n->clip, phi0);
}

sr_status sr_net_gradients(sr_net* n, const float* f, const float* phi_star, int B, double* loss) {
  if (!n || !f || !phi_star || B < 1 || B > n->maxB) return SR_EINVAL;
  NET_TRY(net_forward(n, f, B, 1.f, n->y));
  return net_backward(n, phi_star, B, loss);
}

sr_status sr_net_train_step(sr_net* n, const float* f, const float* phi_star, int B, float lr,
                            double* loss) {
  if (!(lr >= 0.f) || !std::isfinite(lr)) return SR_EINVAL;
  NET_TRY(sr_net_gradients(n, f, phi_star, B, loss));
  ++n->step;
  // 1 - beta^t with beta the float the kernel uses, so that at t = 1 the
  // correction cancels the moments' (1 - beta) factor to rounding
  const float bc1 = 1.f - (float)std::pow((double)kAdamB1, (double)n->step);
  const float bc2 = 1.f - (float)std::pow((double)kAdamB2, (double)n->step);
  k_adam<<<ew_grid(n->P), 256, 0, n->stream>>>(n->theta, n->m, n->v, n->grad, n->P, lr, bc1, bc2);
  NET_CK(n, cudaGetLastError(), "adam");
  ++n->launches;
  n->packed = false;
  return SR_OK;
}

long long sr_net_kernel_launches(sr_net* n, int reset) {
  if (!n) return -1;
  const long long v = n->launches;
  if (reset) n->launches = 0;
  return v;
}

sr_status sr_conv3x3(const uint16_t* x, int B, int H, int W, int cin, const uint16_t* w,
                     const float* bias, int cout, int mode, const uint16_t* ref, void* y,
                     float out_scale, void* cuda_stream) {
  if (!x || !w || !y || B < 1 || H < 1 || W < 1 || !conv_shape_ok(cin, cout) || mode < 0 ||
      mode > SR_CONV_OUT1 || (mode == SR_CONV_MASK && !ref) || (mode == SR_CONV_OUT1 && !bias) ||
      (mode == SR_CONV_RELU && !bias)) {
    g_err = "sr_conv3x3: bad argument";
    return SR_EINVAL;
  }
  ConvArgs a{reinterpret_cast<const bf16*>(x), reinterpret_cast<const bf16*>(w), bias,
             reinterpret_cast<const bf16*>(ref), y, B, H, W, cin, cout, mode, out_scale, 9};
  if (mode == SR_CONV_MASK) a.bias = nullptr;
  cudaError_t e = launch_conv(a, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return net_fail(nullptr, e, "sr_conv3x3");
  return SR_OK;
}

sr_status sr_conv3x3_dgrad(const uint16_t* dy, int B, int H, int W, int cout, const uint16_t* w,
                           int cin, int mode, const uint16_t* ref, uint16_t* dx,
                           void* cuda_stream) {
  if (!dy || !w || !dx || B < 1 || H < 1 || W < 1 || !conv_shape_ok(cout, cin) ||
      (mode != SR_CONV_PLAIN && mode != SR_CONV_MASK) || (mode == SR_CONV_MASK && !ref)) {
    g_err = "sr_conv3x3_dgrad: bad argument";
    return SR_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // flipped, transposed copy of the weights in a stream-ordered scratch buffer
  const long long nw = (long long)cout * 9 * cin;
  bf16* wt = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&wt, sizeof(bf16) * nw, s);
  if (e != cudaSuccess) return net_fail(nullptr, e, "sr_conv3x3_dgrad scratch");
  k_flip_transpose<<<ew_grid(nw), 256, 0, s>>>(reinterpret_cast<const bf16*>(w), wt, cout, cin);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    ConvArgs a{reinterpret_cast<const bf16*>(dy), wt, nullptr, reinterpret_cast<const bf16*>(ref),
               dx, B, H, W, cout, cin, mode, 1.f, 9};
    e = launch_conv(a, s);
  }
  cudaError_t e2 = cudaFreeAsync(wt, s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return net_fail(nullptr, e, "sr_conv3x3_dgrad");
  return SR_OK;
}

sr_status sr_conv3x3_wgrad(const uint16_t* dy, const uint16_t* x, int B, int H, int W, int cin,
                           int cout, int cin_real, int cout_real, float* dw, float* db,
                           void* cuda_stream) {
  if (!dy || !x || !dw || B < 1 || H < 1 || W < 1 || !wgrad_shape_ok(cin, cout) ||
      cin_real < 1 || cin_real > cin || cout_real < 1 || cout_real > cout) {
    g_err = "sr_conv3x3_wgrad: bad argument";
    return SR_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  WgradArgs a{reinterpret_cast<const bf16*>(dy), reinterpret_cast<const bf16*>(x), dw, B, H, W,
              cin, cout, cin_real, cout_real, 0, 9};
  cudaError_t e = launch_wgrad(a, s);
  if (e == cudaSuccess && db)
    e = launch_bias_grad(a.dy, (long long)B * H * W, cout, cout_real, db, s);
  if (e != cudaSuccess) return net_fail(nullptr, e, "sr_conv3x3_wgrad");
  return SR_OK;
}

}  // extern "C"
