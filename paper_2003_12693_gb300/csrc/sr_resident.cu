// Whole outer iterations of Alg. 1 for small images in one launch, with the
// state resident on chip.
//
// An image of M x N pixels is owned by one cluster of C CTAs (8 or 16); CTA q
// holds rows [q M/C, (q+1) M/C) of every plane (phi, w at two parities, e,
// g, div e, the right-hand side, the half spectrum and the column solve's
// output) in its shared memory for all the iterations of the launch.  The
// phases of one outer iteration are those of the tiled kernels, and they use
// the same per-pixel arithmetic (sr_point.cuh):
//   per inner step s (Eq. (37), increment form):
//     right-hand side G of the CTA's rows (window sum of Sec. 4 only when a
//       pixel of the CTA is in the narrow band, exact as in k_prep)
//     row R2C transforms of the CTA's rows                      (local)
//     cluster barrier
//     column solve by the factored recursions of Eq. (32)'s operator
//       (sr_colrec.cu), reading the other CTAs' spectrum rows    (DSMEM)
//     row C2R transforms, psi += result                         (local)
//     cluster barrier
//   w/b update of Eqs. (41), (42), (40), (23) into the other w parity, e in
//   place; on check iterations the FP64 sums of the stopping test
//   cluster barrier; the stopping decision from the C partial sums, taken
//   identically by every CTA.
// Neighbour rows of the stencils and the window halos come from the other
// CTAs' shared memory through the cluster's distributed shared memory.  Global
// memory is read once at the start and written once at the end, so a launch
// costs one load and one store of the state plus the on-chip iterations
// instead of 4S + 1 dependent kernel launches per iteration (right-hand side,
// row pass, column pass and inverse row pass per inner step, then the w/b
// update) with every plane crossing L2.
//
// All control flow that contains a cluster barrier is uniform over the
// cluster: the loop bounds are launch arguments and the stopping decision is
// computed by every CTA from the same partial sums in the same order.
#include <cooperative_groups.h>

#include "sr_dft.cuh"
#include "sr_internal.h"
#include "sr_point.cuh"

namespace cg = cooperative_groups;

namespace srk {
namespace res {

using namespace srk::cdft;

// Shared-memory layout of one CTA, identical across the cluster (offsets in
// floats from the dynamic shared-memory base, each 16-byte aligned).
struct Lay {
  int RPC, PL, SW;  // rows per CTA, floats per plane, staged window row width N + 2R
  int psi, phik, w1[2], w2[2], e1, e2, g, D, G, X, X2, hu1, hu2, scr, part;
  int total;
};

__host__ __device__ inline int lay_take(int& o, int n) {
  const int r = o;
  o += (n + 3) & ~3;
  return r;
}

__host__ __device__ inline Lay make_lay(int M, int N, int R, int rec_R, int C) {
  Lay l;
  l.RPC = M / C;
  l.PL = l.RPC * N;
  l.SW = N + 2 * R;
  int o = 0;
  l.psi = lay_take(o, l.PL);
  l.phik = lay_take(o, l.PL);
  l.w1[0] = lay_take(o, l.PL);
  l.w1[1] = lay_take(o, l.PL);
  l.w2[0] = lay_take(o, l.PL);
  l.w2[1] = lay_take(o, l.PL);
  l.e1 = lay_take(o, l.PL);
  l.e2 = lay_take(o, l.PL);
  l.g = lay_take(o, l.PL);
  l.D = lay_take(o, l.PL);
  l.G = lay_take(o, l.PL);
  l.X = lay_take(o, l.PL);   // RPC x L complex = PL floats
  l.X2 = lay_take(o, l.PL);
  // u = h(psi) w of the CTA's pixels (the window sum's operand), kept up to
  // date where psi or w change, so the window's halo needs no band function
  l.hu1 = lay_take(o, l.PL);
  l.hu2 = lay_take(o, l.PL);
  // scratch, one use per phase: the window's sums v1, v2, staged u planes
  // and vertical sums; the row transforms' exchange rows (+1 row for idle
  // thread slots);
  // the column solve's copy of the rec_R spectrum rows before and after the
  // CTA's rows, then the forward values of the run and the warm-up after it
  const int L = N / 2, RS = L + L / 16;
  const int win = 2 * (l.RPC + 2 * R) * l.SW + 2 * l.RPC * l.SW + 2 * l.PL;
  const int fft = 2 * (l.RPC + 1) * RS;
  const int colu = 2 * rec_R * N + 2 * (l.RPC + rec_R) * L;
  int sc = win > fft ? win : fft;
  sc = sc > colu ? sc : colu;
  l.scr = lay_take(o, sc);
  l.part = lay_take(o, 4);  // two doubles: this CTA's stopping-test sums
  l.total = o;
  return l;
}

// Fixed-order block reduction of two doubles into out[0..1] (thread 0).
__device__ __forceinline__ void block_sum2(double a, double b, double* out) {
  __shared__ double red[2][kResThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  if (lane == 0) {
    red[0][warp] = a;
    red[1][warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kResThreads / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    out[0] = s0;
    out[1] = s1;
  }
}

// Work is spread by rows over warps and by columns over lanes, so that no
// index needs a division by a runtime width.
template <int LOGL>
__global__ void __launch_bounds__(kResThreads, 1) k_resident(const ResArgs a) {
  // the row transforms at 4 values per thread: L / 4 threads per row spread
  // the transforms over more warps than 16 values would, which shortens the
  // chain the other warps wait for at the next barrier
  constexpr int LOGE = 2;
  constexpr int L = 1 << LOGL, N = 2 * L, E = 1 << LOGE, LOGTP = LOGL - LOGE, TP = 1 << LOGTP;
  constexpr int RS = L + L / 16;
  constexpr int T = kResThreads, NW = T / 32;
  constexpr int NJ = N / 32;       // columns per lane of an image row
  constexpr int NJW = NJ + 1;      // of a staged window row (N + 2R <= N + 32)
  extern __shared__ __align__(16) float sm[];
  __shared__ ResMember mb;
  __shared__ float* rbase[kResCMax];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) mb = a.members[blockIdx.x / C];
  if (tid < C) rbase[tid] = cl.map_shared_rank(sm, tid);
  __syncthreads();
  const Model& m = mb.mod;
  const int M = mb.geo.M, R = m.R;
  const Lay ly = make_lay(M, N, R, mb.rec_R, C);
  const int RPC = ly.RPC, PL = ly.PL, r0 = rank * RPC;

  // row gi (0 <= gi < M) of the plane at offset off, in the owner CTA (the
  // CTA's own rows through its own shared-memory window)
  auto row_at = [&](int off, int gi) -> const float* {
    const int q = gi / RPC;
    return (q == rank ? sm : rbase[q]) + off + (gi - q * RPC) * N;
  };

  // ---- load the CTA's rows of the state
  {
    const int c0 = mb.cur;
    const size_t gb = (size_t)r0 * N;
    const float* src[6] = {mb.phi[c0], mb.w1[c0], mb.w2[c0], mb.e1, mb.e2, mb.g};
    const int dst[6] = {ly.psi, ly.w1[0], ly.w2[0], ly.e1, ly.e2, ly.g};
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      const float4* s4 = reinterpret_cast<const float4*>(src[p] + gb);
      float4* d4 = reinterpret_cast<float4*>(sm + dst[p]);
      for (int q = tid; q < PL / 4; q += T) d4[q] = __ldg(s4 + q);
    }
  }
  // u = h(psi) w at one of the CTA's pixels, with the current w (parity wcur)
  auto set_u = [&](int q, float x, int wcur) {
    const float h = in_band(x, m) ? band_h(x, m) : 0.f;
    sm[ly.hu1 + q] = h * sm[ly.w1[wcur] + q];
    sm[ly.hu2 + q] = h * sm[ly.w2[wcur] + q];
  };
  __syncthreads();  // the rows were loaded by other threads of the CTA
  for (int q = tid; q < PL; q += T) set_u(q, sm[ly.psi + q], 0);
  cl.sync();

  // ---- separable window sum of u = h(x) w over the CTA's rows, Sec. 4:
  // v1, v2 ([RPC][N]) at the start of scr.  After the staging barrier each
  // warp sums its own rows (row r by warp r mod NW, the rows the callers'
  // per-pixel loops give the same warp), down the columns, then along the row
  // it just summed, so only warp barriers follow.
  auto window = [&]() {
    const int SW = ly.SW, SH = RPC + 2 * R;
    float* v1 = sm + ly.scr;
    float* v2 = v1 + PL;
    float* u1 = v2 + PL;
    float* u2 = u1 + SH * SW;
    float* V1 = u2 + SH * SW;
    float* V2 = V1 + RPC * SW;
    for (int sr = warp; sr < SH; sr += NW) {
      const int gi = r0 - R + sr;
      const bool in = gi >= 0 && gi < M;
      const float* p1 = in ? row_at(ly.hu1, gi) : sm;
      const float* p2 = in ? row_at(ly.hu2, gi) : sm;
      float a1[NJW], a2[NJW];
#pragma unroll
      for (int c = 0; c < NJW; ++c) {
        const int j = lane + 32 * c - R;
        const bool ok = in && j >= 0 && j < N;
        a1[c] = ok ? p1[j] : 0.f;
        a2[c] = ok ? p2[j] : 0.f;
      }
#pragma unroll
      for (int c = 0; c < NJW; ++c) {
        const int sc = lane + 32 * c;
        if (sc < SW) {
          u1[sr * SW + sc] = a1[c];
          u2[sr * SW + sc] = a2[c];
        }
      }
    }
    __syncthreads();
    for (int r = warp; r < RPC; r += NW) {
      float acc1[NJW], acc2[NJW];
#pragma unroll
      for (int c = 0; c < NJW; ++c) acc1[c] = acc2[c] = 0.f;
      for (int p = 0; p <= 2 * R; ++p) {
        const float kw = m.kw[p];
#pragma unroll
        for (int c = 0; c < NJW; ++c) {
          const int sc = lane + 32 * c;
          if (sc < SW) {
            acc1[c] = fmaf(kw, u1[(r + p) * SW + sc], acc1[c]);
            acc2[c] = fmaf(kw, u2[(r + p) * SW + sc], acc2[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NJW; ++c) {
        const int sc = lane + 32 * c;
        if (sc < SW) {
          V1[r * SW + sc] = acc1[c];
          V2[r * SW + sc] = acc2[c];
        }
      }
      __syncwarp();
      float s1[NJ], s2[NJ];
#pragma unroll
      for (int c = 0; c < NJ; ++c) s1[c] = s2[c] = 0.f;
      for (int p = 0; p <= 2 * R; ++p) {
        const float kw = m.kw[p];
#pragma unroll
        for (int c = 0; c < NJ; ++c) {
          s1[c] = fmaf(kw, V1[r * SW + lane + 32 * c + p], s1[c]);
          s2[c] = fmaf(kw, V2[r * SW + lane + 32 * c + p], s2[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < NJ; ++c) {
        v1[r * N + lane + 32 * c] = s1[c];
        v2[r * N + lane + 32 * c] = s2[c];
      }
      __syncwarp();
    }
  };

  auto any_band = [&](const float* x) {
    int any = 0;
    for (int q = tid; q < PL; q += T) any |= in_band(x[q], m);
    return __syncthreads_or(any) != 0;
  };
  // whether the CTA's psi has narrow-band pixels: from the load, then from
  // each inverse row pass's update (its threads own every row), read after
  // the cluster barrier that follows it; two flags alternate, the one not in
  // use is cleared after that barrier
  __shared__ int bflag[2];
  if (tid < 2) bflag[tid] = 0;
  int bpar = 0;
  bool band_psi = any_band(sm + ly.psi);

  // the row transforms: thread slot t = tid / TP takes row t, whose TP
  // threads are lanes of one warp, so the stages' exchanges synchronise the
  // warp only; whole warps without a row skip the transforms
  const int ft = tid >> LOGTP, fu = tid & (TP - 1);
  const bool flive = ft < RPC;
  const bool fwarp = (tid & ~31) < RPC * TP;
  float2* fbase = reinterpret_cast<float2*>(sm + ly.scr) + (size_t)(flive ? ft : RPC) * RS;

  int wc = 0;    // local parity of the current w
  int done = 0;
  for (int k = 0; k < a.max_outer; ++k) {
    if (k > 0) {  // u with the w of the update just made, seen by the whole cluster
      for (int q = tid; q < PL; q += T) set_u(q, sm[ly.psi + q], wc);
      cl.sync();
    }
    const bool last = k == a.max_outer - 1;
    const bool check = a.tol > 0.0 ? ((k + 1) % a.check_every == 0 || last)
                                   : (last && a.check_last != 0);
    float* psi = sm + ly.psi;
    if (check)
      for (int q = tid; q < PL / 4; q += T)
        reinterpret_cast<float4*>(sm + ly.phik)[q] = reinterpret_cast<const float4*>(psi)[q];
    const float* W1 = sm + ly.w1[wc];
    const float* W2 = sm + ly.w2[wc];
    float* E1 = sm + ly.e1;
    float* E2 = sm + ly.e2;
    const float* Gg = sm + ly.g;
    for (int s = 0; s < mb.inner_S; ++s) {
      // ---- right-hand side of the inner step, Eq. (37) in increment form
      {
        const bool band = band_psi;
        if (band) window();
        const float* v1 = sm + ly.scr;
        const float* v2 = v1 + PL;
        float* G = sm + ly.G;
        float* D = sm + ly.D;
        for (int i = warp; i < RPC; i += NW) {
          const int gi = r0 + i;
          const float* up_row = i > 0 ? psi + (i - 1) * N : row_at(ly.psi, gi == 0 ? M - 1 : gi - 1);
          const float* dn_row = i < RPC - 1 ? psi + (i + 1) * N
                                            : row_at(ly.psi, gi == M - 1 ? 0 : gi + 1);
          const float* e1u_row = i > 0 ? E1 + (i - 1) * N : row_at(ly.e1, gi == 0 ? M - 1 : gi - 1);
          // every load of the row first, then the arithmetic, then the stores
          float x[NJ], up[NJ], dn[NJ], lf[NJ], rt[NJ], dv[NJ];
          float w1[NJ], w2[NJ], gg[NJ], vv1[NJ], vv2[NJ];
#pragma unroll
          for (int c = 0; c < NJ; ++c) {
            const int j = lane + 32 * c, q = i * N + j;
            x[c] = psi[q];
            up[c] = up_row[j];
            dn[c] = dn_row[j];
            lf[c] = psi[i * N + ((j - 1) & (N - 1))];
            rt[c] = psi[i * N + ((j + 1) & (N - 1))];
            if (s == 0)  // div e, fixed over the inner loop
              dv[c] = div_e(E1[q], e1u_row[j], E2[q], E2[i * N + ((j - 1) & (N - 1))]);
            else
              dv[c] = D[q];
            if (band) {
              w1[c] = W1[q];
              w2[c] = W2[q];
              gg[c] = Gg[q];
              vv1[c] = v1[q];
              vv2[c] = v2[q];
            }
          }
#pragma unroll
          for (int c = 0; c < NJ; ++c) {
            const int q = i * N + lane + 32 * c;
            const float f = rhs_bulk(m, x[c], up[c], dn[c], lf[c], rt[c], dv[c]);
            G[q] = band ? rhs_band(m, f, x[c], w1[c], w2[c], gg[c], vv1[c], vv2[c]) : m.tau * f;
            if (s == 0) D[q] = dv[c];
          }
        }
        __syncthreads();
      }
      // ---- row R2C: z[n] = G[2n] + i G[2n+1], FFT_L, even/odd split -> X
      {
        if (fwarp) {
          float2 x[E];
          const float2* row = reinterpret_cast<const float2*>(sm + ly.G + (flive ? ft : 0) * N);
#pragma unroll
          for (int q = 0; q < E; ++q) x[q] = flive ? row[fu + (q << LOGTP)] : make_float2(0.f, 0.f);
          stages<LOGL, LOGE, 0, false, 1, false, true, true>(x, fbase, fu, mb.tws4);
#pragma unroll
          for (int q = 0; q < E; ++q) fbase[pad(fu + (q << LOGTP))] = x[q];
          __syncwarp();
          if (flive) {
          float2* Xrow = reinterpret_cast<float2*>(sm + ly.X) + (size_t)ft * L;
#pragma unroll
          for (int q = 0; q < E; ++q) {
            const int kk = fu + (q << LOGTP);
            const float2 Zk = x[q];
            if (kk == 0) {
              Xrow[0] = make_float2(Zk.x + Zk.y, Zk.x - Zk.y);
              continue;
            }
            const float2 Zm = fbase[pad(L - kk)];
            const float2 Ev = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
            const float2 Dd = make_float2(0.5f * (Zk.x - Zm.x), 0.5f * (Zk.y + Zm.y));
            const float2 O = make_float2(Dd.y, -Dd.x);
            Xrow[kk] = cadd(Ev, cmul(__ldg(&mb.twN[kk]), O));
          }
          }
        }
      }
      cl.sync();
      // ---- column solve: forward and backward recursions per column and
      // real/imaginary part (task = 2 k + part, lane-contiguous) over the
      // CTA's rows.  The warm-ups read the rec_R spectrum rows before and
      // after the CTA's rows (indices modulo M), first copied from the other
      // CTAs into scratch by all warps, so that the recursions' chains read
      // only this CTA's shared memory.
      {
        const int Rr = mb.rec_R;
        float* Hx = sm + ly.scr;          // [2 Rr][N]: the rows before, then after
        float* U = Hx + 2 * Rr * N;       // [(RPC + Rr)][2L]
        float* X2 = sm + ly.X2;
        const float* Xo = sm + ly.X;
        // all of a thread's remote loads are issued before its stores, in
        // batches of HB rows, so that their latencies overlap
        constexpr int NC4 = (N / 4 + 31) / 32, HB = 4;
        for (int hr0 = warp; hr0 < 2 * Rr; hr0 += HB * NW) {
          float4 t[HB][NC4];
#pragma unroll
          for (int b = 0; b < HB; ++b) {
            const int hr = hr0 + b * NW;
            if (hr < 2 * Rr) {
              int gi = hr < Rr ? r0 - Rr + hr : r0 + RPC + (hr - Rr);
              gi %= M;
              if (gi < 0) gi += M;
              const float4* srow = reinterpret_cast<const float4*>(row_at(ly.X, gi));
#pragma unroll
              for (int c = 0; c < NC4; ++c)
                if (lane + 32 * c < N / 4) t[b][c] = srow[lane + 32 * c];
            }
          }
#pragma unroll
          for (int b = 0; b < HB; ++b) {
            const int hr = hr0 + b * NW;
            if (hr < 2 * Rr) {
#pragma unroll
              for (int c = 0; c < NC4; ++c)
                if (lane + 32 * c < N / 4)
                  reinterpret_cast<float4*>(Hx + hr * N)[lane + 32 * c] = t[b][c];
            }
          }
        }
        __syncthreads();
        for (int task = tid; task < 2 * L; task += T) {
          const float4 p = __ldg(mb.rec + (task >> 1));
          const float r = (task & 1) ? p.z : p.x, sc = (task & 1) ? p.w : p.y;
          float uu = 0.f;
#pragma unroll 4
          for (int j = 0; j < Rr; ++j) uu = fmaf(r, uu, Hx[j * N + task]);
#pragma unroll 4
          for (int j = 0; j < RPC; ++j) {
            uu = fmaf(r, uu, Xo[j * N + task]);
            U[j * 2 * L + task] = uu;
          }
#pragma unroll 4
          for (int j = 0; j < Rr; ++j) {
            uu = fmaf(r, uu, Hx[(Rr + j) * N + task]);
            U[(RPC + j) * 2 * L + task] = uu;
          }
          float v = 0.f;
#pragma unroll 4
          for (int j = RPC + Rr - 1; j >= RPC; --j) v = fmaf(r, v, U[j * 2 * L + task]);
#pragma unroll 4
          for (int j = RPC - 1; j >= 0; --j) {
            v = fmaf(r, v, U[j * 2 * L + task]);
            X2[j * 2 * L + task] = sc * v;
          }
        }
        __syncthreads();
      }
      // ---- row C2R of X2, inverse FFT_L, psi += result
      if (fwarp) {
        const float2* Xrow = reinterpret_cast<const float2*>(sm + ly.X2) + (size_t)(flive ? ft : 0) * L;
        float2 x[E];
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int kk = fu + (q << LOGTP);
          const float2 xk = Xrow[kk], xm = Xrow[(L - kk) & (L - 1)];
          if (kk == 0) {
            x[q] = make_float2(xk.x + xk.y, xk.x - xk.y);
            continue;
          }
          const float2 Xe = make_float2(xk.x + xm.x, xk.y - xm.y);
          const float2 Dd = make_float2(xk.x - xm.x, xk.y + xm.y);
          const float2 Xo = cmul(Dd, cconj(__ldg(&mb.twN[kk])));
          x[q] = make_float2(Xe.x - Xo.y, Xe.y + Xo.x);
        }
        stages<LOGL, LOGE, 0, true, 1, false, true, true>(x, fbase, fu, mb.tws4);
        if (flive) {
          float2* prow = reinterpret_cast<float2*>(psi + ft * N);
          int nb = 0;
#pragma unroll
          for (int q = 0; q < E; ++q) {
            const float2 pv = prow[fu + (q << LOGTP)];
            const float2 nv = make_float2(pv.x + x[q].x, pv.y + x[q].y);
            prow[fu + (q << LOGTP)] = nv;
            nb |= in_band(nv.x, m) | in_band(nv.y, m);
            const int qq = ft * N + 2 * (fu + (q << LOGTP));
            set_u(qq, nv.x, wc);
            set_u(qq + 1, nv.y, wc);
          }
          if (nb) bflag[bpar] = 1;
        }
      }
      cl.sync();
      band_psi = bflag[bpar] != 0;
      if (tid == 0) bflag[bpar ^ 1] = 0;
      bpar ^= 1;
    }
    // ---- w and b update, Eqs. (41), (42), (40), (23), into the other w parity
    {
      const bool band = band_psi;
      if (band) window();
      const float* v1 = sm + ly.scr;
      const float* v2 = v1 + PL;
      float* W1o = sm + ly.w1[wc ^ 1];
      float* W2o = sm + ly.w2[wc ^ 1];
      const float* phik = sm + ly.phik;
      double n0 = 0.0, n1 = 0.0;
      for (int i = warp; i < RPC; i += NW) {
        const int gi = r0 + i;
        const float* dn_row = i < RPC - 1 ? psi + (i + 1) * N
                                          : row_at(ly.psi, gi == M - 1 ? 0 : gi + 1);
        float x[NJ], dn[NJ], rt[NJ], e1[NJ], e2[NJ], w1[NJ], w2[NJ], gg[NJ], vv1[NJ], vv2[NJ];
        float pk[NJ];
#pragma unroll
        for (int c = 0; c < NJ; ++c) {
          const int j = lane + 32 * c, q = i * N + j;
          x[c] = psi[q];
          dn[c] = dn_row[j];
          rt[c] = psi[i * N + ((j + 1) & (N - 1))];
          e1[c] = E1[q];
          e2[c] = E2[q];
          w1[c] = W1[q];
          w2[c] = W2[q];
          if (band) {
            gg[c] = Gg[q];
            vv1[c] = v1[q];
            vv2[c] = v2[q];
          }
          if (check) pk[c] = phik[q];
        }
#pragma unroll
        for (int c = 0; c < NJ; ++c) {
          const int q = i * N + lane + 32 * c;
          const float b1 = e1[c] + w1[c], b2 = e2[c] + w2[c];
          float wo1, wo2, eo1, eo2;
          if (band)
            wb_point<true>(m, x[c], dn[c] - x[c], rt[c] - x[c], b1, b2, gg[c], vv1[c], vv2[c], wo1,
                           wo2, eo1, eo2);
          else
            wb_point<false>(m, x[c], dn[c] - x[c], rt[c] - x[c], b1, b2, 0.f, 0.f, 0.f, wo1, wo2,
                            eo1, eo2);
          W1o[q] = wo1;
          W2o[q] = wo2;
          E1[q] = eo1;
          E2[q] = eo2;
          if (check) {
            const double df = (double)x[c] - (double)pk[c];
            n0 += df * df;
            n1 += (double)pk[c] * (double)pk[c];
          }
        }
      }
      if (check) block_sum2(n0, n1, reinterpret_cast<double*>(sm + ly.part));
    }
    cl.sync();
    wc ^= 1;
    done = k + 1;
    if (check) {
      double num = 0.0, den = 0.0;
      for (int q = 0; q < C; ++q) {
        const double* p = reinterpret_cast<const double*>(rbase[q] + ly.part);
        num += p[0];
        den += p[1];
      }
      if (rank == 0 && tid == 0) {
        mb.red[0] = num;
        mb.red[1] = den;
      }
      const double rel = sqrt(num) / (sqrt(den) + 1e-6);
      if (a.tol > 0.0 && rel <= a.tol) break;
    }
  }

  // ---- store the CTA's rows of the state at parity cur ^ (done & 1)
  {
    const int pf = mb.cur ^ (done & 1);
    const size_t gb = (size_t)r0 * N;
    float* dst[5] = {mb.phi[pf], mb.w1[pf], mb.w2[pf], mb.e1, mb.e2};
    const int src[5] = {ly.psi, ly.w1[wc], ly.w2[wc], ly.e1, ly.e2};
#pragma unroll
    for (int p = 0; p < 5; ++p) {
      float4* d4 = reinterpret_cast<float4*>(dst[p] + gb);
      const float4* s4 = reinterpret_cast<const float4*>(sm + src[p]);
      for (int q = tid; q < PL / 4; q += T) d4[q] = s4[q];
    }
  }
  if (rank == 0 && tid == 0) *mb.done = done;
  // no CTA may leave while another can still read its shared memory
  cl.sync();
}

template <int LOGL>
cudaError_t go(const ResArgs& a, int members, int C, size_t smem, cudaStream_t s, bool set_attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kResThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (set_attr) {
    // the largest size any context may use, so that contexts of different
    // sizes can share the kernel; clusters of 16 need the non-portable size
    cudaError_t e = cudaFuncSetAttribute(k_resident<LOGL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kResMaxSmem);
    if (e != cudaSuccess) return e;
    if (C > 8 &&
        cudaFuncSetAttribute(k_resident<LOGL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return cudaErrorNotSupported;
    }
    cfg.gridDim = dim3(C);
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, k_resident<LOGL>, &cfg);
    if (e != cudaSuccess) {
      cudaGetLastError();  // a cluster shape the device refuses is not an error here
      return cudaErrorNotSupported;
    }
    return clusters > 0 ? cudaSuccess : cudaErrorNotSupported;
  }
  cfg.gridDim = dim3(C * members);
  cfg.stream = s;
  return cudaLaunchKernelEx(&cfg, k_resident<LOGL>, a);
}

}  // namespace res

size_t resident_smem(const Geo& geo, int R, int rec_R, int C) {
  const res::Lay l = res::make_lay(geo.M, geo.N, R, rec_R, C);
  return (size_t)l.total * sizeof(float);
}

bool resident_supported(const Geo& geo, int R, int rec_R, int C) {
  if (geo.neumann || rec_R <= 0 || R < 0 || R > kMaxR) return false;
  if (C != 8 && C != 16) return false;
  if (geo.N != 32 && geo.N != 64 && geo.N != 128 && geo.N != 256) return false;
  if (geo.M < 2 * C || geo.M % C) return false;
  // one pass of the row transforms: the CTA's rows at L / 4 threads each
  if ((geo.M / C) * (geo.L / 4) > kResThreads) return false;
  return resident_smem(geo, R, rec_R, C) <= kResMaxSmem;
}

cudaError_t launch_resident(const ResArgs& a, int members, const Geo& geo, int C, size_t smem,
                            cudaStream_t s, bool set_attr) {
  switch (geo.L) {
    case 16: return res::go<4>(a, members, C, smem, s, set_attr);
    case 32: return res::go<5>(a, members, C, smem, s, set_attr);
    case 64: return res::go<6>(a, members, C, smem, s, set_attr);
    case 128: return res::go<7>(a, members, C, smem, s, set_attr);
  }
  return cudaErrorInvalidValue;
}

}  // namespace srk
