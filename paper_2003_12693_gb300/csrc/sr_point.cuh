// Per-pixel arithmetic of one outer iteration, shared by the tiled kernels
// (sr_kernels.cu) and the cluster-resident iteration (sr_resident.cu), so that
// both evaluate the regularised functions, the right-hand side and the w/b
// update with the same FP32 operations.
#pragma once
#include <math.h>

#include "sr_internal.h"

namespace srk {

// ---------------------------------------------------------------------------
// Regularised functions, Eqs. (5), (6), (11), (28), (29), in FP32
// ---------------------------------------------------------------------------
// Arguments are scaled once, y = x / eps (as x times the host-computed 1/eps);
// each branch boundary |y| = 1 is a point of continuity of the function.
constexpr float kInvPi = 0.318309886183790671538f;

__device__ __forceinline__ float heps(float x, const Model& m) {
  const float y = x * m.inv_eps;
  if (y > 1.f) return 1.f;
  if (y < -1.f) return 0.f;
  return 0.5f * (1.f + y + sinpif(y) * kInvPi);
}
__device__ __forceinline__ float deps(float x, const Model& m) {
  const float y = x * m.inv_eps;
  if (fabsf(y) > 1.f) return 0.f;
  return (1.f + cospif(y)) * m.half_inv_eps;
}
// delta_eps and delta'_eps (Eq. (29)) of one argument
__device__ __forceinline__ void dd_eps(float x, const Model& m, float& d, float& dp) {
  const float y = x * m.inv_eps;
  if (fabsf(y) > 1.f) {
    d = dp = 0.f;
    return;
  }
  float sn, cs;
  sincospif(y, &sn, &cs);
  d = (1.f + cs) * m.half_inv_eps;
  dp = -m.dp_scale * sn;
}
// The band functions at x need H_eps and delta_eps at x + l and x - l, and
// the rhs also delta_eps, delta'_eps at x.  All of them come from one
// sincospif of y = x/eps: sin and cos at y +- l/eps follow by angle addition
// with the host constants sin(pi l/eps), cos(pi l/eps) (absolute error a few
// 1e-7, where the separate evaluations give about 1e-7).
struct BandTrig {
  float y, sn, cs;
  __device__ __forceinline__ BandTrig(float x, const Model& m) {
    y = x * m.inv_eps;
    sincospif(y, &sn, &cs);
  }
  // H_eps and delta_eps at x + sign * l
  __device__ __forceinline__ void at_shift(float sign, const Model& m, float& h, float& d) const {
    const float Y = y + sign * m.l_eps;
    const float sY = sn * m.cos_l + sign * cs * m.sin_l;
    const float cY = cs * m.cos_l - sign * sn * m.sin_l;
    const bool in = fabsf(Y) <= 1.f;
    h = in ? 0.5f * (1.f + Y + sY * kInvPi) : (Y > 0.f ? 1.f : 0.f);
    d = in ? (1.f + cY) * m.half_inv_eps : 0.f;
  }
  // delta_eps and delta'_eps at x
  __device__ __forceinline__ void at_zero(const Model& m, float& d, float& dp) const {
    const bool in = fabsf(y) <= 1.f;
    d = in ? (1.f + cs) * m.half_inv_eps : 0.f;
    dp = in ? -m.dp_scale * sn : 0.f;
  }
  // h(x) = H(x + l)(1 - H(x - l)) (Eq. (11)) and h'(x) (Eq. (28)), |x| < l + eps
  __device__ __forceinline__ void band(const Model& m, float& h, float& hp) const {
    float hA, dA, hB, dB;
    at_shift(1.f, m, hA, dA);
    at_shift(-1.f, m, hB, dB);
    h = hA * (1.f - hB);
    hp = dA * (1.f - hB) - hA * dB;
  }
};

__device__ __forceinline__ float band_h(float x, const Model& m) {
  if (fabsf(x) >= m.band_l + m.eps) return 0.f;
  float h, hp;
  BandTrig(x, m).band(m, h, hp);
  return h;
}
__device__ __forceinline__ float band_hp(float x, const Model& m) {
  if (fabsf(x) >= m.band_l + m.eps) return 0.f;
  float h, hp;
  BandTrig(x, m).band(m, h, hp);
  return hp;
}

__device__ __forceinline__ bool in_band(float x, const Model& m) { return fabsf(x) < m.band_l + m.eps; }

// G = tau [ mu (div e + Lap psi) - gamma g |w| delta'(psi) + alpha g delta(psi)
//           + 2 beta h'(psi) (w . v) ] at one pixel (the band terms only where
// |psi| < l + eps; e = b - w, div the backward divergence).
// BAND = false is the form for tiles without narrow-band pixels: the band
// terms are not evaluated at all (rather than predicated off per pixel).
// div(b - w) = div e, backward differences (Eq. (36))
__device__ __forceinline__ float div_e(float e1, float e1u, float e2, float e2l) {
  return (e1 - e1u) + (e2 - e2l);
}
__device__ __forceinline__ float rhs_bulk(const Model& m, float x, float up, float dn, float lf,
                                          float rt, float dv) {
  const float lap = (up + dn) + (lf + rt) - 4.f * x;
  return m.mu * (dv + lap);
}
// the narrow-band terms added to the bulk force f at one pixel; G = tau f
__device__ __forceinline__ float rhs_band(const Model& m, float f, float x, float w1, float w2,
                                          float g, float v1, float v2) {
  if (in_band(x, m)) {
    const float wn = sqrtf(w1 * w1 + w2 * w2);
    const BandTrig bt(x, m);
    float dl, dpl, hh, hp;
    bt.at_zero(m, dl, dpl);
    bt.band(m, hh, hp);
    f += -m.gamma * g * wn * dpl + m.alpha * g * dl + 2.f * m.beta * hp * (w1 * v1 + w2 * v2);
  }
  return m.tau * f;
}

// Eqs. (41), (42), (40), (23) at one pixel: B = grad phi + b + (2 beta/mu) h v,
// t = (gamma/mu) g delta(phi); w = B/|B| if |B| > t else 0; b' = b + grad phi - w;
// returns w' and e' = b' - w'.
template <bool BAND>
__device__ __forceinline__ void wb_point(const Model& m, float x, float d1, float d2, float b1,
                                         float b2, float g, float v1, float v2, float& wo1,
                                         float& wo2, float& eo1, float& eo2) {
  float Bv1 = d1 + b1;
  float Bv2 = d2 + b2;
  float thr = 0.f;
  if (BAND && in_band(x, m)) {
    const BandTrig bt(x, m);
    float h, hp, dl, dpl;
    bt.band(m, h, hp);
    bt.at_zero(m, dl, dpl);
    Bv1 = fmaf(m.beta2_mu * h, v1, Bv1);
    Bv2 = fmaf(m.beta2_mu * h, v2, Bv2);
    thr = m.gamma_mu * g * dl;
  }
  // |B| and B/|B| from one reciprocal square root (a few ulp, against a
  // correctly rounded sqrt and two divisions)
  const float nB2 = Bv1 * Bv1 + Bv2 * Bv2;
  const float r = rsqrtf(nB2);
  float W1 = 0.f, W2 = 0.f;
  if (nB2 > 0.f && nB2 * r > thr) {
    W1 = Bv1 * r;
    W2 = Bv2 * r;
  }
  wo1 = W1;
  wo2 = W2;
  eo1 = ((b1 + d1) - W1) - W1;
  eo2 = ((b2 + d2) - W2) - W2;
}

}  // namespace srk
