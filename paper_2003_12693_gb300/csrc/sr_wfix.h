// Iterated w sub-problem, Eqs. (38)-(40): one sweep w <- B(w) / |B(w)|.
// Internal to the library (sr_api.cu <-> sr_wfix.cu).
#pragma once

#include "sr_internal.h"

namespace srk {

struct WFixArgs {
  Geo geo;
  Model mod;
  const float* phi1;       // phi^{k+1}
  const float* wk1;        // w^k: b^k = e^k + w^k
  const float* wk2;
  const float* ek1;        // e^k = b^k - w^k
  const float* ek2;
  const float* cw1;        // w^{k+1,r}, whose window sum v^{k+1,r} enters B (Eq. (38))
  const float* cw2;
  float* nw1;              // w^{k+1,r+1}; must not alias wk or cw
  float* nw2;
  float* e1o;              // last sweep: e^{k+1} = b^{k+1} - w^{k+1} (may alias ek), else null
  float* e2o;
  const float* phi_old;    // phi^k for the stopping test (last sweep), or null
  double* partials;        // 2 doubles per 32 x 32 tile when phi_old != null
};

cudaError_t launch_wfix_sweep(const WFixArgs& a, cudaStream_t s);

}  // namespace srk
