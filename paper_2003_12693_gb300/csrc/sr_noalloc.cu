// sr_phi_step_noalloc: one inner step of the phi update for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: a host that hands every byte of GPU
// memory out of its own fixed arena (a long-running service with a hard memory
// budget), code that runs while its stream is being captured into a CUDA graph
// in a mode that forbids allocation, or a real-time loop that cannot afford the
// implicit device synchronisation cudaMalloc and cudaFree may cause.  For them
// this file keeps the half spectrum and the FFT / symbol tables of the step in
// a file-scope device array that the module loader reserves once per GPU and
// that stays reserved until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Nothing in it has to start at zero: each call rewrites the
// tables and the whole spectrum before reading them.  Two calls whose work
// overlaps on the GPU (different streams, or one stream used from several
// threads without ordering) race on the array and give wrong results.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "sr.h"
#include "sr_internal.h"

namespace {

// Largest image this entry point accepts: H, W <= 512 (powers of two >= 16).
constexpr int kMaxSide = 512;
constexpr size_t kSpectrumBytes = (size_t)kMaxSide * (kMaxSide / 2) * sizeof(float2);  // 1 MiB
constexpr size_t kTableBytes = 16 * 1024;
constexpr size_t kScratchBytes = kSpectrumBytes + kTableBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_nsm[kMaxDevices] = {};

// Tables of the step, computed in double and rounded once, like sr_create's:
// FFT twiddles of the row (length W/2) and column (length H) transforms, the
// real-row post-processing twiddles exp(-2 pi i k / W), and the two halves of
// the symbol of Eq. (32), tau mu 4 sin^2(pi l / H) and tau mu 4 sin^2(pi k / W).
__global__ void k_noalloc_tables(int H, int W, double taumu, float2* tw_row, float2* tw_col,
                                 float2* tw_n, float* aM, float* aN) {
  const int L = W / 2;
  const int total = L + H + L + H + (L + 1);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    double s, c;
    if (t < L) {
      sincospi(-2.0 * (double)t / (double)L, &s, &c);
      tw_row[t] = make_float2((float)c, (float)s);
    } else if (t < L + H) {
      const int q = t - L;
      sincospi(-2.0 * (double)q / (double)H, &s, &c);
      tw_col[q] = make_float2((float)c, (float)s);
    } else if (t < 2 * L + H) {
      const int k = t - L - H;
      sincospi(-2.0 * (double)k / (double)W, &s, &c);
      tw_n[k] = make_float2((float)c, (float)s);
    } else if (t < 2 * L + 2 * H) {
      const int l = t - 2 * L - H;
      const double sn = sinpi((double)l / (double)H);
      aM[l] = (float)(taumu * 4.0 * sn * sn);
    } else {
      const int k = t - 2 * L - 2 * H;
      const double sn = sinpi((double)k / (double)W);
      aN[k] = (float)(taumu * 4.0 * sn * sn);
    }
  }
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int log2i(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

// Once per device, with that device current: the device address of the
// array (host code may not use the symbol itself as a pointer) and the kernel
// attributes.  Returns nullptr on failure.
unsigned char* scratch_for_current_device(int* nsm) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return nullptr;
    if (srk::configure_kernels() != cudaSuccess) return nullptr;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return nullptr;
    g_nsm[dev] = n;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *nsm = g_nsm[dev];
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" sr_status sr_phi_step_noalloc(int H, int W, const sr_params* p, const float* g,
                                         const float* psi_in, const float* w1, const float* w2,
                                         const float* b1, const float* b2, float* psi_out,
                                         void* cuda_stream) {
  if (!p || !g || !psi_in || !w1 || !w2 || !b1 || !b2 || !psi_out) return SR_EINVAL;
  const float vals[] = {p->alpha, p->beta, p->gamma, p->mu, p->tau, p->eps, p->band_l, p->d};
  for (float v : vals)
    if (!std::isfinite(v)) return SR_EINVAL;
  if (p->mu <= 0.f || p->tau <= 0.f || p->eps <= 0.f || p->band_l < 0.f) return SR_EINVAL;
  if (p->win_radius < 0 || p->win_radius > srk::kMaxR) return SR_EINVAL;
  if (p->win_radius > 0 && p->d <= 0.f) return SR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(psi_in) & 15u) || (reinterpret_cast<uintptr_t>(psi_out) & 15u))
    return SR_EINVAL;
  // the spectrum of a larger image does not fit the fixed array
  if (!pow2(H) || !pow2(W) || H < 16 || W < 16 || H > kMaxSide || W > kMaxSide)
    return SR_EUNSUPPORTED;

  int nsm = 0;
  unsigned char* base = scratch_for_current_device(&nsm);
  if (!base) return SR_ECUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);

  const int L = W / 2;
  float2* X = reinterpret_cast<float2*>(base);
  float2* tw_row = reinterpret_cast<float2*>(base + kSpectrumBytes);
  float2* tw_col = tw_row + kMaxSide / 2;
  float2* tw_n = tw_col + kMaxSide;
  float* aM = reinterpret_cast<float*>(tw_n + kMaxSide / 2);
  float* aN = aM + kMaxSide;

  k_noalloc_tables<<<8, 256, 0, s>>>(H, W, (double)p->tau * (double)p->mu, tw_row, tw_col, tw_n,
                                     aM, aN);
  if (cudaGetLastError() != cudaSuccess) return SR_ECUDA;

  srk::Geo geo{H, W, L, log2i(W)};
  srk::Model m{};
  m.alpha = p->alpha;
  m.beta = p->beta;
  m.gamma = p->gamma;
  m.mu = p->mu;
  m.tau = p->tau;
  m.eps = p->eps;
  m.band_l = p->band_l;
  m.beta2_mu = (float)(2.0 * (double)p->beta / (double)p->mu);
  m.gamma_mu = (float)((double)p->gamma / (double)p->mu);
  m.inv_eps = (float)(1.0 / (double)p->eps);
  m.half_inv_eps = (float)(0.5 / (double)p->eps);
  m.dp_scale = (float)(1.57079632679489661923 / ((double)p->eps * (double)p->eps));
  m.l_eps = (float)((double)p->band_l / (double)p->eps);
  m.sin_l = (float)std::sin(3.14159265358979323846 * (double)p->band_l / (double)p->eps);
  m.cos_l = (float)std::cos(3.14159265358979323846 * (double)p->band_l / (double)p->eps);
  m.R = p->win_radius;
  for (int t = -m.R; t <= m.R; ++t)
    m.kw[t + m.R] = (float)std::exp(-(double)(t * t) / ((double)p->d * (double)p->d));

  // the same row-pass shape as a context of this size uses (one rule for both)
  int NT = 0, T = 0;
  if (!srk::row_shape(H, L, nsm, &NT, &T)) return SR_EUNSUPPORTED;
  // Only the shared-memory passes of sr_kernels.cu (k_rowfwd, k_colsolve,
  // k_rowinv) may run this plan: they read the flat twiddle table `tw` alone.
  // The register passes of sr_fft.cu need the per-stage tables, which this
  // entry point does not build, so they stay null here.
  srk::Fft frow{L, log2i(L), log2i(L) / 4, 1 << (log2i(L) % 4), tw_row, nullptr, nullptr};
  srk::Fft fcol{H, log2i(H), log2i(H) / 4, 1 << (log2i(H) % 4), tw_col, nullptr, nullptr};

  srk::RowFwdArgs fa{};
  fa.geo = geo;
  fa.mod = m;
  fa.fft = frow;
  fa.twN = tw_n;
  fa.psi = psi_in;
  fa.g = g;
  fa.w1 = w1;
  fa.w2 = w2;
  fa.b1 = b1;
  fa.b2 = b2;
  fa.X = X;
  fa.T = T;
  fa.CW = W < 128 ? W : 128;
  if (srk::launch_rowfwd(fa, srk::kRowRHS, NT, s) != cudaSuccess) return SR_ECUDA;
  srk::ColArgs ca{geo, fcol, aM, aN, X};
  if (srk::launch_colsolve(ca, s) != cudaSuccess) return SR_ECUDA;
  srk::RowInvArgs ia{};
  ia.geo = geo;
  ia.fft = frow;
  ia.twN = tw_n;
  ia.X = X;
  ia.psi_in = psi_in;
  ia.out = psi_out;
  ia.T = T;
  if (srk::launch_rowinv(ia, srk::kInvADD, NT, s) != cudaSuccess) return SR_ECUDA;
  return SR_OK;
}
