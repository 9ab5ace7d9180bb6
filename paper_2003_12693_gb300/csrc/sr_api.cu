// Host side of the C-ABI declared in include/sr.h: parameter checks, device
// state, FFT plans and tables, CUDA-graph capture of the outer iteration, and
// the FP64 stopping test.  The kernels live in sr_kernels.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "sr.h"
#include "sr_internal.h"
#include "sr_wfix.h"
#include "sr_inner.h"

using srk::Fft;
using srk::Geo;
using srk::Model;

struct sr_ctx {
  int H = 0, W = 0, L = 0;
  sr_params prm{};
  cudaStream_t stream = nullptr;     // caller's stream
  cudaStream_t cap_stream = nullptr; // private stream used only for graph capture
  int device = 0;
  int nsm = 0;
  Geo geo{};
  Model mod{};
  Fft fft_row{}, fft_col{};
  int row_T = 0, row_NT = 0, row_CW = 0;
  bool fft2 = false;  // register-resident FFT passes (sr_fft.cu) for this size
  bool fftgen = false;  // mixed-radix passes (sr_fftgen.cu): a side is not a power of two
  srk::GenPlan plan_row{}, plan_col{};
  bool gen_batched = false;  // member of a group: launch shapes for many images at once
  bool gen_fft_cols = false; // mixed-radix sides: column FFT instead of the recursions (timed, or SR_GEN_FFT_COLS)
  float2* gen_tab = nullptr;  // stage twiddles and roots of both plans
  sr_schedule sched{};  // schedule of the fft2 passes
  CUtensorMap tm_X{};   // X as a float32 matrix, boxes for the TMA column pass
  bool tm_X_ok = false;
  int col_tma_grid = 0;
  int* err_dev = nullptr;  // device error flag of the bounded waits
  long long stall_cycles = 0;  // failure-path tests: TMA column waits that run out (sr_test_stall_waits)
  int n_tile = 0;    // CTAs of the 32 x 8 tile kernels (energy)
  int n_tile32 = 0;  // CTAs of the 32 x 32 tile kernels (w/b update)

  // device state
  float* phi[2] = {nullptr, nullptr};
  float* w1[2] = {nullptr, nullptr};
  float* w2[2] = {nullptr, nullptr};
  float* e1 = nullptr;  // Bregman variable carried as e = b - w
  float* e2 = nullptr;
  float* g = nullptr;
  float* tmp1 = nullptr;
  float* tmp2 = nullptr;
  float* stage = nullptr;
  float* G = nullptr;         // increment right-hand side of the current inner step
  float* divE = nullptr;      // div e of the current outer iteration (fixed over the inner loop)
  unsigned char* mask_dev = nullptr;
  float2* X = nullptr;
  float2* X2 = nullptr;       // output of the recursion column pass (schedule 7)
  float4* rec = nullptr;      // per-column (r, s) pairs of that pass
  int rec_R = 0;              // its warm-up length; 0 if it is not available
  float2* tw_row = nullptr;
  float2* tw_col = nullptr;
  float2* tw_n = nullptr;
  float2* tws[4] = {nullptr, nullptr, nullptr, nullptr};  // stage twiddles: row16, row8, col16, col8
  float* aM = nullptr;
  float* aN = nullptr;
  double* partials = nullptr;
  double* red = nullptr;       // device: reduction result
  double* red_host = nullptr;  // pinned host copy
  int cur = 0;                 // phi[cur], w*[cur] hold phi^k, w^k
  long long iters = 0;

  // graphs of one outer iteration without the stopping test, per parity
  // w sub-problem: 0 = soft threshold (41)-(42); >= 1 = sweeps of (38)-(40)
  int w_sweeps = 0;
  long long inner_steps = 0;  // inner phi steps run by sr_iterate (all modes)
  float* wfx1 = nullptr;   // sweep ping-pong planes, allocated on first use
  // phi sub-problem solver: 0 = FFT (Eqs. (31)-(33)), 1 = AOS (end of Sec. 4)
  int phi_solver = 0;
  float* aos_T1 = nullptr;  // AOS scratch planes, allocated on first use
  float* aos_X2 = nullptr;
  srk::AosArgs aos{};       // AOS constants (k, r, s, warm-up, powers of r)
  // Neumann reading of Eq. (27) (sr_set_boundary): the solve runs on the even
  // extension of each row (length 2W) and the reflected columns
  srk::Geo geo2{};          // M x 2W, complex row length W
  srk::Fft fft_row2{};
  float2* tw_row2 = nullptr;
  float2* tw_n2 = nullptr;
  float2* tws2[2] = {nullptr, nullptr};  // stage twiddles of length W: 16 and 8 values
  float* G2 = nullptr;      // M x 2W: the extended rows, then the inverse transform
  float2* Xn = nullptr;     // M x W: their half spectrum
  float2* Xn2 = nullptr;    // M x W: after the column solve
  float4* rec2 = nullptr;   // per-column (r, s) of the reflected column solve
  int rec2_R = 0;
  int row2_T = 0, row2_threads = 0;
  float* wfx2 = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_kernels = 0;
  // outer iterations resident in shared memory (sr_set_resident)
  int resident = 0;
  size_t res_smem = 0;
  int res_C = 0;                      // CTAs per cluster (8 or 16)
  float2* res_tws4 = nullptr;         // stage twiddles of the rows, 4 values per thread
  srk::ResMember* res_dev = nullptr;  // the image's description at parity 0 and 1
  int* res_done = nullptr;            // iterations the last launch ran
  int* res_done_host = nullptr;       // pinned copy

  long long launches = 0;
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_pending;  // (kclass, event index of the start)
  double ktime[SR_KCLASS_COUNT] = {0};
  long long kcount[SR_KCLASS_COUNT] = {0};

  std::string err;
};

namespace {

sr_status fail(sr_ctx* c, sr_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

sr_status cuda_fail(sr_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(c, SR_ECUDA, m);
}

#define SR_CUDA(ctx, call)                                      \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);  \
  } while (0)

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

bool finite_f(float v) { return std::isfinite(v); }

sr_status check_params(const sr_params* p, std::string& why) {
  const float vals[] = {p->alpha, p->beta, p->gamma, p->mu, p->tau, p->eps, p->band_l, p->d,
                        p->inner_tol, p->rho, p->sigma};
  for (float v : vals)
    if (!finite_f(v)) {
      why = "parameters must be finite";
      return SR_EINVAL;
    }
  if (p->mu <= 0.f || p->tau <= 0.f || p->eps <= 0.f) {
    why = "mu, tau and eps must be positive";
    return SR_EINVAL;
  }
  if (p->win_radius < 0 || p->win_radius > srk::kMaxR) {
    why = "win_radius must lie in [0, 8]";
    return SR_EINVAL;
  }
  if (p->win_radius > 0 && p->d <= 0.f) {
    why = "d must be positive";
    return SR_EINVAL;
  }
  if (p->band_l < 0.f || p->rho < 0.f || p->sigma < 0.f) {
    why = "band_l, rho and sigma must be non-negative";
    return SR_EINVAL;
  }
  if (p->inner_S < 1) {
    why = "inner_S must be >= 1";
    return SR_EINVAL;
  }
  if (p->s_pow != 1 && p->s_pow != 2) {
    why = "s_pow must be 1 or 2";
    return SR_EINVAL;
  }
  if (p->check_every < 1) {
    why = "check_every must be >= 1";
    return SR_EINVAL;
  }
  if ((int)std::ceil(3.0 * p->sigma) > srk::kMaxGauss) {
    why = "sigma too large (ceil(3 sigma) must be <= 32)";
    return SR_EINVAL;
  }
  if (!std::isfinite(p->inner_tol)) {
    why = "inner_tol must be finite";
    return SR_EINVAL;
  }
  return SR_OK;
}

// Mixed-radix plan of length n: radix-16 stages, one radix 8, 4 or 2 for the
// rest of the power of two, then the odd primes (each at most 31).  Appends
// the stage twiddles exp(-2 pi i t k / (Ns R)) and, for primes without a
// dedicated butterfly, the roots exp(-2 pi i e / R) to tab (FP64, rounded).
bool gen_plan(int n, srk::GenPlan& P, std::vector<float2>& tab, std::vector<int>& root_at) {
  std::vector<int> rad;
  int m = n;
  while (m % 16 == 0) rad.push_back(16), m /= 16;
  if (m % 8 == 0) rad.push_back(8), m /= 8;
  else if (m % 4 == 0) rad.push_back(4), m /= 4;
  else if (m % 2 == 0) rad.push_back(2), m /= 2;
  for (int p = 3; p < srk::kGenMaxRadix && m > 1; p += 2)
    while (m % p == 0) rad.push_back(p), m /= p;
  if (m != 1 || (int)rad.size() > srk::kGenMaxStages) return false;
  P = srk::GenPlan{};
  P.n = n;
  P.nst = (int)rad.size();
  int Ns = 1;
  for (int s = 0; s < P.nst; ++s) {
    const int R = rad[s];
    P.radix[s] = R;
    P.ns[s] = Ns;
    // ceil(2^32 / d) for the device's multiply-high division; 0 stands for d = 1
    auto magic = [](int d) {
      return d == 1 ? 0u : (unsigned)(((1ull << 32) + (unsigned)d - 1) / (unsigned)d);
    };
    P.mag_m[s] = magic(n / R);
    P.mag_ns[s] = magic(Ns);
    P.twoff[s] = (int)tab.size();
    for (int t = 1; t < R; ++t)
      for (int k = 0; k < Ns; ++k) {
        const double a = -2.0 * M_PI * (double)t * (double)k / ((double)Ns * R);
        tab.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
      }
    const bool dedicated = R == 2 || R == 3 || R == 4 || R == 5 || R == 8 || R == 16;
    if (!dedicated) {
      if (root_at[R] < 0) {
        root_at[R] = (int)tab.size();
        for (int e = 0; e < R; ++e) {
          const double a = -2.0 * M_PI * (double)e / (double)R;
          tab.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
      }
      P.rootoff[s] = root_at[R];
    }
    Ns *= R;
  }
  return true;
}

void make_fft(Fft& f, int L, const float2* tw) {
  f.L = L;
  f.logL = ilog2(L);
  f.tw = tw;
  f.n16 = f.logL / 4;
  f.tail = 1 << (f.logL % 4);
}

std::vector<float2> twiddles(int n, int len) { return srk::twiddle_table(n, len); }
using srk::stage_twiddle_table;

// Failure injection for tests (sr_test_fail_allocations): the number of
// device or pinned-host allocations the library may still make before the
// next ones fail as if memory had run out; negative = no limit.
std::atomic<long long> g_alloc_budget{-1};

bool take_alloc() {
  long long b = g_alloc_budget.load();
  while (b >= 0) {
    if (b == 0) return false;
    if (g_alloc_budget.compare_exchange_weak(b, b - 1)) return true;
  }
  return true;
}

cudaError_t dev_alloc(void** p, size_t bytes) {
  if (!take_alloc()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t host_alloc(void** p, size_t bytes) {
  if (!take_alloc()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(p, bytes);
}

template <class T>
sr_status upload(sr_ctx* c, T** dst, const std::vector<T>& v) {
  const cudaError_t e = dev_alloc((void**)dst, v.size() * sizeof(T));
  if (e == cudaErrorMemoryAllocation) return fail(c, SR_ENOMEM, "device allocation failed");
  SR_CUDA(c, e);
  SR_CUDA(c, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SR_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---- launch bookkeeping (per-kernel events in profile mode) ---------------
int ev_take(sr_ctx* c) {
  const int idx = (int)c->ev_pending.size() * 2;
  while ((int)c->ev_pool.size() < idx + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    c->ev_pool.push_back(e);
  }
  return idx;
}

sr_status flush_profile(sr_ctx* c) {
  if (c->ev_pending.empty()) return SR_OK;
  SR_CUDA(c, cudaStreamSynchronize(c->stream));
  for (auto& pr : c->ev_pending) {
    float ms = 0.f;
    SR_CUDA(c, cudaEventElapsedTime(&ms, c->ev_pool[pr.second], c->ev_pool[pr.second + 1]));
    c->ktime[pr.first] += ms;
    c->kcount[pr.first] += 1;
  }
  c->ev_pending.clear();
  return SR_OK;
}

// Run `launch` on stream s; in profile mode bracket it with events.
template <class F>
sr_status run_kernel(sr_ctx* c, int kclass, cudaStream_t s, const char* name, F launch) {
  int ev = -1;
  if (c->profile) {
    if (c->ev_pending.size() >= 4096) {
      sr_status st = flush_profile(c);
      if (st != SR_OK) return st;
    }
    ev = ev_take(c);
    if (ev < 0) return fail(c, SR_ECUDA, "cudaEventCreate failed");
    SR_CUDA(c, cudaEventRecord(c->ev_pool[ev], s));
  }
  cudaError_t e = launch();
  if (e != cudaSuccess) return cuda_fail(c, e, name);
  c->launches += 1;
  if (c->profile) {
    SR_CUDA(c, cudaEventRecord(c->ev_pool[ev + 1], s));
    c->ev_pending.push_back({kclass, ev});
  }
  return SR_OK;
}

// ---- FFT schedule -----------------------------------------------------------
int sched_rows(const sr_ctx* c, const sr_schedule& sc) {
  return sc.row_threads * sc.row_values_per_thread / c->L;
}

bool sched_valid(const sr_ctx* c, const sr_schedule& sc) {
  if (!c->fft2) return false;
  if (sc.row_values_per_thread != 8 && sc.row_values_per_thread != 16) return false;
  if (sc.col_schedule == srk::kColRec) {
    if (c->rec_R <= 0) return false;
  } else if (sc.col_schedule == srk::kColSmall) {
    if (c->rec_R <= 0 || !srk::solve_small_supported(c->geo, c->rec_R)) return false;
  } else {
    if (sc.col_schedule < 0 || sc.col_schedule > 6) return false;
    if (sc.col_schedule == 3 && !c->tm_X_ok) return false;
    if (srk::colsolve2_threads(c->H, sc.col_schedule) > 1024) return false;
  }
  if (sc.row_threads < 1 || sc.row_threads > 512) return false;
  const long long prod = (long long)sc.row_threads * sc.row_values_per_thread;
  if (prod % c->L) return false;
  const int T = (int)(prod / c->L);
  if (T < 1 || T > c->H) return false;
  if (sc.row_threads != T * c->L / sc.row_values_per_thread) return false;
  return srk::rowfft2_smem(T, c->L, sc.row_values_per_thread == 8 ? 3 : 4) <= 200 * 1024;
}

// raise the shared-memory limits of the kernels a schedule uses
cudaError_t sched_configure(sr_ctx* c, const sr_schedule& sc) {
  srk::RowFwdArgs fa{};
  fa.geo = c->geo;
  fa.T = sched_rows(c, sc);
  srk::RowInvArgs ia{};
  ia.geo = c->geo;
  ia.T = fa.T;
  srk::ColArgs ca{};
  ca.geo = c->geo;
  const int le = sc.row_values_per_thread == 8 ? 3 : 4;
  cudaError_t e = srk::launch_rowfft2(fa, le, sc.row_threads, nullptr, true);
  if (e == cudaSuccess) e = srk::launch_rowifft2(ia, true, le, sc.row_threads, nullptr, true);
  if (e != cudaSuccess) return e;
  if (sc.col_schedule == srk::kColRec) return cudaSuccess;
  if (sc.col_schedule == srk::kColSmall) {
    srk::SmallArgs sa{};
    sa.geo = c->geo;
    sa.rec_R = c->rec_R;
    return srk::launch_solve_small(sa, nullptr, true);
  }
  if (sc.col_schedule == 3) {
    e = srk::launch_colsolve_tma(ca, c->tm_X, 0, nullptr, true);
    int per_sm = 0;
    if (e == cudaSuccess) e = srk::colsolve_tma_occupancy(c->H, &per_sm);
    if (e != cudaSuccess) return e;
    const int nb = c->L / srk::colsolve_tma_cb(c->H);
    c->col_tma_grid = std::max(1, std::min(nb, c->nsm * std::max(per_sm, 1)));
    return cudaSuccess;
  }
  return srk::launch_colsolve2(ca, sc.col_schedule, nullptr, true);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D float32 tensor map: rows x cols (cols innermost), row pitch in floats,
// box of box_cols x box_rows, zero fill outside the tensor.
bool make_tensor_map_2d(CUtensorMap* map, const void* base, int rows, int cols, int pitch,
                        int box_cols, int box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// why the calling thread's last sr_create failed (sr_last_error(NULL))
thread_local std::string g_create_err;

std::mutex g_tune_mutex;
// (H, W, warm-up length of the column recursions) -> (device, schedule): the
// recursion passes' availability and cost depend on tau mu through rec_R
std::map<std::tuple<int, int, int>, std::pair<int, sr_schedule>> g_tuned;

// Time the candidate row and column schedules on the context's buffers and
// keep the fastest (once per image size and device in the process).
sr_status autotune(sr_ctx* c) {
  // SR_FFT_SCHEDULE="row_values,row_threads,col_schedule" fixes the schedule
  // (reproducible profiling); invalid values fall back to tuning
  if (const char* env = std::getenv("SR_FFT_SCHEDULE")) {
    sr_schedule sc{};
    if (std::sscanf(env, "%d,%d,%d", &sc.row_values_per_thread, &sc.row_threads,
                    &sc.col_schedule) == 3 &&
        sched_valid(c, sc)) {
      c->sched = sc;
      SR_CUDA(c, sched_configure(c, sc));
      return SR_OK;
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find({c->H, c->W, c->rec_R});
    if (it != g_tuned.end() && it->second.first == c->device) {
      c->sched = it->second.second;
      SR_CUDA(c, sched_configure(c, c->sched));
      return SR_OK;
    }
  }
  const size_t P = (size_t)c->H * c->W;
  SR_CUDA(c, cudaMemset(c->G, 0, P * sizeof(float)));
  SR_CUDA(c, cudaMemset(c->X, 0, (size_t)c->H * c->L * sizeof(float2)));
  SR_CUDA(c, cudaDeviceSynchronize());
  cudaStream_t s = c->cap_stream;
  cudaEvent_t e0, e1;
  SR_CUDA(c, cudaEventCreate(&e0));
  SR_CUDA(c, cudaEventCreate(&e1));
  auto time_it = [&](auto&& launch, float* us) -> cudaError_t {
    cudaError_t e = launch();
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
    const int reps = 10;
    for (int r = 0; r < reps; ++r)
      if ((e = launch()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
    *us = 1000.f * ms / reps;
    return cudaSuccess;
  };
  // bring clocks up before timing: ~20 ms of back-to-back launches
  {
    srk::ColArgs ca{};
    ca.geo = c->geo;
    ca.fft = c->fft_col;
    ca.aM = c->aM;
    ca.aN = c->aN;
    ca.X = c->X;
    sr_schedule sc{16, 0, 0, 0.f};
    SR_CUDA(c, sched_configure(c, sc));
    SR_CUDA(c, cudaEventRecord(e0, s));
    for (int r = 0; r < 4000; ++r) {
      SR_CUDA(c, srk::launch_colsolve2(ca, 0, s, false));
      if (r % 200 == 199) {
        SR_CUDA(c, cudaEventRecord(e1, s));
        SR_CUDA(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        SR_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
        if (ms > 20.f) break;
      }
    }
    SR_CUDA(c, cudaStreamSynchronize(s));
  }
  sr_schedule best{};
  float best_row = 1e30f;
  const int vpts[2] = {16, 8};
  const int threads[4] = {64, 128, 256, 512};
  cudaError_t err = cudaSuccess;
  for (int vi = 0; vi < 2 && err == cudaSuccess; ++vi)
    for (int ti = 0; ti < 4 && err == cudaSuccess; ++ti) {
      sr_schedule sc{vpts[vi], threads[ti], 0, 0.f};
      if (!sched_valid(c, sc)) continue;
      if ((err = sched_configure(c, sc)) != cudaSuccess) break;
      srk::RowFwdArgs fa{};
      fa.geo = c->geo;
      fa.fft = c->fft_row;
      fa.twN = c->tw_n;
      fa.src = c->G;
      fa.X = c->X;
      fa.T = sched_rows(c, sc);
      srk::RowInvArgs ia{};
      ia.geo = c->geo;
      ia.fft = c->fft_row;
      ia.twN = c->tw_n;
      ia.X = c->X;
      ia.psi_in = c->tmp1;
      ia.out = c->tmp2;
      ia.T = fa.T;
      const int le = sc.row_values_per_thread == 8 ? 3 : 4;
      float us = 0.f;
      err = time_it([&] {
        cudaError_t e = srk::launch_rowfft2(fa, le, sc.row_threads, s, false);
        return e != cudaSuccess ? e : srk::launch_rowifft2(ia, true, le, sc.row_threads, s, false);
      }, &us);
      if (err == cudaSuccess && us < best_row) {
        best_row = us;
        best.row_values_per_thread = sc.row_values_per_thread;
        best.row_threads = sc.row_threads;
      }
    }
  float best_col = 1e30f;
  for (int cs = 0; cs <= srk::kColRec && err == cudaSuccess; ++cs) {
    sr_schedule sc = best;
    sc.col_schedule = cs;
    if (!sched_valid(c, sc)) continue;
    if ((err = sched_configure(c, sc)) != cudaSuccess) break;
    srk::ColArgs ca{};
    ca.geo = c->geo;
    ca.fft = c->fft_col;
    ca.aM = c->aM;
    ca.aN = c->aN;
    ca.X = c->X;
    ca.err = c->err_dev;
    ca.rec = c->rec;
    ca.rec_R = c->rec_R;
    ca.Xout = c->X2;
    float us = 0.f;
    err = time_it([&] {
      if (cs == srk::kColRec) return srk::launch_colsolve_rec(ca, s);
      return cs == 3 ? srk::launch_colsolve_tma(ca, c->tm_X, c->col_tma_grid, s, false)
                     : srk::launch_colsolve2(ca, cs, s, false);
    }, &us);
    if (err == cudaSuccess && us < best_col) {
      best_col = us;
      best.col_schedule = cs;
    }
  }
  best.tuned_us = best_row + best_col;
  // the one-CTA solve of small images replaces the row pair and the column
  // pass together: it competes with their sum
  if (err == cudaSuccess) {
    sr_schedule sc = best;
    sc.col_schedule = srk::kColSmall;
    if (sched_valid(c, sc) && (err = sched_configure(c, sc)) == cudaSuccess) {
      srk::SmallArgs sa{};
      sa.geo = c->geo;
      sa.G = c->G;
      sa.psi_in = c->tmp1;
      sa.out = c->tmp2;
      sa.tws16 = c->fft_row.tws16;
      sa.twN = c->tw_n;
      sa.rec = c->rec;
      sa.rec_R = c->rec_R;
      float us = 0.f;
      err = time_it([&] { return srk::launch_solve_small(sa, s, false); }, &us);
      if (err == cudaSuccess && us < best.tuned_us) {
        best.col_schedule = srk::kColSmall;
        best.tuned_us = us;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(c, err, "FFT schedule autotuner");
  c->sched = best;
  SR_CUDA(c, sched_configure(c, best));
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned[{c->H, c->W, c->rec_R}] = {c->device, best};
  return SR_OK;
}

// Sides that are not powers of two: time the two column passes the
// mixed-radix path can use (the recursions of column schedule 7, or the
// mixed-radix column FFT with the symbol of Eq. (32)) and keep the faster,
// once per size, warm-up length and device in the process.
// SR_GEN_FFT_COLS=1 (FFT) or 0 (recursions) fixes the choice.
std::map<std::tuple<int, int, int>, std::pair<int, bool>> g_tuned_gen;

sr_status autotune_gen(sr_ctx* c) {
  if (const char* env = std::getenv("SR_GEN_FFT_COLS")) {
    c->gen_fft_cols = env[0] == '1' || c->rec_R <= 0;
    return SR_OK;
  }
  if (c->rec_R <= 0) {
    c->gen_fft_cols = true;
    return SR_OK;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned_gen.find({c->H, c->W, c->rec_R});
    if (it != g_tuned_gen.end() && it->second.first == c->device) {
      c->gen_fft_cols = it->second.second;
      return SR_OK;
    }
  }
  SR_CUDA(c, cudaMemset(c->X, 0, (size_t)c->H * c->L * sizeof(float2)));
  srk::ColArgs ca{};
  ca.geo = c->geo;
  ca.fft = c->fft_col;
  ca.aM = c->aM;
  ca.aN = c->aN;
  ca.X = c->X;
  ca.err = c->err_dev;
  ca.rec = c->rec;
  ca.rec_R = c->rec_R;
  ca.Xout = c->X2;
  cudaStream_t s = c->cap_stream;
  cudaEvent_t e0, e1;
  SR_CUDA(c, cudaEventCreate(&e0));
  SR_CUDA(c, cudaEventCreate(&e1));
  float best[2] = {1e30f, 1e30f};  // [0] recursions, [1] column FFT
  cudaError_t err = cudaSuccess;
  for (int round = 0; round < 2 && err == cudaSuccess; ++round)
    for (int fftc = 0; fftc < 2 && err == cudaSuccess; ++fftc) {
      auto launch = [&] {
        return fftc ? srk::launch_colsolve_gen(ca, c->plan_col, false, s)
                    : srk::launch_colsolve_rec(ca, s);
      };
      if ((err = launch()) != cudaSuccess) break;
      if ((err = cudaEventRecord(e0, s)) != cudaSuccess) break;
      for (int r = 0; r < 10 && err == cudaSuccess; ++r) err = launch();
      if (err == cudaSuccess) err = cudaEventRecord(e1, s);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err == cudaSuccess) best[fftc] = std::min(best[fftc], ms);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(c, err, "mixed-radix column pass autotuner");
  c->gen_fft_cols = best[1] < best[0];
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned_gen[{c->H, c->W, c->rec_R}] = {c->device, c->gen_fft_cols};
  return SR_OK;
}

// ---- one inner step: psi_out = psi_in + L^{-1} G ---------------------------
// With load_src set, the step solves L out = load_src instead (Eqs. (31)-(33)
// alone).
// div_mode: 0 forms div e in the step, 1 also stores it in divE (first inner
// step of an outer iteration), 2 reads it from divE (later inner steps).
sr_status enqueue_phi_step(sr_ctx* c, cudaStream_t s, const float* psi_in, const float* w1,
                           const float* w2, const float* e1, const float* e2, float* psi_out,
                           const float* load_src, int div_mode = 0) {
  sr_status st;
  const float* src = load_src;
  if (!load_src) {
    srk::PrepArgs pa{};
    pa.geo = c->geo;
    pa.mod = c->mod;
    pa.psi = psi_in;
    pa.g = c->g;
    pa.w1 = w1;
    pa.w2 = w2;
    pa.e1 = e1;
    pa.e2 = e2;
    pa.G = c->G;
    pa.D = div_mode ? c->divE : nullptr;
    pa.D_load = div_mode == 2;
    st = run_kernel(c, SR_KCLASS_PREP, s, "k_prep", [&] { return srk::launch_prep(pa, s); });
    if (st != SR_OK) return st;
    src = c->G;
    if (c->phi_solver == 1) {
      srk::AosArgs aa = c->aos;
      aa.G = c->G;
      aa.psi = psi_in;
      aa.phi = psi_out;
      aa.T1 = c->aos_T1;
      aa.X2 = c->aos_X2;
      // the AOS line solves count as the column pass and the row pass
      c->launches += 1;
      return run_kernel(c, SR_KCLASS_COLSOLVE, s, "k_aos", [&] { return srk::launch_aos(aa, s, false); });
    }
  }
  if (c->geo.neumann) {
    // (1 - tau mu Lap_N) delta = src with the reflective Laplacian: the even
    // extension of each row diagonalises the row direction with the periodic
    // FFT of length 2W (its spectrum is the DCT-II's, rotated), and each
    // column is solved with reflective ends by the recursions on its even
    // extension of length 2M; the first W columns of the result are kept
    st = run_kernel(c, SR_KCLASS_ROWFFT, s, "k_mirror_rows",
                    [&] { return srk::launch_mirror_rows(src, c->G2, c->geo, s); });
    if (st != SR_OK) return st;
    srk::RowFwdArgs na{};
    na.geo = c->geo2;
    na.fft = c->fft_row2;
    na.twN = c->tw_n2;
    na.src = c->G2;
    na.X = c->Xn;
    na.T = c->row2_T;
    st = run_kernel(c, SR_KCLASS_ROWFFT, s, "k_rowfft",
                    [&] { return srk::launch_rowfft2(na, 4, c->row2_threads, s, false); });
    if (st != SR_OK) return st;
    srk::ColArgs nc{};
    nc.geo = c->geo2;
    nc.X = c->Xn;
    nc.Xout = c->Xn2;
    nc.rec = c->rec2;
    nc.rec_R = c->rec2_R;
    nc.mirror = 1;
    st = run_kernel(c, SR_KCLASS_COLSOLVE, s, "k_colsolve_rec",
                    [&] { return srk::launch_colsolve_rec(nc, s); });
    if (st != SR_OK) return st;
    srk::RowInvArgs ni{};
    ni.geo = c->geo2;
    ni.fft = c->fft_row2;
    ni.twN = c->tw_n2;
    ni.X = c->Xn2;
    ni.out = c->G2;
    ni.T = c->row2_T;
    st = run_kernel(c, SR_KCLASS_ROWIFFT, s, "k_rowifft",
                    [&] { return srk::launch_rowifft2(ni, false, 4, c->row2_threads, s, false); });
    if (st != SR_OK) return st;
    return run_kernel(c, SR_KCLASS_ROWIFFT, s, "k_add_half", [&] {
      return srk::launch_add_half(load_src ? nullptr : psi_in, c->G2, psi_out, c->geo, s);
    });
  }
  if (c->fft2 && c->sched.col_schedule == srk::kColSmall) {
    srk::SmallArgs sa{};
    sa.geo = c->geo;
    sa.G = src;
    sa.psi_in = load_src ? nullptr : psi_in;
    sa.out = psi_out;
    sa.tws16 = c->fft_row.tws16;
    sa.twN = c->tw_n;
    sa.rec = c->rec;
    sa.rec_R = c->rec_R;
    return run_kernel(c, SR_KCLASS_COLSOLVE, s, "k_solve_small",
                      [&] { return srk::launch_solve_small(sa, s, false); });
  }
  srk::RowFwdArgs fa{};
  fa.geo = c->geo;
  fa.mod = c->mod;
  fa.fft = c->fft_row;
  fa.twN = c->tw_n;
  fa.src = src;
  fa.X = c->X;
  fa.T = c->fft2 ? sched_rows(c, c->sched) : c->fftgen ? srk::gen_rows_per_cta(c->L, c->H, c->gen_batched) : c->row_T;
  fa.CW = c->row_CW;
  st = run_kernel(c, SR_KCLASS_ROWFFT, s, "k_rowfwd", [&] {
    if (c->fftgen) return srk::launch_rowfft_gen(fa, c->plan_row, c->gen_batched, s);
    return c->fft2 ? srk::launch_rowfft2(fa, c->sched.row_values_per_thread == 8 ? 3 : 4,
                                         c->sched.row_threads, s, false)
                   : srk::launch_rowfwd(fa, srk::kRowLOAD, c->row_NT, s);
  });
  if (st != SR_OK) return st;
  srk::ColArgs ca{};
  ca.geo = c->geo;
  ca.fft = c->fft_col;
  ca.aM = c->aM;
  ca.aN = c->aN;
  ca.X = c->X;
  ca.err = c->err_dev;
  ca.stall_cycles = c->stall_cycles;
  ca.rec = c->rec;
  ca.rec_R = c->rec_R;
  ca.Xout = c->X2;
  // the recursion column pass: chosen by the autotuner for power-of-two sides,
  // always used for other sides (it needs no FFT plan of the column length)
  const bool col_rec = c->rec_R > 0 && ((c->fft2 && c->sched.col_schedule == srk::kColRec) ||
                                        (c->fftgen && !c->gen_fft_cols));
  st = run_kernel(c, SR_KCLASS_COLSOLVE, s, "k_colsolve", [&] {
    if (col_rec) return srk::launch_colsolve_rec(ca, s);
    if (c->fftgen) return srk::launch_colsolve_gen(ca, c->plan_col, c->gen_batched, s);
    if (!c->fft2) return srk::launch_colsolve(ca, s);
    if (col_rec) return srk::launch_colsolve_rec(ca, s);
    if (c->sched.col_schedule == 3)
      return srk::launch_colsolve_tma(ca, c->tm_X, c->col_tma_grid, s, false);
    return srk::launch_colsolve2(ca, c->sched.col_schedule, s, false);
  });
  if (st != SR_OK) return st;
  srk::RowInvArgs ia{};
  ia.geo = c->geo;
  ia.fft = c->fft_row;
  ia.twN = c->tw_n;
  ia.X = col_rec ? c->X2 : c->X;
  ia.psi_in = psi_in;
  ia.out = psi_out;
  ia.T = c->fft2 ? sched_rows(c, c->sched) : c->fftgen ? srk::gen_rows_per_cta(c->L, c->H, c->gen_batched) : c->row_T;
  const int imode = load_src ? srk::kInvSTORE : srk::kInvADD;
  return run_kernel(c, SR_KCLASS_ROWIFFT, s, "k_rowinv", [&] {
    if (c->fftgen)
      return srk::launch_rowifft_gen(ia, c->plan_row, imode == srk::kInvADD, c->gen_batched, s);
    return c->fft2 ? srk::launch_rowifft2(ia, imode == srk::kInvADD,
                                          c->sched.row_values_per_thread == 8 ? 3 : 4,
                                          c->sched.row_threads, s, false)
                   : srk::launch_rowinv(ia, imode, c->row_NT, s);
  });
}

sr_status enqueue_wb(sr_ctx* c, cudaStream_t s, const float* phi1, const float* w1i,
                     const float* w2i, const float* e1i, const float* e2i, float* w1o, float* w2o,
                     float* e1o, float* e2o, const float* phi_old) {
  srk::WBArgs a{};
  a.geo = c->geo;
  a.mod = c->mod;
  a.phi1 = phi1;
  a.g = c->g;
  a.w1 = w1i;
  a.w2 = w2i;
  a.e1 = e1i;
  a.e2 = e2i;
  a.w1o = w1o;
  a.w2o = w2o;
  a.e1o = e1o;
  a.e2o = e2o;
  a.phi_old = phi_old;
  a.partials = c->partials;
  sr_status st = run_kernel(c, SR_KCLASS_WB_UPDATE, s, "k_wb_update",
                            [&] { return srk::launch_wb_update(a, s); });
  if (st != SR_OK || !phi_old) return st;
  return run_kernel(c, SR_KCLASS_REDUCE, s, "k_reduce", [&] {
    return srk::launch_reduce(c->partials, c->n_tile32, 2, c->red, s);
  });
}

// Eqs. (38)-(40) swept `sweeps` times from w^k, then Eq. (23); the sweeps
// alternate between (w1o, w2o) and the context's wfx planes so that the last
// one lands in (w1o, w2o).  (w1o, w2o) must not alias (w1i, w2i).
sr_status enqueue_wb_fixed(sr_ctx* c, cudaStream_t s, const float* phi1, const float* w1i,
                           const float* w2i, const float* e1i, const float* e2i, float* w1o,
                           float* w2o, float* e1o, float* e2o, const float* phi_old, int sweeps) {
  const float* cw1 = w1i;
  const float* cw2 = w2i;
  for (int r = 0; r < sweeps; ++r) {
    const bool last = r == sweeps - 1;
    const bool to_out = (sweeps - 1 - r) % 2 == 0;
    srk::WFixArgs a{};
    a.geo = c->geo;
    a.mod = c->mod;
    a.phi1 = phi1;
    a.wk1 = w1i;
    a.wk2 = w2i;
    a.ek1 = e1i;
    a.ek2 = e2i;
    a.cw1 = cw1;
    a.cw2 = cw2;
    a.nw1 = to_out ? w1o : c->wfx1;
    a.nw2 = to_out ? w2o : c->wfx2;
    a.e1o = last ? e1o : nullptr;
    a.e2o = last ? e2o : nullptr;
    a.phi_old = last ? phi_old : nullptr;
    a.partials = c->partials;
    sr_status st = run_kernel(c, SR_KCLASS_WB_UPDATE, s, "k_wfix_sweep",
                              [&] { return srk::launch_wfix_sweep(a, s); });
    if (st != SR_OK) return st;
    cw1 = a.nw1;
    cw2 = a.nw2;
  }
  if (!phi_old) return SR_OK;
  return run_kernel(c, SR_KCLASS_REDUCE, s, "k_reduce", [&] {
    return srk::launch_reduce(c->partials, c->n_tile32, 2, c->red, s);
  });
}

sr_status alloc_wfix(sr_ctx* c) {
  if (c->wfx1) return SR_OK;
  const size_t P = (size_t)c->H * c->W;
  for (float** pl : {&c->wfx1, &c->wfx2}) {
    const cudaError_t e = dev_alloc((void**)pl, sizeof(float) * P);
    if (e == cudaErrorMemoryAllocation) return fail(c, SR_ENOMEM, "device allocation failed");
    SR_CUDA(c, e);
  }
  return SR_OK;
}

// The w/b update of an outer iteration, by Eqs. (41)-(42) or by sweeps of
// Eqs. (38)-(40).
sr_status enqueue_w_step(sr_ctx* c, cudaStream_t s, int p, bool check) {
  const int q = 1 - p;
  if (c->w_sweeps > 0)
    return enqueue_wb_fixed(c, s, c->phi[q], c->w1[p], c->w2[p], c->e1, c->e2, c->w1[q], c->w2[q],
                            c->e1, c->e2, check ? c->phi[p] : nullptr, c->w_sweeps);
  return enqueue_wb(c, s, c->phi[q], c->w1[p], c->w2[p], c->e1, c->e2, c->w1[q], c->w2[q], c->e1,
                    c->e2, check ? c->phi[p] : nullptr);
}

sr_status read_residual(sr_ctx* c, double* rel);

// One outer iteration with the inner exit of Sec. 4: after each inner step
// the relative change ||psi^{s+1} - psi^s|| / (||psi^s|| + 1e-6) is reduced in
// FP64 and read back; the loop stops once it is <= inner_tol, after at most
// inner_S steps.  Runs eagerly (the step count is data-dependent).
sr_status enqueue_iteration_inner_tol(sr_ctx* c, int p, bool check) {
  const int q = 1 - p;
  const size_t P = (size_t)c->H * c->W;
  const int nblocks = std::max(1, std::min(c->n_tile32, 1024));  // partials hold 2 n_tile32
  for (int it = 0; it < c->prm.inner_S; ++it) {
    const float* in = it == 0 ? c->phi[p] : c->phi[q];
    const float* prev = in;
    if (it > 0) {  // the step overwrites psi in place: keep psi^s
      SR_CUDA(c, cudaMemcpyAsync(c->tmp1, in, sizeof(float) * P, cudaMemcpyDeviceToDevice,
                                 c->stream));
      prev = c->tmp1;
    }
    sr_status st = enqueue_phi_step(c, c->stream, in, c->w1[p], c->w2[p], c->e1, c->e2,
                                    c->phi[q], nullptr, it == 0 ? 1 : 2);
    if (st != SR_OK) return st;
    c->inner_steps += 1;
    c->launches += 2;
    SR_CUDA(c, srk::launch_change_partials(c->phi[q], prev, P, c->partials, nblocks, c->stream));
    SR_CUDA(c, srk::launch_reduce(c->partials, nblocks, 2, c->red, c->stream));
    double rel = 0.0;
    st = read_residual(c, &rel);
    if (st != SR_OK) return st;
    if (rel <= (double)c->prm.inner_tol) break;
  }
  return enqueue_w_step(c, c->stream, p, check);
}

// One outer iteration of Alg. 1 from phi[p], w[p] to phi[1-p], w[1-p].
sr_status enqueue_iteration(sr_ctx* c, cudaStream_t s, int p, bool check) {
  const int q = 1 - p;
  for (int it = 0; it < c->prm.inner_S; ++it) {
    const float* in = it == 0 ? c->phi[p] : c->phi[q];
    sr_status st = enqueue_phi_step(c, s, in, c->w1[p], c->w2[p], c->e1, c->e2, c->phi[q], nullptr,
                                    it == 0 ? 1 : 2);
    if (st != SR_OK) return st;
  }
  return enqueue_w_step(c, s, p, check);
}

void drop_graphs(sr_ctx* c) {
  for (int p = 0; p < 2; ++p)
    if (c->graph[p]) {
      cudaGraphExecDestroy(c->graph[p]);
      c->graph[p] = nullptr;
    }
}

sr_status build_graphs(sr_ctx* c) {
  if (c->graph[0] && c->graph[1]) return SR_OK;
  drop_graphs(c);
  const long long before = c->launches;
  for (int p = 0; p < 2; ++p) {
    cudaGraph_t gph = nullptr;
    SR_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    sr_status st = enqueue_iteration(c, c->cap_stream, p, false);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &gph);
    if (st != SR_OK) {
      if (gph) cudaGraphDestroy(gph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph[p], gph, 0);
    cudaGraphDestroy(gph);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  }
  c->graph_kernels = (int)((c->launches - before) / 2);
  c->launches = before;  // capture enqueues nothing
  return SR_OK;
}

// Device-side bounded waits record timeouts in err_dev; read it at every sync.
sr_status check_device_error(sr_ctx* c) {
  int h = 0;
  SR_CUDA(c, cudaMemcpyAsync(&h, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SR_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h) {
    cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream);
    return fail(c, SR_ETIMEOUT, "a device-side wait for a TMA transfer ran out of time");
  }
  return SR_OK;
}

sr_status read_residual(sr_ctx* c, double* rel) {
  SR_CUDA(c, cudaMemcpyAsync(c->red_host, c->red, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  SR_CUDA(c, cudaStreamSynchronize(c->stream));
  sr_status es = check_device_error(c);
  if (es != SR_OK) return es;
  const double num = c->red_host[0], den = c->red_host[1];
  const double r = std::sqrt(num) / (std::sqrt(den) + 1e-6);
  *rel = r;
  if (!std::isfinite(r)) return fail(c, SR_ENONFINITE, "non-finite value in the stopping test");
  return SR_OK;
}

// the configuration the resident kernel implements
bool resident_base_ok(const sr_ctx* c) {
  return c->fft2 && c->phi_solver == 0 && c->w_sweeps == 0 && c->prm.inner_tol <= 0.f;
}
bool resident_ok(const sr_ctx* c) {
  return resident_base_ok(c) && srk::resident_supported(c->geo, c->mod.R, c->rec_R, c->res_C);
}

// sr_iterate with the state resident in shared memory: one launch runs up to
// max_outer outer iterations with the stopping test of Sec. 4 on the device.
sr_status iterate_resident(sr_ctx* c, int max_outer, double tol, int* outer_done,
                           double* rel_change) {
  srk::ResArgs a{};
  a.members = c->res_dev + c->cur;
  a.max_outer = max_outer;
  a.tol = tol;
  a.check_every = c->prm.check_every;
  a.check_last = rel_change != nullptr;
  sr_status st = run_kernel(c, SR_KCLASS_RESIDENT, c->stream, "k_resident", [&] {
    return srk::launch_resident(a, 1, c->geo, c->res_C, c->res_smem, c->stream, false);
  });
  if (st != SR_OK) return st;
  int done = max_outer;
  double rel = NAN;
  if (tol > 0.0 || rel_change != nullptr) {
    SR_CUDA(c, cudaMemcpyAsync(c->res_done_host, c->res_done, sizeof(int), cudaMemcpyDeviceToHost,
                               c->stream));
    st = read_residual(c, &rel);  // synchronises the stream
    if (st == SR_OK || st == SR_ENONFINITE) done = *c->res_done_host;
  }
  c->cur ^= done & 1;
  c->iters += done;
  c->inner_steps += (long long)done * c->prm.inner_S;
  if (outer_done) *outer_done = done;
  if (rel_change) *rel_change = rel;
  if (st != SR_OK) return st;
  if (c->profile) {
    st = flush_profile(c);
    if (st != SR_OK) return st;
  }
  if (tol > 0.0 && !(rel <= tol)) return SR_ENOTCONVERGED;
  return SR_OK;
}

}  // namespace

// ============================================================================
// C-ABI
// ============================================================================
extern "C" {

const char* sr_status_string(sr_status s) {
  switch (s) {
    case SR_OK: return "ok";
    case SR_EINVAL: return "invalid argument";
    case SR_ENOMEM: return "out of memory";
    case SR_ECUDA: return "CUDA error";
    case SR_ENONFINITE: return "non-finite value";
    case SR_ENOTCONVERGED: return "not converged";
    case SR_ETIMEOUT: return "timeout";
    case SR_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* sr_last_error(const sr_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

sr_status sr_params_default(sr_params* p) {
  if (!p) return SR_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->alpha = 4.f;
  p->beta = 0.2f;
  p->gamma = 4.f;
  p->mu = 8.f;
  p->tau = 0.1f;
  p->eps = 1.f;
  p->band_l = 1.f;
  p->d = 3.f;
  p->win_radius = 3;
  p->inner_S = 3;
  p->inner_tol = 0.f;
  p->rho = 1.f;
  p->sigma = 1.f;
  p->s_pow = 2;
  p->check_every = 10;
  return SR_OK;
}

void sr_destroy(sr_ctx* c) {
  if (!c) return;
  drop_graphs(c);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  void* bufs[] = {c->phi[0], c->phi[1], c->w1[0], c->w1[1], c->w2[0], c->w2[1], c->e1, c->e2,
                  c->g, c->tmp1, c->tmp2, c->stage, c->G, c->divE, c->mask_dev, c->X, c->tw_row, c->tw_col,
                  c->tw_n, c->aM, c->aN, c->partials, c->red, c->err_dev, c->gen_tab,
                  c->tws[0], c->tws[1], c->tws[2], c->tws[3], c->wfx1, c->wfx2,
                  c->X2, c->rec, c->aos_T1, c->aos_X2, c->tw_row2, c->tw_n2,
                  c->tws2[0], c->tws2[1], c->G2, c->Xn, c->Xn2, c->rec2, c->res_dev,
                  c->res_done, c->res_tws4};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->red_host) cudaFreeHost(c->red_host);
  if (c->res_done_host) cudaFreeHost(c->res_done_host);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

sr_status sr_create(int H, int W, const sr_params* p, void* cuda_stream, sr_ctx** out) {
  if (!out || !p) return SR_EINVAL;
  *out = nullptr;
  if (H < 1 || W < 1) return SR_EINVAL;
  std::string why;
  sr_status st = check_params(p, why);
  if (st != SR_OK) return st;
  // powers of two use the register-resident passes; other sides (multiples of
  // 16 whose prime factors are at most 31) the mixed-radix passes
  if (H < 16 || W < 16 || H > 4096 || W > 4096 || H % 16 || W % 16) return SR_EUNSUPPORTED;
  const bool pow2 = is_pow2(H) && is_pow2(W);
  {
    srk::GenPlan tmp;
    std::vector<float2> tab;
    std::vector<int> at(srk::kGenMaxRadix, -1);
    if (!pow2 && (!gen_plan(H, tmp, tab, at) || !gen_plan(W / 2, tmp, tab, at)))
      return SR_EUNSUPPORTED;
  }

  sr_ctx* c = new (std::nothrow) sr_ctx();
  if (!c) return SR_ENOMEM;
  c->H = H;
  c->W = W;
  c->L = W / 2;
  c->prm = *p;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  c->geo.M = H;
  c->geo.N = W;
  c->geo.L = W / 2;
  c->geo.logN = ilog2(W);  // used by the power-of-two paths only

  auto bail = [&](sr_status s) {
    g_create_err = c->err.empty() ? std::string(sr_status_string(s)) : c->err;
    sr_destroy(c);
    return s;
  };
#define CREATE_CUDA(call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) {                               \
      if (e_ == cudaErrorMemoryAllocation) return bail(SR_ENOMEM); \
      return bail(SR_ECUDA);                               \
    }                                                      \
  } while (0)

  CREATE_CUDA(cudaGetDevice(&c->device));
  CREATE_CUDA(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
  CREATE_CUDA(srk::configure_kernels());
  CREATE_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));

  // model constants
  Model& m = c->mod;
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

  // row-pass shape of the fixed small-size passes (powers of two): T rows per
  // CTA with T * (W/2) = 16 * threads
  const int L = c->L;
  if (pow2) {
    int NT = 0, T = 0;
    if (!srk::row_shape(H, L, c->nsm, &NT, &T)) return bail(SR_EUNSUPPORTED);
    c->row_T = T;
    c->row_NT = NT;
  }
  c->row_CW = W < 128 ? W : 128;
  c->n_tile = srk::tile_blocks(c->geo);
  c->n_tile32 = srk::tile32_blocks(c->geo);

  const size_t P = (size_t)H * W;
  float** planes[] = {&c->phi[0], &c->phi[1], &c->w1[0], &c->w1[1], &c->w2[0], &c->w2[1],
                      &c->e1,     &c->e2,     &c->g,     &c->tmp1,  &c->tmp2,  &c->stage,
                      &c->G,      &c->divE};
  for (float** pl : planes) CREATE_CUDA(dev_alloc((void**)pl, P * sizeof(float)));
  CREATE_CUDA(dev_alloc((void**)&c->mask_dev, P));
  CREATE_CUDA(dev_alloc((void**)&c->X, (size_t)H * L * sizeof(float2)));
  CREATE_CUDA(dev_alloc((void**)&c->partials, (size_t)c->n_tile * 3 * sizeof(double)));
  CREATE_CUDA(dev_alloc((void**)&c->red, 4 * sizeof(double)));
  CREATE_CUDA(host_alloc((void**)&c->red_host, 4 * sizeof(double)));
  for (float** pl : planes) CREATE_CUDA(cudaMemset(*pl, 0, P * sizeof(float)));

  // tables: FFT twiddles, the post/pre-processing twiddles of the real row
  // transform, and the two halves of the symbol of Eq. (32)
  if ((st = upload(c, &c->tw_row, twiddles(L, L))) != SR_OK) return bail(st);
  if ((st = upload(c, &c->tw_col, twiddles(H, H))) != SR_OK) return bail(st);
  if ((st = upload(c, &c->tw_n, twiddles(L, W))) != SR_OK) return bail(st);
  std::vector<float> aM(H), aN(L + 1);
  const double tm = (double)p->tau * (double)p->mu;
  for (int l = 0; l < H; ++l) {
    const double s = std::sin(M_PI * (double)l / (double)H);
    aM[l] = (float)(tm * 4.0 * s * s);
  }
  for (int k = 0; k <= L; ++k) {
    const double s = std::sin(M_PI * (double)k / (double)W);
    aN[k] = (float)(tm * 4.0 * s * s);
  }
  if ((st = upload(c, &c->aM, aM)) != SR_OK) return bail(st);
  if ((st = upload(c, &c->aN, aN)) != SR_OK) return bail(st);
  make_fft(c->fft_row, L, c->tw_row);
  make_fft(c->fft_col, H, c->tw_col);
  if (pow2) {
    const int lens[4] = {L, L, H, H}, loges[4] = {4, 3, 4, 3};
    for (int q = 0; q < 4; ++q) {
      std::vector<float2> tb = stage_twiddle_table(lens[q], loges[q]);
      const int want = srk::stage_twiddles(lens[q], loges[q]);
      if (want > 0 && (int)tb.size() != want) return bail(SR_ECUDA);
      if ((st = upload(c, &c->tws[q], tb)) != SR_OK) return bail(st);
    }
    c->fft_row.tws16 = c->tws[0];
    c->fft_row.tws8 = c->tws[1];
    c->fft_col.tws16 = c->tws[2];
    c->fft_col.tws8 = c->tws[3];
  }
  {
    // the recursion column pass (schedule 7): per column the root r in (0, 1)
    // of tau mu r^2 - c r + tau mu = 0, c = 1 + 2 tau mu + tau mu 4 sin^2(pi k / W),
    // and s = r / (tau mu W); column 0 carries k = 0 and k = W / 2
    const double a = tm;
    std::vector<double> rk(L + 1), sk(L + 1);
    for (int k = 0; k <= L; ++k) {
      const double sn = std::sin(M_PI * (double)k / (double)W);
      const double cc = 1.0 + 2.0 * a + a * 4.0 * sn * sn;
      rk[k] = 2.0 * a / (cc + std::sqrt(cc * cc - 4.0 * a * a));
      sk[k] = rk[k] / (a * (double)W);
    }
    c->rec_R = srk::colsolve_rec_radius(rk[0]);
    if (c->rec_R > 0) {
      std::vector<float4> tab(L);
      for (int k = 0; k < L; ++k)
        tab[k] = make_float4((float)rk[k], (float)sk[k], (float)rk[k == 0 ? L : k],
                             (float)sk[k == 0 ? L : k]);
      if ((st = upload(c, &c->rec, tab)) != SR_OK) return bail(st);
      CREATE_CUDA(dev_alloc((void**)&c->X2, (size_t)H * L * sizeof(float2)));
    }
  }
  {
    // AOS constants: k = 2 tau mu, r the root in (0, 1) of k r^2 - (1 + 2k) r + k = 0
    const double k = 2.0 * tm, cc = 1.0 + 2.0 * k;
    const double r = 2.0 * k / (cc + std::sqrt(cc * cc - 4.0 * k * k));
    c->aos.geo = c->geo;
    c->aos.k = (float)k;
    c->aos.tm = (float)tm;
    c->aos.r = (float)r;
    c->aos.s = (float)(r / k);
    c->aos.R = srk::aos_radius(r);
    c->aos.warm_blocks = (c->aos.R + 31) / 32 + 1;
    double pw = 1.0;
    for (int m = 0; m <= 32; ++m) {
      c->aos.pw[m] = (float)pw;
      pw *= r;
    }
  }
  CREATE_CUDA(dev_alloc((void**)&c->err_dev, sizeof(int)));
  CREATE_CUDA(cudaMemset(c->err_dev, 0, sizeof(int)));
  c->fft2 = pow2 && srk::fft2_supported(c->geo);
  if (!pow2) {
    std::vector<float2> tab;
    std::vector<int> at(srk::kGenMaxRadix, -1);
    gen_plan(W / 2, c->plan_row, tab, at);
    gen_plan(H, c->plan_col, tab, at);
    if ((st = upload(c, &c->gen_tab, tab)) != SR_OK) return bail(st);
    c->plan_row.tw = c->plan_row.roots = c->gen_tab;
    c->plan_col.tw = c->plan_col.roots = c->gen_tab;
    CREATE_CUDA(srk::configure_fftgen());
    c->fftgen = true;
    if (autotune_gen(c) != SR_OK) return bail(SR_ECUDA);
  }
  if (c->fft2) {
    const int cb = srk::colsolve_tma_cb(H);
    c->tm_X_ok = make_tensor_map_2d(&c->tm_X, c->X, H, W, W, 2 * cb, H < 256 ? H : 256);
    if (autotune(c) != SR_OK) return bail(SR_ECUDA);
  }

  // g = 1 until sr_edge_function is called
  std::vector<float> ones(P, 1.f);
  CREATE_CUDA(cudaMemcpy(c->g, ones.data(), P * sizeof(float), cudaMemcpyHostToDevice));
  CREATE_CUDA(cudaDeviceSynchronize());
#undef CREATE_CUDA
  *out = c;
  return SR_OK;
}

sr_status sr_edge_function(sr_ctx* c, const float* image, int ld) {
  if (!c) return SR_EINVAL;
  if (!image || ld < c->W) return fail(c, SR_EINVAL, "image must be non-NULL with ld >= W");
  srk::EdgeArgs a{};
  a.geo = c->geo;
  const double sigma = c->prm.sigma;
  a.r = sigma > 0.0 ? (int)std::ceil(3.0 * sigma) : 0;
  std::vector<double> k(2 * a.r + 1);
  double sum = 0.0;
  for (int t = -a.r; t <= a.r; ++t) {
    k[t + a.r] = sigma > 0.0 ? std::exp(-(double)(t * t) / (2.0 * sigma * sigma)) : 1.0;
    sum += k[t + a.r];
  }
  for (int t = 0; t <= 2 * a.r; ++t) a.k[t] = (float)(k[t] / sum);
  a.rho = c->prm.rho;
  a.s_pow = c->prm.s_pow;
  c->launches += 3;
  SR_CUDA(c, srk::launch_edge(a, image, ld, c->tmp1, c->tmp2, c->g, c->stream));
  return SR_OK;
}

sr_status sr_set_phi(sr_ctx* c, const float* phi0, int ld) {
  if (!c) return SR_EINVAL;
  if (!phi0 || ld < c->W) return fail(c, SR_EINVAL, "phi0 must be non-NULL with ld >= W");
  c->cur = 0;
  c->iters = 0;
  SR_CUDA(c, cudaMemcpy2DAsync(c->phi[0], c->W * sizeof(float), phi0, (size_t)ld * sizeof(float),
                               c->W * sizeof(float), c->H, cudaMemcpyDeviceToDevice, c->stream));
  c->launches += 1;
  SR_CUDA(c, srk::launch_init_wb(c->phi[0], c->w1[0], c->w2[0], c->e1, c->e2, c->geo, c->stream));
  return SR_OK;
}

sr_status sr_iterate(sr_ctx* c, int max_outer, double tol, int* outer_done, double* rel_change) {
  if (!c) return SR_EINVAL;
  if (outer_done) *outer_done = 0;
  if (max_outer < 0 || !std::isfinite(tol)) return fail(c, SR_EINVAL, "bad max_outer or tol");
  if (max_outer == 0) return SR_OK;
  if (c->resident && resident_ok(c)) return iterate_resident(c, max_outer, tol, outer_done, rel_change);
  const bool inner_exit = c->prm.inner_tol > 0.f;
  const bool use_graph = !c->profile && !inner_exit;
  if (use_graph) {
    sr_status st = build_graphs(c);
    if (st != SR_OK) return st;
  }
  double rel = NAN;
  int done = 0;
  for (int k = 0; k < max_outer; ++k) {
    const bool last = k == max_outer - 1;
    const bool check = tol > 0.0 ? ((k + 1) % c->prm.check_every == 0 || last)
                                 : (last && rel_change != nullptr);
    sr_status st;
    if (!check && use_graph) {
      cudaError_t e = cudaGraphLaunch(c->graph[c->cur], c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
      c->launches += c->graph_kernels;
      st = SR_OK;
    } else if (inner_exit) {
      st = enqueue_iteration_inner_tol(c, c->cur, check);
    } else {
      st = enqueue_iteration(c, c->stream, c->cur, check);
    }
    if (st != SR_OK) return st;
    if (!inner_exit) c->inner_steps += c->prm.inner_S;
    c->cur ^= 1;
    c->iters += 1;
    done = k + 1;
    if (check) {
      st = read_residual(c, &rel);
      if (rel_change) *rel_change = rel;
      if (outer_done) *outer_done = done;
      if (st != SR_OK) return st;
      if (tol > 0.0 && rel <= tol) break;
    }
  }
  if (outer_done) *outer_done = done;
  if (rel_change) *rel_change = rel;
  if (c->profile) {
    sr_status st = flush_profile(c);
    if (st != SR_OK) return st;
  }
  if (tol > 0.0 && !(rel <= tol)) return SR_ENOTCONVERGED;
  return SR_OK;
}

sr_status sr_mask(sr_ctx* c, unsigned char* mask, int ld) {
  if (!c) return SR_EINVAL;
  if (!mask || ld < c->W) return fail(c, SR_EINVAL, "mask must be non-NULL with ld >= W");
  c->launches += 1;
  SR_CUDA(c, srk::launch_mask(c->phi[c->cur], mask, ld, c->geo, c->stream));
  return SR_OK;
}

sr_status sr_get_phi(sr_ctx* c, float* phi, int ld) {
  if (!c) return SR_EINVAL;
  if (!phi || ld < c->W) return fail(c, SR_EINVAL, "phi must be non-NULL with ld >= W");
  SR_CUDA(c, cudaMemcpy2DAsync(phi, (size_t)ld * sizeof(float), c->phi[c->cur],
                               c->W * sizeof(float), c->W * sizeof(float), c->H,
                               cudaMemcpyDeviceToDevice, c->stream));
  return SR_OK;
}

sr_status sr_get_state(sr_ctx* c, float* phi, float* w1, float* w2, float* b1, float* b2) {
  if (!c) return SR_EINVAL;
  if (!phi || !w1 || !w2 || !b1 || !b2) return fail(c, SR_EINVAL, "NULL state pointer");
  const size_t P = (size_t)c->H * c->W;
  const size_t bytes = P * sizeof(float);
  const float* src[] = {c->phi[c->cur], c->w1[c->cur], c->w2[c->cur]};
  float* dst[] = {phi, w1, w2};
  for (int t = 0; t < 3; ++t)
    SR_CUDA(c, cudaMemcpyAsync(dst[t], src[t], bytes, cudaMemcpyDeviceToDevice, c->stream));
  // b = e + w
  c->launches += 2;
  SR_CUDA(c, srk::launch_axpb(c->e1, c->w1[c->cur], 1.f, b1, P, c->stream));
  SR_CUDA(c, srk::launch_axpb(c->e2, c->w2[c->cur], 1.f, b2, P, c->stream));
  return SR_OK;
}

sr_status sr_set_state(sr_ctx* c, const float* phi, const float* w1, const float* w2,
                       const float* b1, const float* b2) {
  if (!c) return SR_EINVAL;
  if (!phi || !w1 || !w2 || !b1 || !b2) return fail(c, SR_EINVAL, "NULL state pointer");
  const size_t P = (size_t)c->H * c->W;
  const size_t bytes = P * sizeof(float);
  c->cur = 0;
  const float* src[] = {phi, w1, w2};
  float* dst[] = {c->phi[0], c->w1[0], c->w2[0]};
  for (int t = 0; t < 3; ++t)
    SR_CUDA(c, cudaMemcpyAsync(dst[t], src[t], bytes, cudaMemcpyDeviceToDevice, c->stream));
  // e = b - w
  c->launches += 2;
  SR_CUDA(c, srk::launch_axpb(b1, c->w1[0], -1.f, c->e1, P, c->stream));
  SR_CUDA(c, srk::launch_axpb(b2, c->w2[0], -1.f, c->e2, P, c->stream));
  return SR_OK;
}

sr_status sr_get_g(sr_ctx* c, float* g) {
  if (!c) return SR_EINVAL;
  if (!g) return fail(c, SR_EINVAL, "NULL g");
  SR_CUDA(c, cudaMemcpyAsync(g, c->g, (size_t)c->H * c->W * sizeof(float),
                             cudaMemcpyDeviceToDevice, c->stream));
  return SR_OK;
}

sr_status sr_set_g(sr_ctx* c, const float* g) {
  if (!c) return SR_EINVAL;
  if (!g) return fail(c, SR_EINVAL, "NULL g");
  SR_CUDA(c, cudaMemcpyAsync(c->g, g, (size_t)c->H * c->W * sizeof(float),
                             cudaMemcpyDeviceToDevice, c->stream));
  return SR_OK;
}

sr_status sr_energy(sr_ctx* c, double* E, double* Eg, double* Ea, double* Er) {
  if (!c) return SR_EINVAL;
  srk::EnergyArgs a{};
  a.geo = c->geo;
  a.mod = c->mod;
  a.phi = c->phi[c->cur];
  a.g = c->g;
  a.partials = c->partials;
  c->launches += 2;
  SR_CUDA(c, srk::launch_energy(a, c->stream));
  SR_CUDA(c, srk::launch_reduce(c->partials, c->n_tile, 3, c->red, c->stream));
  SR_CUDA(c, cudaMemcpyAsync(c->red_host, c->red, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  SR_CUDA(c, cudaStreamSynchronize(c->stream));
  const double eg = c->red_host[0], ea = c->red_host[1], er = c->red_host[2];
  if (Eg) *Eg = eg;
  if (Ea) *Ea = ea;
  if (Er) *Er = er;
  const double e = (double)c->prm.gamma * eg + (double)c->prm.alpha * ea + (double)c->prm.beta * er;
  if (E) *E = e;
  if (!std::isfinite(e)) return fail(c, SR_ENONFINITE, "non-finite energy");
  return SR_OK;
}

sr_status sr_repulsion_field(sr_ctx* c, const float* phi, const float* w1, const float* w2,
                             float* v1, float* v2) {
  if (!c) return SR_EINVAL;
  if (!phi || !w1 || !w2 || !v1 || !v2) return fail(c, SR_EINVAL, "NULL pointer");
  srk::RepArgs a{};
  a.geo = c->geo;
  a.mod = c->mod;
  a.phi = phi;
  a.w1 = w1;
  a.w2 = w2;
  a.v1 = v1;
  a.v2 = v2;
  c->launches += 1;
  SR_CUDA(c, srk::launch_repulsion(a, c->stream));
  return SR_OK;
}

sr_status sr_phi_step(sr_ctx* c, const float* psi_in, const float* w1, const float* w2,
                      const float* b1, const float* b2, float* psi_out) {
  if (!c) return SR_EINVAL;
  if (!psi_in || !w1 || !w2 || !b1 || !b2 || !psi_out)
    return fail(c, SR_EINVAL, "NULL pointer");
  for (const void* ptr : {(const void*)psi_in, (const void*)w1, (const void*)w2, (const void*)b1,
                          (const void*)b2, (const void*)psi_out})
    if (!aligned16(ptr)) return fail(c, SR_EINVAL, "buffers must be 16-byte aligned");
  const size_t P = (size_t)c->H * c->W;
  c->launches += 2;
  SR_CUDA(c, srk::launch_axpb(b1, w1, -1.f, c->tmp1, P, c->stream));  // e = b - w
  SR_CUDA(c, srk::launch_axpb(b2, w2, -1.f, c->tmp2, P, c->stream));
  return enqueue_phi_step(c, c->stream, psi_in, w1, w2, c->tmp1, c->tmp2, psi_out, nullptr);
}

sr_status sr_fft_solve(sr_ctx* c, const float* rhs, float* out) {
  if (!c) return SR_EINVAL;
  if (!rhs || !out) return fail(c, SR_EINVAL, "NULL pointer");
  if (!aligned16(out)) return fail(c, SR_EINVAL, "out must be 16-byte aligned");
  return enqueue_phi_step(c, c->stream, nullptr, nullptr, nullptr, nullptr, nullptr, out, rhs);
}

sr_status sr_w_b_update(sr_ctx* c, const float* phi1, const float* w1_in, const float* w2_in,
                        const float* b1_in, const float* b2_in, float* w1_out, float* w2_out,
                        float* b1_out, float* b2_out) {
  if (!c) return SR_EINVAL;
  if (!phi1 || !w1_in || !w2_in || !b1_in || !b2_in || !w1_out || !w2_out || !b1_out || !b2_out)
    return fail(c, SR_EINVAL, "NULL pointer");
  if (w1_out == w1_in || w2_out == w2_in || w1_out == w2_in || w2_out == w1_in)
    return fail(c, SR_EINVAL, "w_out must not alias w_in");
  for (const void* ptr : {(const void*)phi1, (const void*)w1_in, (const void*)w2_in,
                          (const void*)b1_in, (const void*)b2_in, (const void*)w1_out,
                          (const void*)w2_out, (const void*)b1_out, (const void*)b2_out})
    if (!aligned16(ptr)) return fail(c, SR_EINVAL, "buffers must be 16-byte aligned");
  const size_t P = (size_t)c->H * c->W;
  c->launches += 4;
  SR_CUDA(c, srk::launch_axpb(b1_in, w1_in, -1.f, c->tmp1, P, c->stream));  // e = b - w
  SR_CUDA(c, srk::launch_axpb(b2_in, w2_in, -1.f, c->tmp2, P, c->stream));
  sr_status st = enqueue_wb(c, c->stream, phi1, w1_in, w2_in, c->tmp1, c->tmp2, w1_out, w2_out,
                            c->tmp1, c->tmp2, nullptr);
  if (st != SR_OK) return st;
  SR_CUDA(c, srk::launch_axpb(c->tmp1, w1_out, 1.f, b1_out, P, c->stream));  // b = e + w
  SR_CUDA(c, srk::launch_axpb(c->tmp2, w2_out, 1.f, b2_out, P, c->stream));
  return SR_OK;
}

sr_status sr_w_b_fixed_point(sr_ctx* c, const float* phi1, const float* w1_in, const float* w2_in,
                             const float* b1_in, const float* b2_in, int sweeps, float* w1_out,
                             float* w2_out, float* b1_out, float* b2_out) {
  if (!c) return SR_EINVAL;
  if (sweeps < 1 || sweeps > 64) return fail(c, SR_EINVAL, "sweeps must be in [1, 64]");
  if (!phi1 || !w1_in || !w2_in || !b1_in || !b2_in || !w1_out || !w2_out || !b1_out || !b2_out)
    return fail(c, SR_EINVAL, "NULL pointer");
  if (w1_out == w1_in || w2_out == w2_in || w1_out == w2_in || w2_out == w1_in)
    return fail(c, SR_EINVAL, "w_out must not alias w_in");
  sr_status st = alloc_wfix(c);
  if (st != SR_OK) return st;
  const size_t P = (size_t)c->H * c->W;
  c->launches += 4;
  SR_CUDA(c, srk::launch_axpb(b1_in, w1_in, -1.f, c->tmp1, P, c->stream));  // e = b - w
  SR_CUDA(c, srk::launch_axpb(b2_in, w2_in, -1.f, c->tmp2, P, c->stream));
  st = enqueue_wb_fixed(c, c->stream, phi1, w1_in, w2_in, c->tmp1, c->tmp2, w1_out, w2_out,
                        c->tmp1, c->tmp2, nullptr, sweeps);
  if (st != SR_OK) return st;
  SR_CUDA(c, srk::launch_axpb(c->tmp1, w1_out, 1.f, b1_out, P, c->stream));  // b = e + w
  SR_CUDA(c, srk::launch_axpb(c->tmp2, w2_out, 1.f, b2_out, P, c->stream));
  return SR_OK;
}

long long sr_inner_steps(sr_ctx* c, int reset) {
  if (!c) return -1;
  const long long v = c->inner_steps;
  if (reset) c->inner_steps = 0;
  return v;
}

sr_status sr_set_w_sweeps(sr_ctx* c, int sweeps) {
  if (!c) return SR_EINVAL;
  if (sweeps < 0 || sweeps > 64) return fail(c, SR_EINVAL, "sweeps must be in [0, 64]");
  if (sweeps > 0 && c->geo.neumann)
    return fail(c, SR_EUNSUPPORTED, "the iterated w variant is built for the periodic reading");
  if (sweeps > 0) {
    sr_status st = alloc_wfix(c);
    if (st != SR_OK) return st;
  }
  if (sweeps != c->w_sweeps) {
    c->w_sweeps = sweeps;
    drop_graphs(c);
  }
  return SR_OK;
}

sr_status sr_get_schedule(sr_ctx* c, sr_schedule* out) {
  if (!c || !out) return SR_EINVAL;
  if (c->fft2) {
    *out = c->sched;
  } else {
    *out = sr_schedule{16, 0, 0, 0.f};
  }
  return SR_OK;
}

sr_status sr_set_schedule(sr_ctx* c, const sr_schedule* sc) {
  if (!c || !sc) return SR_EINVAL;
  if (!c->fft2) return fail(c, SR_EUNSUPPORTED, "this size uses fixed FFT kernels");
  if (!sched_valid(c, *sc)) return fail(c, SR_EINVAL, "invalid FFT schedule for this size");
  SR_CUDA(c, sched_configure(c, *sc));
  c->sched = *sc;
  c->sched.tuned_us = 0.f;
  drop_graphs(c);
  return SR_OK;
}

long long sr_kernel_launches(const sr_ctx* c, int reset) {
  if (!c) return 0;
  const long long n = c->launches;
  if (reset) const_cast<sr_ctx*>(c)->launches = 0;
  return n;
}

sr_status sr_set_resident(sr_ctx* c, int on) {
  if (!c || !(on == 0 || on == 1 || on == 8 || on == 16)) return SR_EINVAL;
  if (!on) {
    c->resident = 0;
    return SR_OK;
  }
  const char* why =
      "resident iterations need W in {32, 64, 128, 256}, H a multiple of 8 (>= 16), the state "
      "within one cluster's shared memory, the periodic FFT solve with the column recursions "
      "and Eqs. (41)-(42)";
  if (!resident_base_ok(c)) return fail(c, SR_EUNSUPPORTED, why);
  // clusters of 16 CTAs where the rows divide and the device schedules them,
  // else 8; SR_RESIDENT_CLUSTER=8 or 16 fixes the choice
  std::vector<int> cands = {16, 8};
  if (on == 8 || on == 16) {
    cands = {on};
  } else if (const char* env = std::getenv("SR_RESIDENT_CLUSTER")) {
    const int v = std::atoi(env);
    if (v == 8 || v == 16) cands = {v};
  }
  int C = 0;
  size_t smem = 0;
  for (int cand : cands) {
    if (!srk::resident_supported(c->geo, c->mod.R, c->rec_R, cand)) continue;
    const size_t sm_c = srk::resident_smem(c->geo, c->mod.R, c->rec_R, cand);
    srk::ResArgs probe{};
    const cudaError_t pe = srk::launch_resident(probe, 1, c->geo, cand, sm_c, nullptr, true);
    if (pe == cudaErrorNotSupported) continue;
    SR_CUDA(c, pe);
    C = cand;
    smem = sm_c;
    break;
  }
  if (!C) return fail(c, SR_EUNSUPPORTED, why);
  if (!c->res_dev) {
    cudaError_t e = dev_alloc((void**)&c->res_dev, 2 * sizeof(srk::ResMember));
    if (e == cudaSuccess) e = dev_alloc((void**)&c->res_done, sizeof(int));
    if (e == cudaSuccess) e = host_alloc((void**)&c->res_done_host, sizeof(int));
    if (e == cudaErrorMemoryAllocation) return fail(c, SR_ENOMEM, "allocation failed");
    SR_CUDA(c, e);
  }
  if (!c->res_tws4) {
    const sr_status st = upload(c, &c->res_tws4, stage_twiddle_table(c->L, 2));
    if (st != SR_OK) return st;
  }
  srk::ResMember mb[2];
  for (int p = 0; p < 2; ++p) {
    srk::ResMember& r = mb[p];
    r = srk::ResMember{};
    r.geo = c->geo;
    r.mod = c->mod;
    r.inner_S = c->prm.inner_S;
    r.rec_R = c->rec_R;
    r.cur = p;
    r.g = c->g;
    for (int q = 0; q < 2; ++q) {
      r.phi[q] = c->phi[q];
      r.w1[q] = c->w1[q];
      r.w2[q] = c->w2[q];
    }
    r.e1 = c->e1;
    r.e2 = c->e2;
    r.tws4 = c->res_tws4;
    r.twN = c->tw_n;
    r.rec = c->rec;
    r.done = c->res_done;
    r.red = c->red;
  }
  SR_CUDA(c, cudaMemcpy(c->res_dev, mb, sizeof(mb), cudaMemcpyHostToDevice));
  c->res_smem = smem;
  c->res_C = C;
  c->resident = 1;
  return SR_OK;
}

sr_status sr_set_phi_solver(sr_ctx* c, int solver) {
  if (!c || solver < 0 || solver > 1) return SR_EINVAL;
  if (solver == 1 && c->geo.neumann)
    return fail(c, SR_EUNSUPPORTED, "the AOS solve is built for the periodic reading");
  if (solver == 1) {
    if (c->aos.R <= 0)
      return fail(c, SR_EUNSUPPORTED, "2 tau mu too large for the AOS recursions' warm-up");
    for (float** pl : {&c->aos_T1, &c->aos_X2}) {
      if (*pl) continue;
      const cudaError_t e = dev_alloc((void**)pl, sizeof(float) * (size_t)c->H * c->W);
      if (e == cudaErrorMemoryAllocation) return fail(c, SR_ENOMEM, "device allocation failed");
      SR_CUDA(c, e);
    }
    SR_CUDA(c, srk::launch_aos(c->aos, nullptr, true));
  }
  c->phi_solver = solver;
  drop_graphs(c);
  return SR_OK;
}

sr_status sr_set_boundary(sr_ctx* c, int neumann) {
  if (!c || neumann < 0 || neumann > 1) return SR_EINVAL;
  if (neumann && (!is_pow2(c->H) || !is_pow2(c->W) || c->W > 2048))
    return fail(c, SR_EUNSUPPORTED, "the Neumann solve needs power-of-two sides with W <= 2048");
  if (neumann && (c->phi_solver != 0 || c->w_sweeps != 0))
    return fail(c, SR_EUNSUPPORTED, "the Neumann reading is built for the FFT solve and Eqs. (41)-(42)");
  if (neumann && !c->G2) {
    const int H = c->H, W = c->W;
    const double a = (double)c->prm.tau * (double)c->prm.mu;
    c->geo2 = srk::Geo{H, 2 * W, W, ilog2(2 * W), 0};
    sr_status st;
    if ((st = upload(c, &c->tw_row2, twiddles(W, W))) != SR_OK) return st;
    if ((st = upload(c, &c->tw_n2, twiddles(W, 2 * W))) != SR_OK) return st;
    const int loges[2] = {4, 3};
    for (int q = 0; q < 2; ++q) {
      std::vector<float2> tb = stage_twiddle_table(W, loges[q]);
      if ((st = upload(c, &c->tws2[q], tb)) != SR_OK) return st;
    }
    make_fft(c->fft_row2, W, c->tw_row2);
    c->fft_row2.tws16 = c->tws2[0];
    c->fft_row2.tws8 = c->tws2[1];
    // column k of the extended rows' half spectrum holds DCT index k (and the
    // packed column 0 holds W in its imaginary part): c = 1 + 2a + a 4 sin^2(pi k / (2W))
    std::vector<double> rk(W + 1), sk(W + 1);
    for (int k = 0; k <= W; ++k) {
      const double sn = std::sin(M_PI * (double)k / (2.0 * (double)W));
      const double cc = 1.0 + 2.0 * a + a * 4.0 * sn * sn;
      rk[k] = 2.0 * a / (cc + std::sqrt(cc * cc - 4.0 * a * a));
      sk[k] = rk[k] / (a * 2.0 * (double)W);
    }
    c->rec2_R = srk::colsolve_rec_radius(rk[0]);
    if (c->rec2_R <= 0) return fail(c, SR_EUNSUPPORTED, "tau mu too large for the recursions' warm-up");
    std::vector<float4> tab(W);
    for (int k = 0; k < W; ++k)
      tab[k] = make_float4((float)rk[k], (float)sk[k], (float)rk[k == 0 ? W : k],
                           (float)sk[k == 0 ? W : k]);
    if ((st = upload(c, &c->rec2, tab)) != SR_OK) return st;
    const size_t P = (size_t)H * W;
    for (void** pl : {(void**)&c->G2, (void**)&c->Xn, (void**)&c->Xn2}) {
      const cudaError_t e = dev_alloc(pl, 2 * P * sizeof(float));
      if (e == cudaErrorMemoryAllocation) return fail(c, SR_ENOMEM, "device allocation failed");
      SR_CUDA(c, e);
    }
    // row passes of length W: 16 values per thread, about 2048 values per CTA
    c->row2_T = std::max(1, std::min(H, 2048 / W));
    c->row2_threads = c->row2_T * W / 16;
    srk::RowFwdArgs fa{};
    fa.geo = c->geo2;
    fa.T = c->row2_T;
    srk::RowInvArgs ia{};
    ia.geo = c->geo2;
    ia.T = c->row2_T;
    SR_CUDA(c, srk::launch_rowfft2(fa, 4, c->row2_threads, nullptr, true));
    SR_CUDA(c, srk::launch_rowifft2(ia, false, 4, c->row2_threads, nullptr, true));
  }
  c->geo.neumann = neumann;
  drop_graphs(c);
  return SR_OK;
}

sr_status sr_aos_solve(sr_ctx* c, const float* rhs, float* out) {
  if (!c) return SR_EINVAL;
  if (!rhs || !out) return fail(c, SR_EINVAL, "NULL buffer");
  if (rhs == out) return fail(c, SR_EINVAL, "rhs and out must not alias");
  if (c->aos.R <= 0)
    return fail(c, SR_EUNSUPPORTED, "2 tau mu too large for the AOS recursions' warm-up");
  if (c->phi_solver != 1) {  // allocates the scratch plane and sets the kernel attributes
    const int keep = c->phi_solver;
    sr_status st = sr_set_phi_solver(c, 1);
    if (st != SR_OK) return st;
    c->phi_solver = keep;
  }
  srk::AosArgs aa = c->aos;
  aa.G = rhs;
  aa.psi = nullptr;
  aa.phi = out;
  aa.T1 = c->aos_T1;
  aa.X2 = c->aos_X2;
  c->launches += 2;
  SR_CUDA(c, srk::launch_aos(aa, c->stream, false));
  return SR_OK;
}

sr_status sr_test_stall_waits(sr_ctx* c, long long cycles) {
  if (!c || cycles < 0) return SR_EINVAL;
  c->stall_cycles = cycles;
  drop_graphs(c);  // the graphs hold the column pass's arguments by value
  return SR_OK;
}

sr_status sr_test_fail_allocations(long long n) {
  g_alloc_budget.store(n < 0 ? -1 : n);
  return SR_OK;
}

sr_status sr_profile_enable(sr_ctx* c, int enable) {
  if (!c) return SR_EINVAL;
  c->profile = enable != 0;
  return SR_OK;
}

sr_status sr_profile_overhead(sr_ctx* c, double* us) {
  if (!c || !us) return SR_EINVAL;
  // the event pair of run_kernel around an empty kernel, 65 times: the median
  const int reps = 65;
  std::vector<cudaEvent_t> ev(2 * reps, nullptr);
  for (auto& e : ev) SR_CUDA(c, cudaEventCreate(&e));
  cudaError_t err = cudaSuccess;
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    err = cudaEventRecord(ev[2 * r], c->stream);
    if (err == cudaSuccess) err = srk::launch_empty(c->stream);
    if (err == cudaSuccess) err = cudaEventRecord(ev[2 * r + 1], c->stream);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
  std::vector<float> ms(reps, 0.f);
  for (int r = 0; r < reps && err == cudaSuccess; ++r)
    err = cudaEventElapsedTime(&ms[r], ev[2 * r], ev[2 * r + 1]);
  for (auto& e : ev) cudaEventDestroy(e);
  if (err != cudaSuccess) return cuda_fail(c, err, "profiling overhead");
  std::nth_element(ms.begin(), ms.begin() + reps / 2, ms.end());
  *us = 1000.0 * ms[reps / 2];
  return SR_OK;
}

sr_status sr_kernel_times(sr_ctx* c, int kclass, double* total_ms, long long* launches) {
  if (!c) return SR_EINVAL;
  if (kclass < 0 || kclass >= SR_KCLASS_COUNT) return fail(c, SR_EINVAL, "bad kernel class");
  sr_status st = flush_profile(c);
  if (st != SR_OK) return st;
  if (total_ms) *total_ms = c->ktime[kclass];
  if (launches) *launches = c->kcount[kclass];
  c->ktime[kclass] = 0.0;
  c->kcount[kclass] = 0;
  return SR_OK;
}

// ---- groups: many contexts iterated by one graph with concurrent branches ----
}  // extern "C"

struct sr_group {
  std::vector<sr_ctx*> m;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // per parity
  int device = 0;
  // sr_group_run: one graph of per-member while-loops, built for a step and
  // a starting parity; per-member loop state in device memory
  cudaGraphExec_t run_graph = nullptr;
  int run_step = 0, run_parity = -1;
  srk::LoopState* loop = nullptr;     // device, one per member
  srk::LoopState* loop_host = nullptr;  // pinned copy
  int lanes = 32;  // concurrent chains of members (sr_group_tune)
  // members with resident iterations (sr_set_resident): one launch per row
  // length runs all of them, one cluster each; the graphs hold the others
  std::vector<int> res;                        // member indices, ordered by row length
  std::vector<int> res_off, res_cnt;           // per row-length class
  std::vector<size_t> res_smem;                // largest shared memory of the class
  std::vector<srk::Geo> res_geo;               // a member's geometry (row length)
  std::vector<int> res_C;                      // the class's cluster size
  srk::ResMember* res_dev = nullptr;           // [2][res.size()] descriptors per parity
  std::vector<char> in_graph;                  // per member: 1 if it runs in the graphs
  int n_graph = 0;
};

namespace {

void group_release(sr_group* g) {
  for (int p = 0; p < 2; ++p)
    if (g->graph[p]) cudaGraphExecDestroy(g->graph[p]);
  if (g->run_graph) cudaGraphExecDestroy(g->run_graph);
  if (g->loop) cudaFree(g->loop);
  if (g->loop_host) cudaFreeHost(g->loop_host);
  if (g->res_dev) cudaFree(g->res_dev);
  delete g;
}

// The resident members' launches, one per row-length class, on the group's
// stream (ResArgs as in iterate_resident, the members' descriptors at the
// group's parity).
cudaError_t group_resident_launch(sr_group* g, int max_outer, double tol, int check_every,
                                  int check_last) {
  const int nres = (int)g->res.size();
  const int p = g->m[0]->cur;
  for (size_t k = 0; k < g->res_off.size(); ++k) {
    srk::ResArgs a{};
    a.members = g->res_dev + (size_t)p * nres + g->res_off[k];
    a.max_outer = max_outer;
    a.tol = tol;
    a.check_every = check_every;
    a.check_last = check_last;
    const cudaError_t e = srk::launch_resident(a, g->res_cnt[k], g->res_geo[k], g->res_C[k],
                                               g->res_smem[k],
                                               g->m[0]->stream, false);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The graph of sr_group_run: for every member a while-node whose body is
// `step` outer iterations (captured as sr_iterate captures them, the last
// one with the FP64 change sums) followed by the member's stopping test
// (k_loop_ctl), which sets the node's condition.  Members converge and leave
// independently; the nodes are spread over lanes like group_build's.
cudaError_t group_build_run(sr_group* g, int step, int parity, std::string& why) {
  const int n = (int)g->m.size();
  int lanes = g->lanes;
  lanes = std::min(lanes, n);
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)g->m[a]->H * g->m[a]->W > (long long)g->m[b]->H * g->m[b]->W;
  });
  std::vector<long long> load(lanes, 0);
  std::vector<cudaGraphNode_t> last(lanes, nullptr);
  cudaGraph_t top = nullptr;
  cudaError_t e = cudaGraphCreate(&top, 0);
  for (int idx = 0; idx < n && e == cudaSuccess; ++idx) {
    const int mi = order[idx];
    if (!g->in_graph[mi]) continue;
    sr_ctx* c = g->m[mi];
    const int lane = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[lane] += (long long)c->H * c->W;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, top, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) break;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, top, last[lane] ? &last[lane] : nullptr, nullptr,
                         last[lane] ? 1 : 0, &np);
    if (e != cudaSuccess) break;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    const long long before = c->launches;
    c->gen_batched = true;
    sr_status st = SR_OK;
    for (int r = 0; r < step && st == SR_OK; ++r)
      st = enqueue_iteration(c, c->cap_stream, (parity + r) & 1, r == step - 1);
    c->gen_batched = false;
    c->launches = before;
    cudaError_t e2 = st == SR_OK ? srk::launch_loop_ctl(h, c->red, g->loop + mi, step, c->cap_stream)
                                 : cudaSuccess;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &captured);
    if (st != SR_OK) {
      why = c->err;
      if (e == cudaSuccess) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) last[lane] = node;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->run_graph, top, 0);
  if (top) cudaGraphDestroy(top);
  return e;
}

// One outer iteration of every member (parity p), each captured on its own
// stream exactly as sr_iterate captures it and placed as a child graph of one
// parent graph.  The members are spread over a bounded number of lanes
// (longest-processing-time first, by pixel count); members of one lane run
// one after another, the lanes run concurrently.  On failure, why holds the
// member's message.
cudaError_t group_build(sr_group* g, int p, std::string& why) {
  const int n = (int)g->m.size();
  int lanes = g->lanes;
  lanes = std::min(lanes, n);
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)g->m[a]->H * g->m[a]->W > (long long)g->m[b]->H * g->m[b]->W;
  });
  std::vector<long long> load(lanes, 0);
  std::vector<cudaGraphNode_t> last(lanes, nullptr);
  cudaGraph_t parent = nullptr;
  cudaError_t e = cudaGraphCreate(&parent, 0);
  for (int idx = 0; idx < n && e == cudaSuccess; ++idx) {
    if (!g->in_graph[order[idx]]) continue;
    sr_ctx* c = g->m[order[idx]];
    const int lane = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[lane] += (long long)c->H * c->W;
    cudaGraph_t child = nullptr;
    e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    const long long before = c->launches;
    c->gen_batched = true;  // same arithmetic, launch shapes for many images at once
    const sr_status st = enqueue_iteration(c, c->cap_stream, p, false);
    c->gen_batched = false;
    c->graph_kernels = (int)(c->launches - before);
    c->launches = before;  // capture enqueues nothing
    e = cudaStreamEndCapture(c->cap_stream, &child);
    if (st != SR_OK) {
      why = c->err;
      if (e == cudaSuccess) e = cudaErrorUnknown;
    }
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess)
      e = cudaGraphAddChildGraphNode(&node, parent, last[lane] ? &last[lane] : nullptr,
                                     last[lane] ? 1 : 0, child);
    if (e == cudaSuccess) last[lane] = node;
    if (child) cudaGraphDestroy(child);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->graph[p], parent, 0);
  if (parent) cudaGraphDestroy(parent);
  return e;
}

}  // namespace

extern "C" {

sr_status sr_group_create(sr_ctx* const* members, int n, sr_group** out) {
  if (!out) return SR_EINVAL;
  *out = nullptr;
  if (!members || n < 1) return SR_EINVAL;
  for (int k = 0; k < n; ++k)
    if (!members[k]) return SR_EINVAL;
  sr_ctx* c0 = members[0];
  for (int k = 0; k < n; ++k)
    if (members[k]->profile) return fail(c0, SR_EINVAL, "group members must not be profiling");
  for (int k = 0; k < n; ++k)
    if (members[k]->prm.inner_tol > 0.f)
      return fail(c0, SR_EUNSUPPORTED, "group members must use a fixed inner_S (inner_tol <= 0)");
  for (int k = 1; k < n; ++k) {
    if (members[k]->stream != c0->stream || members[k]->device != c0->device)
      return fail(c0, SR_EINVAL, "group members must share the device and the stream");
  }
  sr_group* g = new sr_group;
  g->m.assign(members, members + n);
  g->device = c0->device;
  if (const char* env = std::getenv("SR_GROUP_LANES")) g->lanes = std::max(1, std::atoi(env));
  cudaError_t e = cudaSuccess;
  g->in_graph.assign(n, 1);
  for (int k = 0; k < n; ++k)
    if (members[k]->resident && resident_ok(members[k])) g->res.push_back(k);
  // classes of one row length and cluster size: one launch each
  std::stable_sort(g->res.begin(), g->res.end(), [&](int a, int b) {
    return std::make_pair(members[a]->L, members[a]->res_C) <
           std::make_pair(members[b]->L, members[b]->res_C);
  });
  for (size_t j = 0; j < g->res.size(); ++j) {
    sr_ctx* c = members[g->res[j]];
    g->in_graph[g->res[j]] = 0;
    if (j == 0 || members[g->res[j - 1]]->L != c->L || members[g->res[j - 1]]->res_C != c->res_C) {
      g->res_off.push_back((int)j);
      g->res_cnt.push_back(0);
      g->res_smem.push_back(0);
      g->res_geo.push_back(c->geo);
      g->res_C.push_back(c->res_C);
    }
    g->res_cnt.back() += 1;
    g->res_smem.back() = std::max(g->res_smem.back(), c->res_smem);
  }
  g->n_graph = n - (int)g->res.size();
  if (!g->res.empty()) {
    const size_t nres = g->res.size();
    e = dev_alloc((void**)&g->res_dev, 2 * nres * sizeof(srk::ResMember));
    for (int p = 0; p < 2 && e == cudaSuccess; ++p)
      for (size_t j = 0; j < nres && e == cudaSuccess; ++j)
        e = cudaMemcpy(g->res_dev + p * nres + j, members[g->res[j]]->res_dev + p,
                       sizeof(srk::ResMember), cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
      group_release(g);
      if (e == cudaErrorMemoryAllocation) return fail(c0, SR_ENOMEM, "sr_group_create: allocation failed");
      return cuda_fail(c0, e, "sr_group_create");
    }
  }
  std::string why;
  for (int p = 0; p < 2 && e == cudaSuccess && g->n_graph > 0; ++p) e = group_build(g, p, why);
  if (e != cudaSuccess) {
    group_release(g);
    if (!why.empty()) return fail(c0, SR_ECUDA, "sr_group_create: " + why);
    return cuda_fail(c0, e, "sr_group_create");
  }
  *out = g;
  return SR_OK;
}

sr_status sr_group_iterate(sr_group* g, int max_outer) {
  if (!g) return SR_EINVAL;
  sr_ctx* c0 = g->m[0];
  if (max_outer < 0) return fail(c0, SR_EINVAL, "max_outer must be >= 0");
  for (sr_ctx* c : g->m) {
    if (c->cur != c0->cur) return fail(c0, SR_EINVAL, "group members are at different parities");
    if (c->profile) return fail(c0, SR_EINVAL, "group members must not be profiling");
  }
  const int p0 = c0->cur;
  if (!g->res.empty() && max_outer > 0) {
    const cudaError_t e = group_resident_launch(g, max_outer, 0.0, 1, 0);
    if (e != cudaSuccess) return cuda_fail(c0, e, "resident launch (group)");
  }
  for (int k = 0; k < max_outer && g->n_graph > 0; ++k) {
    cudaError_t e = cudaGraphLaunch(g->graph[(p0 + k) & 1], c0->stream);
    if (e != cudaSuccess) return cuda_fail(c0, e, "cudaGraphLaunch (group)");
  }
  for (int k = 0; k < (int)g->m.size(); ++k) {
    sr_ctx* c = g->m[k];
    c->launches += g->in_graph[k] ? (long long)c->graph_kernels * max_outer : (max_outer > 0);
    c->cur ^= max_outer & 1;
    c->iters += max_outer;
    if (!g->in_graph[k]) c->inner_steps += (long long)max_outer * c->prm.inner_S;
  }
  return SR_OK;
}

sr_status sr_group_run(sr_group* g, int max_outer, double tol, int check_every, int* outer_done,
                       double* rel_change) {
  if (!g) return SR_EINVAL;
  sr_ctx* c0 = g->m[0];
  const int n = (int)g->m.size();
  if (check_every < 1 || check_every > 1000 || !std::isfinite(tol) || tol < 0.0)
    return fail(c0, SR_EINVAL, "sr_group_run: check_every in [1, 1000] and tol >= 0 required");
  const int step = check_every + (check_every & 1);  // even: the body keeps the parity
  if (max_outer < step) return fail(c0, SR_EINVAL, "sr_group_run: max_outer below one body");
  for (sr_ctx* c : g->m) {
    if (c->cur != c0->cur) return fail(c0, SR_EINVAL, "group members are at different parities");
    if (c->profile) return fail(c0, SR_EINVAL, "group members must not be profiling");
  }
  if (!g->loop) {
    SR_CUDA(c0, cudaMalloc((void**)&g->loop, sizeof(srk::LoopState) * n));
    SR_CUDA(c0, cudaMallocHost((void**)&g->loop_host, sizeof(srk::LoopState) * n));
  }
  if (g->n_graph > 0 && (!g->run_graph || g->run_step != step || g->run_parity != c0->cur)) {
    if (g->run_graph) cudaGraphExecDestroy(g->run_graph);
    g->run_graph = nullptr;
    std::string why;
    const cudaError_t e = group_build_run(g, step, c0->cur, why);
    if (e != cudaSuccess) {
      if (g->run_graph) cudaGraphExecDestroy(g->run_graph);
      g->run_graph = nullptr;
      if (!why.empty()) return fail(c0, SR_ECUDA, "sr_group_run: " + why);
      return cuda_fail(c0, e, "sr_group_run");
    }
    g->run_step = step;
    g->run_parity = c0->cur;
  }
  for (int k = 0; k < n; ++k) g->loop_host[k] = srk::LoopState{tol, 0.0, max_outer, 0};
  if (!g->res.empty()) {
    // bodies of `step` iterations, the test after each: stop after the first
    // body whose change is <= tol, or when no further body fits
    SR_CUDA(c0, group_resident_launch(g, max_outer - max_outer % step, tol, step, 1));
    for (int k : g->res) {
      sr_ctx* c = g->m[k];
      SR_CUDA(c0, cudaMemcpyAsync(c->res_done_host, c->res_done, sizeof(int),
                                  cudaMemcpyDeviceToHost, c0->stream));
      SR_CUDA(c0, cudaMemcpyAsync(c->red_host, c->red, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                  c0->stream));
    }
  }
  if (g->n_graph > 0) {
    SR_CUDA(c0, cudaMemcpyAsync(g->loop, g->loop_host, sizeof(srk::LoopState) * n,
                                cudaMemcpyHostToDevice, c0->stream));
    SR_CUDA(c0, cudaGraphLaunch(g->run_graph, c0->stream));
    SR_CUDA(c0, cudaMemcpyAsync(g->loop_host, g->loop, sizeof(srk::LoopState) * n,
                                cudaMemcpyDeviceToHost, c0->stream));
  }
  SR_CUDA(c0, cudaStreamSynchronize(c0->stream));
  for (int k : g->res) {
    sr_ctx* c = g->m[k];
    const double num = c->red_host[0], den = c->red_host[1];
    g->loop_host[k] = srk::LoopState{tol, std::sqrt(num) / (std::sqrt(den) + 1e-6), max_outer,
                                     *c->res_done_host};
    c->launches += 1;
  }
  sr_status st = SR_OK;
  for (int k = 0; k < n; ++k) {
    sr_ctx* c = g->m[k];
    const srk::LoopState& L = g->loop_host[k];
    c->iters += L.iters;
    c->inner_steps += (long long)L.iters * c->prm.inner_S;
    if (outer_done) outer_done[k] = L.iters;
    if (rel_change) rel_change[k] = L.rel;
    if (!std::isfinite(L.rel)) st = SR_ENONFINITE;
    else if (st == SR_OK && !(L.rel <= tol)) st = SR_ENOTCONVERGED;
  }
  for (sr_ctx* c : g->m) {
    sr_status es = check_device_error(c);
    if (es != SR_OK) return es;
  }
  if (st == SR_ENONFINITE) return fail(c0, st, "non-finite value in a member's stopping test");
  return st;
}

sr_status sr_group_tune(sr_group* g, int* lanes_out) {
  if (!g) return SR_EINVAL;
  sr_ctx* c0 = g->m[0];
  const int n = (int)g->m.size();
  if (g->n_graph == 0) {  // every member runs resident: no graph lanes to choose
    if (lanes_out) *lanes_out = g->lanes;
    return SR_OK;
  }
  for (sr_ctx* c : g->m)
    if (c->cur != c0->cur) return fail(c0, SR_EINVAL, "group members are at different parities");
  // save every member's state (phi, w at the current parity, e) to restore it
  std::vector<float*> saved;
  auto release = [&] {
    for (float* q : saved) cudaFree(q);
  };
  for (sr_ctx* c : g->m) {
    const size_t bytes = (size_t)c->H * c->W * sizeof(float);
    const float* src[5] = {c->phi[c->cur], c->w1[c->cur], c->w2[c->cur], c->e1, c->e2};
    for (const float* sp : src) {
      float* q = nullptr;
      const cudaError_t e = dev_alloc((void**)&q, bytes);
      if (e != cudaSuccess) {
        release();
        return e == cudaErrorMemoryAllocation ? fail(c0, SR_ENOMEM, "sr_group_tune: no room to save the states")
                                              : cuda_fail(c0, e, "sr_group_tune");
      }
      saved.push_back(q);
      SR_CUDA(c0, cudaMemcpyAsync(q, sp, bytes, cudaMemcpyDeviceToDevice, c0->stream));
    }
  }
  auto restore = [&]() -> cudaError_t {
    size_t k = 0;
    for (sr_ctx* c : g->m) {
      const size_t bytes = (size_t)c->H * c->W * sizeof(float);
      float* dst[5] = {c->phi[c->cur], c->w1[c->cur], c->w2[c->cur], c->e1, c->e2};
      for (float* dp : dst) {
        const cudaError_t e = cudaMemcpyAsync(dp, saved[k++], bytes, cudaMemcpyDeviceToDevice, c0->stream);
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  const int cands[] = {4, 8, 16, 32, 64};
  int best = g->lanes;
  float best_ms = 1e30f;
  const int p = c0->cur;
  for (int L : cands) {
    if (err != cudaSuccess) break;
    if (L > n && L != cands[0]) continue;
    for (int q = 0; q < 2; ++q)
      if (g->graph[q]) {
        cudaGraphExecDestroy(g->graph[q]);
        g->graph[q] = nullptr;
      }
    g->lanes = L;
    std::string why;
    for (int q = 0; q < 2 && err == cudaSuccess; ++q) err = group_build(g, q, why);
    if (err != cudaSuccess) break;
    // one warm-up pair, then a timed pair of outer iterations (both parities)
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
      if (rep == 1) err = cudaEventRecord(e0, c0->stream);
      if (err == cudaSuccess) err = cudaGraphLaunch(g->graph[p], c0->stream);
      if (err == cudaSuccess) err = cudaGraphLaunch(g->graph[1 - p], c0->stream);
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, c0->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) err = restore();
    if (err == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = L;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c0->stream);
  release();
  if (err != cudaSuccess) return cuda_fail(c0, err, "sr_group_tune");
  for (int q = 0; q < 2; ++q)
    if (g->graph[q]) {
      cudaGraphExecDestroy(g->graph[q]);
      g->graph[q] = nullptr;
    }
  if (g->run_graph) {
    cudaGraphExecDestroy(g->run_graph);
    g->run_graph = nullptr;
  }
  g->lanes = best;
  std::string why;
  for (int q = 0; q < 2 && err == cudaSuccess; ++q) err = group_build(g, q, why);
  if (err != cudaSuccess) return cuda_fail(c0, err, "sr_group_tune");
  if (lanes_out) *lanes_out = best;
  return SR_OK;
}

void sr_group_destroy(sr_group* g) {
  if (g) group_release(g);
}

sr_status sr_segment_host(sr_ctx* c, const float* image_host, const float* phi0_host,
                          int max_outer, double tol, unsigned char* mask_host, float* phi_host,
                          int* outer_done, double* rel_change) {
  if (!c) return SR_EINVAL;
  if (!image_host || !phi0_host || !mask_host) return fail(c, SR_EINVAL, "NULL host pointer");
  const size_t P = (size_t)c->H * c->W;
  SR_CUDA(c, cudaMemcpyAsync(c->stage, image_host, P * sizeof(float), cudaMemcpyHostToDevice,
                             c->stream));
  sr_status st = sr_edge_function(c, c->stage, c->W);
  if (st != SR_OK) return st;
  SR_CUDA(c, cudaMemcpyAsync(c->stage, phi0_host, P * sizeof(float), cudaMemcpyHostToDevice,
                             c->stream));
  if ((st = sr_set_phi(c, c->stage, c->W)) != SR_OK) return st;
  sr_status it = sr_iterate(c, max_outer, tol, outer_done, rel_change);
  if (it != SR_OK && it != SR_ENOTCONVERGED) return it;
  if ((st = sr_mask(c, c->mask_dev, c->W)) != SR_OK) return st;
  SR_CUDA(c, cudaMemcpyAsync(mask_host, c->mask_dev, P, cudaMemcpyDeviceToHost, c->stream));
  if (phi_host)
    SR_CUDA(c, cudaMemcpyAsync(phi_host, c->phi[c->cur], P * sizeof(float),
                               cudaMemcpyDeviceToHost, c->stream));
  SR_CUDA(c, cudaStreamSynchronize(c->stream));
  return it;
}

}  // extern "C"
