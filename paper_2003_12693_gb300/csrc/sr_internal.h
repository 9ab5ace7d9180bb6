// Internal interface between the host library (sr_api.cu) and the kernels
// (sr_kernels.cu).  Not part of the public C-ABI.
#pragma once

#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace srk {

constexpr int kMaxR = 8;        // largest repulsion window half width
constexpr int kE = 16;          // complex values each thread holds per FFT stage
constexpr int kColCB = 4;       // columns per CTA in the column pass
constexpr int kTileX = 32;      // 2-D tile of the window-sum kernels
constexpr int kTileY = 8;
constexpr int kMaxGauss = 32;   // taps of the edge-detector Gaussian

// Programmatic dependent launch.  The kernels of the iteration are launched
// with programmatic stream serialization, so a kernel's CTAs may be resident
// while its predecessor on the stream is still finishing.  Every such kernel
// executes pdl_wait() in every CTA before it reads anything a predecessor
// wrote (and before it can exit), then pdl_trigger() to let its own successor
// be scheduled.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// whether hot-path launches carry the attribute (SR_PDL=0 turns it off)
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, const Args&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Scalar model parameters in FP32 as the kernels use them.
struct Model {
  float alpha, beta, gamma, mu, tau, eps, band_l;
  float beta2_mu;   // 2 beta / mu       (Eq. (41))
  float gamma_mu;   // gamma / mu        (Eq. (42))
  float inv_eps;    // 1 / eps
  float half_inv_eps;  // 1 / (2 eps), the scale of delta_eps (Eq. (6))
  float dp_scale;   // pi / (2 eps^2), the scale of delta'_eps (Eq. (29))
  float l_eps;      // l / eps
  float sin_l, cos_l;  // sin(pi l / eps), cos(pi l / eps)
  int R;            // window half width
  float kw[2 * kMaxR + 1];  // k(p) = exp(-p^2 / d^2), p = -R..R at index p + R
};

// Stockham FFT plan of one power-of-two length: n16 radix-16 stages, then
// one stage of radix `tail` (2, 4 or 8) unless tail == 1.
struct Fft {
  int L;                  // transform length
  int logL;
  int n16;
  int tail;
  const float2* tw;       // tw[q] = exp(-2 pi i q / L), q in [0, L)
  const float2* tws16;    // stage twiddles of the register FFT, 16 values per thread
  const float2* tws8;     // stage twiddles of the register FFT, 8 values per thread
};

struct Geo {
  int M, N;     // rows, columns
  int L;        // N / 2: complex length of a row transform
  int logN;
  int neumann;  // 1: Eq. (27) read literally (no difference across the last row /
                // column, reflective Laplacian); 0: periodic (the default reading)
};

// Row pass, forward: build the right-hand side of one inner step (or load it)
// and store the packed half spectrum X[M][L].
struct RowFwdArgs {
  Geo geo;
  Model mod;
  Fft fft;                 // length L
  const float2* twN;       // exp(-2 pi i k / N), k in [0, L)
  const float* psi;
  const float* g;
  const float* w1;
  const float* w2;
  const float* b1;
  const float* b2;
  const float* src;        // LOAD mode: the right-hand side itself
  float2* X;
  int T;                   // rows per CTA
  int CW;                  // column chunk of the window sum
};

// Mixed-radix Stockham plan of one length (sides that are not powers of two).
constexpr int kGenMaxRadix = 32;      // largest radix (primes up to 31)
constexpr int kGenMaxStages = 16;
constexpr int kGenSmemFloat2 = 12288; // shared-memory budget per CTA: 96 KB
struct GenPlan {
  int n;
  int nst;
  int radix[kGenMaxStages];
  int ns[kGenMaxStages];      // product of the earlier radices
  int twoff[kGenMaxStages];   // stage twiddles at tw + twoff[s] + (t-1) ns[s] + k
  int rootoff[kGenMaxStages]; // roots exp(-2 pi i e / R) at roots + rootoff[s] + e
  unsigned mag_m[kGenMaxStages];   // ceil(2^32 / (n / radix)): division by magic multiply
  unsigned mag_ns[kGenMaxStages];  // ceil(2^32 / ns)
  const float2* tw;
  const float2* roots;
};

// Column pass: forward column FFT, divide by the symbol of Eq. (32), inverse.
struct ColArgs {
  Geo geo;
  Fft fft;                 // length M
  const float* aM;         // tau mu 4 sin^2(pi l / M), l in [0, M)
  const float* aN;         // tau mu 4 sin^2(pi k / N), k in [0, L]
  float2* X;
  int* err;                // device error flag (bounded waits), may be null
  long long stall_cycles;  // failure-path tests only: > 0 makes the TMA column pass wait
                           // this long on a barrier nothing arrives on, then time out
  // column solve by recursions (k_colsolve_rec): per column k, (r, s) of the
  // real part and (r, s) of the imaginary part; warm-up length; output buffer
  const float4* rec;
  int rec_R;
  float2* Xout;
  int mirror;              // 1: the column is the even extension of length 2M (Neumann)
};

// Row pass, inverse: half spectrum to real rows; ADD mode adds psi_in.
struct RowInvArgs {
  Geo geo;
  Fft fft;
  const float2* twN;
  const float2* X;
  const float* psi_in;     // ADD mode
  float* out;
  int T;
};

// Right-hand side of one inner step on 2-D tiles (window sum fused in).  The
// Bregman variable is carried as e = b - w, so that div(b - w) needs only e.
struct PrepArgs {
  Geo geo;
  Model mod;
  const float* psi;
  const float* g;
  const float* w1;
  const float* w2;
  const float* e1;         // b1 - w1
  const float* e2;         // b2 - w2
  float* G;                // increment right-hand side, H x W
  // div e is fixed over the inner loop: with D set, the first inner step
  // stores it there (D_load false) and the later ones read it (D_load true)
  float* D;
  bool D_load;
};

// w and b update with the repulsion window sum fused in; b is carried as
// e = b - w on input and output.
struct WBArgs {
  Geo geo;
  Model mod;
  const float* phi1;       // phi^{k+1}
  const float* g;
  const float* w1;         // w^k
  const float* w2;
  const float* e1;         // e^k = b^k - w^k
  const float* e2;
  float* w1o;              // w^{k+1}
  float* w2o;
  float* e1o;              // e^{k+1} = b^{k+1} - w^{k+1} (may alias e1)
  float* e2o;
  const float* phi_old;    // phi^k for the stopping test, or nullptr
  double* partials;        // 2 doubles per 32 x 32 tile when phi_old != nullptr
};

struct RepArgs {
  Geo geo;
  Model mod;
  const float* phi;
  const float* w1;
  const float* w2;
  float* v1;
  float* v2;
};

struct EnergyArgs {
  Geo geo;
  Model mod;
  const float* phi;
  const float* g;
  double* partials;        // 3 doubles per CTA: E_g, E_a, E_r
};

struct EdgeArgs {
  Geo geo;
  int r;                   // Gaussian radius
  float k[2 * kMaxGauss + 1];
  float rho;
  int s_pow;
};

enum { kRowRHS = 0, kRowLOAD = 1 };
enum { kDivCompute = 0, kDivStore = 1, kDivLoad = 2 };
enum { kInvADD = 0, kInvSTORE = 1 };

// Shared-memory bytes of each kernel for the given configuration.
size_t rowfwd_smem(int T, int L, int R, int CW, int mode);
size_t colsolve_smem(int M);
size_t rowinv_smem(int T, int L);
size_t tile_smem(int R);

// Launchers: enqueue on the stream and return the launch error.
cudaError_t launch_rowfwd(const RowFwdArgs& a, int mode, int nthreads, cudaStream_t s);
cudaError_t launch_colsolve(const ColArgs& a, cudaStream_t s);
cudaError_t launch_rowinv(const RowInvArgs& a, int mode, int nthreads, cudaStream_t s);
cudaError_t launch_wb_update(const WBArgs& a, cudaStream_t s);
cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s);
int tile32_blocks(const Geo& geo);  // CTAs of the 32 x 32 tile kernels
// Row-pass shape of the fixed power-of-two passes (k_rowfwd, k_rowinv) for an
// H-row image with row transforms of complex length L on a device with nsm
// SMs: *T rows per CTA and *NT threads, with T * L = 16 * NT.  Returns false
// (and leaves the outputs alone) when no such shape exists.
bool row_shape(int H, int L, int nsm, int* NT, int* T);
cudaError_t launch_empty(cudaStream_t s);  // one warp that only waits and triggers
// per-member state of a group's device-side stopping loop (sr_group_run)
struct LoopState {
  double tol;      // set by the host before the launch
  double rel;      // last relative change
  int max_outer;   // set by the host
  int iters;       // outer iterations run (reset by the host)
};
cudaError_t launch_loop_ctl(cudaGraphConditionalHandle h, const double* red, LoopState* st,
                            int step, cudaStream_t s);
// Host tables (double, rounded once): exp(-2 pi i q / len) for q < n, and the
// per-stage twiddles of the register FFT of length len with 2^logE values
// per thread (the layout TwPlan in sr_dft.cuh describes).
std::vector<float2> twiddle_table(int n, int len);
std::vector<float2> stage_twiddle_table(int len, int logE);
cudaError_t launch_repulsion(const RepArgs& a, cudaStream_t s);
cudaError_t launch_energy(const EnergyArgs& a, cudaStream_t s);
cudaError_t launch_reduce(const double* partials, int nblocks, int ncomp, double* out,
                          cudaStream_t s);
cudaError_t launch_init_wb(const float* phi, float* w1, float* w2, float* e1, float* e2,
                           Geo geo, cudaStream_t s);
// out = a + sign * b elementwise over n floats (b <-> e conversions)
cudaError_t launch_axpb(const float* a, const float* b, float sign, float* out, size_t n,
                        cudaStream_t s);
cudaError_t launch_mask(const float* phi, unsigned char* mask, int ld, Geo geo,
                        cudaStream_t s);
cudaError_t launch_edge(const EdgeArgs& a, const float* f, int ld, float* tmp1, float* tmp2,
                        float* g, cudaStream_t s);
cudaError_t configure_kernels();   // raise dynamic shared-memory limits once

// Register-resident FFT passes (sr_fft.cu) for L = W/2 in [16, 2048] and
// H in [16, 4096].  Rows: 2^logE values per thread (logE 3 or 4), T rows per
// CTA, T * L / 2^logE threads.  Columns: schedule 0 (4 columns per CTA, 16
// values per thread; 2 columns at H = 4096), 1 (2 columns, 8 values),
// 2 (4 columns, 8 values).
bool fft2_supported(const Geo& geo);

// Mixed-radix passes (sr_fftgen.cu) for sides that are not powers of two.
// batched: the launch shapes for a member of a group (fuller CTAs)
int gen_rows_per_cta(int n, int count, bool batched);
cudaError_t configure_fftgen();
cudaError_t launch_rowfft_gen(const RowFwdArgs& a, const GenPlan& P, bool batched, cudaStream_t s);
cudaError_t launch_colsolve_gen(const ColArgs& a, const GenPlan& P, bool batched, cudaStream_t s);
cudaError_t launch_rowifft_gen(const RowInvArgs& a, const GenPlan& P, bool add, bool batched,
                               cudaStream_t s);
size_t rowfft2_smem(int T, int L, int logE);
int stage_twiddles(int L, int logE);  // entries of the stage-twiddle table
cudaError_t launch_rowfft2(const RowFwdArgs& a, int logE, int nthreads, cudaStream_t s,
                           bool set_attr);
cudaError_t launch_rowifft2(const RowInvArgs& a, bool add, int logE, int nthreads, cudaStream_t s,
                            bool set_attr);
cudaError_t launch_colsolve2(const ColArgs& a, int sched, cudaStream_t s, bool set_attr);
int colsolve2_threads(int M, int sched);
// Persistent TMA column pass (schedule 3); tm maps X as a float32 matrix of
// H rows by W floats with boxes of 2 * colsolve_tma_cb(H) x min(H, 256).
cudaError_t launch_colsolve_tma(const ColArgs& a, const CUtensorMap& tm, int grid, cudaStream_t s,
                                bool set_attr);
int colsolve_tma_cb(int M);
cudaError_t colsolve_tma_occupancy(int M, int* blocks_per_sm);  // after set_attr
// Column solve by a forward and a backward first-order recursion per column
// (sr_colrec.cu, column schedule 7): kRecRows rows per thread, kRecChunks
// threads of one column per CTA row; reads a.X, writes a.Xout (a.X != a.Xout).
constexpr int kRecRows = 32;
constexpr int kRecChunks = 4;
constexpr int kColRec = 7;
// warm-up length for the slowest decay r_max (0 if none of the buckets suffices)
int colsolve_rec_radius(double r_max);
cudaError_t launch_colsolve_rec(const ColArgs& a, cudaStream_t s);

// The whole solve of one inner step in one CTA (sr_small.cu, column schedule
// 8), for power-of-two images whose rows fit one pass of kSmallThreads
// threads at 16 values each (M * L / 16 <= kSmallThreads, L <= 512): row R2C,
// column recursions (rec_R in 8..32), row C2R with psi += result.
constexpr int kSmallThreads = 512;
constexpr int kColSmall = 8;
struct SmallArgs {
  Geo geo;
  const float* G;        // right-hand side (increment or the full one)
  const float* psi_in;   // added to the result; null: out = solution
  float* out;            // may alias psi_in
  const float2* tws16;   // stage twiddles of the row transform (16 values per thread)
  const float2* twN;     // exp(-2 pi i k / N), k < L
  const float4* rec;     // per-column (r, s) pairs of the recursions
  int rec_R;
};
bool solve_small_supported(const Geo& geo, int rec_R);
size_t solve_small_smem(const Geo& geo);
cudaError_t launch_solve_small(const SmallArgs& a, cudaStream_t s, bool set_attr);

// Outer iterations with the state resident in shared memory (sr_resident.cu):
// one cluster of C CTAs per image (C = 8, or 16 with the non-portable cluster
// size), CTA q owning rows [q M/C, (q+1) M/C); N in {32, 64, 128, 256}, M a
// multiple of C (>= 2 C), the recursion column solve (rec_R > 0), periodic
// boundary.
constexpr int kResCMax = 16;
constexpr int kResThreads = 256;
constexpr size_t kResMaxSmem = 220 * 1024;
struct ResMember {
  Geo geo;
  Model mod;
  int inner_S;
  int rec_R;
  int cur;               // parity of the state buffers on entry
  const float* g;
  float* phi[2];
  float* w1[2];
  float* w2[2];
  float* e1;             // e = b - w (one buffer, updated in place)
  float* e2;
  const float2* tws4;    // stage twiddles of the row transform (4 values per thread)
  const float2* twN;     // exp(-2 pi i k / N), k < L
  const float4* rec;     // per-column (r, s) pairs of the column recursions
  int* done;             // outer iterations run (written once, at the end)
  double* red;           // last stopping test: ||phi^{k+1} - phi^k||^2, ||phi^k||^2
};
struct ResArgs {
  const ResMember* members;  // one per cluster
  int max_outer;
  double tol;                // > 0: stop at the first check with rel <= tol
  int check_every;           // checks after every check_every-th and the last iteration
  int check_last;            // tol <= 0: evaluate the test after the last iteration
};
size_t resident_smem(const Geo& geo, int R, int rec_R, int C);
bool resident_supported(const Geo& geo, int R, int rec_R, int C);
// set_attr: raise the shared-memory limit and check that a cluster of C fits
// (cudaErrorNotSupported if not); otherwise launch `members` clusters of C.
cudaError_t launch_resident(const ResArgs& a, int members, const Geo& geo, int C, size_t smem,
                            cudaStream_t s, bool set_attr);
// Neumann solve helpers: the even extension of each row (out is M x 2N) and
// out = psi + T[:, :N] (T is M x 2N; psi may be null)
cudaError_t launch_mirror_rows(const float* in, float* out, const Geo& geo, cudaStream_t s);
cudaError_t launch_add_half(const float* psi, const float* T, float* out, const Geo& geo,
                            cudaStream_t s);

// AOS solve of the phi sub-problem (sr_aos.cu): phi = psi + 1/2 [T1 + T2],
// T1 = (I - k A_1)^{-1} (G + tau mu (A_1 - A_2) psi), T2 the same with A_1 and
// A_2 swapped, k = 2 tau mu, A_1 / A_2 the periodic second differences down
// the columns / along the rows.  psi may be null (then
// phi = 1/2 [(I - k A_1)^{-1} G + (I - k A_2)^{-1} G]).
constexpr int kAosRowWarps = 4;
struct AosArgs {
  Geo geo;
  const float* G;
  const float* psi;
  float* T1;          // H x W scratch: the column-direction solve
  float* X2;          // H x W scratch: the row-direction input
  float* phi;         // output; may alias psi (the row pass reads psi only at the element it writes)
  float k;            // 2 tau mu
  float tm;           // tau mu
  float r, s;         // factor root and scale r / k
  int R;              // warm-up of the column recursion (template bucket)
  int warm_blocks;    // warm-up blocks of 32 of the row recursion
  float pw[33];       // r^m, m = 0..32
};
int aos_radius(double r);  // 0 if no bucket suffices
cudaError_t launch_aos(const AosArgs& a, cudaStream_t s, bool set_attr);

int tile_blocks(const Geo& geo);   // CTAs of the 2-D tile kernels

}  // namespace srk
