/*
 * sr.h - C-ABI of the GB300 Split Bregman self-repelling snake (SR).
 *
 * The library runs the Split Bregman iteration for the self-repelling snake
 * of Pan et al. (Alg. 1, Secs. 3-4) on one GPU with hand-written sm_103a
 * kernels.  It takes plain pointers and sizes; nothing here depends on a
 * framework's tensor types.
 *
 * Layout.  Every image-sized buffer is a float32 (or uint8 for masks) plane
 * of H rows by W columns, row-major, with a leading dimension ld >= W
 * elements between rows.  Row index i (the paper's x1), column index j (x2).
 * Unless a function says "host", pointers are device pointers on the device
 * that was current when the context was created.
 *
 * Ownership.  The caller owns every buffer it passes; no call keeps a caller
 * pointer after it returns.  The context owns its state (phi, w, b, g), the
 * FFT workspace and the CUDA graphs, and frees them in sr_destroy.
 *
 * Streams.  All work is enqueued on the stream given to sr_create (0 means
 * the legacy default stream).  Calls return once the work is enqueued,
 * except where a function says it synchronises.
 *
 * Errors.  Every call returns an sr_status; none exits, aborts or traps the
 * device.  SR_ECUDA means a CUDA runtime call failed; sr_last_error gives the
 * message.  A context that returned SR_ECUDA should be destroyed.
 */
#ifndef SR_H
#define SR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sr_status {
  SR_OK = 0,
  SR_EINVAL = 1,          /* bad argument: size, pointer, parameter value */
  SR_ENOMEM = 2,          /* device or host allocation failed */
  SR_ECUDA = 3,           /* a CUDA runtime call failed (see sr_last_error) */
  SR_ENONFINITE = 4,      /* NaN or Inf met in the state or the stopping test */
  SR_ENOTCONVERGED = 5,   /* tol > 0 and max_outer reached before convergence */
  SR_ETIMEOUT = 6,        /* a bounded device-side wait (TMA transfer) ran out of time */
  SR_EUNSUPPORTED = 7     /* size or option this build does not implement */
} sr_status;

/* Model and solver parameters.  Defaults (sr_params_default) are the Fig. 1
 * set of Sec. 5: alpha=4, gamma=4, beta=0.2, mu=8, eps=1, l=1, tau=0.1, S=3. */
typedef struct sr_params {
  float alpha;       /* balloon (area) weight, Eq. (7) */
  float beta;        /* repulsion weight, Eq. (7) */
  float gamma;       /* geodesic-length weight, Eq. (7) */
  float mu;          /* splitting penalty, Eq. (22) */
  float tau;         /* time step of the semi-implicit scheme, Eq. (30) */
  float eps;         /* width of the regularised Heaviside / Dirac, Eqs. (5)-(6) */
  float band_l;      /* narrow-band half width l of h, Eq. (11) */
  float d;           /* Gaussian scale of the repulsion window, Sec. 4 */
  int win_radius;    /* window half width R: offsets p, q in [-R, R], 0 <= R <= 8 */
  int inner_S;       /* inner semi-implicit steps per outer iteration, Eq. (37) */
  float inner_tol;   /* inner exit of Sec. 4: > 0 stops the inner loop once the relative
                        change of phi between inner steps is <= inner_tol (at most
                        inner_S steps; eager, no graph); <= 0 runs exactly inner_S */
  float rho;         /* edge-detector scale, Eq. (1) */
  float sigma;       /* Gaussian smoothing of the image in Eq. (1); 0 disables */
  int s_pow;         /* exponent s in Eq. (1): 1 or 2 */
  int check_every;   /* outer iterations between FP64 stopping tests (>= 1) */
} sr_params;

typedef struct sr_ctx sr_ctx;

/* Fill *p with the Fig. 1 defaults (and d = 3, R = 3, rho = 1, sigma = 1,
 * s = 2, check_every = 10).  Returns SR_EINVAL if p is NULL. */
sr_status sr_params_default(sr_params* p);

/* Create a solver for H x W images.  Validates the parameters (finite, mu,
 * tau, eps > 0, 0 <= R <= 8, S >= 1, s in {1, 2}), allocates the device state
 * and FFT workspace and builds the twiddle and symbol tables of Eq. (32).
 * Supported sizes: H and W multiples of 16 in [16, 4096] such that H and
 * W/2 have no prime factor above 31 (SR_EUNSUPPORTED otherwise).  Powers of
 * two use register-resident FFT passes with an autotuned schedule, other
 * sides (e.g. 96, 160, 224) mixed-radix shared-memory row passes with radices
 * 16, 8, 4, 2, 3, 5 and direct DFTs of the other primes, and for the column
 * solve the faster, timed at sr_create (once per size and tau mu in the
 * process), of the recursions of column schedule 7 and a mixed-radix column
 * FFT with the symbol's division (the environment variable SR_GEN_FFT_COLS =
 * 1 or 0 at sr_create fixes the column FFT or the recursions).
 * cuda_stream is a cudaStream_t (may be 0). */
sr_status sr_create(int H, int W, const sr_params* p, void* cuda_stream, sr_ctx** out);

/* Release everything the context owns.  NULL is ignored. */
void sr_destroy(sr_ctx* ctx);

/* Message of the last failing call on this context ("" if none); with NULL,
 * why the calling thread's last sr_create failed. */
const char* sr_last_error(const sr_ctx* ctx);
const char* sr_status_string(sr_status s);

/* Eq. (1): g = 1 / (1 + rho |grad(G_sigma * f)|^s) from the image f
 * (device, H x W, leading dimension ld).  The Gaussian is sampled on
 * |t| <= ceil(3 sigma), normalised, with a replicated border; the gradient
 * uses central differences inside and one-sided ones on the border.  Alg. 1
 * computes g once per image, before the iterations. */
sr_status sr_edge_function(sr_ctx* ctx, const float* image, int ld);

/* Alg. 1 initialisation: phi^0 = phi0 (device, a signed distance function,
 * Eq. (3): negative inside), w^0 = grad phi^0 (forward differences, Eq. (35),
 * periodic), b^0 = 0.  Resets the iteration counter. */
sr_status sr_set_phi(sr_ctx* ctx, const float* phi0, int ld);

/* Alg. 1 outer loop.  Each outer iteration runs inner_S semi-implicit steps
 * of Eq. (37) (repulsion window sum, right-hand side, FFT solve of Eqs.
 * (31)-(33)) and then the w update of Eqs. (41), (42), (40) and the Bregman
 * update of Eq. (23).
 *   tol <= 0: run exactly max_outer iterations; asynchronous unless
 *             rel_change is non-NULL, in which case the last iteration also
 *             computes the relative change (FP64) and the call synchronises.
 *   tol  > 0: every check_every iterations the relative change
 *             ||phi^{k+1} - phi^k|| / (||phi^k|| + 1e-6) (the form of the
 *             inner stopping rule of Sec. 4) is reduced in FP64 on the GPU
 *             and read back; the loop stops once it is <= tol.  Returns
 *             SR_ENOTCONVERGED if max_outer is reached first.
 * outer_done (may be NULL) receives the iterations run by this call;
 * rel_change (may be NULL) the last relative change computed.  A NaN or Inf
 * in the stopping test returns SR_ENONFINITE. */
sr_status sr_iterate(sr_ctx* ctx, int max_outer, double tol, int* outer_done,
                     double* rel_change);

/* Eq. (3): mask[i, j] = 1 where phi < 0 (inside the contour), else 0.
 * mask is a device uint8 plane with leading dimension ld. */
sr_status sr_mask(sr_ctx* ctx, unsigned char* mask, int ld);

/* Copy the current phi to a device buffer (leading dimension ld). */
sr_status sr_get_phi(sr_ctx* ctx, float* phi, int ld);

/* Checkpoint / resume: copy the full iteration state (phi, w1, w2, b1, b2;
 * device, contiguous H x W each) out of / into the context.  Iterating from a
 * restored state gives bit-identical results to an uninterrupted run. */
sr_status sr_get_state(sr_ctx* ctx, float* phi, float* w1, float* w2, float* b1, float* b2);
sr_status sr_set_state(sr_ctx* ctx, const float* phi, const float* w1, const float* w2,
                       const float* b1, const float* b2);

/* Copy g out of / into the context (device, contiguous H x W). */
sr_status sr_get_g(sr_ctx* ctx, float* g);
sr_status sr_set_g(sr_ctx* ctx, const float* g);

/* Discrete energy of Eqs. (7)-(10) at the current phi, accumulated in FP64 on
 * the GPU: E = gamma E_g + alpha E_a + beta E_r with E_g = sum g |grad phi|
 * delta(phi), E_a = sum g (1 - H(phi)), E_r = -sum_x h(phi_x) grad phi_x .
 * sum_y K(x - y) h(phi_y) grad phi_y over the repulsion window (forward
 * differences, terms outside the image dropped).  Synchronises.  Any output
 * pointer may be NULL. */
sr_status sr_energy(sr_ctx* ctx, double* E, double* Eg, double* Ea, double* Er);

/* ---- Single steps of the hot path (device buffers, contiguous H x W) ----
 * These run one row of the iteration on caller buffers with the context's
 * parameters and g; they exist so each step can be checked on its own.
 * sr_phi_step, sr_fft_solve (out) and sr_w_b_update need 16-byte aligned
 * buffers (SR_EINVAL otherwise). */

/* Sec. 4 repulsion field: v = sum_{p,q=-R..R} exp(-(p^2+q^2)/d^2)
 * w_{i+p,j+q} h(phi_{i+p,j+q}), terms outside the image dropped. */
sr_status sr_repulsion_field(sr_ctx* ctx, const float* phi, const float* w1, const float* w2,
                             float* v1, float* v2);

/* One inner step of Eq. (37): psi_out = phi^{k+1,s+1} from psi_in =
 * phi^{k+1,s} and the frozen w^k, b^k.  psi_out may alias psi_in. */
sr_status sr_phi_step(sr_ctx* ctx, const float* psi_in, const float* w1, const float* w2,
                      const float* b1, const float* b2, float* psi_out);

/* Eqs. (31)-(33) alone: out = Re F^{-1}[F(rhs) / F(1 - tau mu Laplacian)]. */
sr_status sr_fft_solve(sr_ctx* ctx, const float* rhs, float* out);

/* Eqs. (41), (42), (40), (23) after the inner loop: from phi^{k+1}, w^k, b^k
 * compute w^{k+1} and b^{k+1}.  b_out may alias b_in; w_out must not alias
 * w_in (the window sum reads w^k around every pixel). */
sr_status sr_w_b_update(sr_ctx* ctx, const float* phi1, const float* w1_in,
                        const float* w2_in, const float* b1_in, const float* b2_in,
                        float* w1_out, float* w2_out, float* b1_out, float* b2_out);

/* The iterated w sub-problem, Eqs. (38)-(40), then Eq. (23): from
 * w^{k+1,0} = w^k, `sweeps` times (1 <= sweeps <= 64)
 *     w <- B / |B|,  B = grad phi^{k+1} + b^k + (2 beta / mu) h(phi^{k+1}) v(w),
 * v(w) the window sum of Eq. (38) over h(phi^{k+1}) w (terms outside the
 * image dropped), the zero vector kept at zero; then b^{k+1} = b^k +
 * grad phi^{k+1} - w^{k+1}.  The denominator gamma g delta + mu of Eq. (39) is
 * a positive scalar, so the projection (40) removes it: this variant has no
 * threshold, unlike Eqs. (41)-(42).  Aliasing rules as sr_w_b_update.  The
 * first call allocates two image planes in the context. */
sr_status sr_w_b_fixed_point(sr_ctx* ctx, const float* phi1, const float* w1_in,
                             const float* w2_in, const float* b1_in, const float* b2_in,
                             int sweeps, float* w1_out, float* w2_out, float* b1_out,
                             float* b2_out);

/* Choose how sr_iterate (and a group created afterwards) solves the w
 * sub-problem: sweeps = 0 the generalised soft threshold of Eqs. (41)-(42)
 * (the default), 1 <= sweeps <= 64 that many sweeps of Eqs. (38)-(40) as in
 * sr_w_b_fixed_point.  The context's graphs are rebuilt on the next
 * sr_iterate; groups capture the setting when they are created. */
sr_status sr_set_w_sweeps(sr_ctx* ctx, int sweeps);

/* How the phi sub-problem of each inner step is solved: solver 0 = the FFT
 * solve of Eqs. (31)-(33) (the default); 1 = additive operator splitting, the
 * alternative named at the end of Sec. 4 in the form of Eqs. (19)-(20):
 *     phi = 1/2 [ (I - 2 tau mu A_1)^{-1} F + (I - 2 tau mu A_2)^{-1} F ],
 * A_1, A_2 the periodic second differences down the columns and along the
 * rows; each factor is a cyclic tridiagonal solve with constant coefficients,
 * factored once into a forward and a backward first-order recursion.  AOS is
 * a first-order splitting of the exact solve, so its phi differs from the FFT
 * solve's by O((tau mu)^2).  The first call with solver 1 allocates two image
 * planes.  SR_EUNSUPPORTED if 2 tau mu is so large (above about 30) that the
 * recursions' warm-up would exceed 128 places; graphs are rebuilt on the next
 * sr_iterate. */
sr_status sr_set_phi_solver(sr_ctx* ctx, int solver);

/* Boundary reading.  neumann = 0 (the default): periodic differences, as the
 * symbol of Eq. (32) diagonalises.  neumann = 1: Eq. (27) read literally with
 * the homogeneous condition d phi / dn = 0 -- forward differences are zero
 * across the last row and the last column, the backward divergence is minus
 * the adjoint of that gradient, the Laplacian their product (the reflective
 * 5-point stencil), and (1 - tau mu Lap) phi = F is solved in the basis of the
 * type-II DCT, which diagonalises it with the symbol
 * 1 + tau mu (4 sin^2(pi l / 2M) + 4 sin^2(pi k / 2N)).  On the GPU the row
 * direction is transformed by the periodic FFT of each row's even extension
 * (length 2W) and each column is solved with reflective ends by the
 * recursions of column schedule 7 on its even extension; sr_fft_solve,
 * sr_phi_step, sr_w_b_update, sr_set_phi (w^0 = grad phi^0), sr_energy and
 * sr_iterate all follow the setting.  The window sum of Sec. 4 drops the
 * terms outside the image either way.  SR_EUNSUPPORTED unless H and W are
 * powers of two with W <= 2048, or together with the AOS solver or the
 * iterated w variant.  The first call with neumann = 1 allocates about five
 * image planes; graphs are rebuilt on the next sr_iterate. */
sr_status sr_set_boundary(sr_ctx* ctx, int neumann);

/* Resident outer iterations for small images.  on = 1: sr_iterate runs its
 * outer iterations of Alg. 1 in ONE launch per call, with the whole state
 * (phi, w at both parities, e, g, div e, the right-hand side and the half
 * spectrum) held in the shared memory of one cluster of C CTAs -- CTA q owns
 * rows [q H/C, (q+1) H/C); with on = 1, C = 16 where H/16 >= 2 rows and
 * the device schedules clusters of 16, else 8 (the environment variable
 * SR_RESIDENT_CLUSTER = 8 or 16 fixes it); on = 8 or 16 asks for that C
 * (SR_EUNSUPPORTED if it does not fit).  16 gives one image the shortest
 * iterations; 8 lets twice as many images run at once, which serves a group
 * of many small images better -- for all the iterations of the call;
 * neighbour
 * rows, window halos and the column recursions' warm-ups are read from the
 * other CTAs' shared memory (distributed shared memory), and the phases of an
 * iteration are separated by cluster barriers instead of kernel boundaries.
 * Global memory is read once and written once per call.  The stopping test
 * of Sec. 4 (FP64 sums, every check_every iterations and after the last) is
 * evaluated on the device; sr_iterate reads the iteration count and the
 * residual back only when tol > 0 or rel_change is requested.  The
 * per-pixel arithmetic is that of the tiled kernels; the column solve is
 * the recursion pass of column schedule 7 with one run per CTA, so results
 * agree with the default path to rounding, not bit for bit.
 * Supported: W in {32, 64, 128, 256}, H a multiple of 8 with H >= 16, the
 * state within 220 KB of shared memory per CTA (H * W <= 16384 at R <= 8),
 * the periodic FFT solve with the column recursions available (tau mu <=
 * about 8), the soft-threshold w update and no inner exit; otherwise
 * SR_EUNSUPPORTED.  While the context's configuration is changed to one of
 * those (sr_set_boundary, sr_set_phi_solver, sr_set_w_sweeps) sr_iterate
 * uses the default path.  In a group (sr_group_create), members with
 * resident iterations on run together in one launch per row length and
 * cluster size, one cluster each, with their own stopping tests in sr_group_run; the other
 * members run in the group's graphs.  on = 0 restores the default path. */
sr_status sr_set_resident(sr_ctx* ctx, int on);

/* The AOS solve alone (device buffers, contiguous H x W, not aliased):
 * out = 1/2 [ (I - 2 tau mu A_1)^{-1} rhs + (I - 2 tau mu A_2)^{-1} rhs ].
 * The first call allocates two image planes in the context. */
sr_status sr_aos_solve(sr_ctx* ctx, const float* rhs, float* out);

/* Inner phi steps sr_iterate has run on this context (all outer iterations;
 * with inner_tol > 0 the count per iteration depends on the data); reset to
 * zero when reset != 0.  -1 for a NULL context. */
long long sr_inner_steps(sr_ctx* ctx, int reset);

/* One inner step of the phi update, like sr_phi_step, for callers that
 * cannot allocate device memory.  The paper has no counterpart: this entry
 * point exists for hosts that hand out all GPU memory from their own fixed
 * arena, for code running while its stream is captured into a CUDA graph in a
 * mode that forbids allocation, and for real-time loops that cannot afford
 * the device synchronisation cudaMalloc / cudaFree may cause.
 * It takes no context and allocates nothing: the half spectrum and the FFT and
 * symbol tables live in a file-scope device array of 1 MiB + 16 KiB that the
 * library reserves on every GPU that loads it, until the process exits.
 *   H, W:  powers of two with 16 <= H, W <= 512; larger sizes return
 *          SR_EUNSUPPORTED and launch nothing.
 *   p:     model parameters (inner_S, inner_tol, rho, sigma, s_pow and
 *          check_every are ignored); invalid values return SR_EINVAL.
 *   g, psi_in, w1, w2, b1, b2: device inputs, contiguous H x W float32;
 *          psi_out: device output, may alias psi_in; psi_in and psi_out must
 *          be 16-byte aligned.
 *   cuda_stream: cudaStream_t the work is enqueued on (0: legacy stream).
 * The first call on a device looks up the array's device address and sets
 * kernel attributes, so make that first call before any stream capture.
 * Every call rewrites the whole array before reading it, so nothing carries
 * over between calls, but calls whose work overlaps on the GPU race on the
 * array: order them on one stream.  SR_ECUDA if a CUDA call fails. */
sr_status sr_phi_step_noalloc(int H, int W, const sr_params* p, const float* g,
                              const float* psi_in, const float* w1, const float* w2,
                              const float* b1, const float* b2, float* psi_out,
                              void* cuda_stream);

/* FFT schedule of the phi solve: how the row and column passes of Eqs.
 * (31)-(33) are laid out on the GPU.  sr_create picks it by timing the
 * candidates once per image size in the process (the result is cached), so
 * it depends on the device.  Every schedule computes the same transform.
 *   row_values_per_thread: 8 or 16 (radix-8 or radix-16 stages)
 *   row_threads: threads per CTA of the row passes; rows per CTA =
 *                row_threads * row_values_per_thread / (W / 2)
 *   col_schedule: 0 = 4 columns per CTA, 16 values per thread (2 columns at
 *                 H = 4096); 1 = 2 columns, 8 values; 2 = 4 columns, 8 values;
 *                 3 = persistent CTAs fed by TMA (tensor-memory-accelerator
 *                 box loads/stores, double buffered), 4 columns, 16 values;
 *                 4 = 2 columns, 16 values; 5 = 4 columns, 16 values with
 *                 double-buffered exchanges; 6 = 4 columns, 16 values with
 *                 registers capped for two CTAs per SM; 7 = no column FFT:
 *                 the column operator of Eq. (32) for row frequency k is
 *                 the periodic tridiagonal c_k - tau mu (S + S^-1), solved
 *                 exactly by its scalar factorisation into a forward and a
 *                 backward first-order recursion (warm-up long enough that
 *                 the truncated start is below 2^-27 relative; available
 *                 when tau mu <= about 8); 8 = the whole solve of one inner
 *                 step in one CTA (row transforms, the recursions of 7 and
 *                 the inverse row transforms, the half spectrum kept in
 *                 shared memory) for power-of-two images with
 *                 H * W / 32 <= 512 and W <= 1024, where launches and not
 *                 bytes bound the step; the autotuner compares it with the
 *                 best row pair plus column pass
 *   tuned_us: measured microseconds of one row pair plus one column pass
 *             when the autotuner chose the schedule, else 0.
 * Sizes below W = 32 use fixed kernels and report row_threads = 0.
 * The environment variable SR_FFT_SCHEDULE="row_values,row_threads,
 * col_schedule" makes sr_create use that schedule (when valid for the size)
 * instead of tuning, e.g. for reproducible profiling.
 * sr_set_schedule validates the fields (SR_EINVAL) and rebuilds the
 * iteration graphs. */
typedef struct sr_schedule {
  int row_values_per_thread;
  int row_threads;
  int col_schedule;
  float tuned_us;
} sr_schedule;
sr_status sr_get_schedule(sr_ctx* ctx, sr_schedule* out);
sr_status sr_set_schedule(sr_ctx* ctx, const sr_schedule* sched);

/* Kernel launches enqueued by this context since creation (or the last
 * reset).  Graph launches count every kernel node they run. */
long long sr_kernel_launches(const sr_ctx* ctx, int reset);

/* Per-kernel timing: when enabled, sr_iterate launches without graphs and
 * records CUDA events around every kernel on the context's stream.
 * sr_kernel_times synchronises and returns, for kernel class c (see
 * SR_KCLASS_*), the summed milliseconds and the launch count, then clears
 * the accumulators. */
#define SR_KCLASS_ROWFFT 0       /* row R2C FFT of the right-hand side */
#define SR_KCLASS_COLSOLVE 1     /* column FFT, divide by the symbol, inverse */
#define SR_KCLASS_ROWIFFT 2      /* row C2R FFT + phi update */
#define SR_KCLASS_WB_UPDATE 3    /* repulsion + shrink + projection + Bregman */
#define SR_KCLASS_REDUCE 4       /* FP64 stopping-test reduction */
#define SR_KCLASS_PREP 5         /* repulsion window sum + right-hand side */
#define SR_KCLASS_RESIDENT 6     /* whole outer iterations resident on chip */
#define SR_KCLASS_COUNT 7
sr_status sr_profile_enable(sr_ctx* ctx, int enable);
/* Microseconds the profiling mode's event pair adds to a kernel's measured
 * time: the median over 65 event pairs around an empty kernel launched the
 * same way on the context's stream.  Synchronises. */
sr_status sr_profile_overhead(sr_ctx* ctx, double* us);
sr_status sr_kernel_times(sr_ctx* ctx, int kclass, double* total_ms, long long* launches);

/* ---- Failure-path test hooks (not needed in normal use) ----
 * They let tests drive the library's error paths without faulting, hanging
 * or exhausting a GPU.
 *
 * sr_test_stall_waits: with cycles > 0, every CTA of the TMA column pass
 * (col_schedule 3 of sr_schedule) makes its first wait on a shared-memory
 * barrier that no transfer arrives on, gives up after `cycles` clock cycles,
 * records a timeout in the context's device error flag, waits (bounded by the
 * normal limit of about 2^31 cycles) for its own transfers in flight, and
 * returns.  The next synchronising call (sr_iterate with tol > 0 or a
 * rel_change pointer) then returns SR_ETIMEOUT and clears the flag; the
 * context stays usable, and cycles = 0 restores normal waits.  Other column
 * schedules have no device-side waits and ignore the setting.  SR_EINVAL for
 * a NULL context or cycles < 0.
 *
 * sr_test_fail_allocations: process-wide; after n more successful device or
 * pinned-host allocations by the library, every further one fails as if
 * memory had run out, so the calling entry point returns SR_ENOMEM after
 * freeing what it had allocated.  n < 0 removes the limit (the default). */
sr_status sr_test_stall_waits(sr_ctx* ctx, long long cycles);
sr_status sr_test_fail_allocations(long long n);

/* Batched iteration (many images, uneven sizes).  A group holds n contexts
 * created on the same device with the same stream (sizes may differ; every
 * size sr_create accepts).  sr_group_iterate runs max_outer outer iterations
 * of Alg. 1 on every member: one CUDA graph per parity holds the members'
 * iterations as concurrent branches (each a chain of its own kernels), so
 * small images share the GPU instead of running one after another.  Each
 * member's results are bit-identical to sr_iterate(member, max_outer, 0, ...)
 * on that member alone.  Members with resident iterations (sr_set_resident)
 * are not in the graphs: all of them run in one launch per row length and
 * cluster size (one cluster per member, the same kernel as sr_iterate's, so
 * also bit for bit), on the group's stream before the graphs.  The group
 * takes each member's mode (resident or not, sweeps, solver, boundary) as it
 * is at sr_group_create: change a member's mode before creating the group.  There is no stopping test inside the group call
 * (tol = 0 semantics); sr_iterate on a member afterwards gives its relative
 * change.  The members must be at the same parity: created or reset with
 * sr_set_phi / sr_set_state together and iterated only through the group, or
 * by the same counts.
 *   Errors: SR_EINVAL for n < 1, a NULL member, members on different streams
 *   or devices, or members at different parities; SR_ECUDA as usual.  The
 *   group does not own the contexts: destroy the group first. */
typedef struct sr_group sr_group;
sr_status sr_group_create(sr_ctx* const* members, int n, sr_group** out);
sr_status sr_group_iterate(sr_group* group, int max_outer);

/* Run every member until its own stopping test passes, in one graph launch.
 * The launched graph holds, per member, a device-side while-loop (a CUDA
 * graph conditional node) whose body is B outer iterations (B = check_every
 * rounded up to an even number, so a body leaves the member at its parity)
 * followed by the member's stopping test: the relative change
 * ||phi^{k+1} - phi^k|| / (||phi^k|| + 1e-6) of the body's last iteration,
 * reduced in FP64 on the GPU as sr_iterate's, decides on the device whether
 * the member runs another body (change > tol and another body fits under
 * max_outer).  Members stop independently; the others keep the GPU.  Each
 * member's state equals sr_iterate(member, outer_done[k], 0, ...) bit for bit.
 * Synchronises.  outer_done and rel_change (n entries each, may be NULL)
 * receive each member's iterations and last relative change.  Returns
 * SR_ENOTCONVERGED if some member reached max_outer first, SR_ENONFINITE if a
 * member's change was NaN or Inf (that member stops), SR_EINVAL for
 * check_every outside [1, 1000], tol < 0 or max_outer < B.  The first call
 * (and a call with another check_every or parity) builds the graph. */
sr_status sr_group_run(sr_group* group, int max_outer, double tol, int check_every,
                       int* outer_done, double* rel_change);
/* Choose how many members run concurrently in the group's graphs (its
 * "lanes": 4, 8, 16, 32 or 64, at most the member count) by timing two outer
 * iterations of the whole group with each and keeping the fastest; the
 * members' states are saved before and restored after every timing, so the
 * call leaves them as it found them (it allocates room for five image planes
 * per member for the time of the call).  Synchronises.  lanes_out (may be
 * NULL) receives the choice.  Without this call a group uses 32 lanes, or the
 * count in the environment variable SR_GROUP_LANES at sr_group_create. */
sr_status sr_group_tune(sr_group* group, int* lanes_out);
void sr_group_destroy(sr_group* group);

/* Convenience for callers with host buffers: copy the image and phi0 from
 * host memory (pinned memory gives asynchronous copies), compute g, set
 * phi0, run max_outer iterations (tol as in sr_iterate), and copy the mask
 * (uint8, H x W contiguous) and, if phi_host is non-NULL, phi back to host
 * memory.  Synchronises.  outer_done / rel_change as in sr_iterate. */
sr_status sr_segment_host(sr_ctx* ctx, const float* image_host, const float* phi0_host,
                          int max_outer, double tol, unsigned char* mask_host,
                          float* phi_host, int* outer_done, double* rel_change);

#ifdef __cplusplus
}
#endif
#endif /* SR_H */
