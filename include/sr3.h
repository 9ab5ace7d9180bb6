/*
 * sr3.h - C-ABI of the Split Bregman self-repelling snake on volumes.
 *
 * The paper applies the method to a 3-D CT volume (Fig. 6, Sec. 5); its
 * iteration is Alg. 1 with a third axis everywhere.  This library runs it on
 * one GPU under the readings of the 2-D library (sr.h): periodic forward
 * differences and backward divergence (Eqs. (35)-(36)); the repulsion window
 * sum (Sec. 4, Eq. (38)) over the cube |p|, |q|, |r| <= R with weight
 * exp(-(p^2 + q^2 + r^2) / d^2), terms outside the volume dropped; one
 * semi-implicit step of Eq. (37) with the 3-D Laplacian, whose system
 * (1 - tau mu Lap) phi = F is diagonalised by the 3-D DFT with the symbol
 * 1 + tau mu (4 sin^2(pi l_z / Z) + 4 sin^2(pi l_y / M) + 4 sin^2(pi l_x / N))
 * (Eq. (32) with a third term); the soft threshold and projection of Eqs.
 * (41), (42), (40) on 3-vectors and the Bregman update of Eq. (23).
 *
 * Layout.  A volume is a float32 array of Z x M x N values, row-major (the
 * last index fastest), contiguous, on the device that was current at
 * sr3_create.  Vector fields (w, b, v) are passed as three such volumes, the
 * z, y (M) and x (N) components, as an array of three pointers.
 *
 * Ownership and streams as in sr.h: the caller owns every buffer; the context
 * owns its state and scratch (about 27 volumes of 4 bytes per voxel, two of
 * 8) and frees them in sr3_destroy; work is enqueued on the stream given to
 * sr3_create and the calls return once it is enqueued.
 *
 * Errors: SR_EINVAL for bad arguments, SR_EUNSUPPORTED for sizes outside M,
 * N in {16, 32, ..., 1024} (powers of two), 1 <= Z <= 4096, or tau mu so
 * large that the z-recursions' warm-up would exceed 64 planes; SR_ENOMEM,
 * SR_ECUDA as usual.  Nothing exits or traps.
 */
#ifndef SR3_H
#define SR3_H

#include "sr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sr3_ctx sr3_ctx;

/* Create a solver for Z x M x N volumes with the parameters of sr_params
 * (rho, sigma, s_pow, check_every and inner_tol are not used; g is given by
 * sr3_set_g, 1 until then). */
sr_status sr3_create(int Z, int M, int N, const sr_params* p, void* cuda_stream, sr3_ctx** out);
void sr3_destroy(sr3_ctx* ctx);

/* The edge weight g of Eq. (1) (device volume), copied into the context. */
sr_status sr3_set_g(sr3_ctx* ctx, const float* g);

/* Alg. 1 initialisation: phi^0 = phi0, w^0 = grad phi^0 (forward, periodic),
 * b^0 = 0. */
sr_status sr3_set_phi(sr3_ctx* ctx, const float* phi0);

/* Copy the iteration state (phi, w[3], b[3]) into / out of the context. */
sr_status sr3_set_state(sr3_ctx* ctx, const float* phi, const float* const w[3],
                        const float* const b[3]);
sr_status sr3_get_state(sr3_ctx* ctx, float* phi, float* const w[3], float* const b[3]);

/* Alg. 1 outer loop: max_outer iterations of inner_S steps of Eq. (37) and
 * the w / b update of Eqs. (41), (42), (40), (23). */
sr_status sr3_iterate(sr3_ctx* ctx, int max_outer);

/* Single steps on caller buffers, for checking each on its own:
 * the window sum v = sum K h(phi) w over the cube (Eq. (38));
 * (1 - tau mu Lap) out = rhs (out must not alias rhs);
 * one inner step of Eq. (37), psi_out from psi_in with w, b frozen (psi_out may
 * alias psi_in);
 * the w / b update from phi^{k+1}, w^k, b^k (outputs must not alias w). */
sr_status sr3_window_sum(sr3_ctx* ctx, const float* phi, const float* const w[3], float* const v[3]);
sr_status sr3_fft_solve(sr3_ctx* ctx, const float* rhs, float* out);
sr_status sr3_phi_step(sr3_ctx* ctx, const float* psi_in, const float* const w[3],
                       const float* const b[3], float* psi_out);
sr_status sr3_w_b_update(sr3_ctx* ctx, const float* phi1, const float* const w[3],
                         const float* const b[3], float* const w_out[3], float* const b_out[3]);

/* Kernel launches enqueued by this context (-1 for NULL). */
long long sr3_kernel_launches(const sr3_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SR3_H */
