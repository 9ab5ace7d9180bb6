/*
 * FP64 CPU oracle for the Split Bregman iteration of the self-repelling snake
 * (Pan, Song, Liu, Li, Zhou, Tan, Chen, "Using the Split Bregman Algorithm to
 * Solve the Self-repelling Snake Model").
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path; it
 * shares no code with it.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.
 *
 * Every routine works on row-major float64 planes of M rows by N columns
 * (index i*N + j), takes its steps in the order the paper states them, and
 * uses no blocking, fusion or reordering beyond that.  Points where the paper
 * is silent or garbled follow the readings listed with each function.
 *
 * Parity status: every function below is pinned by the CPU tests (closed
 * forms, brute force, a dense direct solve, numpy's FFT, the minimiser of the
 * w sub-problem, the gradient of the discrete energy).  The full K-iteration
 * trajectory has no such pin: the method is sensitive to rounding at pixels
 * where |B| is near zero or near the threshold, so multi-iteration runs are
 * compared through invariants only.
 */
#ifndef SR_ORACLE_H
#define SR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double alpha;   /* balloon weight, Eq. (7) */
  double beta;    /* repulsion weight, Eq. (7) */
  double gamma;   /* geodesic-length weight, Eq. (7) */
  double mu;      /* splitting penalty, Eq. (22) */
  double tau;     /* time step, Eq. (30) */
  double eps;     /* regularisation width of H and delta, Eqs. (5)-(6) */
  double band_l;  /* narrow-band half width l of h, Eq. (11) */
  double d;       /* Gaussian scale of the repulsion window, Sec. 4 */
  int R;          /* repulsion window half width: p, q in [-R, R] */
  int S;          /* inner semi-implicit steps per outer iteration, Eq. (37) */
} oc_params;

/* Scalar functions: Eqs. (5), (6), (29), (11), (28). */
double oc_heaviside(double phi, double eps);
double oc_delta(double phi, double eps);
double oc_delta_prime(double phi, double eps);
double oc_band(double phi, double eps, double l);
double oc_band_prime(double phi, double eps, double l);

/* Edge detector g of Eq. (1); sigma <= 0 skips the Gaussian. */
void oc_edge(int M, int N, const double* f, double rho, double sigma, int s_pow, double* g);

/* Forward differences of Eq. (35), periodic. */
void oc_grad(int M, int N, const double* phi, double* d1, double* d2);
/* Backward-difference divergence of Eq. (36), periodic. */
void oc_div(int M, int N, const double* a1, const double* a2, double* out);

/* Unnormalised 2-D DFT in place (sign -1 forward, +1 inverse). */
void oc_fft2(int M, int N, double* re, double* im, int sign);
/* 1-D transform of length n with the given stride (exported for the tests). */
void oc_fft1(int n, double* re, double* im, int stride, int sign);

/* phi = Re F^{-1}[ F(rhs) / F(1 - tau mu Laplacian) ], Eqs. (31)-(33). */
void oc_solve(int M, int N, double tau, double mu, const double* rhs, double* phi);

/* Repulsion field v of Sec. 4: window sum of K(p,q) w h(phi); zero outside. */
void oc_repulsion(int M, int N, const oc_params* p, const double* phi,
                  const double* w1, const double* w2, double* v1, double* v2);

/* Right-hand side F^{k,s} of Eq. (37), with v given. */
void oc_rhs(int M, int N, const oc_params* p, const double* psi, const double* g,
            const double* w1, const double* w2, const double* b1, const double* b2,
            const double* v1, const double* v2, double* F);

/* One semi-implicit inner step: v from psi, F, then the FFT solve. */
void oc_phi_step(int M, int N, const oc_params* p, const double* psi, const double* g,
                 const double* w1, const double* w2, const double* b1, const double* b2,
                 double* psi_next);

/* Generalised soft threshold of Eq. (42) on one vector. */
void oc_soft_threshold(double B1, double B2, double t, double* o1, double* o2);

/* w and b updates after the inner loop: Eqs. (41), (42), (40), (23).
 * w1,w2 hold w^k on entry and w^{k+1} on exit; b1,b2 likewise.  If wt1 is not
 * NULL the shrunk vector before the projection is stored in wt1, wt2. */
void oc_w_b_update(int M, int N, const oc_params* p, const double* phi1, const double* g,
                   double* w1, double* w2, double* b1, double* b2,
                   double* wt1, double* wt2);

/* Alg. 1 initialisation: w0 = grad phi0 (forward differences), b0 = 0. */
void oc_init(int M, int N, const double* phi0, double* w1, double* w2, double* b1, double* b2);

/* Alg. 1 iterations: K outer iterations with exactly S inner steps each.
 * rel (length K, may be NULL) receives ||phi^{k+1}-phi^k|| / (||phi^k|| + 1e-6). */
void oc_iterate(int M, int N, const oc_params* p, const double* g, double* phi,
                double* w1, double* w2, double* b1, double* b2, int K, double* rel);

/* Discrete energy of Eqs. (7)-(10) with the gradient replaced by forward
 * differences and the double integral by the same window sum as v.
 * out = {E, E_g, E_a, E_r} with E = gamma E_g + alpha E_a + beta E_r. */
void oc_energy(int M, int N, const oc_params* p, const double* phi, const double* g, double* out);

/* 1 where phi < 0 (inside the contour, Eq. (3)). */
void oc_mask(int M, int N, const double* phi, unsigned char* mask);

#ifdef __cplusplus
}
#endif
#endif
