/*
 * FP64 CPU oracle for the Split Bregman self-repelling snake.
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark; never by the product path.
 *
 * The code is plain on purpose: direct loops, the steps of Alg. 1 in the
 * paper's order, a textbook recursive mixed-radix FFT, and the window sum of
 * the repulsion field written as the double sum it is.  OpenMP only splits
 * independent output rows or columns across threads; each output value is
 * produced by one thread in a fixed order, so results do not depend on the
 * thread count.
 */
#include "sr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define IDX(i, j) ((size_t)(i) * (size_t)N + (size_t)(j))

static double* alloc_d(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

/* ------------------------------------------------------------------------ */
/* Scalar functions                                                          */
/* ------------------------------------------------------------------------ */

/* Eq. (5): compactly supported regularised Heaviside. */
double oc_heaviside(double phi, double eps) {
  if (phi > eps) return 1.0;
  if (phi < -eps) return 0.0;
  return 0.5 * (1.0 + phi / eps + sin(M_PI * phi / eps) / M_PI);
}

/* Eq. (6): its derivative, the regularised Dirac function. */
double oc_delta(double phi, double eps) {
  if (fabs(phi) > eps) return 0.0;
  return (1.0 + cos(M_PI * phi / eps)) / (2.0 * eps);
}

/* Eq. (29): derivative of delta. */
double oc_delta_prime(double phi, double eps) {
  if (fabs(phi) > eps) return 0.0;
  return -M_PI / (2.0 * eps * eps) * sin(M_PI * phi / eps);
}

/* Eq. (11): narrow band h = H(phi + l) (1 - H(phi - l)). */
double oc_band(double phi, double eps, double l) {
  return oc_heaviside(phi + l, eps) * (1.0 - oc_heaviside(phi - l, eps));
}

/* Eq. (28): h' = delta(phi + l)(1 - H(phi - l)) - H(phi + l) delta(phi - l). */
double oc_band_prime(double phi, double eps, double l) {
  return oc_delta(phi + l, eps) * (1.0 - oc_heaviside(phi - l, eps)) -
         oc_heaviside(phi + l, eps) * oc_delta(phi - l, eps);
}

/* ------------------------------------------------------------------------ */
/* Edge detector, Eq. (1)                                                    */
/* ------------------------------------------------------------------------ */

/* g = 1 / (1 + rho |grad(G_sigma * f)|^s).  The paper does not state how the
 * Gaussian or the gradient are discretised; the reading used here: a sampled
 * Gaussian on |t| <= ceil(3 sigma), normalised to sum 1, replicated border;
 * central differences inside, one-sided differences on the border rows and
 * columns. */
void oc_edge(int M, int N, const double* f, double rho, double sigma, int s_pow, double* g) {
  double* a = alloc_d((size_t)M * N);
  double* b = alloc_d((size_t)M * N);
  int r = sigma > 0.0 ? (int)ceil(3.0 * sigma) : 0;
  double* k = alloc_d(2 * r + 1);
  double ksum = 0.0;
  for (int t = -r; t <= r; ++t) {
    k[t + r] = sigma > 0.0 ? exp(-(double)(t * t) / (2.0 * sigma * sigma)) : 1.0;
    ksum += k[t + r];
  }
  for (int t = 0; t <= 2 * r; ++t) k[t] /= ksum;
  /* blur along rows (index i), then along columns (index j) */
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
      for (int t = -r; t <= r; ++t) {
        int ii = i + t;
        if (ii < 0) ii = 0;
        if (ii > M - 1) ii = M - 1;
        s += k[t + r] * f[IDX(ii, j)];
      }
      a[IDX(i, j)] = s;
    }
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
      for (int t = -r; t <= r; ++t) {
        int jj = j + t;
        if (jj < 0) jj = 0;
        if (jj > N - 1) jj = N - 1;
        s += k[t + r] * a[IDX(i, jj)];
      }
      b[IDX(i, j)] = s;
    }
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      double gi, gj;
      if (M == 1) gi = 0.0;
      else if (i == 0) gi = b[IDX(1, j)] - b[IDX(0, j)];
      else if (i == M - 1) gi = b[IDX(M - 1, j)] - b[IDX(M - 2, j)];
      else gi = 0.5 * (b[IDX(i + 1, j)] - b[IDX(i - 1, j)]);
      if (N == 1) gj = 0.0;
      else if (j == 0) gj = b[IDX(i, 1)] - b[IDX(i, 0)];
      else if (j == N - 1) gj = b[IDX(i, N - 1)] - b[IDX(i, N - 2)];
      else gj = 0.5 * (b[IDX(i, j + 1)] - b[IDX(i, j - 1)]);
      double mag = sqrt(gi * gi + gj * gj);
      g[IDX(i, j)] = 1.0 / (1.0 + rho * pow(mag, (double)s_pow));
    }
  free(a);
  free(b);
  free(k);
}

/* ------------------------------------------------------------------------ */
/* Discrete operators, Eqs. (35)-(36)                                        */
/* ------------------------------------------------------------------------ */

/* Forward differences; the boundary wraps periodically, the reading that makes
 * the Fourier symbol of Eq. (32) exact. */
void oc_grad(int M, int N, const double* phi, double* d1, double* d2) {
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      d1[IDX(i, j)] = phi[IDX((i + 1) % M, j)] - phi[IDX(i, j)];
      d2[IDX(i, j)] = phi[IDX(i, (j + 1) % N)] - phi[IDX(i, j)];
    }
}

/* Backward-difference divergence, periodic. */
void oc_div(int M, int N, const double* a1, const double* a2, double* out) {
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j)
      out[IDX(i, j)] = (a1[IDX(i, j)] - a1[IDX((i + M - 1) % M, j)]) +
                       (a2[IDX(i, j)] - a2[IDX(i, (j + N - 1) % N)]);
}

/* ------------------------------------------------------------------------ */
/* FFT: recursive mixed-radix decimation in time                              */
/* ------------------------------------------------------------------------ */

static int smallest_factor(int n) {
  for (int p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

/* y[k] = sum_n x[n s] exp(sign 2 pi i n k / n_len) for n_len = n.  With
 * n = p m and n = p n2 + n1 the sum splits into p transforms of length m over
 * the sub-sequences x[p n2 + n1], combined with the twiddles W_n^{n1 k}.
 * tc/ts hold cos/sin(2 pi e / tn) for the top-level length tn. */
static void fft_rec(int n, const double* xr, const double* xi, int s, double* yr, double* yi,
                    int sign, const double* tc, const double* ts, int tn) {
  if (n == 1) {
    yr[0] = xr[0];
    yi[0] = xi[0];
    return;
  }
  int p = smallest_factor(n), m = n / p;
  double* sr = alloc_d(n);
  double* si = alloc_d(n);
  for (int n1 = 0; n1 < p; ++n1)
    fft_rec(m, xr + (size_t)n1 * s, xi + (size_t)n1 * s, s * p, sr + n1 * m, si + n1 * m, sign,
            tc, ts, tn);
  int step = tn / n;
  for (int k = 0; k < n; ++k) {
    double accr = 0.0, acci = 0.0;
    for (int n1 = 0; n1 < p; ++n1) {
      long e = ((long)n1 * k) % n;
      double c = tc[e * step], sn = sign * ts[e * step];
      double ar = sr[n1 * m + k % m], ai = si[n1 * m + k % m];
      accr += ar * c - ai * sn;
      acci += ar * sn + ai * c;
    }
    yr[k] = accr;
    yi[k] = acci;
  }
  free(sr);
  free(si);
}

void oc_fft1(int n, double* re, double* im, int stride, int sign) {
  double* tc = alloc_d(n);
  double* ts = alloc_d(n);
  for (int e = 0; e < n; ++e) {
    tc[e] = cos(2.0 * M_PI * (double)e / (double)n);
    ts[e] = sin(2.0 * M_PI * (double)e / (double)n);
  }
  double* xr = alloc_d(n);
  double* xi = alloc_d(n);
  double* yr = alloc_d(n);
  double* yi = alloc_d(n);
  for (int t = 0; t < n; ++t) {
    xr[t] = re[(size_t)t * stride];
    xi[t] = im[(size_t)t * stride];
  }
  fft_rec(n, xr, xi, 1, yr, yi, sign, tc, ts, n);
  for (int t = 0; t < n; ++t) {
    re[(size_t)t * stride] = yr[t];
    im[(size_t)t * stride] = yi[t];
  }
  free(tc);
  free(ts);
  free(xr);
  free(xi);
  free(yr);
  free(yi);
}

void oc_fft2(int M, int N, double* re, double* im, int sign) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < M; ++i) oc_fft1(N, re + (size_t)i * N, im + (size_t)i * N, 1, sign);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < N; ++j) oc_fft1(M, re + j, im + j, N, sign);
}

/* Eqs. (31)-(33): divide the spectrum by the symbol of (1 - tau mu Laplacian),
 * 1 - tau mu (2 cos z1 + 2 cos z2 - 4) with z1 = 2 pi l1 / M, z2 = 2 pi l2 / N
 * (zero-based l1, l2; the printed brace in the symbol is misplaced), invert,
 * keep the real part.  The inverse transform is scaled by 1/(MN). */
void oc_solve(int M, int N, double tau, double mu, const double* rhs, double* phi) {
  size_t P = (size_t)M * N;
  double* re = alloc_d(P);
  double* im = alloc_d(P);
  memcpy(re, rhs, P * sizeof(double));
  oc_fft2(M, N, re, im, -1);
  for (int l1 = 0; l1 < M; ++l1)
    for (int l2 = 0; l2 < N; ++l2) {
      double z1 = 2.0 * M_PI * l1 / M, z2 = 2.0 * M_PI * l2 / N;
      double lam = 1.0 - tau * mu * (2.0 * cos(z1) + 2.0 * cos(z2) - 4.0);
      re[IDX(l1, l2)] /= lam;
      im[IDX(l1, l2)] /= lam;
    }
  oc_fft2(M, N, re, im, +1);
  for (size_t t = 0; t < P; ++t) phi[t] = re[t] / (double)P;
  free(re);
  free(im);
}

/* ------------------------------------------------------------------------ */
/* Repulsion field, Sec. 4                                                   */
/* ------------------------------------------------------------------------ */

/* v_ij = sum_{p,q=-R..R} exp(-(p^2+q^2)/d^2) w_{i+p,j+q} h(phi_{i+p,j+q}).
 * Terms with (i+p, j+q) outside the image are dropped: the window integral runs
 * over Omega only. */
void oc_repulsion(int M, int N, const oc_params* p, const double* phi, const double* w1,
                  const double* w2, double* v1, double* v2) {
  size_t P = (size_t)M * N;
  double* u1 = alloc_d(P);
  double* u2 = alloc_d(P);
  for (size_t t = 0; t < P; ++t) {
    double h = oc_band(phi[t], p->eps, p->band_l);
    u1[t] = h * w1[t];
    u2[t] = h * w2[t];
  }
  int R = p->R;
  double d2 = p->d * p->d;
  int side = 2 * R + 1;
  double* K = alloc_d((size_t)side * side); /* K(p, q) = exp(-(p^2 + q^2) / d^2) */
  for (int pp = -R; pp <= R; ++pp)
    for (int qq = -R; qq <= R; ++qq)
      K[(pp + R) * side + (qq + R)] = exp(-(double)(pp * pp + qq * qq) / d2);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      double s1 = 0.0, s2 = 0.0;
      for (int pp = -R; pp <= R; ++pp) {
        int ii = i + pp;
        if (ii < 0 || ii >= M) continue;
        for (int qq = -R; qq <= R; ++qq) {
          int jj = j + qq;
          if (jj < 0 || jj >= N) continue;
          double kw = K[(pp + R) * side + (qq + R)];
          s1 += kw * u1[IDX(ii, jj)];
          s2 += kw * u2[IDX(ii, jj)];
        }
      }
      v1[IDX(i, j)] = s1;
      v2[IDX(i, j)] = s2;
    }
  free(K);
  free(u1);
  free(u2);
}

/* ------------------------------------------------------------------------ */
/* phi sub-problem, Eqs. (26), (30), (37)                                     */
/* ------------------------------------------------------------------------ */

/* F = psi + tau [ -gamma g |w| delta'(psi) + alpha g delta(psi)
 *                 + 2 beta h'(psi) (w . v) + mu div(b - w) ].
 * psi is the current inner iterate phi^{k+1,s} (the printed phi^{k,s} read as
 * the inner iterate, since the loop starts from phi^{k+1,0} = phi^k). */
void oc_rhs(int M, int N, const oc_params* p, const double* psi, const double* g,
            const double* w1, const double* w2, const double* b1, const double* b2,
            const double* v1, const double* v2, double* F) {
  size_t P = (size_t)M * N;
  double* a1 = alloc_d(P);
  double* a2 = alloc_d(P);
  double* dv = alloc_d(P);
  for (size_t t = 0; t < P; ++t) {
    a1[t] = b1[t] - w1[t];
    a2[t] = b2[t] - w2[t];
  }
  oc_div(M, N, a1, a2, dv);
  for (size_t t = 0; t < P; ++t) {
    double x = psi[t];
    double wn = sqrt(w1[t] * w1[t] + w2[t] * w2[t]);
    double force = -p->gamma * g[t] * wn * oc_delta_prime(x, p->eps) +
                   p->alpha * g[t] * oc_delta(x, p->eps) +
                   2.0 * p->beta * oc_band_prime(x, p->eps, p->band_l) *
                       (w1[t] * v1[t] + w2[t] * v2[t]) +
                   p->mu * dv[t];
    F[t] = x + p->tau * force;
  }
  free(a1);
  free(a2);
  free(dv);
}

void oc_phi_step(int M, int N, const oc_params* p, const double* psi, const double* g,
                 const double* w1, const double* w2, const double* b1, const double* b2,
                 double* psi_next) {
  size_t P = (size_t)M * N;
  double* v1 = alloc_d(P);
  double* v2 = alloc_d(P);
  double* F = alloc_d(P);
  oc_repulsion(M, N, p, psi, w1, w2, v1, v2);
  oc_rhs(M, N, p, psi, g, w1, w2, b1, b2, v1, v2, F);
  oc_solve(M, N, p->tau, p->mu, F, psi_next);
  free(v1);
  free(v2);
  free(F);
}

/* ------------------------------------------------------------------------ */
/* w sub-problem and Bregman update, Eqs. (41), (42), (40), (23)             */
/* ------------------------------------------------------------------------ */

/* Eq. (42): max(|B| - t, 0) B / |B|, with 0 (0/|0|) = 0. */
void oc_soft_threshold(double B1, double B2, double t, double* o1, double* o2) {
  double n = sqrt(B1 * B1 + B2 * B2);
  double s = n - t;
  if (s < 0.0) s = 0.0;
  if (n == 0.0 || s == 0.0) {
    *o1 = 0.0;
    *o2 = 0.0;
    return;
  }
  *o1 = s * B1 / n;
  *o2 = s * B2 / n;
}

void oc_w_b_update(int M, int N, const oc_params* p, const double* phi1, const double* g,
                   double* w1, double* w2, double* b1, double* b2, double* wt1, double* wt2) {
  size_t P = (size_t)M * N;
  double* v1 = alloc_d(P);
  double* v2 = alloc_d(P);
  double* d1 = alloc_d(P);
  double* d2 = alloc_d(P);
  /* Eq. (41) uses w^k and h(phi^{k+1}) inside the window integral. */
  oc_repulsion(M, N, p, phi1, w1, w2, v1, v2);
  oc_grad(M, N, phi1, d1, d2);
  for (size_t t = 0; t < P; ++t) {
    double h = oc_band(phi1[t], p->eps, p->band_l);
    double B1 = d1[t] + b1[t] + (2.0 * p->beta / p->mu) * h * v1[t];
    double B2 = d2[t] + b2[t] + (2.0 * p->beta / p->mu) * h * v2[t];
    double thr = (p->gamma / p->mu) * g[t] * oc_delta(phi1[t], p->eps);
    double s1, s2;
    oc_soft_threshold(B1, B2, thr, &s1, &s2);
    if (wt1) {
      wt1[t] = s1;
      wt2[t] = s2;
    }
    /* Eq. (40): projection onto |w| = 1, with the zero vector kept at zero. */
    double n = sqrt(s1 * s1 + s2 * s2);
    double n1 = n > 0.0 ? s1 / n : 0.0;
    double n2 = n > 0.0 ? s2 / n : 0.0;
    w1[t] = n1;
    w2[t] = n2;
    /* Eq. (23) */
    b1[t] = b1[t] + d1[t] - n1;
    b2[t] = b2[t] + d2[t] - n2;
  }
  free(v1);
  free(v2);
  free(d1);
  free(d2);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1                                                               */
/* ------------------------------------------------------------------------ */

void oc_init(int M, int N, const double* phi0, double* w1, double* w2, double* b1, double* b2) {
  oc_grad(M, N, phi0, w1, w2);
  memset(b1, 0, (size_t)M * N * sizeof(double));
  memset(b2, 0, (size_t)M * N * sizeof(double));
}

void oc_iterate(int M, int N, const oc_params* p, const double* g, double* phi, double* w1,
                double* w2, double* b1, double* b2, int K, double* rel) {
  size_t P = (size_t)M * N;
  double* psi = alloc_d(P);
  double* nxt = alloc_d(P);
  for (int k = 0; k < K; ++k) {
    memcpy(psi, phi, P * sizeof(double)); /* phi^{k+1,0} = phi^k */
    for (int s = 0; s < p->S; ++s) {
      oc_phi_step(M, N, p, psi, g, w1, w2, b1, b2, nxt);
      memcpy(psi, nxt, P * sizeof(double));
    }
    oc_w_b_update(M, N, p, psi, g, w1, w2, b1, b2, NULL, NULL);
    double num = 0.0, den = 0.0;
    for (size_t t = 0; t < P; ++t) {
      num += (psi[t] - phi[t]) * (psi[t] - phi[t]);
      den += phi[t] * phi[t];
    }
    if (rel) rel[k] = sqrt(num) / (sqrt(den) + 1e-6);
    memcpy(phi, psi, P * sizeof(double));
  }
  free(psi);
  free(nxt);
}

/* ------------------------------------------------------------------------ */
/* Energy, Eqs. (7)-(10), and mask, Eq. (3)                                  */
/* ------------------------------------------------------------------------ */

void oc_energy(int M, int N, const oc_params* p, const double* phi, const double* g, double* out) {
  size_t P = (size_t)M * N;
  double* d1 = alloc_d(P);
  double* d2 = alloc_d(P);
  double* v1 = alloc_d(P);
  double* v2 = alloc_d(P);
  oc_grad(M, N, phi, d1, d2);
  oc_repulsion(M, N, p, phi, d1, d2, v1, v2);
  double Eg = 0.0, Ea = 0.0, Er = 0.0;
  for (size_t t = 0; t < P; ++t) {
    Eg += g[t] * sqrt(d1[t] * d1[t] + d2[t] * d2[t]) * oc_delta(phi[t], p->eps);
    Ea += g[t] * (1.0 - oc_heaviside(phi[t], p->eps));
    Er -= oc_band(phi[t], p->eps, p->band_l) * (d1[t] * v1[t] + d2[t] * v2[t]);
  }
  out[0] = p->gamma * Eg + p->alpha * Ea + p->beta * Er;
  out[1] = Eg;
  out[2] = Ea;
  out[3] = Er;
  free(d1);
  free(d2);
  free(v1);
  free(v2);
}

void oc_mask(int M, int N, const double* phi, unsigned char* mask) {
  for (size_t t = 0; t < (size_t)M * N; ++t) mask[t] = phi[t] < 0.0 ? 1 : 0;
}
