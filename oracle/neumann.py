"""FP64 oracle of the Neumann-boundary variant of the phi sub-problem.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests may import
it; the product path never does.  The CUDA path's version (sr_set_boundary)
is checked against it by tests/test_gpu_neumann.py.

Eq. (27) states a Neumann-type boundary condition, while the symbol of
Eq. (32) diagonalises the periodic Laplacian (the default reading).  This
module takes Eq. (27) literally with the homogeneous condition d phi / dn = 0
(the (w - b).n part is dropped with the boundary differences of w - b):

* forward differences with a zero difference across the last row / column;
* the backward divergence that is exactly minus the adjoint of that gradient;
* the Laplacian as their composition (the reflective 5-point stencil);
* (1 - tau mu Lap_N) phi = F solved with the orthonormal type-II DCT, whose
  basis cos(pi k (i + 1/2) / M) diagonalises Lap_N with eigenvalues
  -4 sin^2(pi k / (2M)) per axis (a library transform used as one step);
* the right-hand side of Eq. (37) and the w/b update of Eqs. (41), (42),
  (40), (23) with these differences, from the pinned scalar functions and
  window sum of the C oracle.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

from . import Params, _f64, band, band_prime, delta, delta_prime, repulsion, soft_threshold


def grad(phi):
    """Forward differences, zero across the last row (d1) and column (d2)."""
    phi = _f64(phi)
    d1 = np.zeros_like(phi)
    d2 = np.zeros_like(phi)
    d1[:-1, :] = phi[1:, :] - phi[:-1, :]
    d2[:, :-1] = phi[:, 1:] - phi[:, :-1]
    return d1, d2


def div(a1, a2):
    """Backward divergence with a1[-1, :] = a2[:, -1] = 0 and nothing before
    the first row / column: div = -grad^T."""
    a1, a2 = _f64(a1), _f64(a2)
    out = np.zeros_like(a1)
    out[0, :] += a1[0, :]
    out[1:-1, :] += a1[1:-1, :] - a1[:-2, :]
    out[-1, :] += -a1[-2, :]
    out[:, 0] += a2[:, 0]
    out[:, 1:-1] += a2[:, 1:-1] - a2[:, :-2]
    out[:, -1] += -a2[:, -2]
    return out


def laplacian(phi):
    return div(*grad(phi))


def symbol(M, N, tau, mu):
    """Eigenvalues of 1 - tau mu Lap_N on the DCT-II basis."""
    k = np.arange(M)[:, None]
    l = np.arange(N)[None, :]
    return 1.0 + tau * mu * (4.0 * np.sin(np.pi * k / (2 * M)) ** 2 +
                             4.0 * np.sin(np.pi * l / (2 * N)) ** 2)


def solve(rhs, tau, mu):
    """(1 - tau mu Lap_N) phi = rhs by the orthonormal DCT-II."""
    rhs = _f64(rhs)
    c = scipy.fft.dctn(rhs, type=2, norm="ortho")
    return scipy.fft.idctn(c / symbol(*rhs.shape, tau, mu), type=2, norm="ortho")


def _vec(f, x, *args):
    return np.array([f(v, *args) for v in np.ravel(x)]).reshape(np.shape(x))


def rhs(psi, g, w1, w2, b1, b2, p: Params):
    """F of Eq. (37) with the Neumann divergence (v from the pinned window sum)."""
    psi, g = _f64(psi), _f64(g)
    w1, w2, b1, b2 = (_f64(a) for a in (w1, w2, b1, b2))
    v1, v2 = repulsion(psi, w1, w2, p)
    nw = np.hypot(w1, w2)
    force = (-p.gamma * g * nw * _vec(delta_prime, psi, p.eps)
             + p.alpha * g * _vec(delta, psi, p.eps)
             + 2.0 * p.beta * _vec(band_prime, psi, p.eps, p.band_l) * (w1 * v1 + w2 * v2)
             + p.mu * div(b1 - w1, b2 - w2))
    return psi + p.tau * force


def phi_step(psi, g, w1, w2, b1, b2, p: Params):
    return solve(rhs(psi, g, w1, w2, b1, b2, p), p.tau, p.mu)


def w_b_update(phi1, g, w1, w2, b1, b2, p: Params):
    """Eqs. (41), (42), (40), (23) with the Neumann forward differences."""
    phi1, g = _f64(phi1), _f64(g)
    w1, w2, b1, b2 = (_f64(a) for a in (w1, w2, b1, b2))
    v1, v2 = repulsion(phi1, w1, w2, p)
    d1, d2 = grad(phi1)
    h = _vec(band, phi1, p.eps, p.band_l)
    B1 = d1 + b1 + (2.0 * p.beta / p.mu) * h * v1
    B2 = d2 + b2 + (2.0 * p.beta / p.mu) * h * v2
    t = (p.gamma / p.mu) * g * _vec(delta, phi1, p.eps)
    n1 = np.empty_like(B1)
    n2 = np.empty_like(B2)
    for idx in np.ndindex(B1.shape):
        s1, s2 = soft_threshold(B1[idx], B2[idx], t[idx])
        n = np.hypot(s1, s2)
        n1[idx], n2[idx] = (s1 / n, s2 / n) if n > 0.0 else (0.0, 0.0)
    return n1, n2, b1 + d1 - n1, b2 + d2 - n2
