"""FP64 oracle of the Split Bregman SR iteration on volumes (the 3-D use of
Fig. 6).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).  The CUDA path's
version (include/sr3.h, sr3.cu) is checked against it by tests/test_gpu_sr3.py.

The method is the 2-D one with a third axis everywhere, under the same
readings: periodic forward differences (Eq. (35)) and backward divergence
(Eq. (36)); the window sum of Eq. (38) over the cube |p|, |q|, |r| <= R with
the separable weight exp(-(p^2 + q^2 + r^2) / d^2), terms outside the volume
dropped; Eq. (37) with the 3-D Laplacian, solved by the 3-D FFT with the
symbol 1 + tau mu sum_a 4 sin^2(pi l_a / n_a) (Eq. (32) with a third term);
Eqs. (41), (42), (40), (23) on 3-vectors.  Arrays are (Z, M, N); w and b are
tuples of three arrays.  Scalar functions come from the pinned C oracle.
"""
from __future__ import annotations

import numpy as np

from . import Params, band, band_prime, delta, delta_prime


def _vec(f, x, *args):
    return np.array([f(v, *args) for v in np.ravel(x)]).reshape(np.shape(x))


def grad(phi):
    return tuple(np.roll(phi, -1, axis=a) - phi for a in range(3))


def div(a):
    return sum(a[k] - np.roll(a[k], 1, axis=k) for k in range(3))


def window_sum(phi, w, p: Params):
    """v = sum over the cube of exp(-(p^2+q^2+r^2)/d^2) h(phi) w at the
    shifted voxel, terms outside the volume dropped (direct triple sum)."""
    h = _vec(band, phi, p.eps, p.band_l)
    u = [h * wk for wk in w]
    Z, M, N = phi.shape
    R = p.R
    v = [np.zeros_like(phi) for _ in range(3)]
    pad = [np.pad(uk, R) for uk in u]
    for dz in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                k = np.exp(-(dz * dz + dy * dy + dx * dx) / (p.d * p.d))
                for c in range(3):
                    v[c] += k * pad[c][R + dz:R + dz + Z, R + dy:R + dy + M, R + dx:R + dx + N]
    return tuple(v)


def symbol(shape, tau, mu):
    Z, M, N = shape
    lz = np.arange(Z)[:, None, None]
    lm = np.arange(M)[None, :, None]
    ln = np.arange(N)[None, None, :]
    return 1.0 + tau * mu * 4.0 * (np.sin(np.pi * lz / Z) ** 2 + np.sin(np.pi * lm / M) ** 2 +
                                   np.sin(np.pi * ln / N) ** 2)


def solve(rhs, tau, mu):
    """(1 - tau mu Lap) phi = rhs, periodic, by the 3-D FFT."""
    return np.real(np.fft.ifftn(np.fft.fftn(rhs) / symbol(rhs.shape, tau, mu)))


def rhs(psi, g, w, b, p: Params):
    v = window_sum(psi, w, p)
    nw = np.sqrt(sum(wk * wk for wk in w))
    wv = sum(wk * vk for wk, vk in zip(w, v))
    force = (-p.gamma * g * nw * _vec(delta_prime, psi, p.eps)
             + p.alpha * g * _vec(delta, psi, p.eps)
             + 2.0 * p.beta * _vec(band_prime, psi, p.eps, p.band_l) * wv
             + p.mu * div(tuple(bk - wk for bk, wk in zip(b, w))))
    return psi + p.tau * force


def phi_step(psi, g, w, b, p: Params):
    return solve(rhs(psi, g, w, b, p), p.tau, p.mu)


def shrink(B, t):
    """Eq. (42) on 3-vectors: max(|B| - t, 0) B / |B|, zero for B = 0."""
    n = np.sqrt(sum(Bk * Bk for Bk in B))
    scale = np.where(n > 0.0, np.maximum(n - t, 0.0) / np.where(n > 0.0, n, 1.0), 0.0)
    return tuple(scale * Bk for Bk in B)


def w_b_update(phi1, g, w, b, p: Params):
    v = window_sum(phi1, w, p)
    d = grad(phi1)
    h = _vec(band, phi1, p.eps, p.band_l)
    B = tuple(dk + bk + (2.0 * p.beta / p.mu) * h * vk for dk, bk, vk in zip(d, b, v))
    t = (p.gamma / p.mu) * g * _vec(delta, phi1, p.eps)
    s = shrink(B, t)
    n = np.sqrt(sum(sk * sk for sk in s))
    wn = tuple(np.where(n > 0.0, sk / np.where(n > 0.0, n, 1.0), 0.0) for sk in s)
    bn = tuple(bk + dk - wk for bk, dk, wk in zip(b, d, wn))
    return wn, bn


def outer_iteration(phi, g, w, b, p: Params):
    """One outer iteration of Alg. 1 on a volume; returns (phi, w, b)."""
    psi = phi
    for _ in range(p.S):
        psi = phi_step(psi, g, w, b, p)
    wn, bn = w_b_update(psi, g, w, b, p)
    return psi, wn, bn
