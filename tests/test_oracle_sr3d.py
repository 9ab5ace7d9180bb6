"""Pins of the volume (3-D) oracle: the solve against a dense solve, the
window sum against a brute force over voxel pairs and against the pinned 2-D
window sum on z-constant fields, the 3-vector shrink against its closed
cases, and a whole outer iteration that reduces to the 2-D oracle on
z-constant volumes."""
import numpy as np
import pytest

import oracle
from oracle import Params
from oracle import sr3d


def test_solve_matches_a_dense_solve():
    Z, M, N = 3, 4, 5
    tau, mu = 0.1, 8.0
    P = Z * M * N

    def lap(x):
        return sum(np.roll(x, 1, a) + np.roll(x, -1, a) - 2 * x for a in range(3))
    A = np.zeros((P, P))
    for k in range(P):
        e = np.zeros(P)
        e[k] = 1.0
        A[:, k] = e - tau * mu * lap(e.reshape(Z, M, N)).ravel()
    rhs = np.random.default_rng(0).normal(size=(Z, M, N))
    ref = np.linalg.solve(A, rhs.ravel()).reshape(Z, M, N)
    assert np.allclose(sr3d.solve(rhs, tau, mu), ref, atol=1e-12)


def test_window_sum_matches_brute_force(oracle_lib):
    rng = np.random.default_rng(1)
    shape = (4, 5, 6)
    phi = rng.uniform(-1.5, 1.5, shape)
    w = tuple(rng.normal(size=shape) for _ in range(3))
    p = Params(R=1, d=1.5)
    v = sr3d.window_sum(phi, w, p)
    h = np.vectorize(lambda x: oracle.band(x, p.eps, p.band_l))(phi)
    ref = [np.zeros(shape) for _ in range(3)]
    for x in np.ndindex(shape):
        for y in np.ndindex(shape):
            dz, dy, dx = (y[0] - x[0], y[1] - x[1], y[2] - x[2])
            if max(abs(dz), abs(dy), abs(dx)) <= p.R:
                k = np.exp(-(dz * dz + dy * dy + dx * dx) / p.d ** 2)
                for c in range(3):
                    ref[c][x] += k * h[y] * w[c][y]
    for a, r in zip(v, ref):
        assert np.allclose(a, r, atol=1e-12)


def test_window_sum_on_z_constant_fields_scales_the_2d_sum(oracle_lib):
    rng = np.random.default_rng(2)
    Z, M, N = 9, 12, 10
    phi2 = rng.uniform(-2, 2, (M, N))
    w1, w2 = rng.normal(size=(2, M, N))
    p = Params(R=3, d=3.0)
    rep = lambda a: np.repeat(a[None], Z, axis=0)  # noqa: E731
    v = sr3d.window_sum(rep(phi2), (rep(w1), rep(w2), np.zeros((Z, M, N))), p)
    v1, v2 = oracle.repulsion(phi2, w1, w2, p)
    for z in range(Z):
        kz = sum(np.exp(-dz * dz / p.d ** 2) for dz in range(-p.R, p.R + 1) if 0 <= z + dz < Z)
        assert np.allclose(v[0][z], kz * v1, atol=1e-12)
        assert np.allclose(v[1][z], kz * v2, atol=1e-12)
        assert np.allclose(v[2][z], 0.0)


def test_shrink_closed_cases():
    B = (np.array([3.0, 0.0, 0.3]), np.array([4.0, 0.0, 0.0]), np.array([0.0, 0.0, 0.4]))
    s = sr3d.shrink(B, np.array([2.5, 1.0, 0.6]))
    assert np.allclose([s[0][0], s[1][0], s[2][0]], [1.5, 2.0, 0.0])   # |B| = 5 -> 2.5
    assert s[0][1] == 0.0 and s[1][1] == 0.0                           # B = 0 -> 0
    assert np.allclose([s[0][2], s[2][2]], [0.0, 0.0])                 # |B| = 0.5 <= t


def test_outer_iteration_reduces_to_2d_on_z_constant_volumes(oracle_lib):
    """beta = 0 (the window sum is the only term that sees the volume's
    extent in z): every slice follows the pinned 2-D Alg. 1."""
    from paper_2003_12693_gb300 import synth
    phi, w1, w2, b1, b2, g = synth.random_state(16, 12, seed=4)
    Z = 3
    p = Params(R=2, d=2.0, beta=0.0, S=2)
    rep = lambda a: np.repeat(a[None], Z, axis=0)  # noqa: E731
    zero = np.zeros((Z,) + phi.shape)
    phi3, w3, b3 = sr3d.outer_iteration(rep(phi), rep(g), (zero, rep(w1), rep(w2)),
                                        (zero, rep(b1), rep(b2)), p)
    st = oracle.State(phi.copy(), w1.copy(), w2.copy(), b1.copy(), b2.copy())
    oracle.iterate(st, g, 1, p)
    for z in range(Z):
        assert np.allclose(phi3[z], st.phi, atol=1e-10)
        assert np.allclose(w3[1][z], st.w1, atol=1e-9) and np.allclose(w3[2][z], st.w2, atol=1e-9)
        assert np.allclose(b3[1][z], st.b1, atol=1e-9) and np.allclose(b3[2][z], st.b2, atol=1e-9)
        assert np.allclose(w3[0][z], 0.0) and np.allclose(b3[0][z], 0.0)
