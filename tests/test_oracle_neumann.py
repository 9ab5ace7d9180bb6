"""Pins of the Neumann-boundary oracle (the variant that reads Eq. (27)
literally) against what the mathematics fixes: the adjoint pair, a dense
solve, the DCT eigenvectors, conservation, and agreement with the pinned
periodic oracle wherever the boundary plays no part."""
import numpy as np
import pytest

import oracle
from oracle import Params
from oracle import neumann as nm


def test_divergence_is_minus_the_adjoint_of_the_gradient():
    rng = np.random.default_rng(0)
    phi = rng.normal(size=(7, 9))
    a1, a2 = rng.normal(size=(2, 7, 9))
    d1, d2 = nm.grad(phi)
    assert abs(np.vdot(d1, a1) + np.vdot(d2, a2) + np.vdot(phi, nm.div(a1, a2))) < 1e-12
    assert np.all(d1[-1] == 0) and np.all(d2[:, -1] == 0)


def test_laplacian_is_the_reflective_stencil_and_conserves_mass():
    rng = np.random.default_rng(1)
    phi = rng.normal(size=(6, 5))
    lap = nm.laplacian(phi)
    pad = np.pad(phi, 1, mode="edge")          # reflective: the ghost equals the edge value
    ref = pad[2:, 1:-1] + pad[:-2, 1:-1] + pad[1:-1, 2:] + pad[1:-1, :-2] - 4 * phi
    assert np.allclose(lap, ref, atol=1e-13)
    assert abs(lap.sum()) < 1e-12
    assert np.allclose(nm.laplacian(np.full((4, 4), 3.0)), 0.0)


@pytest.mark.parametrize("shape", [(8, 8), (6, 9), (5, 7)])
def test_solve_matches_a_dense_solve(shape):
    M, N = shape
    tau, mu = 0.1, 8.0
    P = M * N
    A = np.zeros((P, P))
    for k in range(P):
        e = np.zeros(P)
        e[k] = 1.0
        A[:, k] = e - tau * mu * nm.laplacian(e.reshape(M, N)).ravel()
    rhs = np.random.default_rng(M * N).normal(size=(M, N))
    ref = np.linalg.solve(A, rhs.ravel()).reshape(M, N)
    assert np.allclose(nm.solve(rhs, tau, mu), ref, atol=1e-12)


def test_dct_basis_functions_are_eigenvectors():
    M, N = 8, 6
    i = np.arange(M)[:, None] + 0.5
    j = np.arange(N)[None, :] + 0.5
    sym = nm.symbol(M, N, 0.1, 8.0)
    for k, l in [(0, 0), (1, 0), (3, 2), (7, 5)]:
        v = np.cos(np.pi * k * i / M) * np.cos(np.pi * l * j / N)
        assert np.allclose(v - 0.8 * nm.laplacian(v), sym[k, l] * v, atol=1e-12)
        assert np.allclose(nm.solve(v, 0.1, 8.0), v / sym[k, l], atol=1e-12)


def _interior_state(M=40, N=36, seed=3):
    """Fields that vanish within 10 px of the border (phi constant there)."""
    rng = np.random.default_rng(seed)
    mask = np.zeros((M, N))
    mask[10:-10, 10:-10] = 1.0
    phi = 3.0 + mask * rng.normal(size=(M, N))
    w1, w2, b1, b2 = (mask * rng.normal(size=(M, N)) for _ in range(4))
    g = 1.0 / (1.0 + rng.uniform(0, 1, (M, N)))
    return phi, g, w1, w2, b1, b2


def test_rhs_and_w_update_match_the_periodic_oracle_away_from_the_border(oracle_lib):
    """With every field constant near the border, no difference crosses it,
    so the Neumann and periodic operators coincide (the periodic oracle is
    pinned elsewhere): a dropped term or a sign error would show here."""
    phi, g, w1, w2, b1, b2 = _interior_state()
    p = Params(R=3, d=3.0)
    v1, v2 = oracle.repulsion(phi, w1, w2, p)
    Fp = oracle.rhs(phi, g, w1, w2, b1, b2, v1, v2, p)
    Fn = nm.rhs(phi, g, w1, w2, b1, b2, p)
    assert np.allclose(Fn, Fp, atol=1e-12)
    a = nm.w_b_update(phi, g, w1, w2, b1, b2, p)
    r = oracle.w_b_update(phi, g, w1, w2, b1, b2, p)
    for x, y in zip(a, r):
        assert np.allclose(x, y, atol=1e-12)


def test_constant_level_set_is_a_fixed_point_of_the_solve():
    c = np.full((12, 10), -2.5)
    assert np.allclose(nm.solve(c, 0.1, 8.0), c)
