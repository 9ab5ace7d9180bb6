"""Pins of the AOS oracle: each directional solve against a dense solve of
its cyclic tridiagonal matrix, the splitting formula itself, constants, and
first-order agreement with the exact (FFT) solve of Eqs. (31)-(33) as
tau -> 0."""
import numpy as np
import pytest

import oracle
from oracle import aos


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 31])
def test_cyclic_solve_matches_dense(n):
    rng = np.random.default_rng(n)
    d = rng.normal(size=(n, 4))
    k = 1.6
    A = np.diag(np.full(n, 1.0 + 2.0 * k))
    for i in range(n):
        A[i, (i + 1) % n] += -k
        A[i, (i - 1) % n] += -k
    x = aos.solve_cyclic(n, -k, 1.0 + 2.0 * k, d)
    assert np.allclose(A @ x, d, atol=1e-11)


def test_aos_step_is_the_mean_of_the_two_directional_solves():
    rng = np.random.default_rng(2)
    F = rng.normal(size=(6, 7))
    tau, mu = 0.1, 8.0
    k = 2 * tau * mu

    def lap1d(n):
        A = -2.0 * np.eye(n)
        for i in range(n):
            A[i, (i + 1) % n] += 1.0
            A[i, (i - 1) % n] += 1.0
        return A
    v = np.linalg.solve(np.eye(6) - k * lap1d(6), F)
    w = np.linalg.solve(np.eye(7) - k * lap1d(7), F.T).T
    assert np.allclose(aos.solve(F, tau, mu), 0.5 * (v + w), atol=1e-12)


def test_constants_are_preserved():
    assert np.allclose(aos.solve(np.full((8, 5), 2.5), 0.1, 8.0), 2.5)


def test_splitting_error_vanishes_to_second_order(oracle_lib):
    """AOS and the exact solve agree to O((tau mu)^2) on a smooth field."""
    i = np.arange(32)[:, None]
    j = np.arange(32)[None, :]
    F = np.sin(2 * np.pi * i / 32) * np.cos(4 * np.pi * j / 32) + 0.3 * np.cos(2 * np.pi * j / 32)
    errs = []
    for tau in (0.04, 0.02, 0.01):
        errs.append(np.abs(aos.solve(F, tau, 8.0) - oracle.solve(F, tau, 8.0)).max())
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0
