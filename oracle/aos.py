"""FP64 oracle of the AOS solve of the phi sub-problem (the alternative the
paper mentions at the end of Sec. 4).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).  The CUDA path's
version (sr_aos.cu) is checked against it by tests/test_gpu_aos.py.

The semi-implicit step (1 - tau mu Lap) phi = F of Eqs. (30)-(33) is replaced
by additive operator splitting in the form of Eqs. (19)-(20): with A_1, A_2
the constant one-dimensional second differences along the rows' and the
columns' direction (periodic, as the default reading of the boundary),

    phi = 1/2 [ (I - 2 tau mu A_1)^{-1} F + (I - 2 tau mu A_2)^{-1} F ].

Each factor is a cyclic tridiagonal system per column (A_1) or per row (A_2)
whose matrix is the same for every line and every iteration, so it is
factorised once.  Here each line is solved by LU of the plain tridiagonal
part (the Thomas recursion, written out) with the two wrap-around corners
handled by the Sherman-Morrison formula.
"""
from __future__ import annotations

import numpy as np


def _thomas(a, b, c, d):
    """Solve the tridiagonal system with sub-diagonal a[1:], diagonal b,
    super-diagonal c[:-1] for every column of d (axis 0 is the line)."""
    n = b.shape[0]
    cp = np.empty(n)
    dp = np.empty_like(d)
    cp[0] = c[0] / b[0]
    dp[0] = d[0] / b[0]
    for i in range(1, n):
        m = b[i] - a[i] * cp[i - 1]
        cp[i] = c[i] / m if i < n - 1 else 0.0
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m
    x = np.empty_like(d)
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def solve_cyclic(n, off, diag, d):
    """(diag on the diagonal, off on both neighbours, off in the two wrap
    corners) x = d, along axis 0 of d, by Sherman-Morrison on the Thomas
    solve: the cyclic matrix is T + u v^T with u = (gamma, 0, ..., 0, off),
    v = (1, 0, ..., 0, off / gamma)."""
    if n == 1:
        return d / (diag + 2.0 * off)
    if n == 2:
        A = np.array([[diag, 2.0 * off], [2.0 * off, diag]])
        return np.linalg.solve(A, d.reshape(2, -1)).reshape(d.shape)
    gamma = -diag
    a = np.full(n, off)
    c = np.full(n, off)
    b = np.full(n, diag)
    b[0] = diag - gamma
    b[-1] = diag - off * off / gamma
    u = np.zeros((n,) + (1,) * (d.ndim - 1))
    u[0] = gamma
    u[-1] = off
    y = _thomas(a, b, c, d)
    z = _thomas(a, b, c, u)
    vy = y[0] + (off / gamma) * y[-1]
    vz = z[0] + (off / gamma) * z[-1]
    return y - z * (vy / (1.0 + vz))


def solve(rhs, tau, mu):
    """The AOS step for (1 - tau mu Lap) phi = rhs."""
    rhs = np.asarray(rhs, dtype=np.float64)
    M, N = rhs.shape
    k = 2.0 * tau * mu
    v = solve_cyclic(M, -k, 1.0 + 2.0 * k, rhs)              # along axis 0 (A_1)
    w = solve_cyclic(N, -k, 1.0 + 2.0 * k, rhs.T).T          # along axis 1 (A_2)
    return 0.5 * (v + w)
