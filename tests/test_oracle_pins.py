"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle routine against something other than itself: a
closed form, a finite-difference derivative, a library routine (numpy's FFT),
a dense direct solve, a brute-force double sum over all pixel pairs, the
numerical minimiser of the pointwise w sub-problem, or the gradient of the
discrete energy.  None of them re-types the routine's own formula.
"""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
from oracle import Params

EPS_SET = [0.5, 1.0, 2.0]


# --------------------------------------------------------------------------
# Scalar functions, Eqs. (5), (6), (11), (28), (29)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("eps", EPS_SET)
def test_heaviside_special_values_and_limits(oracle_lib, eps):
    assert oracle.heaviside(0.0, eps) == pytest.approx(0.5, abs=1e-15)
    assert oracle.heaviside(eps, eps) == pytest.approx(1.0, abs=1e-15)
    assert oracle.heaviside(-eps, eps) == pytest.approx(0.0, abs=1e-15)
    assert oracle.heaviside(3 * eps, eps) == 1.0
    assert oracle.heaviside(-3 * eps, eps) == 0.0
    # odd symmetry about 1/2: H(x) + H(-x) = 1
    for x in np.linspace(-2 * eps, 2 * eps, 41):
        assert oracle.heaviside(x, eps) + oracle.heaviside(-x, eps) == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("eps", EPS_SET)
def test_delta_is_derivative_of_heaviside(oracle_lib, eps):
    hstep = 1e-5
    for x in np.linspace(-1.5 * eps, 1.5 * eps, 61):
        fd = (oracle.heaviside(x + hstep, eps) - oracle.heaviside(x - hstep, eps)) / (2 * hstep)
        assert oracle.delta(x, eps) == pytest.approx(fd, abs=1e-8)


@pytest.mark.parametrize("eps", EPS_SET)
def test_delta_prime_is_derivative_of_delta(oracle_lib, eps):
    hstep = 1e-5
    for x in np.linspace(-1.5 * eps, 1.5 * eps, 61):
        if abs(abs(x) - eps) < 1e-9:
            continue  # delta'' jumps at |phi| = eps; the central difference is O(h) there
        fd = (oracle.delta(x + hstep, eps) - oracle.delta(x - hstep, eps)) / (2 * hstep)
        assert oracle.delta_prime(x, eps) == pytest.approx(fd, abs=1e-7 / eps ** 3)


@pytest.mark.parametrize("eps", EPS_SET)
def test_delta_unit_mass_and_support(oracle_lib, eps):
    xs = np.linspace(-eps, eps, 20001)
    vals = np.array([oracle.delta(x, eps) for x in xs])
    assert np.trapezoid(vals, xs) == pytest.approx(1.0, abs=1e-7)
    assert oracle.delta(1.0001 * eps, eps) == 0.0
    assert oracle.delta(0.0, eps) == pytest.approx(1.0 / eps)


@pytest.mark.parametrize("eps,l", [(1.0, 1.0), (0.5, 1.0), (1.0, 2.0), (1.0, 0.5)])
def test_band_and_its_derivative(oracle_lib, eps, l):
    hstep = 1e-5
    for x in np.linspace(-(l + 2 * eps), l + 2 * eps, 81):
        fd = (oracle.band(x + hstep, eps, l) - oracle.band(x - hstep, eps, l)) / (2 * hstep)
        assert oracle.band_prime(x, eps, l) == pytest.approx(fd, abs=1e-8)
        if abs(x) >= l + eps:
            # zero up to the rounding of sin(pi) at the support edge
            assert abs(oracle.band(x, eps, l)) < 1e-15
    # for l >= eps the band is exactly 1 on |phi| <= l - eps, in particular at phi = 0
    if l >= eps:
        assert oracle.band(0.0, eps, l) == pytest.approx(1.0, abs=1e-15)
        assert oracle.band(l - eps, eps, l) == pytest.approx(1.0, abs=1e-15)
    # symmetric profile
    for x in np.linspace(0, l + eps, 17):
        assert oracle.band(x, eps, l) == pytest.approx(oracle.band(-x, eps, l), abs=1e-15)


# --------------------------------------------------------------------------
# Edge detector, Eq. (1)
# --------------------------------------------------------------------------

def test_edge_constant_image_gives_one(oracle_lib):
    g = oracle.edge(np.full((20, 17), 0.37), rho=2.0, sigma=1.0, s_pow=2)
    assert np.abs(g - 1.0).max() < 1e-14


@pytest.mark.parametrize("s_pow", [1, 2])
@pytest.mark.parametrize("axis", [0, 1])
def test_edge_linear_ramp(oracle_lib, s_pow, axis):
    """A ramp of slope a is unchanged by a normalised symmetric blur away from the
    border, and its central difference is exactly a: g = 1/(1 + rho |a|^s)."""
    a, rho, H, W = 0.35, 1.7, 24, 30
    i, j = np.mgrid[0:H, 0:W].astype(float)
    f = a * (i if axis == 0 else j) + 0.2
    g = oracle.edge(f, rho=rho, sigma=1.0, s_pow=s_pow)
    r = 3 + 1
    inner = g[r:H - r, r:W - r]
    assert np.abs(inner - 1.0 / (1.0 + rho * a ** s_pow)).max() < 1e-13


def test_edge_without_blur_uses_central_and_one_sided_differences(oracle_lib):
    """sigma = 0: numpy.gradient (library) gives the same finite differences."""
    rng = np.random.default_rng(3)
    f = rng.normal(size=(11, 13))
    g = oracle.edge(f, rho=0.8, sigma=0.0, s_pow=2)
    gi, gj = np.gradient(f)
    assert np.abs(g - 1.0 / (1.0 + 0.8 * (gi ** 2 + gj ** 2))).max() < 1e-14


def test_edge_blur_matches_library_gaussian(oracle_lib):
    """scipy.ndimage.correlate1d with the sampled, normalised kernel and 'nearest'
    border gives the same blurred image; g then follows from numpy.gradient."""
    from scipy import ndimage
    rng = np.random.default_rng(4)
    f = rng.normal(size=(19, 23))
    sigma = 1.3
    r = math.ceil(3 * sigma)
    t = np.arange(-r, r + 1)
    k = np.exp(-t * t / (2 * sigma * sigma))
    k /= k.sum()
    fb = ndimage.correlate1d(ndimage.correlate1d(f, k, axis=0, mode="nearest"), k, axis=1,
                             mode="nearest")
    gi, gj = np.gradient(fb)
    ref = 1.0 / (1.0 + 1.0 * np.sqrt(gi ** 2 + gj ** 2) ** 1)
    g = oracle.edge(f, rho=1.0, sigma=sigma, s_pow=1)
    assert np.abs(g - ref).max() < 1e-13


# --------------------------------------------------------------------------
# Discrete operators, Eqs. (35)-(36)
# --------------------------------------------------------------------------

def test_divergence_is_negative_adjoint_of_gradient(oracle_lib):
    """Summation by parts on the periodic grid: <div a, phi> = -<a, grad phi>."""
    rng = np.random.default_rng(5)
    M, N = 9, 14
    phi, a1, a2 = rng.normal(size=(3, M, N))
    d1, d2 = oracle.grad(phi)
    lhs = np.sum(oracle.div(a1, a2) * phi)
    rhs = -np.sum(a1 * d1 + a2 * d2)
    assert lhs == pytest.approx(rhs, rel=1e-13, abs=1e-12)


def test_div_grad_is_five_point_laplacian(oracle_lib):
    rng = np.random.default_rng(6)
    phi = rng.normal(size=(10, 7))
    lap = sum(np.roll(phi, s, ax) for s in (1, -1) for ax in (0, 1)) - 4 * phi
    d1, d2 = oracle.grad(phi)
    assert np.abs(oracle.div(d1, d2) - lap).max() < 1e-13


def test_gradient_of_ramp(oracle_lib):
    i, j = np.mgrid[0:8, 0:9].astype(float)
    d1, d2 = oracle.grad(2.5 * i - 0.5 * j)
    assert np.allclose(d1[:-1], 2.5) and np.allclose(d2[:, :-1], -0.5)
    # periodic wrap at the last row / column
    assert np.allclose(d1[-1], -2.5 * 7) and np.allclose(d2[:, -1], 0.5 * 8)


# --------------------------------------------------------------------------
# FFT and the phi solve, Eqs. (31)-(33)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", list(range(1, 70)) + [32 * m for m in range(2, 33)])
def test_fft1_matches_numpy(oracle_lib, n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    ref = np.fft.fft(x)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(oracle.fft1(x, -1) - ref).max() / scale < 1e-12
    assert np.abs(oracle.fft1(x, +1) - np.fft.ifft(x) * n).max() / scale < 1e-12


@pytest.mark.parametrize("shape", [(8, 8), (8, 6), (7, 5), (64, 96), (96, 992), (128, 128)])
def test_fft2_matches_numpy(oracle_lib, shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    ref = np.fft.fft2(x)
    assert np.abs(oracle.fft2(x, -1) - ref).max() / np.abs(ref).max() < 1e-12


def _periodic_second_difference(n):
    D = -2.0 * np.eye(n)
    for k in range(n):
        D[k, (k + 1) % n] += 1.0
        D[k, (k - 1) % n] += 1.0
    return D


@pytest.mark.parametrize("shape", [(8, 8), (8, 6), (5, 7)])
def test_solve_matches_dense_direct_solve(oracle_lib, shape):
    """(I - tau mu Laplacian_periodic) phi = F solved by dense LU (numpy)."""
    M, N = shape
    tau, mu = 0.1, 8.0
    lap = np.kron(_periodic_second_difference(M), np.eye(N)) + \
        np.kron(np.eye(M), _periodic_second_difference(N))
    A = np.eye(M * N) - tau * mu * lap
    rng = np.random.default_rng(M * 100 + N)
    F = rng.normal(size=(M, N))
    ref = np.linalg.solve(A, F.ravel()).reshape(M, N)
    assert np.abs(oracle.solve(F, tau, mu) - ref).max() < 1e-12


def test_solve_eigenfunction_and_constant(oracle_lib):
    """cos(2 pi (a i/M + b j/N)) is an eigenfunction of the periodic 5-point
    Laplacian with eigenvalue -4 sin^2(pi a/M) - 4 sin^2(pi b/N)."""
    M, N, tau, mu = 16, 12, 0.1, 8.0
    i, j = np.mgrid[0:M, 0:N].astype(float)
    for a, b in [(0, 0), (1, 0), (0, 5), (3, 4), (8, 6), (15, 11)]:
        F = np.cos(2 * np.pi * (a * i / M + b * j / N))
        lam = 1.0 + tau * mu * (4 * np.sin(np.pi * a / M) ** 2 + 4 * np.sin(np.pi * b / N) ** 2)
        assert np.abs(oracle.solve(F, tau, mu) - F / lam).max() < 1e-13
    assert np.abs(oracle.solve(np.full((M, N), 2.5), tau, mu) - 2.5).max() < 1e-13


# --------------------------------------------------------------------------
# Repulsion field (Sec. 4 window sum)
# --------------------------------------------------------------------------

def _brute_force_v(phi, w1, w2, R, d, eps, l):
    """O(P^2) sum over every pair (x, y) of the image: weight
    exp(-|x-y|^2/d^2) restricted to the (2R+1)^2 window."""
    M, N = phi.shape
    hb = np.vectorize(lambda x: oracle.band(x, eps, l))(phi)
    ys = [(a, b) for a in range(M) for b in range(N)]
    v1, v2 = np.zeros_like(phi), np.zeros_like(phi)
    for x1 in range(M):
        for x2 in range(N):
            s1 = s2 = 0.0
            for y1, y2 in ys:
                if abs(x1 - y1) <= R and abs(x2 - y2) <= R:
                    k = math.exp(-((x1 - y1) ** 2 + (x2 - y2) ** 2) / d ** 2)
                    s1 += k * w1[y1, y2] * hb[y1, y2]
                    s2 += k * w2[y1, y2] * hb[y1, y2]
            v1[x1, x2], v2[x1, x2] = s1, s2
    return v1, v2


@pytest.mark.parametrize("shape,R,d", [((9, 9), 3, 3.0), ((12, 16), 4, 4.0), ((16, 13), 2, 5.0)])
def test_repulsion_matches_brute_force(oracle_lib, shape, R, d):
    from paper_2003_12693_gb300.synth import random_state
    phi, w1, w2, _, _, _ = random_state(*shape, seed=11, phi_scale=2.5)
    p = Params(R=R, d=d)
    v1, v2 = oracle.repulsion(phi, w1, w2, p)
    r1, r2 = _brute_force_v(phi, w1, w2, R, d, p.eps, p.band_l)
    assert np.abs(v1 - r1).max() < 1e-12 and np.abs(v2 - r2).max() < 1e-12


@pytest.mark.parametrize("R,d", [(3, 3.0), (4, 4.0), (8, 8.0), (2, 5.0)])
def test_repulsion_closed_form_on_the_band(oracle_lib, R, d):
    """phi = 0, w = (1, 0): h = 1, so interior v1 = (sum_p e^{-p^2/d^2})^2 and a
    corner keeps one quadrant, (sum_{p>=0} e^{-p^2/d^2})^2."""
    M = N = 2 * R + 9
    p = Params(R=R, d=d)
    phi = np.zeros((M, N))
    v1, v2 = oracle.repulsion(phi, np.ones((M, N)), np.zeros((M, N)), p)
    s_full = sum(math.exp(-q * q / d ** 2) for q in range(-R, R + 1))
    s_half = sum(math.exp(-q * q / d ** 2) for q in range(0, R + 1))
    assert v1[M // 2, N // 2] == pytest.approx(s_full ** 2, rel=1e-14)
    assert v1[0, 0] == pytest.approx(s_half ** 2, rel=1e-14)
    assert np.abs(v2).max() == 0.0
    # outside the band (|phi| >= l + eps) nothing repels
    v1, _ = oracle.repulsion(np.full((M, N), 2.0), np.ones((M, N)), np.zeros((M, N)), p)
    assert np.abs(v1).max() == 0.0


# --------------------------------------------------------------------------
# Right-hand side F of Eq. (37): gradient of the split energy
# --------------------------------------------------------------------------

def _split_energy(phi, g, w1, w2, b1, b2, p):
    """E(phi, w) of Eq. (22) discretised with the Sec. 4 operators: geodesic,
    area, windowed repulsion (both orderings of each pair) and the splitting
    penalty mu/2 |w - grad phi - b|^2 with forward differences."""
    M, N = phi.shape
    H = np.vectorize(lambda x: oracle.heaviside(x, p.eps))(phi)
    D = np.vectorize(lambda x: oracle.delta(x, p.eps))(phi)
    hb = np.vectorize(lambda x: oracle.band(x, p.eps, p.band_l))(phi)
    Eg = np.sum(g * np.sqrt(w1 ** 2 + w2 ** 2) * D)
    Ea = np.sum(g * (1.0 - H))
    Er = 0.0
    for q1 in range(-p.R, p.R + 1):
        for q2 in range(-p.R, p.R + 1):
            k = math.exp(-(q1 * q1 + q2 * q2) / p.d ** 2)
            # pairs (x, x + q) with both points inside the image
            xs1 = slice(max(0, -q1), min(M, M - q1))
            xs2 = slice(max(0, -q2), min(N, N - q2))
            ys1 = slice(max(0, q1), min(M, M + q1))
            ys2 = slice(max(0, q2), min(N, N + q2))
            Er -= k * np.sum((w1[xs1, xs2] * w1[ys1, ys2] + w2[xs1, xs2] * w2[ys1, ys2]) *
                             hb[xs1, xs2] * hb[ys1, ys2])
    d1 = np.roll(phi, -1, 0) - phi
    d2 = np.roll(phi, -1, 1) - phi
    Emu = 0.5 * p.mu * np.sum((w1 - d1 - b1) ** 2 + (w2 - d2 - b2) ** 2)
    return p.gamma * Eg + p.alpha * Ea + p.beta * Er + Emu


def test_rhs_is_descent_direction_of_split_energy(oracle_lib):
    """(F - psi)/tau + mu Lap psi = -dE/dphi: Eq. (26) is the gradient flow of
    Eq. (24).  Checked by central finite differences of the energy."""
    from paper_2003_12693_gb300.synth import random_state
    M, N = 12, 11
    phi, w1, w2, b1, b2, g = random_state(M, N, seed=21, phi_scale=2.0)
    p = Params(alpha=4.0, beta=0.7, gamma=3.0, mu=8.0, tau=0.1, R=3, d=3.0)
    v1, v2 = oracle.repulsion(phi, w1, w2, p)
    F = oracle.rhs(phi, g, w1, w2, b1, b2, v1, v2, p)
    lap = sum(np.roll(phi, s, ax) for s in (1, -1) for ax in (0, 1)) - 4 * phi
    descent = (F - phi) / p.tau + p.mu * lap
    hstep = 1e-6
    rng = np.random.default_rng(0)
    # avoid the kinks of delta'' at |phi| = eps and of h'' at |phi +- l| = eps
    for _ in range(30):
        i, j = int(rng.integers(M)), int(rng.integers(N))
        x = phi[i, j]
        if min(abs(abs(x) - p.eps), abs(abs(x - p.band_l) - p.eps),
               abs(abs(x + p.band_l) - p.eps)) < 1e-3:
            continue
        e = np.zeros_like(phi)
        e[i, j] = hstep
        fd = (_split_energy(phi + e, g, w1, w2, b1, b2, p) -
              _split_energy(phi - e, g, w1, w2, b1, b2, p)) / (2 * hstep)
        assert descent[i, j] == pytest.approx(-fd, abs=2e-5 * max(1.0, abs(fd)))


# --------------------------------------------------------------------------
# w sub-problem, Eqs. (41), (42), (40), and the Bregman update, Eq. (23)
# --------------------------------------------------------------------------

def _argmin_shrink(B, t):
    """Minimiser of t|w| + 1/2 |w - B|^2 by numerical optimisation."""
    fun = lambda w: t * math.hypot(w[0], w[1]) + 0.5 * ((w[0] - B[0]) ** 2 + (w[1] - B[1]) ** 2)
    best = None
    for start in ([0.0, 0.0], list(B), [B[0] * 0.5, B[1] * 0.5]):
        r = optimize.minimize(fun, start, method="Nelder-Mead",
                              options=dict(xatol=1e-12, fatol=1e-15, maxiter=20000))
        if best is None or r.fun < best.fun:
            best = r
    return best.x


def test_soft_threshold_is_the_prox_of_the_norm(oracle_lib):
    rng = np.random.default_rng(7)
    cases = [((0.0, 0.0), 0.3), ((0.3, -0.4), 0.0), ((0.3, 0.4), 0.5), ((3.0, 4.0), 5.0)]
    cases += [((float(a), float(b)), float(t)) for a, b, t in
              zip(rng.normal(size=20), rng.normal(size=20), rng.uniform(0, 1.5, 20))]
    for B, t in cases:
        o = oracle.soft_threshold(B[0], B[1], t)
        ref = _argmin_shrink(B, t)
        assert abs(o[0] - ref[0]) < 1e-6 and abs(o[1] - ref[1]) < 1e-6, (B, t, o, ref)
    # ties and near ties: |B| = t gives zero; just above gives a short vector along B
    t = 0.5
    for scale, zero in [(1.0, True), (1 - 2.0 ** -20, True), (1 + 2.0 ** -20, False)]:
        o = oracle.soft_threshold(0.3 * scale, 0.4 * scale, t)
        assert (o == (0.0, 0.0)) == zero
        if not zero:
            assert o[0] / o[1] == pytest.approx(0.75, rel=1e-12)


def test_w_update_minimises_the_linearised_w_subproblem(oracle_lib):
    """Before the projection, w~ minimises, pixel by pixel,
    gamma g delta(phi) |w| - 2 beta h(phi) w . v + mu/2 |w - grad phi - b|^2,
    with v the window sum over w^k (the one-sweep reading of Eq. (41))."""
    from paper_2003_12693_gb300.synth import random_state
    M, N = 10, 9
    phi, w1, w2, b1, b2, g = random_state(M, N, seed=31, phi_scale=1.5)
    p = Params(alpha=4.0, beta=0.6, gamma=4.0, mu=8.0, R=2, d=2.0)
    nw1, nw2, nb1, nb2, wt1, wt2 = oracle.w_b_update(phi, g, w1, w2, b1, b2, p,
                                                     return_shrunk=True)
    v1, v2 = oracle.repulsion(phi, w1, w2, p)
    d1 = np.roll(phi, -1, 0) - phi
    d2 = np.roll(phi, -1, 1) - phi
    for i in range(M):
        for j in range(N):
            D = oracle.delta(phi[i, j], p.eps)
            h = oracle.band(phi[i, j], p.eps, p.band_l)
            c = np.array([d1[i, j] + b1[i, j], d2[i, j] + b2[i, j]])
            vv = np.array([v1[i, j], v2[i, j]])

            def fun(w):
                return (p.gamma * g[i, j] * D * math.hypot(w[0], w[1])
                        - 2 * p.beta * h * (w[0] * vv[0] + w[1] * vv[1])
                        + 0.5 * p.mu * ((w[0] - c[0]) ** 2 + (w[1] - c[1]) ** 2))

            best = None
            for start in ([0.0, 0.0], list(c), [wt1[i, j] + 0.1, wt2[i, j] - 0.1]):
                r = optimize.minimize(fun, start, method="Nelder-Mead",
                                      options=dict(xatol=1e-12, fatol=1e-15, maxiter=20000))
                if best is None or r.fun < best.fun:
                    best = r
            assert abs(best.x[0] - wt1[i, j]) < 1e-5 and abs(best.x[1] - wt2[i, j]) < 1e-5
            # Eq. (40): unit vector along w~, or zero
            n = math.hypot(wt1[i, j], wt2[i, j])
            if n > 0:
                assert math.hypot(nw1[i, j], nw2[i, j]) == pytest.approx(1.0, abs=1e-14)
                assert nw1[i, j] * wt2[i, j] - nw2[i, j] * wt1[i, j] == pytest.approx(0, abs=1e-14)
            else:
                assert nw1[i, j] == 0.0 and nw2[i, j] == 0.0


def test_bregman_iteration_enforces_the_eikonal_constraint(oracle_lib):
    """With only the splitting term (alpha = beta = gamma = 0) the iteration
    pursues |grad phi| = 1 (Eqs. (13), (22)-(23)).  The constraint defect
    |grad phi - w| must shrink; a Bregman update with the wrong sign or a
    dropped term lets it grow."""
    i, j = np.mgrid[0:32, 0:32].astype(float)
    phi0 = 0.3 * (np.sin(2 * np.pi * i / 32) * 6 + np.cos(2 * np.pi * j / 32) * 4)
    st = oracle.initial_state(phi0)
    # start w on the unit circle so that the defect is pure constraint violation
    n = np.hypot(st.w1, st.w2)
    st.w1, st.w2 = st.w1 / n, st.w2 / n
    p = Params(alpha=0.0, beta=0.0, gamma=0.0, mu=8.0, tau=0.1, R=2, d=2.0)

    def defect(s):
        d1, d2 = oracle.grad(s.phi)
        return float(np.sqrt(np.mean((d1 - s.w1) ** 2 + (d2 - s.w2) ** 2)))

    g = np.ones_like(phi0)
    d0 = defect(st)
    oracle.iterate(st, g, 60, p)
    assert defect(st) < 0.25 * d0
    # |grad phi| moves toward 1 in the mean
    d1, d2 = oracle.grad(st.phi)
    m0 = np.mean(np.abs(np.hypot(*oracle.grad(phi0)) - 1))
    assert np.mean(np.abs(np.hypot(d1, d2) - 1)) < 0.5 * m0


# --------------------------------------------------------------------------
# Whole iteration (Alg. 1): invariants
# --------------------------------------------------------------------------

def test_transpose_equivariance_over_a_few_iterations(oracle_lib):
    """Every operator is symmetric under swapping the axes (forward differences,
    the window, the symbol of Eq. (32)), so running on f^T, phi0^T gives phi^T.
    Over longer runs rounding differences grow (the gate |B| > t and the
    direction B/|B| at small |B| amplify them), so only 2 iterations are checked."""
    from paper_2003_12693_gb300 import synth
    wl = synth.WORKLOADS["two_disks_128"]
    f, phi0 = wl.image()[:64, 10:74], wl.phi0()[:64, 10:74]
    # a tie-free init: shift one rectangle edge by half a pixel
    phi0 = synth.rect_sdf(64, 64, 20.5, 50, 6, 58)
    p = Params.from_dict(wl.params())
    g = oracle.edge(f)
    a = oracle.initial_state(phi0)
    b = oracle.initial_state(phi0.T.copy())
    oracle.iterate(a, g, 2, p)
    oracle.iterate(b, g.T.copy(), 2, p)
    assert np.abs(a.phi - b.phi.T).max() < 1e-9
    assert np.abs(a.w1 - b.w2.T).max() < 1e-6
    assert np.abs(a.b1 - b.b2.T).max() < 1e-6


@pytest.fixture(scope="module")
def two_disks_run(oracle_lib):
    from paper_2003_12693_gb300 import synth
    wl = synth.WORKLOADS["two_disks_128"]
    p = Params.from_dict(wl.params())
    f, phi0 = wl.image(), wl.phi0()
    g = oracle.edge(f)
    st = oracle.initial_state(phi0)
    e0 = oracle.energy(phi0, g, p)
    rel = oracle.iterate(st, g, wl.K, p)
    return dict(p=p, g=g, phi0=phi0, st=st, e0=e0, rel=rel)


def test_two_disks_topology_is_preserved(two_disks_run):
    """The contour enclosing both disks must not split (Fig. 1): {phi < 0}
    stays one 4-connected component and {phi >= 0} one 8-connected one."""
    from scipy import ndimage
    phi, phi0 = two_disks_run["st"].phi, two_disks_run["phi0"]
    for field in (phi0, phi):
        assert ndimage.label(field < 0)[1] == 1
        assert ndimage.label(field >= 0, structure=np.ones((3, 3)))[1] == 1
    # the contour has moved onto the disks: most of the rectangle is now outside
    assert (phi < 0).sum() < 0.7 * (phi0 < 0).sum()


def test_two_disks_w_is_unit_or_zero(two_disks_run):
    st = two_disks_run["st"]
    n = np.hypot(st.w1, st.w2)
    assert np.all((n == 0.0) | (np.abs(n - 1.0) < 1e-12))


def test_two_disks_energy_decreases(two_disks_run):
    e0 = two_disks_run["e0"]
    e1 = oracle.energy(two_disks_run["st"].phi, two_disks_run["g"], two_disks_run["p"])
    assert e1[0] < e0[0]


# --------------------------------------------------------------------------
# Discrete energy, Eqs. (7)-(10)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,R,d,seed", [((12, 11), 3, 3.0, 31), ((16, 16), 4, 4.0, 32),
                                            ((9, 14), 2, 5.0, 33)])
def test_energy_is_the_split_energy_on_the_constraint(oracle_lib, shape, R, d, seed):
    """With w = grad phi (forward differences) and b = 0 the splitting penalty
    of Eq. (22) vanishes and the split energy is the energy of Eq. (7).  The
    split energy is pinned independently: its finite-difference gradient is
    the right-hand side of Eq. (37) (test_rhs_is_descent_direction_of_split_energy)."""
    from paper_2003_12693_gb300.synth import random_state
    phi, _, _, _, _, g = random_state(*shape, seed=seed, phi_scale=2.0)
    p = Params(alpha=3.0, beta=0.6, gamma=2.5, mu=8.0, tau=0.1, R=R, d=d)
    d1 = np.roll(phi, -1, 0) - phi
    d2 = np.roll(phi, -1, 1) - phi
    z = np.zeros_like(phi)
    ref = _split_energy(phi, g, d1, d2, z, z, p)
    E, Eg, Ea, Er = oracle.energy(phi, g, p)
    assert E == pytest.approx(ref, rel=1e-12, abs=1e-12)
    assert E == pytest.approx(p.gamma * Eg + p.alpha * Ea + p.beta * Er, rel=1e-13, abs=1e-13)
    # each term alone, by switching the other weights off
    for a, b_, c in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)):
        q = Params(alpha=a, beta=b_, gamma=c, mu=8.0, tau=0.1, R=R, d=d)
        assert oracle.energy(phi, g, q)[0] == pytest.approx(
            _split_energy(phi, g, d1, d2, z, z, q), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("shape,R,d", [((10, 12), 3, 3.0), ((14, 9), 2, 2.5)])
def test_energy_repulsion_term_matches_pair_sum(oracle_lib, shape, R, d):
    """E_r = -sum over all ordered pixel pairs (x, y), both inside the image and
    within the R-window, of K(x - y) h(phi_x) h(phi_y) grad phi_x . grad phi_y:
    an O(P^2) loop over every pair."""
    from paper_2003_12693_gb300.synth import random_state
    phi, _, _, _, _, g = random_state(*shape, seed=41, phi_scale=1.5)
    p = Params(R=R, d=d)
    M, N = shape
    d1 = np.roll(phi, -1, 0) - phi
    d2 = np.roll(phi, -1, 1) - phi
    hb = np.vectorize(lambda x: oracle.band(x, p.eps, p.band_l))(phi)
    pts = [(i, j) for i in range(M) for j in range(N)]
    Er = 0.0
    for x1, x2 in pts:
        for y1, y2 in pts:
            if abs(x1 - y1) <= R and abs(x2 - y2) <= R:
                k = math.exp(-((x1 - y1) ** 2 + (x2 - y2) ** 2) / d ** 2)
                Er -= k * hb[x1, x2] * hb[y1, y2] * (d1[x1, x2] * d1[y1, y2] +
                                                     d2[x1, x2] * d2[y1, y2])
    assert oracle.energy(phi, g, p)[3] == pytest.approx(Er, rel=1e-12, abs=1e-12)


def test_energy_of_constant_level_sets(oracle_lib):
    """Far from the contour (|phi| > eps) delta and h vanish, so E_g = E_r = 0;
    E_a counts the g-weighted inside: sum g where phi < -eps, 0 where phi > eps."""
    rng = np.random.default_rng(5)
    g = rng.uniform(0.1, 1.0, (11, 13))
    p = Params()
    for c, area in ((-3.0, g.sum()), (3.0, 0.0)):
        E, Eg, Ea, Er = oracle.energy(np.full(g.shape, c), g, p)
        assert Eg == 0.0 and Er == 0.0
        assert Ea == pytest.approx(area, rel=1e-14)
        assert E == pytest.approx(p.alpha * area, rel=1e-14)


@pytest.mark.parametrize("eps,offset", [(1.0, 0.5), (1.0, 0.3), (2.0, 0.5)])
def test_energy_of_a_straight_edge(oracle_lib, eps, offset):
    """phi = j - c, a signed distance to the vertical line j = c (inside to the
    left).  With g = 1 the geodesic term is the contour's length: the raised
    cosine delta of Eq. (6) sampled at unit spacing sums to exactly 1 across the
    edge when 2 eps is an integer, so E_g = M (rows).  The area term is the
    inside's area, c + 1/2 per row: its derivative in c is that same delta sum
    (= 1), and at a half-integer c the samples of the odd function
    1 - H(x) - [x < 0] cancel in pairs.  Periodic forward differences wrap only
    at the last column, where phi is far outside the band."""
    M, N = 10, 24
    c = 9 + offset
    phi = np.tile(np.arange(N, dtype=np.float64) - c, (M, 1))
    g = np.ones((M, N))
    p = Params(eps=eps)
    _, Eg, Ea, _ = oracle.energy(phi, g, p)
    assert Eg == pytest.approx(M * 1.0, rel=1e-13)
    assert Ea == pytest.approx(M * (c + 0.5), rel=1e-13)


def test_mask_is_sign_of_phi(oracle_lib):
    phi = np.array([[-1.0, 0.0], [1e-300, -1e-300]])
    assert oracle.mask(phi).tolist() == [[1, 0], [0, 1]]


# ----------------------------------------------------------------------------
# The iterated w sub-problem, Eqs. (38)-(40)
# ----------------------------------------------------------------------------
def _wb_inputs(seed, H=24, W=20):
    from paper_2003_12693_gb300 import synth
    phi, w1, w2, b1, b2, g = synth.random_state(H, W, seed=seed)
    return phi, g, w1, w2, b1, b2


def test_fixed_point_one_sweep_is_the_unthresholded_shrink(oracle_lib):
    """With gamma = 0 the threshold of Eq. (42) vanishes and Eqs. (41)-(42)
    reduce to B / |B| with v from w^k: one sweep of Eqs. (38)-(40)."""
    phi, g, w1, w2, b1, b2 = _wb_inputs(1)
    p = Params(gamma=0.0, R=3, d=3.0)
    a = oracle.w_b_fixed_point(phi, g, w1, w2, b1, b2, p, 1)
    r = oracle.w_b_update(phi, g, w1, w2, b1, b2, p)
    for x, y in zip(a, r):
        assert np.allclose(x, y, atol=1e-12)


def test_fixed_point_denominator_cancels(oracle_lib):
    """The positive scalar gamma g delta + mu of Eq. (39) drops out under the
    projection (40): the result does not depend on gamma or g."""
    phi, g, w1, w2, b1, b2 = _wb_inputs(2)
    a = oracle.w_b_fixed_point(phi, g, w1, w2, b1, b2, Params(gamma=4.0, R=3, d=3.0), 2)
    b = oracle.w_b_fixed_point(phi, 0.3 * g, w1, w2, b1, b2, Params(gamma=0.5, R=3, d=3.0), 2)
    for x, y in zip(a, b):
        assert np.allclose(x, y, atol=1e-12)


def test_fixed_point_without_repulsion_is_one_sweep(oracle_lib):
    """beta = 0: v does not enter, so every sweep gives the same w."""
    phi, g, w1, w2, b1, b2 = _wb_inputs(3)
    p = Params(beta=0.0, R=3, d=3.0)
    one = oracle.w_b_fixed_point(phi, g, w1, w2, b1, b2, p, 1)
    five = oracle.w_b_fixed_point(phi, g, w1, w2, b1, b2, p, 5)
    for x, y in zip(one, five):
        assert np.allclose(x, y, atol=1e-13)


def test_fixed_point_sweeps_converge_for_weak_repulsion(oracle_lib):
    """For small beta the map w -> B(w)/|B(w)| contracts: the sweeps settle
    on a fixed point, unit vectors (or zero) with b from Eq. (23)."""
    phi, g, w1, w2, b1, b2 = _wb_inputs(4)
    p = Params(beta=0.02, R=3, d=3.0)
    a = oracle.w_b_fixed_point(phi, g, w1, w2, b1, b2, p, 30)
    b = oracle.w_b_fixed_point(phi, g, w1, w2, b1, b2, p, 31)
    assert np.abs(a[0] - b[0]).max() < 1e-9 and np.abs(a[1] - b[1]).max() < 1e-9
    n = np.hypot(a[0], a[1])
    assert np.all((n == 0) | (np.abs(n - 1) < 1e-12))
    d1, d2 = oracle.grad(phi)
    assert np.allclose(a[2], b1 + d1 - a[0]) and np.allclose(a[3], b2 + d2 - a[1])


def test_outer_iteration_with_one_sweep_and_no_threshold_is_alg1(oracle_lib):
    """gamma = 0, one sweep: the variant's outer iteration equals Alg. 1's."""
    phi, g, w1, w2, b1, b2 = _wb_inputs(5, 32, 32)
    p = Params(gamma=0.0, R=3, d=3.0)
    st = oracle.State(phi.copy(), w1.copy(), w2.copy(), b1.copy(), b2.copy())
    ref = st.copy()
    oracle.outer_iteration_fixed_point(st, g, p, 1)
    oracle.iterate(ref, g, 1, p)
    for x, y in zip((st.phi, st.w1, st.w2, st.b1, st.b2), (ref.phi, ref.w1, ref.w2, ref.b1, ref.b2)):
        assert np.allclose(x, y, atol=1e-11)


# ----------------------------------------------------------------------------
# The inner exit of Sec. 4
# ----------------------------------------------------------------------------
def _inner_state(seed=8, H=32, W=32):
    from paper_2003_12693_gb300 import synth
    phi, w1, w2, b1, b2, g = synth.random_state(H, W, seed=seed)
    return oracle.State(phi, w1, w2, b1, b2), g


def test_inner_exit_with_zero_tolerance_is_alg1(oracle_lib):
    st, g = _inner_state()
    p = Params(R=3, d=3.0)
    ref = st.copy()
    rels = oracle.outer_iteration_inner_tol(st, g, p, 0.0)
    oracle.iterate(ref, g, 1, p)
    assert len(rels) == p.S
    for x, y in zip((st.phi, st.w1, st.w2, st.b1, st.b2), (ref.phi, ref.w1, ref.w2, ref.b1, ref.b2)):
        assert np.allclose(x, y, atol=1e-12)


def test_inner_exit_with_a_loose_tolerance_takes_one_step(oracle_lib):
    st, g = _inner_state()
    p = Params(R=3, d=3.0, S=5)
    ref = st.copy()
    rels = oracle.outer_iteration_inner_tol(st, g, p, 1e9)
    assert len(rels) == 1
    psi = oracle.phi_step(ref.phi, g, ref.w1, ref.w2, ref.b1, ref.b2, p)
    assert np.allclose(st.phi, psi, atol=1e-13)
    assert rels[0] == pytest.approx(np.linalg.norm(psi - ref.phi) / (np.linalg.norm(ref.phi) + 1e-6))


def test_inner_exit_steps_grow_as_the_tolerance_shrinks(oracle_lib):
    st, g = _inner_state()
    p = Params(R=3, d=3.0, S=8)
    full = oracle.outer_iteration_inner_tol(st.copy(), g, p, 0.0)
    assert all(b < a for a, b in zip(full, full[1:]))          # the inner steps contract
    counts = [len(oracle.outer_iteration_inner_tol(st.copy(), g, p, t))
              for t in (full[0] * 1.01, full[2] * 1.01, full[5] * 1.01, 0.0)]
    assert counts == [1, 3, 6, 8]
