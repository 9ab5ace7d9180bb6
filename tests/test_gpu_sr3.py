"""The SR iteration on volumes (Fig. 6's 3-D use) on the GPU against its FP64
oracle, oracle/sr3d.py (pinned by a dense solve, a brute-force window sum
over voxel pairs, the 3-vector shrink's closed cases and the reduction to the
2-D oracle on z-constant volumes).  Through the C-ABI of include/sr3.h:
the window sum, the solve (complex FFTs on the two inner axes, recursions
along z), one inner step, the w/b update and one outer iteration."""
import pytest

from gpu_common import *  # noqa: F401,F403
from oracle import sr3d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _vol(shape, **kw):
    from paper_2003_12693_gb300 import sr3
    return sr3.Volume(*shape, sr.make_params(**kw))


def _state(shape, seed, phi_scale=2.0):
    """Smooth phi with many zero crossings, O(1) w and b, g in (0, 1]."""
    rng = np.random.default_rng(seed)
    Z, M, N = shape
    z, i, j = np.meshgrid(np.arange(Z), np.arange(M), np.arange(N), indexing="ij")
    phi = phi_scale * (np.sin(2 * np.pi * (z / Z + 0.3)) + np.cos(2 * np.pi * i / M * 2)
                       + np.sin(2 * np.pi * j / N * 3)) + rng.normal(0, 0.3, shape)
    w = tuple(rng.normal(0, 0.6, shape) for _ in range(3))
    b = tuple(rng.normal(0, 0.4, shape) for _ in range(3))
    g = rng.uniform(0.1, 1.0, shape)
    return f32(phi), tuple(f32(a) for a in w), tuple(f32(a) for a in b), f32(g)


@pytest.mark.parametrize("shape,R,d", [((8, 16, 32), 2, 2.0), ((12, 32, 16), 3, 3.0),
                                       ((6, 16, 16), 4, 4.0)])
def test_window_sum_matches_oracle(shape, R, d):
    phi, w, _, _ = _state(shape, seed=R)
    V = _vol(shape, win_radius=R, d=d)
    v = [host(t) for t in V.window_sum(dev(phi), [dev(a) for a in w])]
    ref = sr3d.window_sum(phi, w, oparams(R=R, d=d))
    err = max(np.abs(a - b).max() for a, b in zip(v, ref))
    report("sr3_window_sum", shape=str(shape), R=R, max_abs_err=err)
    assert err <= 2e-6 * (2 * R + 1) ** 3
    V.close()


@pytest.mark.parametrize("shape", [(8, 16, 16), (16, 32, 64), (5, 64, 32), (3, 16, 128),
                                   (32, 128, 128)])
@pytest.mark.parametrize("tau,mu", [(0.1, 8.0), (1.0, 8.0)])
def test_solve_matches_oracle(shape, tau, mu):
    """(1 - tau mu Lap) phi = rhs: FP32 FFTs, eps_32 log2(P) max|rhs|."""
    rng = np.random.default_rng(sum(shape))
    rhs = f32(rng.normal(size=shape) * 3.0 + 1.0)
    V = _vol(shape, tau=tau, mu=mu)
    out = host(V.fft_solve(dev(rhs)))
    ref = sr3d.solve(rhs, tau, mu)
    err = np.abs(out - ref).max()
    tol = 4e-7 * math.log2(np.prod(shape)) * np.abs(rhs).max()
    report("sr3_solve", shape=str(shape), tau_mu=tau * mu, max_abs_err=err, tol=tol)
    assert err <= tol
    V.close()


def test_solve_divides_fourier_modes_by_their_symbol():
    shape = (6, 32, 16)
    V = _vol(shape)
    z, i, j = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    for a, b, c in [(0, 0, 0), (1, 0, 0), (3, 16, 8), (5, 31, 15), (0, 1, 0), (2, 3, 7)]:
        F = np.cos(2 * np.pi * (a * z / shape[0] + b * i / shape[1] + c * j / shape[2]))
        lam = sr3d.symbol(shape, 0.1, 8.0)[a, b, c]
        out = host(V.fft_solve(dev(F)))
        assert np.abs(out - f32(F) / lam).max() < 2e-6, (a, b, c)
    V.close()


@pytest.mark.parametrize("shape,R,d", [((8, 32, 32), 2, 2.0), ((16, 64, 32), 3, 3.0)])
def test_phi_step_matches_oracle(shape, R, d):
    phi, w, b, g = _state(shape, seed=10 + R)
    p = oparams(R=R, d=d)
    V = _vol(shape, win_radius=R, d=d)
    V.set_g(dev(g))
    out = host(V.phi_step(dev(phi), [dev(a) for a in w], [dev(a) for a in b]))
    ref = sr3d.phi_step(phi, g, w, b, p)
    err = np.abs(out - ref).max()
    report("sr3_phi_step", shape=str(shape), R=R, max_abs_dphi=err)
    assert err <= PHI_TOL
    V.close()


def _conditioning(phi1, g, w, b, p):
    v = sr3d.window_sum(phi1, w, p)
    d = sr3d.grad(phi1)
    h = np.vectorize(lambda x: oracle.band(x, p.eps, p.band_l))(phi1)
    B = [dk + bk + (2 * p.beta / p.mu) * h * vk for dk, bk, vk in zip(d, b, v)]
    D = np.vectorize(lambda x: oracle.delta(x, p.eps))(phi1)
    return np.sqrt(sum(x * x for x in B)), (p.gamma / p.mu) * g * D


@pytest.mark.parametrize("shape,R,d", [((8, 32, 32), 2, 2.0), ((6, 16, 64), 3, 3.0)])
def test_w_b_update_matches_oracle(shape, R, d):
    """Element-wise where |B| is well away from 0 and from t (FP32 and FP64
    may take different branches at near-ties); valid everywhere."""
    phi, w, b, g = _state(shape, seed=20 + R)
    p = oparams(R=R, d=d)
    V = _vol(shape, win_radius=R, d=d)
    V.set_g(dev(g))
    wo, bo = V.w_b_update(dev(phi), [dev(a) for a in w], [dev(a) for a in b])
    wo, bo = [host(t) for t in wo], [host(t) for t in bo]
    rw, rb = sr3d.w_b_update(phi, g, w, b, p)
    nB, t = _conditioning(phi, g, w, b, p)
    dB = 5e-6
    cond = (nB > 50 * dB) & (np.abs(nB - t) > 4 * dB)
    tol = 1e-5 + 2.0 * dB / np.maximum(nB, 1e-30)
    for a, r in zip(wo + bo, list(rw) + list(rb)):
        assert not (cond & (np.abs(a - r) > tol + 1e-5)).any()
    n = np.sqrt(sum(x * x for x in wo))
    assert np.all((n == 0) | (np.abs(n - 1) < 1e-5))
    report("sr3_w_b_update", shape=str(shape), R=R, exempt_voxels=int((~cond).sum()))
    assert (~cond).sum() < 0.01 * np.prod(shape)
    V.close()


def test_outer_iteration_matches_oracle():
    """One outer iteration through sr3_iterate from an oracle-reached state of
    a two-ball volume (radius 6, 4 voxels apart, noise 0.05, a box around
    both)."""
    Z, M, N = 16, 32, 64
    z, i, j = np.meshgrid(np.arange(Z), np.arange(M), np.arange(N), indexing="ij")
    rng = np.random.default_rng(7)
    balls = (((z - 8) ** 2 + (i - 16) ** 2 + (j - 24) ** 2 <= 36) |
             ((z - 8) ** 2 + (i - 16) ** 2 + (j - 40) ** 2 <= 36)).astype(float)
    f = balls + rng.normal(0, 0.05, balls.shape)
    # g = 1 / (1 + |grad f|^2) with central differences (the 2-D reading per axis)
    gz, gi, gj = np.gradient(f)
    g = f32(1.0 / (1.0 + gz ** 2 + gi ** 2 + gj ** 2))
    # signed distance of the box [1.25, 14.5] x [8.25, 24.5] x [16, 48.25] (tie-free)
    lo, hi = np.array([1.25, 8.25, 16.0]), np.array([14.5, 24.5, 48.25])
    X = np.stack([z, i, j]).astype(float)
    dlo = X - lo[:, None, None, None]
    dhi = hi[:, None, None, None] - X
    inside = np.minimum(dlo, dhi).min(axis=0)
    out = np.maximum(np.maximum(-dlo, -dhi), 0.0)
    phi = np.where(inside > 0, -inside, np.sqrt((out ** 2).sum(axis=0)))
    phi = f32(phi)
    p = oparams(R=2, d=2.0)
    w = sr3d.grad(phi)
    b = tuple(np.zeros_like(phi) for _ in range(3))
    for _ in range(3):
        state = (f32(phi), tuple(f32(a) for a in w), tuple(f32(a) for a in b))
        phi, w, b = sr3d.outer_iteration(*state[:1], g, state[1], state[2], p)
    V = _vol((Z, M, N), win_radius=2, d=2.0)
    V.set_g(dev(g))
    V.set_state(dev(state[0]), [dev(a) for a in state[1]], [dev(a) for a in state[2]])
    V.iterate(1)
    gphi, gw, gb = V.get_state()
    err = float(np.abs(host(gphi) - phi).max())
    report("sr3_one_iteration", shape=str((Z, M, N)), max_abs_dphi=err)
    assert err <= PHI_TOL
    n = np.sqrt(sum(host(t) ** 2 for t in gw))
    assert np.all((n == 0) | (np.abs(n - 1) < 1e-5))
    V.close()


def test_unsupported_and_invalid_sizes():
    from paper_2003_12693_gb300 import sr3
    with pytest.raises(sr.SRError) as e:
        sr3.Volume(8, 24, 32, sr.make_params())
    assert e.value.status == sr.SR_EUNSUPPORTED
    with pytest.raises(sr.SRError) as e:
        sr3.Volume(0, 32, 32, sr.make_params())
    assert e.value.status == sr.SR_EINVAL
