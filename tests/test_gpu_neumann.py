"""The Neumann reading of Eq. (27) on the GPU against its FP64 oracle.

oracle/neumann.py (pinned by the adjoint identity, a dense solve and the DCT
eigenvectors) takes d phi / dn = 0 literally: no forward difference across
the last row / column, the divergence minus the gradient's adjoint, and the
solve by the orthonormal type-II DCT.  The GPU transforms each row's even
extension with the periodic FFT of length 2W and solves each column with
reflective ends by the recursions on its even extension.  Checked: the solve
alone (random right-hand sides and pure DCT modes), one inner step, the w/b
update, one outer iteration through sr_iterate, the initial w of Alg. 1.
"""
import pytest

from gpu_common import *  # noqa: F401,F403
from oracle import neumann

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ctx(H, W, **kw):
    ctx = context(H, W, **kw)
    ctx.set_boundary("neumann")
    return ctx


@pytest.mark.parametrize("shape", [(16, 16), (32, 64), (128, 128), (256, 512), (64, 2048),
                                   (2048, 2048)])
@pytest.mark.parametrize("tau,mu", [(0.1, 8.0), (1.0, 8.0)])
def test_neumann_solve_matches_oracle(shape, tau, mu):
    H, W = shape
    rng = np.random.default_rng(H + 7 * W)
    rhs = f32(rng.normal(size=shape) * 3.0 + 1.0)
    ctx = _ctx(H, W, tau=tau, mu=mu)
    out = host(ctx.fft_solve(dev(rhs)))
    ref = neumann.solve(rhs, tau, mu)
    err = np.abs(out - ref).max()
    tol = 4e-7 * math.log2(4 * H * W) * np.abs(rhs).max()
    report("neumann_solve", shape=f"{H}x{W}", tau_mu=tau * mu, max_abs_err=err, tol=tol)
    assert err <= tol
    ctx.close()


def test_neumann_solve_divides_dct_modes_by_their_symbol():
    """cos(pi a (i + 1/2) / M) cos(pi b (j + 1/2) / N) is an eigenvector of the
    reflective Laplacian: the solve returns it over 1 + tau mu (4 sin^2(pi a /
    2M) + 4 sin^2(pi b / 2N)), written out here from the DCT-II basis."""
    H, W = 64, 128
    tau, mu = 0.1, 8.0
    ctx = _ctx(H, W, tau=tau, mu=mu)
    i = (np.arange(H)[:, None] + 0.5) / H
    j = (np.arange(W)[None, :] + 0.5) / W
    for a, b in [(0, 0), (1, 0), (0, 1), (63, 127), (32, 64), (5, 17), (0, 127), (63, 0)]:
        F = np.cos(np.pi * a * i) * np.cos(np.pi * b * j)
        lam = 1 + tau * mu * (4 * np.sin(np.pi * a / (2 * H)) ** 2 + 4 * np.sin(np.pi * b / (2 * W)) ** 2)
        out = host(ctx.fft_solve(dev(F)))
        assert np.abs(out - f32(F) / lam).max() < 2e-6, (a, b)
    ctx.close()


@pytest.mark.parametrize("shape,R,d", [((128, 128), 3, 3.0), ((256, 64), 4, 4.0),
                                       ((512, 512), 8, 8.0), ((2048, 2048), 4, 4.0)])
def test_neumann_phi_step_matches_oracle(shape, R, d):
    H, W = shape
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=H + 3 * R))
    p = oparams(R=R, d=d)
    ctx = _ctx(H, W, R=R, d=d)
    ctx.set_g(dev(g))
    out = host(ctx.phi_step(*[dev(a) for a in (phi, w1, w2, b1, b2)]))
    ref = neumann.phi_step(phi, g, w1, w2, b1, b2, p)
    err = np.abs(out - ref).max()
    report("neumann_phi_step", shape=f"{H}x{W}", R=R, max_abs_dphi=err)
    assert err <= PHI_TOL
    ctx.close()


def _conditioning(phi1, g, w1, w2, b1, b2, p):
    v1, v2 = oracle.repulsion(phi1, w1, w2, p)
    d1, d2 = neumann.grad(phi1)
    h = np.vectorize(lambda x: oracle.band(x, p.eps, p.band_l))(phi1)
    D = np.vectorize(lambda x: oracle.delta(x, p.eps))(phi1)
    B1 = d1 + b1 + (2 * p.beta / p.mu) * h * v1
    B2 = d2 + b2 + (2 * p.beta / p.mu) * h * v2
    return np.hypot(B1, B2), (p.gamma / p.mu) * g * D


@pytest.mark.parametrize("shape,R,d", [((128, 128), 3, 3.0), ((256, 64), 8, 8.0)])
def test_neumann_w_b_update_matches_oracle(shape, R, d):
    H, W = shape
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=5 * H + R))
    p = oparams(R=R, d=d)
    ctx = _ctx(H, W, R=R, d=d)
    ctx.set_g(dev(g))
    outs = [host(t) for t in ctx.w_b_update(*[dev(a) for a in (phi, w1, w2, b1, b2)])]
    rw1, rw2, rb1, rb2 = neumann.w_b_update(phi, g, w1, w2, b1, b2, p)
    nB, t = _conditioning(phi, g, w1, w2, b1, b2, p)
    dB = 2e-6
    cond = (nB > 50 * dB) & (np.abs(nB - t) > 4 * dB)
    tol = 1e-5 + 2.0 * dB / np.maximum(nB, 1e-30)
    for a, r in zip(outs, (rw1, rw2, rb1, rb2)):
        assert not (cond & (np.abs(a - r) > tol + 1e-5)).any()
    # the last row's d1 and the last column's d2 are zero: b' = b - w' there
    assert np.allclose(outs[2][-1, :], b1[-1, :] - outs[0][-1, :], atol=1e-5)
    assert np.allclose(outs[3][:, -1], b2[:, -1] - outs[1][:, -1], atol=1e-5)
    report("neumann_w_b_update", shape=f"{H}x{W}", R=R, exempt_pixels=int((~cond).sum()))
    assert (~cond).sum() < 0.01 * H * W
    ctx.close()


@pytest.mark.parametrize("workload,K0", [("two_disks_128", 4), ("ellipses_512", 2)])
def test_neumann_outer_iteration_matches_oracle(workload, K0):
    """One outer iteration through sr_iterate from a state that the Neumann
    oracle iteration reached (S = 3 steps of neumann.phi_step, then
    neumann.w_b_update, from the Neumann initial state of Alg. 1)."""
    wl = synth.WORKLOADS[workload]
    p = oracle.Params.from_dict(wl.params())
    g64 = f32(oracle.edge(wl.image()))
    phi = f32(wl.phi0())
    w1, w2 = neumann.grad(phi)
    b1, b2 = np.zeros_like(phi), np.zeros_like(phi)
    state = None
    for _ in range(K0 + 1):
        state = [f32(a) for a in (phi, w1, w2, b1, b2)]
        psi = state[0]
        for _ in range(p.S):
            psi = neumann.phi_step(psi, g64, *state[1:], p)
        w1, w2, b1, b2 = neumann.w_b_update(psi, g64, *state[1:], p)
        phi = psi
    ctx = _ctx(wl.H, wl.W, R=wl.R, d=wl.d)
    ctx.set_g(dev(g64))
    ctx.set_state(*[dev(a) for a in state])
    ctx.iterate(1)
    gpu = [host(t) for t in ctx.get_state()]
    ctx.close()
    err = float(np.abs(gpu[0] - phi).max())
    report("neumann_one_iteration", workload=workload, max_abs_dphi=err)
    assert err <= PHI_TOL, err


def test_neumann_initial_w_is_the_reflective_gradient():
    H, W = 64, 128
    phi0 = f32(synth.rect_sdf(H, W, 10.25, 50.5, 12, 100.25))
    ctx = _ctx(H, W)
    ctx.set_phi(dev(phi0))
    _, w1, w2, b1, b2 = [host(t) for t in ctx.get_state()]
    d1, d2 = neumann.grad(phi0)
    assert np.abs(w1 - d1).max() < 1e-5 and np.abs(w2 - d2).max() < 1e-5
    assert np.all(w1[-1, :] == 0) and np.all(w2[:, -1] == 0)
    assert np.abs(b1).max() == 0 and np.abs(b2).max() == 0
    ctx.close()


def test_neumann_unsupported_combinations():
    ctx = context(96, 96)
    with pytest.raises(sr.SRError) as e:
        ctx.set_boundary("neumann")
    assert e.value.status == sr.SR_EUNSUPPORTED
    ctx.close()
    ctx = _ctx(64, 64)
    with pytest.raises(sr.SRError) as e:
        ctx.set_phi_solver("aos")
    assert e.value.status == sr.SR_EUNSUPPORTED
    ctx.set_boundary("periodic")
    ctx.set_phi_solver("aos")
    ctx.close()
