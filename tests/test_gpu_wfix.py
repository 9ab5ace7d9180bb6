"""The iterated w sub-problem, Eqs. (38)-(40), against the FP64 oracle.

The GPU kernel drops the positive denominator of Eq. (39) before the
projection (40); the oracle evaluates Eq. (39) literally.  Where |B| is close
to zero the direction of w is ill-conditioned in FP32: one sweep uses the
same exemption rule as the soft-threshold update (compare_wb with no
threshold); after several sweeps such a pixel's w enters its neighbours'
window sums, so pixels within R of an ill-conditioned pixel of an earlier
sweep are exempt too (their values must still be valid)."""
import numpy as np
import pytest
from scipy import ndimage

from gpu_common import *  # noqa: F401,F403

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


SHAPES = [(96, 80), (64, 64), (48, 144)]


@pytest.mark.parametrize("shape", SHAPES)
def test_one_sweep_matches_oracle(shape):
    H, W = shape
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=H + W))
    p = oparams(R=4, d=4.0)
    ctx = context(H, W, R=4, d=4.0)
    ctx.set_g(dev(g))
    out = [host(t) for t in ctx.w_b_fixed_point(*[dev(a) for a in (phi, w1, w2, b1, b2)], 1)]
    ref = oracle.w_b_fixed_point(phi, g, w1, w2, b1, b2, p, 1)
    nB, _ = wb_conditioning(phi, g, w1, w2, b1, b2, p)
    nex = compare_wb((out[0], out[1]), (out[2], out[3]), ref[:2], ref[2:], nB, np.zeros_like(nB),
                     phi, (b1, b2))
    report("w_fixed_point_1", shape=f"{H}x{W}", exempt=nex,
           max_dw=float(np.abs(out[0] - ref[0]).max()))
    ctx.close()


def _sweep_bound(phi, g, w1, w2, b1, b2, p, sweeps, R):
    """Per-pixel bound on |w_gpu - w_oracle| after ``sweeps`` sweeps: a sweep
    turns an FP32 error dB ~ 2e-6 of B into 2 dB / |B| in the direction, and
    a pixel's error reaches every pixel within R at the next sweep through the
    window sum (with a gain of at most 2 per sweep here: 2 beta / mu times the
    window's weight sum, 0.05 x 40)."""
    inv = np.zeros(phi.shape)
    cw1, cw2 = w1, w2
    for r in range(sweeps):
        nB, _ = wb_conditioning(phi, g, cw1, cw2, b1, b2, p)
        spread = 2 * R * (sweeps - 1 - r) + 1
        inv = np.maximum(inv, 2.0 ** (sweeps - r) *
                         ndimage.maximum_filter(1.0 / np.maximum(nB, 1e-12), size=spread,
                                                mode="constant"))
        cw1, cw2, _, _ = oracle.w_b_fixed_point(phi, g, w1, w2, b1, b2, p, r + 1)
    return 1e-5 + 2.0 * 2e-6 * inv


@pytest.mark.parametrize("sweeps", [2, 4])
def test_several_sweeps_match_oracle(sweeps):
    H, W = 96, 80
    R = 4
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=7 + sweeps))
    p = oparams(R=R, d=4.0)
    ctx = context(H, W, R=R, d=4.0)
    ctx.set_g(dev(g))
    out = [host(t) for t in ctx.w_b_fixed_point(*[dev(a) for a in (phi, w1, w2, b1, b2)], sweeps)]
    ref = oracle.w_b_fixed_point(phi, g, w1, w2, b1, b2, p, sweeps)
    tol = _sweep_bound(phi, g, w1, w2, b1, b2, p, sweeps, R)
    dw = np.maximum(np.abs(out[0] - ref[0]), np.abs(out[1] - ref[1]))
    report("w_fixed_point_n", sweeps=sweeps, max_dw=float(dw.max()),
           median_tol=float(np.median(tol)))
    assert np.all(dw <= tol)
    assert np.median(tol) < 5e-3
    n = np.hypot(out[0], out[1])
    assert np.all((n == 0) | (np.abs(n - 1) < 1e-5))
    d1 = np.roll(phi, -1, 0) - phi
    d2 = np.roll(phi, -1, 1) - phi
    assert np.abs(out[2] - (b1 + d1 - out[0])).max() < 1e-5
    assert np.abs(out[3] - (b2 + d2 - out[1])).max() < 1e-5
    ctx.close()


def _ellipse_state(H, W, K, p):
    img = synth.ellipse_scene(11, H=H, W=W, scale=min(H, W) / 512.0)
    g64 = f32(oracle.edge(img))
    st = oracle_state_after(synth.inset_rect_sdf(H, W), g64, K, p)
    return g64, rounded_state(st)


@pytest.mark.parametrize("sweeps", [1, 3])
def test_outer_iteration_with_sweeps_matches_oracle(sweeps):
    """One outer iteration of Alg. 1 with the w sub-problem by Eqs. (38)-(40),
    through sr_iterate's graph, from the oracle's state after 5 iterations."""
    H, W = 128, 96
    p = oparams(R=4, d=4.0)
    g64, state = _ellipse_state(H, W, 5, p)
    ctx = context(H, W, R=4, d=4.0)
    ctx.set_w_sweeps(sweeps)
    ctx.set_g(dev(g64))
    ctx.set_state(*[dev(a) for a in state])
    ctx.iterate(1)
    gpu = [host(t) for t in ctx.get_state()]
    ref = oracle.State(*(a.copy() for a in state))
    oracle.outer_iteration_fixed_point(ref, g64, p, sweeps)
    err = float(np.abs(gpu[0] - ref.phi).max())
    report("w_fixed_point_outer", sweeps=sweeps, max_abs_dphi=err)
    assert err <= PHI_TOL
    n = np.hypot(gpu[1], gpu[2])
    assert np.all((n == 0) | (np.abs(n - 1) < 1e-5))
    # w: phi^{k+1} differs by up to err, which moves B by about 5 err; a
    # formula error would show at most pixels, so at least 99 % agree to 1e-3
    dw = np.maximum(np.abs(gpu[1] - ref.w1), np.abs(gpu[2] - ref.w2))
    report("w_fixed_point_outer_w", sweeps=sweeps, frac_over_1e3=float((dw > 1e-3).mean()))
    assert (dw > 1e-3).mean() <= 0.01
    d1 = np.roll(gpu[0], -1, 0) - gpu[0]
    d2 = np.roll(gpu[0], -1, 1) - gpu[0]
    assert np.abs(gpu[3] - (state[3] + d1 - gpu[1])).max() < 1e-4
    assert np.abs(gpu[4] - (state[4] + d2 - gpu[2])).max() < 1e-4
    ctx.close()


def test_sweeps_in_a_group_match_alone_and_zero_restores_default():
    sizes = [(64, 64), (96, 64)]
    alone, grouped = [], []
    for k, (H, W) in enumerate(sizes):
        img = synth.ellipse_scene(300 + k, H=H, W=W, scale=0.125)
        phi0 = synth.inset_rect_sdf(H, W)
        for lst in (alone, grouped):
            ctx = context(H, W, R=4, d=4.0)
            ctx.set_w_sweeps(2)
            ctx.edge_function(dev(img))
            ctx.set_phi(dev(phi0))
            lst.append(ctx)
    grp = sr.Group(grouped)
    grp.iterate(7)
    for ctx in alone:
        ctx.iterate(7)
    for a, b in zip(alone, grouped):
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(host(x), host(y))
    grp.close()
    # back to Eqs. (41)-(42): bit-identical to a context that never swept
    H, W = sizes[0]
    img = synth.ellipse_scene(300, H=H, W=W, scale=0.125)
    fresh = context(H, W, R=4, d=4.0)
    for c in (alone[0], fresh):
        c.set_w_sweeps(0)
        c.edge_function(dev(img))
        c.set_phi(dev(synth.inset_rect_sdf(H, W)))
        c.iterate(5)
    for x, y in zip(alone[0].get_state(), fresh.get_state()):
        assert np.array_equal(host(x), host(y))
    for ctx in alone + grouped + [fresh]:
        ctx.close()


def test_sweep_argument_checks():
    ctx = context(64, 64)
    with pytest.raises(sr.SRError):
        ctx.set_w_sweeps(-1)
    with pytest.raises(sr.SRError):
        ctx.set_w_sweeps(65)
    z = torch.zeros((64, 64), device="cuda")
    with pytest.raises(sr.SRError):
        ctx.w_b_fixed_point(z, z, z, z, z, 0)
    ctx.close()
