"""Sides that are not powers of two: the mixed-radix FFT passes.

Same comparisons as test_gpu_parity.py, on shapes whose FFT lengths (H and
W/2) have the factors 3, 5, 7 and 31 (a direct length-31 DFT), against the
FP64 oracle, whose transform handles any length.  Every test runs twice: with
the recursion column pass these sizes use by default, and with the
mixed-radix column FFT (SR_GEN_FFT_COLS=1)."""
import pytest

from gpu_common import *  # noqa: F401,F403

pytestmark = pytest.mark.gpu

# (H, W): FFT lengths H and W/2
MIXED = [(48, 96),     # 16*3, 48 = 16*3
         (96, 160),    # 32*3, 80 = 16*5
         (224, 64),    # 32*7, 32
         (160, 992),   # 32*5, 496 = 16*31
         (64, 1120)]   # 64, 560 = 16*5*7


@pytest.fixture(autouse=True, params=["recursion_columns", "fft_columns"])
def _column_pass(request, monkeypatch):
    monkeypatch.setenv("SR_GEN_FFT_COLS", "1" if request.param == "fft_columns" else "0")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("shape", MIXED)
def test_mixed_radix_fft_solve(shape):
    """Eqs. (31)-(33) alone through the mixed-radix passes."""
    H, W = shape
    rng = np.random.default_rng(H * 5 + W)
    rhs = f32(rng.normal(size=shape) * 3.0 + 1.0)
    ctx = context(H, W)
    assert ctx.get_schedule()["row_threads"] == 0  # no register-FFT schedule at this size
    out = host(ctx.fft_solve(dev(rhs)))
    ref = oracle.solve(rhs, 0.1, 8.0)
    tol = 4e-7 * math.log2(H * W) * np.abs(rhs).max()
    report("fft_solve_mixed", shape=f"{H}x{W}", max_abs_err=np.abs(out - ref).max(), tol=tol)
    assert np.abs(out - ref).max() <= tol
    ctx.close()


def test_mixed_radix_eigenfunctions():
    """Pure modes: each Fourier mode is divided by its own symbol."""
    H, W = 96, 160
    ctx = context(H, W)
    i, j = np.mgrid[0:H, 0:W].astype(float)
    for a, b in [(0, 0), (1, 0), (0, 80), (48, 80), (5, 17), (95, 159), (32, 0), (7, 33)]:
        F = np.cos(2 * np.pi * (a * i / H + b * j / W))
        ref = oracle.solve(f32(F), 0.1, 8.0)
        out = host(ctx.fft_solve(dev(F)))
        assert np.abs(out - ref).max() < 2e-6, (a, b)
    ctx.close()


@pytest.mark.parametrize("shape", MIXED)
def test_mixed_radix_phi_step(shape):
    """One semi-implicit step of Eq. (37) (window sum, right-hand side, solve)."""
    H, W = shape
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=H + 3 * W))
    p = oparams(R=4, d=4.0)
    ctx = context(H, W, R=4, d=4.0)
    ctx.set_g(dev(g))
    out = host(ctx.phi_step(*[dev(a) for a in (phi, w1, w2, b1, b2)]))
    ref = oracle.phi_step(phi, g, w1, w2, b1, b2, p)
    report("phi_step_mixed", shape=f"{H}x{W}", max_abs_dphi=np.abs(out - ref).max())
    assert np.abs(out - ref).max() <= PHI_TOL
    ctx.close()


@pytest.mark.parametrize("shape", [(96, 160), (224, 64)])
def test_mixed_radix_one_outer_iteration(shape):
    """One outer iteration of Alg. 1 from the oracle's state after 5 iterations
    of a six-ellipse scene (inset-rectangle start)."""
    H, W = shape
    img = synth.ellipse_scene(11, H=H, W=W, scale=min(H, W) / 512.0)
    p = oparams(R=4, d=4.0)
    g64 = f32(oracle.edge(img))
    st = oracle_state_after(synth.inset_rect_sdf(H, W), g64, 5, p)
    state = rounded_state(st)
    ctx = context(H, W, R=4, d=4.0)
    gpu, ref = one_iteration_both(ctx, state, g64, p)
    check_one_iteration(gpu, ref, state, g64, p)
    ctx.close()


def test_group_with_mixed_radix_members():
    """A group of power-of-two and other sides: each member ends bit-identical
    to the same member iterated alone."""
    sizes = [(96, 160), (128, 128), (224, 64), (64, 96)]
    alone, grouped = [], []
    for k, (H, W) in enumerate(sizes):
        img = synth.ellipse_scene(200 + k, H=H, W=W, scale=max(min(H, W) / 512.0, 0.125))
        phi0 = synth.inset_rect_sdf(H, W)
        for lst in (alone, grouped):
            ctx = context(H, W, R=4, d=4.0)
            ctx.edge_function(dev(img))
            ctx.set_phi(dev(phi0))
            lst.append(ctx)
    grp = sr.Group(grouped)
    grp.iterate(9)
    for ctx in alone:
        ctx.iterate(9)
    for a, b in zip(alone, grouped):
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(host(x), host(y))
    grp.close()
    for ctx in alone + grouped:
        ctx.close()
