"""GPU vs FP64 oracle, element by element, through the C-ABI.

Inputs come from the seeded generators (synth) or from the oracle itself
(states reached by oracle iterations, rounded to FP32); expected values come
from the oracle only.  Tolerances: phi within 1e-4 (the target's bar); the
other fields within bounds derived from FP32 arithmetic, stated per test.
"""
import pytest

from gpu_common import *  # noqa: F401,F403

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (32, 64), (128, 128), (64, 256), (256, 128), (512, 512)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


# ---------------------------------------------------------------- step (b) alone
@pytest.mark.parametrize("shape", SHAPES + [(2048, 2048), (16, 4096), (4096, 32)])
def test_fft_solve_matches_oracle(shape):
    """Eqs. (31)-(33) alone.  FP32 FFT error ~ eps_32 * log2(P) * max|rhs|."""
    H, W = shape
    rng = np.random.default_rng(H * 7 + W)
    rhs = f32(rng.normal(size=shape) * 3.0 + 1.0)
    ctx = context(H, W)
    out = host(ctx.fft_solve(dev(rhs)))
    ref = oracle.solve(rhs, 0.1, 8.0)
    tol = 4e-7 * math.log2(H * W) * np.abs(rhs).max()
    report("fft_solve", shape=f"{H}x{W}", max_abs_err=np.abs(out - ref).max(), tol=tol)
    assert np.abs(out - ref).max() <= tol
    ctx.close()


def test_fft_solve_eigenfunctions():
    """Pure modes: the solve divides each Fourier mode by its own symbol."""
    H, W = 64, 128
    ctx = context(H, W)
    i, j = np.mgrid[0:H, 0:W].astype(float)
    for a, b in [(0, 0), (1, 0), (0, 64), (32, 64), (5, 17), (63, 127), (32, 0), (0, 1)]:
        F = np.cos(2 * np.pi * (a * i / H + b * j / W))
        ref = oracle.solve(f32(F), 0.1, 8.0)
        out = host(ctx.fft_solve(dev(F)))
        assert np.abs(out - ref).max() < 2e-6, (a, b)
    ctx.close()


@pytest.mark.parametrize("shape", [(64, 32), (128, 256), (512, 512), (256, 2048), (4096, 64),
                                   (1024, 256), (2048, 64), (128, 128), (16, 1024)])
def test_every_fft_schedule_matches_oracle(shape):
    """The autotuner may pick any schedule; each one must compute the same solve."""
    H, W = shape
    rng = np.random.default_rng(H + W)
    rhs = f32(rng.normal(size=shape) * 3.0)
    ref = oracle.solve(rhs, 0.1, 8.0)
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=W))
    ref_step = oracle.phi_step(phi, g, w1, w2, b1, b2, oparams())
    ctx = context(H, W)
    ctx.set_g(dev(g))
    tuned = ctx.get_schedule()
    assert tuned["tuned_us"] > 0
    tried = 0
    for vpt in (16, 8):
        for threads in (32, 64, 128, 256, 512):
            for col in range(9):
                try:
                    ctx.set_schedule(vpt, threads, col)
                except sr.SRError as e:
                    assert e.status == sr.SR_EINVAL
                    continue
                tried += 1
                out = host(ctx.fft_solve(dev(rhs)))
                assert np.abs(out - ref).max() <= 4e-7 * math.log2(H * W) * np.abs(rhs).max()
                step = host(ctx.phi_step(*[dev(a) for a in (phi, w1, w2, b1, b2)]))
                assert np.abs(step - ref_step).max() <= PHI_TOL
    assert tried >= 6
    report("schedules", shape=f"{H}x{W}", tried=tried, tuned=str(tuned))
    ctx.close()


@pytest.mark.parametrize("shape", [(16, 32), (48, 32), (64, 32), (256, 64), (2048, 32),
                                   (4096, 32), (128, 128), (16, 1024), (32, 64)])
@pytest.mark.parametrize("tau,mu", [(0.1, 8.0), (1.0, 8.0), (0.01, 1.0)])
@pytest.mark.parametrize("col", [7, 8])
def test_column_recursion_eigenfunctions(shape, tau, mu, col):
    """Column schedule 7 replaces the column FFT by the forward and backward
    recursions that factor the column operator; schedule 8 runs the row
    transforms and the same recursions in one CTA.  Pure Fourier modes must
    come out divided by their own symbol of Eq. (32), including the packed DC
    and Nyquist column (b = 0, W/2), the Nyquist row (a = H/2) and conjugate
    partners (a, H - a); tau mu = 8 needs the longest warm-up (r_0 = 0.70),
    and H = 16 or 48 is shorter than the warm-up (it wraps)."""
    H, W = shape
    ctx = context(H, W, tau=tau, mu=mu)
    tuned = ctx.get_schedule()
    if tuned["row_threads"] == 0:
        pytest.skip("sizes below W = 32 use the fixed passes")
    try:
        ctx.set_schedule(tuned["row_values_per_thread"], tuned["row_threads"], col)
    except sr.SRError as e:
        assert e.status == sr.SR_EINVAL
        pytest.skip("schedule not available at this size and tau mu")
    i, j = np.mgrid[0:H, 0:W].astype(float)
    modes = [(0, 0), (1, 0), (0, W // 2), (H // 2, W // 2), (H // 2, 0), (5, 3), (H - 5, 3),
             (H - 1, W // 2 - 1), (3, W // 2), (H // 3, 1)]
    for a, b in modes:
        ph = 2 * np.pi * (a * i / H + b * j / W)
        F = np.cos(ph) + 0.5 * np.sin(ph)
        ref = oracle.solve(f32(F), tau, mu)
        out = host(ctx.fft_solve(dev(F)))
        assert np.abs(out - ref).max() < 2e-6, (a, b, np.abs(out - ref).max())
    rng = np.random.default_rng(H + W)
    rhs = f32(rng.normal(size=shape) * 3.0 + 1.0)
    ref = oracle.solve(rhs, tau, mu)
    out = host(ctx.fft_solve(dev(rhs)))
    assert np.abs(out - ref).max() <= 4e-7 * math.log2(H * W) * np.abs(rhs).max()
    ctx.close()


# ---------------------------------------------------------------- step (a) alone
@pytest.mark.parametrize("shape", SHAPES[:5])
@pytest.mark.parametrize("R,d", [(0, 1.0), (3, 3.0), (4, 4.0), (8, 8.0), (2, 5.0)])
def test_repulsion_matches_oracle(shape, R, d):
    """Sec. 4 window sum; FP32 sum of (2R+1)^2 terms of size <= 1."""
    H, W = shape
    phi, w1, w2, _, _, _ = synth.random_state(H, W, seed=H + W + R, phi_scale=2.5)
    phi, w1, w2 = f32(phi), f32(w1), f32(w2)
    ctx = context(H, W, R=R, d=d)
    v1, v2 = ctx.repulsion_field(dev(phi), dev(w1), dev(w2))
    r1, r2 = oracle.repulsion(phi, w1, w2, oparams(R=R, d=d))
    tol = 2e-6 * (2 * R + 1) ** 2
    report("repulsion", shape=f"{H}x{W}", R=R,
           max_abs_err=max(np.abs(host(v1) - r1).max(), np.abs(host(v2) - r2).max()))
    assert np.abs(host(v1) - r1).max() <= tol
    assert np.abs(host(v2) - r2).max() <= tol
    ctx.close()


# ---------------------------------------------------------------- edge function
@pytest.mark.parametrize("shape", [(16, 16), (128, 128), (64, 256), (512, 512)])
@pytest.mark.parametrize("s_pow,sigma", [(2, 1.0), (1, 1.0), (2, 0.0), (2, 2.5)])
def test_edge_function_matches_oracle(shape, s_pow, sigma):
    H, W = shape
    rng = np.random.default_rng(H + 3 * W)
    f = f32(rng.uniform(0, 1, shape) + (np.arange(W)[None, :] > W // 2))
    ctx = context(H, W, s_pow=s_pow, sigma=sigma, rho=1.5)
    ctx.edge_function(dev(f))
    g = host(ctx.get_g())
    ref = oracle.edge(f, rho=1.5, sigma=sigma, s_pow=s_pow)
    assert np.abs(g - ref).max() <= 2e-6
    ctx.close()


# ---------------------------------------------------------------- step (b): one inner step
@pytest.mark.parametrize("shape", SHAPES + [(2048, 2048)])
@pytest.mark.parametrize("R,d", [(3, 3.0), (4, 4.0), (8, 8.0)])
def test_phi_step_matches_oracle(shape, R, d):
    """One semi-implicit step of Eq. (37): v, F, FFT solve."""
    H, W = shape
    if H * W > 512 * 512 and R != 4:
        pytest.skip("full size checked at the workload's window only")
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=R * 100 + H))
    p = oparams(R=R, d=d)
    ctx = context(H, W, R=R, d=d)
    ctx.set_g(dev(g))
    out = host(ctx.phi_step(*[dev(a) for a in (phi, w1, w2, b1, b2)]))
    ref = oracle.phi_step(phi, g, w1, w2, b1, b2, p)
    report("phi_step", shape=f"{H}x{W}", R=R, max_abs_dphi=np.abs(out - ref).max())
    assert np.abs(out - ref).max() <= PHI_TOL
    ctx.close()


# ---------------------------------------------------------------- steps (c)-(e)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("R,d,beta", [(3, 3.0, 0.2), (4, 4.0, 0.2), (8, 8.0, 0.6), (3, 3.0, 0.0)])
def test_w_b_update_matches_oracle(shape, R, d, beta):
    H, W = shape
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=H * 3 + R))
    p = oparams(R=R, d=d, beta=beta)
    ctx = context(H, W, R=R, d=d, beta=beta)
    ctx.set_g(dev(g))
    outs = [host(t) for t in ctx.w_b_update(*[dev(a) for a in (phi, w1, w2, b1, b2)])]
    rw1, rw2, rb1, rb2 = oracle.w_b_update(phi, g, w1, w2, b1, b2, p)
    nB, t = wb_conditioning(phi, g, w1, w2, b1, b2, p)
    nex = compare_wb((outs[0], outs[1]), (outs[2], outs[3]), (rw1, rw2), (rb1, rb2), nB, t, phi,
                     (b1, b2))
    report("w_b_update", shape=f"{H}x{W}", R=R, exempt_pixels=nex)
    assert nex < 0.01 * H * W


# ---------------------------------------------------------------- one outer iteration
@pytest.mark.parametrize("K0", [0, 1, 10, 60, 199])
def test_one_outer_iteration_two_disks(K0):
    """Alg. 1, one outer iteration (S = 3 inner steps, w, b) on the 128x128
    two-disk workload, from oracle states along the oracle's own trajectory."""
    wl = synth.WORKLOADS["two_disks_128"]
    p = oracle.Params.from_dict(wl.params())
    g64 = f32(oracle.edge(wl.image()))
    st = oracle_state_after(wl.phi0(), g64, K0, p)
    state = rounded_state(st)
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
    gpu, ref = one_iteration_both(ctx, state, g64, p)
    err, nex = check_one_iteration(gpu, ref, state, g64, p)
    assert nex < 200
    ctx.close()


@pytest.mark.parametrize("K0", [0, 20])
def test_one_outer_iteration_ellipses_512(K0):
    wl = synth.WORKLOADS["ellipses_512"]
    p = oracle.Params.from_dict(wl.params())
    g64 = f32(oracle.edge(wl.image()))
    st = oracle_state_after(wl.phi0(), g64, K0, p)
    state = rounded_state(st)
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
    gpu, ref = one_iteration_both(ctx, state, g64, p)
    check_one_iteration(gpu, ref, state, g64, p)
    ctx.close()


def test_one_outer_iteration_full_size_2048():
    """The benchmark's own workload and launch configuration (2048^2, R = d = 4):
    one outer iteration from phi0, every pixel compared."""
    wl = synth.WORKLOADS["ellipses_2048"]
    p = oracle.Params.from_dict(wl.params())
    g64 = f32(oracle.edge(wl.image()))
    st = oracle_state_after(wl.phi0(), g64, 0, p)
    state = rounded_state(st)
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
    gpu, ref = one_iteration_both(ctx, state, g64, p)
    check_one_iteration(gpu, ref, state, g64, p)
    ctx.close()


def test_one_outer_iteration_full_size_4096():
    """The largest single image (4096^2 blob pairs 1-3 px apart, R = d = 8, the
    17 x 17 window): one outer iteration from phi0, every pixel compared."""
    wl = synth.WORKLOADS["blobs_4096"]
    p = oracle.Params.from_dict(wl.params())
    g64 = f32(oracle.edge(wl.image()))
    st = oracle_state_after(wl.phi0(), g64, 0, p)
    state = rounded_state(st)
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
    gpu, ref = one_iteration_both(ctx, state, g64, p)
    check_one_iteration(gpu, ref, state, g64, p)
    ctx.close()


# ---------------------------------------------------------------- whole run
@pytest.fixture(scope="module")
def two_disks_full():
    wl = synth.WORKLOADS["two_disks_128"]
    p = oracle.Params.from_dict(wl.params())
    f = wl.image()
    phi0 = f32(wl.phi0())
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
    ctx.edge_function(dev(f))
    ctx.set_phi(dev(phi0))
    e0 = ctx.energy()
    ctx.iterate(wl.K)
    e1 = ctx.energy()
    gpu = [host(t) for t in ctx.get_state()]
    mask = host(ctx.mask())
    g = host(ctx.get_g())
    ctx.close()
    ref = oracle_state_after(phi0, f32(oracle.edge(f32(f))), wl.K, p)
    # the oracle's own sensitivity to rounding: the same run on the transposed input
    refT = oracle_state_after(phi0.T.copy(), f32(oracle.edge(f32(f).T.copy())), wl.K, p)
    return dict(gpu=gpu, mask=mask, g=g, e0=e0, e1=e1, ref=ref, refT=refT, phi0=phi0, p=p)


def test_two_disks_run_preserves_topology(two_disks_full):
    """Fig. 1: splitting prevented.  {phi < 0} stays one component."""
    r = two_disks_full
    assert components(r["gpu"][0]) == components(r["phi0"]) == (1, 1)
    assert components(r["ref"].phi) == (1, 1)


def test_two_disks_run_invariants(two_disks_full):
    r = two_disks_full
    n = np.hypot(r["gpu"][1], r["gpu"][2])
    assert np.all((n == 0) | (np.abs(n - 1) < 1e-5))
    assert r["e1"][0] < r["e0"][0]
    assert np.array_equal(r["mask"], (r["gpu"][0] < 0).astype(np.float64))
    # the segmentation against the oracle's, bounded by the oracle's own
    # rounding sensitivity, is checked in test_gpu_whole_run.py; recorded here
    m_gpu = r["gpu"][0] < 0
    m_ref = r["ref"].phi < 0
    m_refT = r["refT"].phi.T < 0
    report("two_disks_200_iterations", mask_diff_gpu_vs_oracle=int((m_gpu != m_ref).sum()),
           mask_diff_oracle_vs_transposed_oracle=int((m_ref != m_refT).sum()),
           max_abs_dphi=np.abs(r["gpu"][0] - r["ref"].phi).max(),
           max_abs_dphi_oracle_vs_transposed=np.abs(r["ref"].phi - r["refT"].phi.T).max())


def test_energy_matches_oracle(two_disks_full):
    r = two_disks_full
    e_ref = oracle.energy(r["gpu"][0], r["g"], r["p"])
    for a, b in zip(r["e1"], e_ref):
        assert a == pytest.approx(b, rel=1e-5, abs=1e-3)


# ---------------------------------------------------------------- library behaviour
def test_checkpoint_resume_is_bit_identical():
    wl = synth.WORKLOADS["two_disks_128"]
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
    ctx.edge_function(dev(wl.image()))
    ctx.set_phi(dev(wl.phi0()))
    ctx.iterate(7)
    saved = [t.clone() for t in ctx.get_state()]
    ctx.iterate(9)
    a = [host(t) for t in ctx.get_state()]
    ctx.set_state(*saved)
    ctx.iterate(9)
    b = [host(t) for t in ctx.get_state()]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    ctx.close()


def test_graph_and_direct_launches_agree():
    """The CUDA-graph path and the per-kernel (profiling) path are the same work."""
    wl = synth.WORKLOADS["two_disks_128"]
    outs = []
    for prof in (False, True):
        ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
        ctx.edge_function(dev(wl.image()))
        ctx.set_phi(dev(wl.phi0()))
        ctx.profile_enable(prof)
        ctx.iterate(5)
        outs.append([host(t) for t in ctx.get_state()])
        if prof:
            ms, n = ctx.kernel_times("prep")
            assert n == 15 and ms > 0
        ctx.close()
    for x, y in zip(*outs):
        assert np.array_equal(x, y)


def test_stopping_test_and_statuses():
    wl = synth.WORKLOADS["two_disks_128"]
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d, check_every=5)
    ctx.edge_function(dev(wl.image()))
    ctx.set_phi(dev(wl.phi0()))
    done, rel, ok = ctx.iterate(12, tol=1e-12)
    assert done == 12 and not ok and rel > 0
    # relative change against the oracle's definition on the same two states
    phi_a = host(ctx.get_phi())
    done, rel, ok = ctx.iterate(1, want_rel=True)
    phi_b = host(ctx.get_phi())
    expect = np.linalg.norm(phi_b - phi_a) / (np.linalg.norm(phi_a) + 1e-6)
    assert rel == pytest.approx(expect, rel=1e-5)
    done, rel, ok = ctx.iterate(50, tol=1.0)
    assert ok and done == 5
    # a non-finite state is reported, not propagated silently
    phi, w1, w2, b1, b2 = ctx.get_state()
    phi[3, 4] = float("nan")
    ctx.set_state(phi, w1, w2, b1, b2)
    with pytest.raises(sr.SRError) as e:
        ctx.iterate(3, tol=1e-9)
    assert e.value.status == sr.SR_ENONFINITE
    ctx.close()


def test_segment_host_matches_device_path():
    wl = synth.WORKLOADS["two_disks_128"]
    f = np.ascontiguousarray(wl.image().astype(np.float32))
    phi0 = np.ascontiguousarray(wl.phi0().astype(np.float32))
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
    mask_h = torch.empty((wl.H, wl.W), dtype=torch.uint8).pin_memory()
    phi_h = torch.empty((wl.H, wl.W), dtype=torch.float32).pin_memory()
    ctx.segment_host(torch.from_numpy(f).pin_memory(), torch.from_numpy(phi0).pin_memory(), 20,
                     0.0, mask_h, phi_h)
    ctx.edge_function(dev(f))
    ctx.set_phi(dev(phi0))
    ctx.iterate(20)
    assert np.array_equal(host(ctx.get_phi()), phi_h.numpy().astype(np.float64))
    assert np.array_equal(host(ctx.mask()), mask_h.numpy().astype(np.float64))
    ctx.close()


def test_degenerate_inputs():
    """Constant phi far from the contour (no narrow band): w, b follow the
    gradient alone; a constant image gives g = 1; R = 0 leaves v = h w."""
    H, W = 32, 32
    ctx = context(H, W, R=0, d=1.0)
    ctx.edge_function(dev(np.full((H, W), 0.3)))
    assert np.all(host(ctx.get_g()) == 1.0)
    phi = np.full((H, W), 7.0)
    ctx.set_phi(dev(phi))
    ctx.iterate(3)
    out = [host(t) for t in ctx.get_state()]
    assert np.abs(out[0] - 7.0).max() < 1e-5
    assert np.all(out[1] == 0) and np.all(out[2] == 0)
    p1, w1, w2, _, _, _ = synth.random_state(H, W, seed=5)
    v1, v2 = ctx.repulsion_field(dev(p1), dev(w1), dev(w2))
    h = np.vectorize(lambda x: oracle.band(x))(f32(p1))
    assert np.abs(host(v1) - h * f32(w1)).max() < 1e-6
    ctx.close()


# ---------------------------------------------------------------- batched groups
GROUP_SIZES = [(64, 128), (128, 128), (256, 64), (512, 512), (128, 256), (1024, 64)]


def _group_inputs(H, W, seed):
    scale = min(H, W) / 512.0
    img = synth.ellipse_scene(seed, H=H, W=W, scale=max(scale, 0.125))
    return img, synth.inset_rect_sdf(H, W)


def test_group_iterate_matches_members_alone():
    """Batched iteration of images of uneven sizes: every member of the group
    ends bit-identical to the same member iterated alone, for an odd count
    (both graph parities) and again after a second call."""
    alone, grouped = [], []
    for k, (H, W) in enumerate(GROUP_SIZES):
        img, phi0 = _group_inputs(H, W, 100 + k)
        for lst in (alone, grouped):
            ctx = context(H, W, R=4, d=4.0)
            ctx.edge_function(dev(img))
            ctx.set_phi(dev(phi0))
            lst.append(ctx)
    grp = sr.Group(grouped)
    grp.iterate(7)
    grp.iterate(4)
    for ctx in alone:
        ctx.iterate(11)
    for a, b in zip(alone, grouped):
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(host(x), host(y))
    # members at different parities are refused
    grouped[0].iterate(1)
    with pytest.raises(sr.SRError) as e:
        grp.iterate(1)
    assert e.value.status == sr.SR_EINVAL
    grp.close()
    for ctx in alone + grouped:
        ctx.close()
