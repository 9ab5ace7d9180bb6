"""The AOS solve of the phi sub-problem on the GPU against its FP64 oracle.

oracle/aos.py solves each cyclic tridiagonal line system by the Thomas
recursion with Sherman-Morrison for the corners (pinned by dense solves); the
GPU factors the same constant-coefficient operator into two first-order
recursions (sr_aos.cu).  Checked: the solve alone on square, oblong, tiny
(lines shorter than the recursions' warm-up) and non-power-of-two shapes and
three values of tau mu; one inner step of Eq. (37) with the AOS solve; one
outer iteration of Alg. 1 with it, through sr_iterate's graph.
"""
import pytest

from gpu_common import *  # noqa: F401,F403
from oracle import aos

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("shape", [(16, 16), (16, 48), (64, 96), (128, 128), (96, 160),
                                   (512, 512), (1024, 256), (2048, 2048)])
@pytest.mark.parametrize("tau,mu", [(0.1, 8.0), (0.5, 8.0), (0.01, 1.0)])
def test_aos_solve_matches_oracle(shape, tau, mu):
    """FP32 recursions: rounding ~ eps_32 / (1 - r)^2 relative to max|rhs|."""
    H, W = shape
    rng = np.random.default_rng(H * 3 + W)
    rhs = f32(rng.normal(size=shape) * 3.0 + 1.0)
    ctx = context(H, W, tau=tau, mu=mu)
    out = host(ctx.aos_solve(dev(rhs)))
    ref = aos.solve(rhs, tau, mu)
    err = np.abs(out - ref).max()
    tol = 2e-6 * np.abs(rhs).max()
    report("aos_solve", shape=f"{H}x{W}", tau_mu=tau * mu, max_abs_err=err, tol=tol)
    assert err <= tol
    ctx.close()


def _oracle_aos_step(psi, g, w1, w2, b1, b2, p):
    v1, v2 = oracle.repulsion(psi, w1, w2, p)
    return aos.solve(oracle.rhs(psi, g, w1, w2, b1, b2, v1, v2, p), p.tau, p.mu)


@pytest.mark.parametrize("shape,R,d", [((128, 128), 3, 3.0), ((256, 96), 4, 4.0),
                                       ((512, 512), 8, 8.0)])
def test_aos_inner_step_matches_oracle(shape, R, d):
    H, W = shape
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=H + R))
    p = oparams(R=R, d=d)
    ctx = context(H, W, R=R, d=d)
    ctx.set_phi_solver("aos")
    ctx.set_g(dev(g))
    out = host(ctx.phi_step(*[dev(a) for a in (phi, w1, w2, b1, b2)]))
    ref = _oracle_aos_step(phi, g, w1, w2, b1, b2, p)
    err = np.abs(out - ref).max()
    report("aos_phi_step", shape=f"{H}x{W}", R=R, max_abs_dphi=err)
    assert err <= PHI_TOL
    ctx.close()


@pytest.mark.parametrize("workload,K0", [("two_disks_128", 10), ("ellipses_512", 5)])
def test_aos_outer_iteration_matches_oracle(workload, K0):
    """One outer iteration (S = 3 AOS inner steps, then Eqs. (41), (42), (40),
    (23)) through sr_iterate, from a state the AOS oracle iteration reached."""
    wl = synth.WORKLOADS[workload]
    p = oracle.Params.from_dict(wl.params())
    g64 = f32(oracle.edge(wl.image()))
    st = oracle.initial_state(f32(wl.phi0()))
    for _ in range(K0 + 1):
        state = [f32(a) for a in (st.phi, st.w1, st.w2, st.b1, st.b2)]
        psi = state[0]
        for _ in range(p.S):
            psi = _oracle_aos_step(psi, g64, *state[1:], p)
        w1, w2, b1, b2 = oracle.w_b_update(psi, g64, *state[1:], p)
        st = oracle.State(psi, w1, w2, b1, b2)
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
    ctx.set_phi_solver("aos")
    ctx.set_g(dev(g64))
    ctx.set_state(*[dev(a) for a in state])
    ctx.iterate(1)
    gpu = [host(t) for t in ctx.get_state()]
    ctx.close()
    err = float(np.abs(gpu[0] - st.phi).max())
    assert err <= PHI_TOL, err
    nB, t = wb_conditioning(gpu[0], g64, *state[1:], p)
    nex = compare_wb((gpu[1], gpu[2]), (gpu[3], gpu[4]), (st.w1, st.w2), (st.b1, st.b2), nB, t,
                     gpu[0], (state[3], state[4]), err_phi=err)
    report("aos_one_iteration", workload=workload, max_abs_dphi=err, exempt_pixels=nex)


def test_aos_solver_switch_rebuilds_the_graph():
    """Switching to AOS and back to FFT before iterating gives the FFT
    iteration bit for bit; switching to AOS changes the iteration."""
    wl = synth.WORKLOADS["two_disks_128"]
    outs = []
    for solvers in (["fft"], ["aos", "fft"], ["aos"]):
        ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
        ctx.edge_function(dev(wl.image()))
        ctx.set_phi(dev(wl.phi0()))
        ctx.iterate(2)  # builds the graphs with the default solver
        for sv in solvers:
            ctx.set_phi_solver(sv)
        ctx.iterate(3)
        outs.append(host(ctx.get_phi()))
        ctx.close()
    assert np.array_equal(outs[0], outs[1])
    assert not np.array_equal(outs[0], outs[2])
