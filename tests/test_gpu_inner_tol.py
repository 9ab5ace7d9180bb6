"""The inner-loop exit of Sec. 4 on the GPU against the FP64 oracle.

The tolerance of each case is placed between two successive relative changes
of the oracle (at their geometric mean, 7 % or more from both here), so that
both sides take the same number of inner steps although their values differ
in the last bits."""
import numpy as np
import pytest

from gpu_common import *  # noqa: F401,F403

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _state(H, W, K, p):
    img = synth.ellipse_scene(11, H=H, W=W, scale=min(H, W) / 512.0)
    g64 = f32(oracle.edge(img))
    st = oracle_state_after(synth.inset_rect_sdf(H, W), g64, K, p)
    return g64, rounded_state(st)


@pytest.mark.parametrize("steps", [1, 2, 4])
def test_inner_exit_matches_oracle(steps):
    H, W = 128, 96
    S = 6
    p = oparams(R=4, d=4.0, S=S)
    g64, state = _state(H, W, 5, p)
    full = oracle.outer_iteration_inner_tol(oracle.State(*(a.copy() for a in state)), g64, p, 0.0)
    # stop after `steps` steps: the change of step `steps` is <= tol < that of the step before
    tol = 1.5 * full[0] if steps == 1 else math.sqrt(full[steps - 1] * full[steps - 2])
    ref = oracle.State(*(a.copy() for a in state))
    rels = oracle.outer_iteration_inner_tol(ref, g64, p, tol)
    assert len(rels) == steps
    ctx = context(H, W, R=4, d=4.0, inner_S=S, inner_tol=tol)
    ctx.set_g(dev(g64))
    ctx.set_state(*[dev(a) for a in state])
    ctx.inner_steps(reset=True)
    ctx.iterate(1)
    assert ctx.inner_steps() == steps
    gpu = [host(t) for t in ctx.get_state()]
    err = float(np.abs(gpu[0] - ref.phi).max())
    report("inner_exit", steps=steps, tol=tol, max_abs_dphi=err)
    assert err <= PHI_TOL
    nB, t = wb_conditioning(gpu[0], g64, state[1], state[2], state[3], state[4], p)
    compare_wb((gpu[1], gpu[2]), (gpu[3], gpu[4]), (ref.w1, ref.w2), (ref.b1, ref.b2), nB, t,
               gpu[0], (state[3], state[4]), err_phi=err)
    ctx.close()


def test_zero_tolerance_counts_fixed_steps_and_groups_reject_the_exit():
    ctx = context(64, 64, inner_S=3)
    img = synth.ellipse_scene(4, H=64, W=64, scale=0.125)
    ctx.edge_function(dev(img))
    ctx.set_phi(dev(synth.inset_rect_sdf(64, 64)))
    ctx.inner_steps(reset=True)
    ctx.iterate(5)
    assert ctx.inner_steps() == 15
    tol_ctx = context(64, 64, inner_S=3, inner_tol=1e-3)
    with pytest.raises(sr.SRError):
        sr.Group([tol_ctx])
    ctx.close()
    tol_ctx.close()
