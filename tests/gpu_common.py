"""Shared helpers of the GPU tests (inputs, oracle references, comparisons)."""
import math

import numpy as np
import torch

import oracle
from paper_2003_12693_gb300 import sr, synth

# The tolerance the target states for phi: max |dphi| <= 1e-4 against FP64.
PHI_TOL = 1e-4


def f32(a):
    """Round to FP32 (the inputs both sides receive) and back to float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def context(H, W, R=3, d=3.0, **kw):
    return sr.Context(H, W, sr.make_params(win_radius=R, d=d, **kw))


def oparams(R=3, d=3.0, **kw):
    return oracle.Params(R=R, d=d, **kw)


def wb_conditioning(phi1, g, w1, w2, b1, b2, p):
    """|B| and t of Eqs. (41)-(42) from the (pinned) oracle building blocks."""
    v1, v2 = oracle.repulsion(phi1, w1, w2, p)
    d1, d2 = oracle.grad(phi1)
    h = np.vectorize(lambda x: oracle.band(x, p.eps, p.band_l))(phi1)
    D = np.vectorize(lambda x: oracle.delta(x, p.eps))(phi1)
    B1 = d1 + b1 + (2 * p.beta / p.mu) * h * v1
    B2 = d2 + b2 + (2 * p.beta / p.mu) * h * v2
    nB = np.hypot(B1, B2)
    t = (p.gamma / p.mu) * g * D
    return nB, t


def compare_wb(w_gpu, b_gpu, w_ref, b_ref, nB, t, phi1_gpu, b_in, err_phi=0.0):
    """Element-wise comparison of w^{k+1}, b^{k+1} where the result is unique
    to FP32 accuracy; validity checks elsewhere.

    Error propagation from phi^{k+1}: B = grad phi + b + (2 beta/mu) h v moves
    by dB <= 5 |dphi| + 2e-6 (forward differences, and h' v with |h'| < 1.6,
    sum k < 30, 2 beta/mu <= 0.15), the threshold t by less than that, and the
    unit vector B/|B| by dw <= 2 dB / |B|.  Where |B| is within dB of t (the
    shrink gate) or of 0 (the direction), FP32 and FP64 may legitimately take
    different branches; there the GPU value must still be valid: |w| in {0, 1}
    and b^{k+1} = b^k + grad phi^{k+1} - w^{k+1} with its own w.
    Returns the number of exempted pixels.
    """
    dB = 5.0 * err_phi + 2e-6
    cond = (nB > 50 * dB) & (np.abs(nB - t) > 4 * dB)
    tol_w = 1e-5 + 2.0 * dB / np.maximum(nB, 1e-30)
    for a, r in zip(w_gpu, w_ref):
        bad = cond & (np.abs(a - r) > tol_w)
        assert not bad.any(), f"w mismatch at {int(bad.sum())} pixels"
    tol_b = tol_w + 2.0 * err_phi + 1e-5
    for a, r in zip(b_gpu, b_ref):
        bad = cond & (np.abs(a - r) > tol_b)
        assert not bad.any(), f"b mismatch at {int(bad.sum())} pixels"
    n = np.hypot(*w_gpu)
    assert np.all((n == 0) | (np.abs(n - 1) < 1e-5)), "w must be a unit vector or zero"
    d1 = np.roll(phi1_gpu, -1, 0) - phi1_gpu
    d2 = np.roll(phi1_gpu, -1, 1) - phi1_gpu
    scale = max(1.0, float(np.abs(phi1_gpu).max())) * 1e-6
    assert np.abs(b_gpu[0] - (b_in[0] + d1 - w_gpu[0])).max() <= 4 * scale + 1e-6
    assert np.abs(b_gpu[1] - (b_in[1] + d2 - w_gpu[1])).max() <= 4 * scale + 1e-6
    return int((~cond).sum())


_REPORT = {}


def report(key, **vals):
    """Record measured errors; written to $SR_PARITY_REPORT at session end."""
    _REPORT.setdefault(key, []).append({k: (float(v) if not isinstance(v, (int, str)) else v)
                                        for k, v in vals.items()})


def write_report():
    import json
    import os
    path = os.environ.get("SR_PARITY_REPORT")
    if path and _REPORT:
        with open(path, "w") as fh:
            json.dump(_REPORT, fh, indent=1)


def components(phi):
    from scipy import ndimage
    inside = ndimage.label(phi < 0)[1]
    outside = ndimage.label(phi >= 0, structure=np.ones((3, 3)))[1]
    return inside, outside


def oracle_state_after(phi0, g, K, p):
    st = oracle.initial_state(phi0)
    if K:
        oracle.iterate(st, g, K, p)
    return st


def rounded_state(st):
    return [f32(a) for a in (st.phi, st.w1, st.w2, st.b1, st.b2)]


def one_iteration_both(ctx, state64, g64, p):
    """Run one outer iteration from the same FP32 state on the GPU and in the
    oracle; return (gpu state, oracle state) as float64 arrays."""
    ctx.set_g(dev(g64))
    ctx.set_state(*[dev(a) for a in state64])
    ctx.iterate(1)
    gpu = [host(t) for t in ctx.get_state()]
    ref = oracle.State(*(a.copy() for a in state64))
    oracle.iterate(ref, g64, 1, p)
    return gpu, ref


def check_one_iteration(gpu, ref, state64, g64, p):
    err = float(np.abs(gpu[0] - ref.phi).max())
    assert err <= PHI_TOL, f"max |dphi| = {err:.3e}"
    nB, t = wb_conditioning(gpu[0], g64, state64[1], state64[2], state64[3], state64[4], p)
    nexempt = compare_wb((gpu[1], gpu[2]), (gpu[3], gpu[4]), (ref.w1, ref.w2), (ref.b1, ref.b2),
                         nB, t, gpu[0], (state64[3], state64[4]), err_phi=err)
    report(f"one_iteration_{gpu[0].shape[0]}x{gpu[0].shape[1]}",
           max_abs_dphi=err, exempt_pixels=nexempt)
    return err, nexempt


__all__ = ["PHI_TOL", "f32", "dev", "host", "context", "oparams", "wb_conditioning",
           "compare_wb", "components", "oracle_state_after", "rounded_state",
           "one_iteration_both", "check_one_iteration", "report", "write_report", "math", "np", "torch", "oracle",
           "sr", "synth"]
