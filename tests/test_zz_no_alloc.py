"""sr_phi_step_noalloc: the inner phi step for callers that cannot allocate.

Some hosts own all GPU memory through their own arena, capture streams into
CUDA graphs in modes that forbid allocation, or run real-time loops that
cannot take the device synchronisation of cudaMalloc / cudaFree.  This entry
point serves them from a fixed device array inside the library.  The test
calls it through the C-ABI several times in a row, with different sizes and
windows (down to 16 x 16 and up to the array's limit of 512 x 512, and the
ragged 512 x 16), and checks each result against the FP64 oracle's inner step
and against the context-based sr_phi_step, within the tolerance the other
tests use for phi (1e-4).  It is collected last so that a run stopping at the
first failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

PHI_TOL = 1e-4


@pytest.fixture(scope="module")
def srmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build, sr
    build.build()
    torch.cuda.set_device(0)
    return sr


def _inputs(H, W, seed):
    """Seeded fields (phi, w1, w2, b1, b2, g), rounded to FP32 once so that the
    oracle and the GPU start from the same numbers."""
    from paper_2003_12693_gb300 import synth
    return [np.ascontiguousarray(a, dtype=np.float32) for a in synth.random_state(H, W, seed=seed)]


# (H, W, R, d, seed): the smallest side, the array's largest image with the
# widest window (the largest shared-memory footprint of the fused row pass),
# a ragged 512 x 16 (rows of complex length 8), and two middle shapes
CASES = [(128, 128, 3, 3.0, 1), (16, 16, 0, 3.0, 3), (512, 512, 8, 8.0, 4),
         (512, 16, 4, 4.0, 5), (256, 64, 4, 4.0, 2)]


def test_noalloc_step_matches_oracle_and_context_step_on_calls_in_a_row(srmod):
    import oracle
    lib = srmod.lib()
    stream = torch.cuda.current_stream()
    for H, W, R, d, seed in CASES:
        arrs = _inputs(H, W, seed)
        phi, w1, w2, b1, b2, g = [torch.from_numpy(a).cuda() for a in arrs]
        params = srmod.make_params(win_radius=R, d=d)
        out = torch.full_like(phi, float("nan"))
        st = lib.sr_phi_step_noalloc(H, W, C.byref(params),
                                     *[C.c_void_p(t.data_ptr())
                                       for t in (g, phi, w1, w2, b1, b2, out)],
                                     C.c_void_p(stream.cuda_stream))
        assert st == srmod.SR_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        a64 = [a.astype(np.float64) for a in arrs]
        ref = oracle.phi_step(a64[0], a64[5], a64[1], a64[2], a64[3], a64[4],
                              oracle.Params(R=R, d=d))
        err = float(np.abs(got - ref).max())
        assert err <= PHI_TOL, (H, W, R, "vs oracle", err)
        ctx = srmod.Context(H, W, params)
        ctx.set_g(g)
        alt = ctx.phi_step(phi, w1, w2, b1, b2)
        err_ctx = float((out - alt).abs().max())
        assert err_ctx <= PHI_TOL, (H, W, R, "vs sr_phi_step", err_ctx)
        ctx.close()


def test_noalloc_step_rejects_sizes_beyond_the_array(srmod):
    lib = srmod.lib()
    params = srmod.make_params()
    dummy = torch.zeros(16, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    for H, W in [(1024, 512), (512, 1024), (48, 64)]:
        st = lib.sr_phi_step_noalloc(H, W, C.byref(params), p, p, p, p, p, p, p, None)
        assert st == srmod.SR_EUNSUPPORTED
    with pytest.raises(srmod.SRError, match="512 x 512"):
        big = torch.zeros((1024, 1024), device="cuda")
        srmod.phi_step_noalloc(params, big, big, big, big, big, big)
