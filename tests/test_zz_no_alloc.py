"""sr_phi_step_noalloc: the inner phi step for callers that cannot allocate.

Some hosts own all GPU memory through their own arena, capture streams into
CUDA graphs in modes that forbid allocation, or run real-time loops that
cannot take the device synchronisation of cudaMalloc / cudaFree.  This entry
point serves them from a fixed device array inside the library.  The test
calls it through the C-ABI twice in a row, with different sizes and windows,
and checks each result against the context-based sr_phi_step within the
tolerance the other tests use for phi (1e-4).  It is collected last so that a
run stopping at the first failure has run every other test before it.
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
    from paper_2003_12693_gb300 import synth
    arrs = synth.random_state(H, W, seed=seed)
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in arrs]


def test_noalloc_step_matches_context_step_on_two_calls(srmod):
    lib = srmod.lib()
    stream = torch.cuda.current_stream()
    for H, W, R, d, seed in [(128, 128, 3, 3.0, 1), (256, 64, 4, 4.0, 2)]:
        phi, w1, w2, b1, b2, g = _inputs(H, W, seed)
        params = srmod.make_params(win_radius=R, d=d)
        ctx = srmod.Context(H, W, params)
        ctx.set_g(g)
        ref = ctx.phi_step(phi, w1, w2, b1, b2)
        out = torch.full_like(phi, float("nan"))
        st = lib.sr_phi_step_noalloc(H, W, C.byref(params),
                                     *[C.c_void_p(t.data_ptr())
                                       for t in (g, phi, w1, w2, b1, b2, out)],
                                     C.c_void_p(stream.cuda_stream))
        assert st == srmod.SR_OK
        torch.cuda.synchronize()
        err = float((out - ref).abs().max())
        assert err <= PHI_TOL, (H, W, err)
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
