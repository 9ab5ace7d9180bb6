"""Failure detection on the GPU without faulting, hanging or exhausting it.

* A bounded device-side wait that runs out: the TMA column pass is told to
  wait on a shared-memory barrier that nothing arrives on, with a short
  limit; the kernel records a timeout, drains its own transfers and returns,
  and the host sees SR_ETIMEOUT.  The context stays usable: with normal
  waits the same iterations from the same state give bit-identical results.
* An allocation failure: the library's allocation hook makes the n-th
  allocation of sr_create fail as if memory had run out; sr_create returns
  SR_ENOMEM, frees what it had allocated, and a later sr_create succeeds.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_common import context, dev, host
from paper_2003_12693_gb300 import sr, synth

pytestmark = pytest.mark.gpu


def _scene_context(H, W):
    ctx = context(H, W, R=4, d=4.0)
    ctx.edge_function(dev(synth.ellipse_scene(2, H, W)))
    ctx.set_phi(dev(synth.inset_rect_sdf(H, W)))
    return ctx


def test_stalled_tma_wait_returns_timeout_and_context_recovers():
    H = W = 512
    ctx = _scene_context(H, W)
    sc = ctx.get_schedule()
    ctx.set_schedule(sc["row_values_per_thread"], sc["row_threads"], 3)  # the TMA column pass
    ctx.iterate(2)
    state0 = [t.clone() for t in ctx.get_state()]
    ctx.iterate(3, want_rel=True)
    ref = host(ctx.get_phi())

    ctx.set_state(*state0)
    assert sr.lib().sr_test_stall_waits(ctx.handle, 2000) == sr.SR_OK
    with pytest.raises(sr.SRError) as err:
        ctx.iterate(1, want_rel=True)
    assert err.value.status == sr.SR_ETIMEOUT
    # the error flag was cleared by the call that reported it
    assert sr.lib().sr_test_stall_waits(ctx.handle, 0) == sr.SR_OK
    ctx.set_state(*state0)
    done, rel, ok = ctx.iterate(3, want_rel=True)
    assert ok and done == 3 and np.isfinite(rel)
    assert np.array_equal(host(ctx.get_phi()), ref)
    ctx.close()


def test_allocation_failure_returns_enomem_and_frees_everything():
    L = sr.lib()
    H = W = 2048
    p = sr.make_params(win_radius=4, d=4.0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for n in (0, 1, 7, 14, 18, 22, 28):
            assert L.sr_test_fail_allocations(n) == sr.SR_OK
            h = C.c_void_p()
            st = L.sr_create(H, W, C.byref(p), None, C.byref(h))
            assert st == sr.SR_ENOMEM, (n, st)
            assert not h.value
    finally:
        L.sr_test_fail_allocations(-1)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # one leaked image plane would be 16 MiB
    assert abs(free0 - free1) < 4 * 2 ** 20, (free0, free1)
    ctx = sr.Context(H, W, p)
    ctx.close()
