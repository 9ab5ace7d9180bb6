"""Resident outer iterations (sr_set_resident): whole iterations of Alg. 1 in
one launch, the state held in the shared memory of one cluster of 8 or 16
CTAs.

Against the FP64 oracle: one outer iteration from oracle states along the
128^2 workload's trajectory and from random states with narrow-band pixels
everywhere (every pixel of phi within 1e-4, w and b by the propagation bound
of the default path's tests), on shapes that put the window halo, the
stencil neighbours and the column recursions' warm-ups across several CTAs
(rows per CTA from 2 to 64, R from 0 to 8).  Against the default path: the
stopping test's residual over several calls (odd and even iteration counts)
and a run stopped by a tolerance, with the test evaluated on the device.
The unsupported configurations are refused."""
import os
import sys

import pytest

from gpu_common import *  # noqa: F401,F403

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_oracle_runs as refs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("K0", [0, 10, 60, 199])
def test_resident_one_iteration_two_disks(K0):
    wl = synth.WORKLOADS["two_disks_128"]
    p = oracle.Params.from_dict(wl.params())
    g64 = f32(oracle.edge(wl.image()))
    state = rounded_state(oracle_state_after(wl.phi0(), g64, K0, p))
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
    ctx.set_resident(True)
    gpu, ref = one_iteration_both(ctx, state, g64, p)
    err, nex = check_one_iteration(gpu, ref, state, g64, p)
    report("resident_one_iteration", shape="128x128", K0=K0, max_abs_dphi=err,
           exempt_pixels=nex)
    assert nex < 200
    ctx.close()


@pytest.mark.parametrize("shape,R,d", [((64, 256), 4, 4.0), ((256, 64), 8, 8.0),
                                       ((512, 32), 3, 3.0), ((16, 32), 0, 1.0),
                                       ((32, 128), 2, 2.0), ((128, 128), 8, 8.0)])
@pytest.mark.parametrize("cluster", ["8", "16"])
def test_resident_one_iteration_random_states(shape, R, d, cluster, monkeypatch):
    """Both cluster sizes (SR_RESIDENT_CLUSTER): 2 to 64 rows per CTA."""
    H, W = shape
    phi, w1, w2, b1, b2, g = (f32(a) for a in synth.random_state(H, W, seed=H + 7 * W + R))
    p = oparams(R=R, d=d)
    ctx = context(H, W, R=R, d=d)
    monkeypatch.setenv("SR_RESIDENT_CLUSTER", cluster)
    if H < 2 * int(cluster):
        with pytest.raises(sr.SRError) as e:
            ctx.set_resident(True)
        assert e.value.status == sr.SR_EUNSUPPORTED
        ctx.close()
        return
    ctx.set_resident(True)
    state = [phi, w1, w2, b1, b2]
    gpu, ref = one_iteration_both(ctx, state, g, p)
    err, nex = check_one_iteration(gpu, ref, state, g, p)
    report("resident_one_iteration", shape=f"{H}x{W}", R=R, cluster=cluster, max_abs_dphi=err,
           exempt_pixels=nex)
    assert nex < 0.01 * H * W
    ctx.close()


def _start(resident, **kw):
    """The 128^2 two-disk workload from the tie-free rectangle (no pixel
    equidistant from two edges, so that the early iterations are unique to
    rounding; see tests/golden/make_oracle_runs.py)."""
    wl = synth.WORKLOADS["two_disks_128"]
    ctx = context(wl.H, wl.W, R=wl.R, d=wl.d, **kw)
    if resident:
        ctx.set_resident(True)
    ctx.edge_function(dev(wl.image()))
    ctx.set_phi(dev(refs.tie_free_phi0("two_disks_128", wl.H, wl.W)))
    return ctx


def _run_checks(resident, calls, n):
    """Residual after each of `calls` calls of n iterations."""
    ctx = _start(resident, check_every=5)
    trace = [ctx.iterate(n, want_rel=True)[1] for _ in range(calls)]
    return ctx, trace


def test_resident_stopping_test_matches_default_path():
    """The residual of Sec. 4's stopping test after calls of 1, 5 and 6
    iterations (odd and even counts: the state's parity alternates), and a
    run stopped by a tolerance placed between two checks: the resident run
    stops after the same number of iterations as the default path, with the
    same residual to rounding (global norms: 5 % relative over 30 iterations,
    where single pixels already differ by more)."""
    for n in (1, 5, 6):
        a, ta = _run_checks(False, 5, n)
        b, tb = _run_checks(True, 5, n)
        for x, y in zip(ta, tb):
            assert abs(x - y) <= 5e-2 * abs(x), (n, ta, tb)
        report("resident_vs_default", iterations=5 * n, rel_default=ta[-1], rel_resident=tb[-1],
               max_abs_dphi=float(np.abs(host(a.get_phi()) - host(b.get_phi())).max()))
        a.close()
        b.close()
    # the default path's residual every 5 iterations; the tolerance goes
    # between the first check that falls clearly below all earlier ones and
    # those earlier ones
    ref, tr = _run_checks(False, 12, 5)
    ref.close()
    delta = 0.05
    js = [j for j in range(1, len(tr)) if tr[j] * (1 + delta) ** 2 < min(tr[:j])]
    assert js, f"no check with a clear drop in the residual trace {tr}"
    j = js[0]
    tol = tr[j] * (1 + delta)
    out = {}
    for resident in (False, True):
        ctx = _start(resident, check_every=5)
        out[resident] = ctx.iterate(5 * len(tr), tol=tol)
        ctx.close()
    assert out[True][0] == out[False][0] == 5 * (j + 1), (out, tr, tol)
    assert out[True][2] and out[False][2]
    assert abs(out[True][1] - out[False][1]) <= 5e-2 * out[False][1]
    report("resident_stop", tol=tol, outer_done=out[True][0], rel_default=out[False][1],
           rel_resident=out[True][1])


def test_resident_switching_keeps_the_state():
    """An iteration on each path gives the state of the default path alone to
    rounding (phi within 1e-4 after two iterations from the tie-free start,
    the early-iteration bar at 128^2; w unit or zero)."""
    out = []
    for order in ((True, False), (False, True), (True, True), (False, False)):
        ctx = _start(False)
        for resident in order:
            ctx.set_resident(resident)
            ctx.iterate(1)
        out.append([host(t) for t in ctx.get_state()])
        ctx.close()
    for k, st in enumerate(out[:3]):
        err = float(np.abs(st[0] - out[3][0]).max())
        report("resident_switching", order=k, max_abs_dphi=err)
        assert err <= PHI_TOL, (k, err)
        n = np.hypot(st[1], st[2])
        assert np.all((n == 0) | (np.abs(n - 1) < 1e-5))


def test_resident_cluster_size_by_argument():
    """sr_set_resident(ctx, 8 or 16) fixes the cluster size: the two runs
    agree with the oracle's one-iteration bar and are refused where the rows
    do not divide (16 CTAs need H >= 32)."""
    wl = synth.WORKLOADS["two_disks_128"]
    p = oracle.Params.from_dict(wl.params())
    g64 = f32(oracle.edge(wl.image()))
    state = rounded_state(oracle_state_after(wl.phi0(), g64, 10, p))
    for cl in (8, 16):
        ctx = context(wl.H, wl.W, R=wl.R, d=wl.d)
        ctx.set_resident(True, cluster=cl)
        gpu, ref = one_iteration_both(ctx, state, g64, p)
        check_one_iteration(gpu, ref, state, g64, p)
        ctx.close()
    ctx = context(16, 32)
    with pytest.raises(sr.SRError) as e:
        ctx.set_resident(True, cluster=16)
    assert e.value.status == sr.SR_EUNSUPPORTED
    assert sr.lib().sr_set_resident(ctx.handle, 4) == sr.SR_EINVAL  # only 0, 1, 8, 16
    ctx.close()


def test_resident_unsupported_configurations():
    for shape in [(16, 512), (128, 512)]:
        ctx = context(*shape)
        with pytest.raises(sr.SRError) as e:
            ctx.set_resident(True)
        assert e.value.status == sr.SR_EUNSUPPORTED
        ctx.close()
    ctx = context(64, 64)
    ctx.set_w_sweeps(2)
    with pytest.raises(sr.SRError) as e:
        ctx.set_resident(True)
    assert e.value.status == sr.SR_EUNSUPPORTED
    ctx.close()
    # tau mu beyond the recursions' warm-up buckets
    ctx = context(64, 64, tau=1.0, mu=40.0)
    with pytest.raises(sr.SRError) as e:
        ctx.set_resident(True)
    assert e.value.status == sr.SR_EUNSUPPORTED
    ctx.close()
