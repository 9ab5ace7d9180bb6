"""sr_group_run: many images of uneven sizes in one graph launch, each with its
own device-side stopping test (a CUDA graph while-loop per member).

The stopping decisions are taken on the GPU from the same FP64 sums that
sr_iterate's stopping test reads, so they are predictable exactly: each member
is first iterated alone in bodies of B outer iterations, reading its
relative change after every body; a tolerance between those traces makes the
members stop after different numbers of bodies.  The group run must stop each
member exactly where its own trace crosses the tolerance and leave it
bit-identical to the member iterated alone for that many iterations."""
import pytest

from gpu_common import *  # noqa: F401,F403

pytestmark = pytest.mark.gpu

SIZES = [(128, 128), (96, 160), (256, 64), (64, 96), (160, 224), (64, 64)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


# members that take resident iterations when the group is built with them
RESIDENT_OK = {(128, 128), (256, 64), (64, 64)}


def _members(seed0, resident=False):
    ctxs = []
    for k, (H, W) in enumerate(SIZES):
        img = synth.ellipse_scene(seed0 + k, H=H, W=W, scale=max(min(H, W) / 512.0, 0.125))
        ctx = context(H, W, R=4, d=4.0)
        if resident and (H, W) in RESIDENT_OK:
            ctx.set_resident(True)
        ctx.edge_function(dev(img))
        ctx.set_phi(dev(synth.inset_rect_sdf(H, W)))
        ctxs.append(ctx)
    return ctxs


@pytest.mark.parametrize("resident", [False, True])
def test_group_run_stops_each_member_at_its_own_tolerance(resident):
    """With resident, three members run in the resident launch (one cluster
    each, two row lengths) and three in the graph."""
    B, bodies = 4, 6
    # traces: relative change after every body of B iterations, member alone
    alone = _members(300, resident)
    traces = []
    for ctx in alone:
        tr = []
        for _ in range(bodies):
            _, rel, _ = ctx.iterate(B, want_rel=True)
            tr.append(rel)
        traces.append(tr)
    for ctx in alone:
        ctx.close()
    # a tolerance that the members cross at different bodies
    flat = sorted(r for tr in traces for r in tr)
    tol = flat[len(flat) // 2]
    expect = []
    for tr in traces:
        n = next((b + 1 for b, r in enumerate(tr) if r <= tol), bodies)
        expect.append(n * B)
    assert len(set(expect)) > 1, "the members should stop at different iterations"
    grouped = _members(300, resident)
    grp = sr.Group(grouped)
    done, rel, converged = grp.run(bodies * B, tol, check_every=B)
    assert done == expect, (done, expect)
    for k, (d, r) in enumerate(zip(done, rel)):
        assert r == traces[k][d // B - 1]
    assert converged == all(tr[e // B - 1] <= tol for tr, e in zip(traces, expect))
    # each member equals the member iterated alone for as many iterations
    ref = _members(300, resident)
    for ctx, d in zip(ref, done):
        ctx.iterate(d)
    for a, b in zip(ref, grouped):
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(host(x), host(y))
    report("group_run", members=len(SIZES), resident=int(resident), tol=tol,
           outer_done=str(done))
    grp.close()
    for ctx in ref + grouped:
        ctx.close()


def test_group_run_reports_unconverged_and_odd_check_every():
    grouped = _members(400)
    grp = sr.Group(grouped)
    # check_every 3 runs bodies of 4 (parity-neutral); tol 0 never converges
    done, rel, converged = grp.run(8, 0.0, check_every=3)
    assert done == [8] * len(SIZES) and not converged
    assert all(np.isfinite(r) and r > 0 for r in rel)
    with pytest.raises(sr.SRError) as e:
        grp.run(2, 1e-3, check_every=3)  # max_outer below one body
    assert e.value.status == sr.SR_EINVAL
    grp.close()
    for ctx in grouped:
        ctx.close()


@pytest.mark.parametrize("n_iter", [5, 6])
def test_group_iterate_with_resident_members_matches_members_alone(n_iter):
    """sr_group_iterate with resident members: odd and even counts (the
    parity of the state), every member bit-identical to running alone."""
    grouped = _members(600, resident=True)
    grp = sr.Group(grouped)
    grp.iterate(n_iter)
    grp.iterate(3)
    alone = _members(600, resident=True)
    for c in alone:
        c.iterate(n_iter)
        c.iterate(3)
    for a, b in zip(alone, grouped):
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(host(x), host(y))
    grp.close()
    for c in alone + grouped:
        c.close()


def test_group_of_resident_members_only():
    """Every member resident: no graph at all, one launch per row length
    (two here); run and iterate still match the members alone bit for bit."""
    sizes = [(128, 128), (64, 64), (256, 64), (64, 64)]

    def members():
        out = []
        for k, (H, W) in enumerate(sizes):
            img = synth.ellipse_scene(700 + k, H=H, W=W, scale=0.125)
            ctx = context(H, W, R=4, d=4.0)
            ctx.set_resident(True)
            ctx.edge_function(dev(img))
            ctx.set_phi(dev(synth.inset_rect_sdf(H, W)))
            out.append(ctx)
        return out
    grouped = members()
    grp = sr.Group(grouped)
    assert grp.tune() in (4, 8, 16, 32, 64)
    grp.iterate(3)
    done, rel, _ = grp.run(8, 0.0, check_every=4)
    assert done == [8] * len(sizes)
    alone = members()
    for c in alone:
        c.iterate(3)
        c.iterate(8)
    for a, b in zip(alone, grouped):
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(host(x), host(y))
    grp.close()
    for c in alone + grouped:
        c.close()


def test_group_tune_picks_a_lane_count_and_leaves_the_states():
    """sr_group_tune times the group at several lane counts; the members'
    states come back bit for bit, and the tuned group still iterates every
    member exactly as alone."""
    grouped = _members(500)
    before = [[host(t) for t in c.get_state()] for c in grouped]
    grp = sr.Group(grouped)
    lanes = grp.tune()
    assert lanes in (4, 8, 16, 32, 64)
    for c, ref in zip(grouped, before):
        for x, y in zip(c.get_state(), ref):
            assert np.array_equal(host(x), y)
    grp.iterate(5)
    alone = _members(500)
    for c in alone:
        c.iterate(5)
    for a, b in zip(alone, grouped):
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(host(x), host(y))
    report("group_tune", members=len(SIZES), lanes=lanes)
    grp.close()
    for c in alone + grouped:
        c.close()
