"""Host logic of the warm-start module on CPU, with fake solver contexts and
a fake network (no GPU): the convergence rules and the training loop's
batching and learning-rate schedule."""
import numpy as np
import torch

from paper_2003_12693_gb300 import warmstart as wsm


class FakeCtx:
    """A context whose mask is a scripted function of its iteration count."""

    def __init__(self, script):
        self.it = 0
        self.script = script

    def iterate(self, n):
        self.it += n

    def mask(self):
        return self.script(self.it)


class FakeGroup:
    def __init__(self, ctxs):
        self.ctxs = ctxs

    def iterate(self, n):
        for c in self.ctxs:
            c.iterate(n)


def shrinking(stop_at, side=64):
    """A square mask that loses a row every 10 iterations until stop_at."""
    def f(it):
        rows = min(it, stop_at) // 10
        m = torch.zeros((side, side), dtype=torch.uint8)
        m[rows:, :] = 1
        return m
    return f


def test_mask_change_rule_settles_after_the_motion_stops():
    ctx = FakeCtx(shrinking(300))
    iters, masks, done = wsm.converge_group([ctx], None, check=50, thr=10, max_iters=2000)
    # rows change by 5 per check (320 px) until 300; the check at 350 sees no change
    assert done == [True] and iters == [350]
    assert int(masks[0].sum()) == (64 - 30) * 64


def test_reference_rule_stops_at_the_first_close_check():
    ref = [shrinking(300)(10_000)]
    ctx = FakeCtx(shrinking(300))
    iters, _, done = wsm.converge_group([ctx], None, check=50, thr=0, max_iters=2000, ref=ref,
                                        iou=0.9)
    # IoU = (64 - 30) / (64 - rows) >= 0.9 first when rows >= 27, i.e. it >= 270 -> check 300
    assert done == [True] and iters == [300]


def test_cap_reports_not_settled():
    ctx = FakeCtx(shrinking(10_000))
    iters, _, done = wsm.converge_group([ctx], None, check=100, thr=10, max_iters=500)
    assert done == [False] and iters == [500]


def test_group_members_keep_their_own_settling_check():
    ctxs = [FakeCtx(shrinking(100)), FakeCtx(shrinking(400))]
    iters, _, done = wsm.converge_group(ctxs, FakeGroup(ctxs), check=50, thr=10, max_iters=2000)
    assert done == [True, True] and iters == [150, 450]


def test_iou_helper():
    a = torch.zeros((4, 4), dtype=torch.uint8)
    b = torch.zeros((4, 4), dtype=torch.uint8)
    assert wsm._iou(a, b) == 1.0
    a[:2] = 1
    b[1:3] = 1
    assert wsm._iou(a, b) == 4 / 12


class FakeNet:
    def __init__(self):
        self.lrs, self.batches = [], []

    def train_step(self, f, phi, lr, loss):
        self.lrs.append(lr)
        self.batches.append((f.clone(), phi.clone()))
        loss.fill_(1.0 / len(self.lrs))


def test_train_batches_pairs_and_decays_the_rate():
    n, H = 10, 4
    imgs = torch.arange(n, dtype=torch.float32)[:, None, None].expand(n, H, H).contiguous()
    phis = -imgs
    net = FakeNet()
    hist = wsm.train(net, imgs, phis, steps=50, batch=3, lr=1e-2, seed=1)
    assert len(hist) == 50 and hist[0] == 1.0
    assert net.lrs[0] == 1e-2 and abs(net.lrs[-1] - 5e-4) < 1e-12
    assert all(a >= b - 1e-15 for a, b in zip(net.lrs, net.lrs[1:]))      # monotone cosine
    for f, p in net.batches:
        assert f.shape == (3, H, H) and torch.equal(p, -f)                 # pairs stay paired
    seen = {int(v) for f, _ in net.batches for v in f[:, 0, 0].tolist()}
    assert len(seen) >= 8                                                  # random batches
    net2 = FakeNet()
    wsm.train(net2, imgs, phis, steps=50, batch=3, lr=1e-2, seed=1)
    assert all(torch.equal(a[0], b[0]) for a, b in zip(net.batches, net2.batches))  # seeded
