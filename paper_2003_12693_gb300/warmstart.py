"""Learned warm start: generate (image, converged phi) pairs with the plain
solver, train the network of include/sr_net.h on them, and segment new images
from the network's phi0 with the plain iteration finishing the solve.

Orchestration only: the iterations, the network's passes and its optimiser
run in libsr.so's kernels.  The host side chooses batches and decides
convergence the same way for every start: every ``check`` outer iterations
the mask {phi < 0} (sr_mask) is compared either with a reference mask (the
image counts as converged once the intersection over union reaches ``iou``)
or, without a reference, with the previous check's mask (converged once at
most ``thr`` pixels changed).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import sr, sr_net


@dataclasses.dataclass
class Converged:
    iters: list[int]          # outer iterations until the mask settled, per image
    seconds: float            # wall time of the whole run (GPU work and checks)
    masks: list[torch.Tensor]
    settled: list[bool]       # False where max_iters ran out first


def _members(H, W, n, params):
    return [sr.Context(H, W, params) for _ in range(n)]


def _iou(a: torch.Tensor, b: torch.Tensor) -> float:
    inter = torch.logical_and(a > 0, b > 0).sum().item()
    union = torch.logical_or(a > 0, b > 0).sum().item()
    return 1.0 if union == 0 else inter / union


def converge_group(ctxs: list, group: "sr.Group | None", check: int, thr: int, max_iters: int,
                   ref=None, iou: float = 0.98) -> tuple[list[int], list[torch.Tensor], list[bool]]:
    """Iterate ``ctxs`` (all set up) in steps of ``check`` until every member
    has converged; with ``group`` the members advance together in one graph,
    else one after the other.  Returns per-member iterations, masks and
    whether each converged before ``max_iters``."""
    n = len(ctxs)
    prev = [c.mask() for c in ctxs]
    iters = [0] * n
    done = [False] * n
    if ref is not None:
        done = [_iou(prev[k], ref[k]) >= iou for k in range(n)]
    it = 0
    while it < max_iters and not all(done):
        if group is not None:
            group.iterate(check)
        else:
            for c, d in zip(ctxs, done):
                if not d:
                    c.iterate(check)
        it += check
        for k, c in enumerate(ctxs):
            if done[k]:
                continue
            m = c.mask()
            if ref is None:
                ok = int((m != prev[k]).sum().item()) <= thr
            else:
                ok = _iou(m, ref[k]) >= iou
            prev[k] = m
            iters[k] = it
            done[k] = ok
    return iters, prev, done


def solve_plain(images: torch.Tensor, phi0: torch.Tensor, params, check=50, thr=10,
                max_iters=8000, ref=None, iou=0.98) -> Converged:
    """One image after the other, each its own context (the plain GPU solver)."""
    B, H, W = images.shape
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters, masks, settled = [], [], []
    ctx = sr.Context(H, W, params)
    for k in range(B):
        ctx.edge_function(images[k])
        ctx.set_phi(phi0 if phi0.dim() == 2 else phi0[k])
        it, m, ok = converge_group([ctx], None, check, thr, max_iters,
                                   None if ref is None else [ref[k]], iou)
        iters += it
        masks += [m[0].clone()]
        settled += ok
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ctx.close()
    return Converged(iters, dt, masks, settled)


def solve_batched(images: torch.Tensor, phi0: torch.Tensor, params, check=50, thr=10,
                  max_iters=8000, ctxs=None, group=None, ref=None, iou=0.98) -> Converged:
    """All images in one group graph (sr_group_iterate); a member that
    converged keeps iterating with the others (its reported iteration count
    and mask are those of the check where it converged)."""
    B, H, W = images.shape
    own = ctxs is None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if own:
        ctxs = _members(H, W, B, params)
    for k, c in enumerate(ctxs):
        c.edge_function(images[k])
        c.set_phi(phi0 if phi0.dim() == 2 else phi0[k])
    if group is None:
        group = sr.Group(ctxs)
    iters, masks, settled = converge_group(ctxs, group, check, thr, max_iters, ref, iou)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if own:
        group.close()
        for c in ctxs:
            c.close()
    return Converged(iters, dt, masks, settled)


def generate_pairs(images: torch.Tensor, phi0: torch.Tensor, params, iters: int,
                   group_size: int = 64) -> torch.Tensor:
    """Converged level sets of the plain solver (``iters`` outer iterations
    from ``phi0``) for every image, in groups of ``group_size`` contexts whose
    graph is captured once and reused for every batch."""
    B, H, W = images.shape
    out = torch.empty_like(images)
    n = min(group_size, B)
    ctxs = _members(H, W, n, params)
    group = sr.Group(ctxs)
    for s in range(0, B, n):
        k_end = min(B, s + n)
        for k in range(s, s + n):
            c = ctxs[k - s]
            src = min(k, k_end - 1)          # a short last batch repeats its last image
            c.edge_function(images[src])
            c.set_phi(phi0 if phi0.dim() == 2 else phi0[src])
        group.iterate(iters)
        for k in range(s, k_end):
            ctxs[k - s].get_phi(out[k])
    group.close()
    for c in ctxs:
        c.close()
    return out


def train(net: "sr_net.Net", images: torch.Tensor, phi_star: torch.Tensor, steps: int,
          batch: int, lr: float, seed: int = 0, lr_final: float | None = None) -> list[float]:
    """Adam on random mini-batches (seeded), learning rate decayed by a cosine
    from ``lr`` to ``lr_final``.  Returns the loss of every step."""
    g = torch.Generator().manual_seed(seed)
    n = images.shape[0]
    lr_final = lr * 0.05 if lr_final is None else lr_final
    loss = torch.zeros(steps, dtype=torch.float64, device=images.device)
    fb = torch.empty((batch,) + tuple(images.shape[1:]), dtype=images.dtype, device=images.device)
    pb = torch.empty_like(fb)
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).to(images.device)
        torch.index_select(images, 0, idx, out=fb)
        torch.index_select(phi_star, 0, idx, out=pb)
        a = 0.5 * (1.0 + np.cos(np.pi * s / max(1, steps - 1)))
        net.train_step(fb, pb, lr_final + (lr - lr_final) * a, loss[s:s + 1])
    return loss.cpu().tolist()


# ----------------------------------------------------------------------------
# Experiment: what the trained network gains over the rectangle start
# ----------------------------------------------------------------------------
def _scene(args):
    from paper_2003_12693_gb300 import synth
    seed, n, noise = args
    return synth.ellipse_scene(seed, n, n, scale=n / 512.0, noise=noise).astype(np.float32)


def experiment(n: int = 128, n_train: int = 2048, n_eval: int = 32, t_ref: int = 3000,
               steps: int = 4000, batch: int = 32, lr: float = 2e-3, rho: float = 1e4,
               sigma: float = 3.0, check: int = 100, procs: int = 16) -> dict:
    """Generate n_train (image, phi after t_ref iterations) pairs of n x n
    ellipse scenes with the plain solver from the inset rectangle, train the
    network on them, then run n_eval held-out images (a) plain, one image per
    context, from the rectangle and (b) batched in one group from the
    network's phi0, each until its mask settles (at most 0.2 % of the pixels
    change over ``check`` iterations; at most 3 t_ref iterations)."""
    import multiprocessing as mp

    from scipy import ndimage

    from paper_2003_12693_gb300 import synth
    from paper_2003_12693_gb300 import warmstart as this   # picklable by module path
    with mp.get_context("spawn").Pool(procs) as pool:
        tr = np.stack(pool.map(this._scene, [(20000 + k, n, 0.1) for k in range(n_train)], 16))
        ev = np.stack(pool.map(this._scene, [(90000 + k, n, 0.1) for k in range(n_eval)], 2))
    torch.cuda.set_device(torch.cuda.current_device())
    prm = dict(synth.WORKLOADS["ellipses_512"].params())
    prm.update(rho=rho, sigma=sigma)
    p = sr.make_params(**prm)
    rect = torch.from_numpy(synth.inset_rect_sdf(n, n).astype(np.float32)).cuda()
    trd, evd = torch.from_numpy(tr).cuda(), torch.from_numpy(ev).cuda()
    t0 = time.perf_counter()
    phis = generate_pairs(trd, rect, p, t_ref)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    net = sr_net.Net(n, n, max_batch=max(batch, n_eval), phi_clip=4.0)
    layers = sr_net.layers()
    net.set_params(torch.from_numpy(synth.net_init(7, layers).astype(np.float32)).cuda())
    t0 = time.perf_counter()
    hist = train(net, trd, phis, steps, batch, lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    ref_phi = generate_pairs(evd, rect, p, t_ref)
    lossd = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.gradients(evd, ref_phi, lossd)
    tgt = torch.clamp(ref_phi, -4.0, 4.0) / 4.0
    rect_loss = 0.5 * torch.mean((torch.clamp(rect, -4.0, 4.0) / 4.0 - tgt) ** 2).item()
    thr = int(0.002 * n * n)
    mx = 3 * t_ref
    plain = solve_plain(evd, rect, p, check=check, thr=thr, max_iters=mx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phi0 = net.forward(evd)
    lb = solve_batched(evd, phi0, p, check=check, thr=thr, max_iters=mx)
    torch.cuda.synchronize()
    t_lb = time.perf_counter() - t0
    rb = solve_batched(evd, rect, p, check=check, thr=thr, max_iters=mx)
    ref_m = [(ref_phi[k] < 0).to(torch.uint8) for k in range(n_eval)]
    rect_m = (rect < 0).to(torch.uint8)
    comps = lambda m: ndimage.label(m.cpu().numpy() > 0)[1]  # noqa: E731
    return dict(
        size=n, train_pairs=n_train, t_ref=t_ref, train_steps=steps, batch=batch,
        pairs_s=t_pairs, train_s=t_train, loss_first=hist[0], loss_last=float(np.mean(hist[-50:])),
        heldout_loss=lossd.item(), rect_loss=rect_loss,
        start_iou_net=float(np.mean([_iou((phi0[k] < 0).to(torch.uint8), ref_m[k])
                                     for k in range(n_eval)])),
        start_iou_rect=float(np.mean([_iou(rect_m, ref_m[k]) for k in range(n_eval)])),
        settle_thr_px=thr, check=check, max_iters=mx,
        plain_iters=float(np.mean(plain.iters)), plain_settled=int(sum(plain.settled)),
        plain_s_per_image=plain.seconds / n_eval,
        learned_batched_iters=float(np.mean(lb.iters)), learned_batched_settled=int(sum(lb.settled)),
        learned_batched_s_per_image=t_lb / n_eval,
        rect_batched_iters=float(np.mean(rb.iters)), rect_batched_settled=int(sum(rb.settled)),
        rect_batched_s_per_image=rb.seconds / n_eval,
        final_iou_learned_vs_plain=float(np.mean([_iou(a, b) for a, b in
                                                  zip(plain.masks, lb.masks)])),
        topology_agree=int(sum(comps(a) == comps(b) for a, b in zip(plain.masks, lb.masks))))


def experiment_scale(n: int = 256, n_train: int = 20000, n_heldout: int = 1000, n_solve: int = 64,
                     t_ref: int = 3000, steps: int = 6000, batch: int = 32, lr: float = 2e-3,
                     rho: float = 1e4, sigma: float = 3.0, check: int = 50, iou: float = 0.9,
                     procs: int = 16) -> dict:
    """The warm start at its configured scale: n_train (image, phi after t_ref
    plain iterations) pairs of n x n six-ellipse scenes (seeds 20000 + k,
    noise drawn from U[0.05, 0.15]), training on all of them, then
    * on n_heldout held-out scenes (seeds 40000 + k): the network's loss and
      the overlap (IoU) of its start mask with the plain solver's mask after
      t_ref iterations, against the inset rectangle's;
    * on the first n_solve of them, "the same accuracy" read as reaching IoU
      >= iou with that plain mask: outer iterations and GPU-seconds per image
      until each image gets there, (a) plain from the rectangle one image at a
      time, (b) batched from the rectangle, (c) batched from the network's
      phi0 (network time included), at most 2 t_ref iterations; and the
      component counts of the final masks against the plain ones."""
    import multiprocessing as mp

    from scipy import ndimage

    from paper_2003_12693_gb300 import synth
    from paper_2003_12693_gb300 import warmstart as this
    rng = np.random.default_rng(12)
    noises = rng.uniform(0.05, 0.15, n_train + n_heldout)
    with mp.get_context("spawn").Pool(procs) as pool:
        tr = np.stack(pool.map(this._scene, [(20000 + k, n, float(noises[k])) for k in range(n_train)], 64))
        ev = np.stack(pool.map(this._scene, [(40000 + k, n, float(noises[n_train + k]))
                                             for k in range(n_heldout)], 16))
    prm = dict(synth.WORKLOADS["ellipses_512"].params())
    prm.update(rho=rho, sigma=sigma)
    p = sr.make_params(**prm)
    rect = torch.from_numpy(synth.inset_rect_sdf(n, n).astype(np.float32)).cuda()
    trd, evd = torch.from_numpy(tr).cuda(), torch.from_numpy(ev).cuda()
    del tr, ev
    t0 = time.perf_counter()
    phis = generate_pairs(trd, rect, p, t_ref)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    net = sr_net.Net(n, n, max_batch=max(batch, n_solve), phi_clip=4.0)
    layers = sr_net.layers()
    net.set_params(torch.from_numpy(synth.net_init(7, layers).astype(np.float32)).cuda())
    t0 = time.perf_counter()
    hist = train(net, trd, phis, steps, batch, lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del phis
    ref_phi = generate_pairs(evd, rect, p, t_ref)
    ref_m = (ref_phi < 0).to(torch.uint8)
    rect_m = (rect < 0).to(torch.uint8)
    losses, start_iou_net, start_iou_rect, rect_losses = [], [], [], []
    tgt = torch.clamp(ref_phi, -4.0, 4.0) / 4.0
    lossd = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s in range(0, n_heldout, n_solve):
        e = min(n_heldout, s + n_solve)
        phi0 = net.forward(evd[s:e])
        net.gradients(evd[s:e], ref_phi[s:e], lossd)
        losses.append(lossd.item() * (e - s))
        for k in range(e - s):
            start_iou_net.append(_iou((phi0[k] < 0).to(torch.uint8), ref_m[s + k]))
            start_iou_rect.append(_iou(rect_m, ref_m[s + k]))
        rect_losses.append(0.5 * torch.mean((torch.clamp(rect, -4.0, 4.0) / 4.0 - tgt[s:e]) ** 2).item()
                           * (e - s))
    mx = 2 * t_ref
    ev_s, ref_s = evd[:n_solve], [ref_m[k] for k in range(n_solve)]
    plain = solve_plain(ev_s, rect, p, check=check, thr=0, max_iters=mx, ref=ref_s, iou=iou)
    rb = solve_batched(ev_s, rect, p, check=check, thr=0, max_iters=mx, ref=ref_s, iou=iou)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phi0 = net.forward(ev_s)
    lb = solve_batched(ev_s, phi0, p, check=check, thr=0, max_iters=mx, ref=ref_s, iou=iou)
    torch.cuda.synchronize()
    t_lb = time.perf_counter() - t0
    comps = lambda m: ndimage.label(m.cpu().numpy() > 0)[1]  # noqa: E731
    return dict(
        size=n, train_pairs=n_train, heldout=n_heldout, solved=n_solve, t_ref=t_ref,
        train_steps=steps, batch=batch, rho=rho, sigma=sigma, pairs_s=t_pairs, train_s=t_train,
        loss_first=hist[0], loss_last=float(np.mean(hist[-100:])),
        heldout_loss=sum(losses) / n_heldout, heldout_rect_loss=sum(rect_losses) / n_heldout,
        start_iou_net=float(np.mean(start_iou_net)), start_iou_rect=float(np.mean(start_iou_rect)),
        accuracy=f"IoU >= {iou} with the plain mask after {t_ref} iterations", check=check,
        max_iters=mx,
        plain_iters=float(np.mean(plain.iters)), plain_reached=int(sum(plain.settled)),
        plain_s_per_image=plain.seconds / n_solve,
        rect_batched_iters=float(np.mean(rb.iters)), rect_batched_reached=int(sum(rb.settled)),
        rect_batched_s_per_image=rb.seconds / n_solve,
        learned_batched_iters=float(np.mean(lb.iters)), learned_batched_reached=int(sum(lb.settled)),
        learned_batched_s_per_image=t_lb / n_solve,
        speedup_learned_batched_vs_plain=(plain.seconds / n_solve) / (t_lb / n_solve),
        topology_agree=int(sum(comps(a) == comps(b) for a, b in zip(plain.masks, lb.masks))))


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned warm start versus the rectangle start")
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--train", type=int, default=2048)
    ap.add_argument("--t-ref", type=int, default=3000)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--scale", action="store_true",
                    help="the configured scale: 20k pairs at 256^2, 1000 held-out images")
    a = ap.parse_args()
    if a.scale:
        print(json.dumps(experiment_scale(n=a.size, n_train=a.train, t_ref=a.t_ref, steps=a.steps)))
    else:
        print(json.dumps(experiment(n=a.size, n_train=a.train, t_ref=a.t_ref, steps=a.steps)))
