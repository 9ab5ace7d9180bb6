"""Learned warm start: generate (image, converged phi) pairs with the plain
solver, train the network of include/sr_net.h on them, and segment new images
from the network's phi0 with the plain iteration finishing the solve.

Orchestration only: the iterations, the network's passes and its optimiser
run in libsr.so's kernels.  The host side chooses batches and judges
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
