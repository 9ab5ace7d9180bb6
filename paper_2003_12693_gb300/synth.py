"""Seeded synthetic inputs for the Split Bregman self-repelling snake.

This module holds no step of the method: it only draws images f and initial
level sets phi0, so that the FP64 oracle and the CUDA path consume the very
same arrays.  The paper's own images (two circles and the synthetic hand of
its Figs. 1 and 3, the cells of Fig. 4, the wheat grains of Fig. 5, the CT
mandible of Fig. 6) are not available; the scenes below reproduce their
geometry instead: objects separated by thin gaps that a plain geodesic active
contour would bridge, and thin ribbons that it would cut (Sec. 5).

Conventions: arrays are float64, row-major, shape (H, W); row index i, column
index j; pixel (i, j) sits at the point (i, j).  The initial level set is the
signed distance of Sec. 2, Eq. (3): negative inside the contour, positive
outside (Alg. 1 initialises phi0 as a signed distance function).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Fig. 1 parameter set (Sec. 5): alpha=4, gamma=4, beta=0.2, mu=8, l=1,
# S=3, eps=1, tau=0.1, Tol=1e-5.
FIG1_PARAMS = dict(alpha=4.0, beta=0.2, gamma=4.0, mu=8.0, tau=0.1, eps=1.0,
                   band_l=1.0, inner_S=3, rho=1.0, sigma=1.0, s_pow=2)


def rect_sdf(H: int, W: int, r0: float, r1: float, c0: float, c1: float,
             clip: float | None = None) -> np.ndarray:
    """Exact Euclidean signed distance to the box [r0, r1] x [c0, c1].

    Negative inside, zero on the edges, positive outside (Eq. (3)).  Inside a
    convex box the distance to the boundary is the distance to the nearest
    edge; outside it is the distance to the box.  ``clip`` optionally limits
    |phi|; it is off by default because a clipped distance has flat regions
    where the forward gradient is exactly zero.
    """
    i = np.arange(H, dtype=np.float64)[:, None]
    j = np.arange(W, dtype=np.float64)[None, :]
    dx = np.maximum(np.maximum(r0 - i, i - r1), 0.0)
    dy = np.maximum(np.maximum(c0 - j, j - c1), 0.0)
    outside = np.sqrt(dx * dx + dy * dy)
    inside = np.minimum(np.minimum(i - r0, r1 - i), np.minimum(j - c0, c1 - j))
    phi = np.where(outside > 0.0, outside, -inside)
    if clip is not None:
        phi = np.clip(phi, -clip, clip)
    return np.ascontiguousarray(phi)


def inset_rect_sdf(H: int, W: int, inset: int = 8, clip: float | None = None) -> np.ndarray:
    """Signed distance of the rectangle inset ``inset`` pixels from the border."""
    return rect_sdf(H, W, inset, H - 1 - inset, inset, W - 1 - inset, clip)


# ----------------------------------------------------------------------------
# Scenes
# ----------------------------------------------------------------------------

def two_disks(seed: int = 1, H: int = 128, W: int = 128, radius: float = 20.0,
              centres=((64, 42), (64, 86)), noise: float = 0.05) -> np.ndarray:
    """Two disks of intensity 1 on 0 plus N(0, noise^2) (Fig. 1 stand-in).

    With radius 20 and centres 44 px apart the disks leave a 4 px gap.
    """
    rng = np.random.default_rng(seed)
    i = np.arange(H)[:, None]
    j = np.arange(W)[None, :]
    img = np.zeros((H, W))
    for ci, cj in centres:
        img[(i - ci) ** 2 + (j - cj) ** 2 <= radius * radius] = 1.0
    return img + rng.normal(0.0, noise, (H, W))


@dataclasses.dataclass
class Ellipse:
    ci: float
    cj: float
    a: float          # semi-axis along the rotated row direction
    b: float          # semi-axis along the rotated column direction
    theta: float
    value: float
    ribbon: float = 0.0   # >0: ring of this width instead of a filled ellipse

    def _local(self, H: int, W: int, i0: int = 0, j0: int = 0):
        i = np.arange(i0, i0 + H, dtype=np.float64)[:, None] - self.ci
        j = np.arange(j0, j0 + W, dtype=np.float64)[None, :] - self.cj
        c, s = math.cos(self.theta), math.sin(self.theta)
        x = c * i + s * j
        y = -s * i + c * j
        return x, y

    def mask(self, H: int, W: int, i0: int = 0, j0: int = 0) -> np.ndarray:
        """Rasterise on the H x W window whose top-left pixel is (i0, j0)."""
        x, y = self._local(H, W, i0, j0)
        q = (x / self.a) ** 2 + (y / self.b) ** 2
        if self.ribbon <= 0.0:
            return q <= 1.0
        # first-order distance to the boundary curve q = 1
        gx = 2.0 * x / (self.a * self.a)
        gy = 2.0 * y / (self.b * self.b)
        dist = (q - 1.0) / np.maximum(np.sqrt(gx * gx + gy * gy), 1e-12)
        return np.abs(dist) <= 0.5 * self.ribbon

    def half_extent(self) -> tuple[float, float]:
        c, s = math.cos(self.theta), math.sin(self.theta)
        ei = math.hypot(self.a * c, self.b * s)
        ej = math.hypot(self.a * s, self.b * c)
        pad = 0.5 * self.ribbon
        return ei + pad, ej + pad


def _fits(e: Ellipse, H: int, W: int, margin: int) -> bool:
    ei, ej = e.half_extent()
    return (e.ci - ei >= margin and e.ci + ei <= H - 1 - margin
            and e.cj - ej >= margin and e.cj + ej <= W - 1 - margin)


def _random_ellipse(rng, H, W, semi, margin, value, ribbon=0.0, tries=200):
    for _ in range(tries):
        a = rng.uniform(*semi)
        b = rng.uniform(*semi)
        theta = rng.uniform(0.0, math.pi)
        e = Ellipse(0.0, 0.0, a, b, theta, value, ribbon)
        ei, ej = e.half_extent()
        lo_i, hi_i = margin + ei, H - 1 - margin - ei
        lo_j, hi_j = margin + ej, W - 1 - margin - ej
        if lo_i > hi_i or lo_j > hi_j:
            continue
        e.ci = rng.uniform(lo_i, hi_i)
        e.cj = rng.uniform(lo_j, hi_j)
        return e
    raise RuntimeError("could not place an ellipse; image too small for the semi-axis range")


def _partner(rng, first: Ellipse, H, W, semi, margin, gap, value, tries=60):
    """Place a second ellipse so that ``gap`` background pixels separate the two.

    Bisection on the centre offset along a random direction until the closest
    pixels of the two rasterised ellipses are gap + 1 apart (gap pixels lie
    between them on the closest line).  The distance map of the first ellipse
    is computed once on a window around the pair; the second is rasterised on
    its own bounding box only.
    """
    from scipy import ndimage
    for _ in range(tries):
        a = rng.uniform(*semi)
        b = rng.uniform(*semi)
        theta = rng.uniform(0.0, math.pi)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        di, dj = math.cos(ang), math.sin(ang)
        d_max = first.a + first.b + a + b + gap + 4.0
        reach = int(math.ceil(d_max + max(a, b) + 4))
        i0, j0 = int(first.ci) - reach, int(first.cj) - reach
        size = 2 * reach + 1
        dist_a = ndimage.distance_transform_edt(~first.mask(size, size, i0, j0))

        def make(D):
            return Ellipse(first.ci + D * di, first.cj + D * dj, a, b, theta, value)

        def separated(D):
            e = make(D)
            ei, ej = e.half_extent()
            bi0, bj0 = int(math.floor(e.ci - ei)) - 1, int(math.floor(e.cj - ej)) - 1
            bi1, bj1 = int(math.ceil(e.ci + ei)) + 1, int(math.ceil(e.cj + ej)) + 1
            mb = e.mask(bi1 - bi0 + 1, bj1 - bj0 + 1, bi0, bj0)
            sub = dist_a[bi0 - i0:bi1 - i0 + 1, bj0 - j0:bj1 - j0 + 1]
            return (not mb.any()) or float(sub[mb].min()) >= gap + 1

        lo, hi = 0.0, d_max
        if not separated(hi):
            continue
        for _ in range(30):
            mid = 0.5 * (lo + hi)
            if separated(mid):
                hi = mid
            else:
                lo = mid
        e = make(hi)
        if _fits(e, H, W, margin):
            return e
    return None


def ellipse_scene(seed: int, H: int = 512, W: int = 512, scale: float = 1.0,
                  semi=(10.0, 80.0), n_ribbons: int = 2, n_gap_pairs: int = 2,
                  gap: int = 2, ribbon_width: float = 3.0, noise: float = 0.1,
                  margin: int = 8, min_semi: float = 4.0) -> np.ndarray:
    """Six ellipses: ``n_ribbons`` thin rings and ``n_gap_pairs`` pairs ``gap`` px apart.

    Objects take intensities U[0.5, 1] on a background U[0, 0.2] in painter's
    order, then N(0, noise^2) is added.  ``scale`` multiplies the semi-axes
    (not the ribbon width or the gap), clamped below at ``min_semi``.
    """
    rng = np.random.default_rng(seed)
    lo = max(semi[0] * scale, min_semi)
    hi = max(semi[1] * scale, lo + 1.0)
    semi_s = (lo, hi)
    bg = rng.uniform(0.0, 0.2)
    img = np.full((H, W), bg)
    objects: list[Ellipse] = []
    for _ in range(n_ribbons):
        objects.append(_random_ellipse(rng, H, W, semi_s, margin,
                                       rng.uniform(0.5, 1.0), ribbon=ribbon_width))
    for _ in range(n_gap_pairs):
        for _attempt in range(50):
            first = _random_ellipse(rng, H, W, semi_s, margin, rng.uniform(0.5, 1.0))
            second = _partner(rng, first, H, W, semi_s, margin, gap, rng.uniform(0.5, 1.0))
            if second is not None:
                objects += [first, second]
                break
        else:
            raise RuntimeError("could not place a gap pair")
    for e in objects:
        img[e.mask(H, W)] = e.value
    return img + rng.normal(0.0, noise, (H, W))


def blob_pairs_scene(seed: int = 5, H: int = 4096, W: int = 4096, grid: int = 10,
                     semi=(15.0, 60.0), gaps=(1, 2, 3), noise: float = 0.15,
                     margin: int = 8) -> np.ndarray:
    """grid x grid jittered cells, each holding a pair of ellipses 1-3 px apart."""
    rng = np.random.default_rng(seed)
    bg = rng.uniform(0.0, 0.2)
    img = np.full((H, W), bg)
    ch, cw = (H - 2 * margin) / grid, (W - 2 * margin) / grid
    for gi in range(grid):
        for gj in range(grid):
            i0 = int(margin + gi * ch)
            j0 = int(margin + gj * cw)
            sh, sw = int(ch), int(cw)
            gap = int(rng.choice(gaps))
            # place the pair inside the cell's own sub-image (cheap rasterisation)
            for _attempt in range(50):
                first = _random_ellipse(rng, sh, sw, semi, 4, rng.uniform(0.5, 1.0))
                second = _partner(rng, first, sh, sw, semi, 4, gap, rng.uniform(0.5, 1.0))
                if second is not None:
                    break
            else:
                raise RuntimeError("could not place a blob pair")
            # jitter the pair inside the cell
            sub = np.zeros((sh, sw), dtype=bool)
            sub_val = np.zeros((sh, sw))
            for e in (first, second):
                m = e.mask(sh, sw)
                sub[m] = True
                sub_val[m] = e.value
            rows = np.nonzero(sub.any(1))[0]
            cols = np.nonzero(sub.any(0))[0]
            si = int(rng.integers(-rows[0] + 1, sh - rows[-1] - 1)) if rows[0] > 1 and sh - rows[-1] > 2 else 0
            sj = int(rng.integers(-cols[0] + 1, sw - cols[-1] - 1)) if cols[0] > 1 and sw - cols[-1] > 2 else 0
            sub = np.roll(sub, (si, sj), (0, 1))
            sub_val = np.roll(sub_val, (si, sj), (0, 1))
            view = img[i0:i0 + sh, j0:j0 + sw]
            view[sub] = sub_val[sub]
    return img + rng.normal(0.0, noise, (H, W))


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    H: int
    W: int
    R: int          # repulsion window half-width (the workload's "l")
    d: float        # Gaussian scale of the window
    K: int          # outer iterations
    description: str

    def image(self) -> np.ndarray:
        return _IMAGES[self.name]()

    def phi0(self) -> np.ndarray:
        return _PHI0[self.name]()

    def params(self) -> dict:
        p = dict(FIG1_PARAMS)
        p.update(d=float(self.d), win_radius=int(self.R))
        return p


WORKLOADS = {
    "two_disks_128": Workload(
        "two_disks_128", 128, 128, 3, 3.0, 200,
        "128x128 two disks r=20, 4 px gap, noise 0.05, seed 1; rectangle rows 36..92 x cols 14..114; l=3"),
    "ellipses_512": Workload(
        "ellipses_512", 512, 512, 4, 4.0, 1000,
        "512x512 six ellipses (2 ribbons 3 px, 2 pairs 2 px apart), noise 0.1, seed 2; inset rectangle; l=4"),
    "ellipses_2048": Workload(
        "ellipses_2048", 2048, 2048, 4, 4.0, 200,
        "2048x2048 six ellipses at 4x scale (ribbons 3 px, gaps 2 px), noise 0.1, seed 22; inset rectangle; l=4"),
    "blobs_4096": Workload(
        "blobs_4096", 4096, 4096, 8, 8.0, 2000,
        "4096x4096 100 ellipse pairs 1-3 px apart on a jittered 10x10 grid, noise 0.15, seed 5; inset rectangle; l=8"),
}

_IMAGES = {
    "two_disks_128": lambda: two_disks(1),
    "ellipses_512": lambda: ellipse_scene(2, 512, 512),
    "ellipses_2048": lambda: ellipse_scene(22, 2048, 2048, scale=4.0),
    "blobs_4096": lambda: blob_pairs_scene(5),
}

_PHI0 = {
    "two_disks_128": lambda: rect_sdf(128, 128, 36, 92, 14, 114),
    "ellipses_512": lambda: inset_rect_sdf(512, 512),
    "ellipses_2048": lambda: inset_rect_sdf(2048, 2048),
    "blobs_4096": lambda: inset_rect_sdf(4096, 4096),
}


def random_state(H: int, W: int, seed: int, phi_scale: float = 3.0):
    """Random fields (phi, w1, w2, b1, b2, g) for operator-level tests.

    phi is smooth with many zero crossings so that the narrow band (Eq. (11))
    covers a large share of the pixels; w, b are O(1); g in (0, 1].
    """
    rng = np.random.default_rng(seed)
    i = np.arange(H)[:, None]
    j = np.arange(W)[None, :]
    phi = np.zeros((H, W))
    for _ in range(6):
        fi, fj = rng.uniform(0.02, 0.12, 2)
        ph1, ph2 = rng.uniform(0, 2 * math.pi, 2)
        phi += np.sin(2 * math.pi * fi * i + ph1) * np.cos(2 * math.pi * fj * j + ph2)
    phi = phi_scale * phi / np.abs(phi).max() + 0.05 * rng.normal(size=(H, W))
    ang = rng.uniform(0, 2 * math.pi, (H, W))
    mag = rng.choice([0.0, 1.0, 1.0, 1.0], size=(H, W))
    w1 = mag * np.cos(ang)
    w2 = mag * np.sin(ang)
    b1 = 0.5 * rng.normal(size=(H, W))
    b2 = 0.5 * rng.normal(size=(H, W))
    g = 1.0 / (1.0 + 4.0 * rng.uniform(0, 1, (H, W)) ** 2)
    return phi, w1, w2, b1, b2, g


# ----------------------------------------------------------------------------
# Warm-start network: seeded parameters and bf16-representable test values
# ----------------------------------------------------------------------------
def net_init(seed: int, layers) -> np.ndarray:
    """Flat He-normal parameters of a stack of 3x3 convolutions.

    ``layers`` lists (Cin, Cout); per layer the flat vector holds W in
    (Cout, 3, 3, Cin) order, W ~ N(0, 2 / (9 Cin)), then Cout zero biases.
    The last layer's weights are scaled by 0.1 so that the initial output is
    small.
    """
    rng = np.random.default_rng(seed)
    parts = []
    for k, (ci, co) in enumerate(layers):
        w = rng.normal(0.0, math.sqrt(2.0 / (9 * ci)), co * 9 * ci)
        if k == len(layers) - 1:
            w *= 0.1
        parts += [w, np.zeros(co)]
    return np.concatenate(parts)


def bf16_exact(a) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even), returned as float64,
    so that a test can hand both sides values that bf16 holds exactly."""
    x = np.ascontiguousarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)
