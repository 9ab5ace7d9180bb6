"""FP64 CPU oracle of the Split Bregman self-repelling snake (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2003_12693_gb300``) never does.  It shares no code with the CUDA
path: the two meet only in the seeded inputs of
``paper_2003_12693_gb300.synth``.

All arrays are float64, C-contiguous, shape (M, N).  Each wrapper names the
equation of the paper it computes.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

_lib = None


class OcParams(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("mu", C.c_double), ("tau", C.c_double), ("eps", C.c_double),
                ("band_l", C.c_double), ("d", C.c_double), ("R", C.c_int), ("S", C.c_int)]


@dataclasses.dataclass
class Params:
    """Model parameters; defaults are the Fig. 1 set (Sec. 5)."""
    alpha: float = 4.0
    beta: float = 0.2
    gamma: float = 4.0
    mu: float = 8.0
    tau: float = 0.1
    eps: float = 1.0
    band_l: float = 1.0
    d: float = 3.0
    R: int = 3
    S: int = 3

    def c(self) -> OcParams:
        return OcParams(self.alpha, self.beta, self.gamma, self.mu, self.tau, self.eps,
                        self.band_l, self.d, int(self.R), int(self.S))

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        return cls(alpha=d.get("alpha", 4.0), beta=d.get("beta", 0.2), gamma=d.get("gamma", 4.0),
                   mu=d.get("mu", 8.0), tau=d.get("tau", 0.1), eps=d.get("eps", 1.0),
                   band_l=d.get("band_l", 1.0), d=d.get("d", 3.0),
                   R=d.get("win_radius", d.get("R", 3)), S=d.get("inner_S", d.get("S", 3)))


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        L = _lib
        for name in ("oc_heaviside", "oc_delta", "oc_delta_prime"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double, C.c_double]
        for name in ("oc_band", "oc_band_prime"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double, C.c_double, C.c_double]
        L.oc_edge.argtypes = [C.c_int, C.c_int, _D, C.c_double, C.c_double, C.c_int, _D]
        L.oc_grad.argtypes = [C.c_int, C.c_int, _D, _D, _D]
        L.oc_div.argtypes = [C.c_int, C.c_int, _D, _D, _D]
        L.oc_fft2.argtypes = [C.c_int, C.c_int, _D, _D, C.c_int]
        L.oc_fft1.argtypes = [C.c_int, _D, _D, C.c_int, C.c_int]
        L.oc_solve.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _D, _D]
        P = C.POINTER(OcParams)
        L.oc_repulsion.argtypes = [C.c_int, C.c_int, P, _D, _D, _D, _D, _D]
        L.oc_rhs.argtypes = [C.c_int, C.c_int, P] + [_D] * 9
        L.oc_phi_step.argtypes = [C.c_int, C.c_int, P] + [_D] * 7
        L.oc_soft_threshold.argtypes = [C.c_double, C.c_double, C.c_double, _D, _D]
        L.oc_w_b_update.argtypes = [C.c_int, C.c_int, P] + [_D] * 8
        L.oc_init.argtypes = [C.c_int, C.c_int] + [_D] * 5
        L.oc_iterate.argtypes = [C.c_int, C.c_int, P, _D, _D, _D, _D, _D, _D, C.c_int, _D]
        L.oc_energy.argtypes = [C.c_int, C.c_int, P, _D, _D, _D]
        L.oc_mask.argtypes = [C.c_int, C.c_int, _D, C.POINTER(C.c_ubyte)]
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- scalars
def heaviside(phi, eps=1.0):
    """Eq. (5)."""
    return lib().oc_heaviside(float(phi), float(eps))


def delta(phi, eps=1.0):
    """Eq. (6)."""
    return lib().oc_delta(float(phi), float(eps))


def delta_prime(phi, eps=1.0):
    """Eq. (29)."""
    return lib().oc_delta_prime(float(phi), float(eps))


def band(phi, eps=1.0, l=1.0):
    """Eq. (11)."""
    return lib().oc_band(float(phi), float(eps), float(l))


def band_prime(phi, eps=1.0, l=1.0):
    """Eq. (28)."""
    return lib().oc_band_prime(float(phi), float(eps), float(l))


# ---------------------------------------------------------------- fields
def edge(f, rho=1.0, sigma=1.0, s_pow=2):
    """Eq. (1)."""
    f = _f64(f)
    g = np.empty_like(f)
    lib().oc_edge(f.shape[0], f.shape[1], _p(f), rho, sigma, s_pow, _p(g))
    return g


def grad(phi):
    """Forward differences, Eq. (35), periodic."""
    phi = _f64(phi)
    d1, d2 = np.empty_like(phi), np.empty_like(phi)
    lib().oc_grad(phi.shape[0], phi.shape[1], _p(phi), _p(d1), _p(d2))
    return d1, d2


def div(a1, a2):
    """Backward-difference divergence, Eq. (36), periodic."""
    a1, a2 = _f64(a1), _f64(a2)
    out = np.empty_like(a1)
    lib().oc_div(a1.shape[0], a1.shape[1], _p(a1), _p(a2), _p(out))
    return out


def fft2(x, sign=-1):
    """Unnormalised 2-D DFT with the oracle's own FFT."""
    x = np.asarray(x)
    re, im = _f64(x.real), _f64(x.imag if np.iscomplexobj(x) else np.zeros(x.shape))
    lib().oc_fft2(re.shape[0], re.shape[1], _p(re), _p(im), int(sign))
    return re + 1j * im


def fft1(x, sign=-1):
    x = np.asarray(x)
    re, im = _f64(x.real), _f64(x.imag if np.iscomplexobj(x) else np.zeros(x.shape))
    lib().oc_fft1(re.shape[0], _p(re), _p(im), 1, int(sign))
    return re + 1j * im


def solve(rhs, tau, mu):
    """Eqs. (31)-(33)."""
    rhs = _f64(rhs)
    out = np.empty_like(rhs)
    lib().oc_solve(rhs.shape[0], rhs.shape[1], tau, mu, _p(rhs), _p(out))
    return out


def repulsion(phi, w1, w2, p: Params):
    """Window sum v of Sec. 4."""
    phi, w1, w2 = _f64(phi), _f64(w1), _f64(w2)
    v1, v2 = np.empty_like(phi), np.empty_like(phi)
    pc = p.c()
    lib().oc_repulsion(phi.shape[0], phi.shape[1], C.byref(pc), _p(phi), _p(w1), _p(w2),
                       _p(v1), _p(v2))
    return v1, v2


def rhs(psi, g, w1, w2, b1, b2, v1, v2, p: Params):
    """F^{k,s} of Eq. (37)."""
    arrs = [_f64(a) for a in (psi, g, w1, w2, b1, b2, v1, v2)]
    F = np.empty_like(arrs[0])
    pc = p.c()
    lib().oc_rhs(arrs[0].shape[0], arrs[0].shape[1], C.byref(pc), *[_p(a) for a in arrs], _p(F))
    return F


def phi_step(psi, g, w1, w2, b1, b2, p: Params):
    """One inner step of Eq. (37): v, F, FFT solve."""
    arrs = [_f64(a) for a in (psi, g, w1, w2, b1, b2)]
    out = np.empty_like(arrs[0])
    pc = p.c()
    lib().oc_phi_step(arrs[0].shape[0], arrs[0].shape[1], C.byref(pc),
                      *[_p(a) for a in arrs], _p(out))
    return out


def soft_threshold(B1, B2, t):
    """Eq. (42) on one vector."""
    o1, o2 = C.c_double(), C.c_double()
    lib().oc_soft_threshold(float(B1), float(B2), float(t), C.byref(o1), C.byref(o2))
    return o1.value, o2.value


def w_b_update(phi1, g, w1, w2, b1, b2, p: Params, return_shrunk=False):
    """Eqs. (41), (42), (40), (23): returns w^{k+1}, b^{k+1} (and the shrunk vector)."""
    phi1, g = _f64(phi1), _f64(g)
    w1, w2, b1, b2 = (_f64(a).copy() for a in (w1, w2, b1, b2))
    wt1, wt2 = np.empty_like(phi1), np.empty_like(phi1)
    pc = p.c()
    lib().oc_w_b_update(phi1.shape[0], phi1.shape[1], C.byref(pc), _p(phi1), _p(g), _p(w1),
                        _p(w2), _p(b1), _p(b2), _p(wt1), _p(wt2))
    if return_shrunk:
        return w1, w2, b1, b2, wt1, wt2
    return w1, w2, b1, b2


def w_b_fixed_point(phi1, g, w1, w2, b1, b2, p: Params, sweeps: int):
    """Eqs. (38)-(40) swept ``sweeps`` times from w^{k+1,0} = w^k, then
    Eq. (23): returns w^{k+1}, b^{k+1}.

    Each sweep forms v^{k+1,r} from the current w (Eq. (38), the window sum of
    Sec. 4 with h(phi^{k+1})), evaluates Eq. (39) with its denominator
    gamma g delta + mu, and projects by Eq. (40) (the zero vector kept at
    zero)."""
    phi1, g = _f64(phi1), _f64(g)
    w1, w2, b1, b2 = (_f64(a) for a in (w1, w2, b1, b2))
    d1, d2 = grad(phi1)
    flat = phi1.ravel()
    h = np.array([band(x, p.eps, p.band_l) for x in flat]).reshape(phi1.shape)
    dl = np.array([delta(x, p.eps) for x in flat]).reshape(phi1.shape)
    c1, c2 = w1, w2
    for _ in range(int(sweeps)):
        v1, v2 = repulsion(phi1, c1, c2, p)
        den = p.gamma * g * dl + p.mu
        t1 = (p.mu * d1 + p.mu * b1 + 2.0 * p.beta * h * v1) / den
        t2 = (p.mu * d2 + p.mu * b2 + 2.0 * p.beta * h * v2) / den
        n = np.hypot(t1, t2)
        safe = np.where(n > 0.0, n, 1.0)
        c1 = np.where(n > 0.0, t1 / safe, 0.0)
        c2 = np.where(n > 0.0, t2 / safe, 0.0)
    return c1, c2, b1 + d1 - c1, b2 + d2 - c2


def outer_iteration_fixed_point(state: "State", g, p: Params, sweeps: int) -> None:
    """One outer iteration of Alg. 1 in place with the w sub-problem solved
    by Eqs. (38)-(40) (``sweeps`` sweeps) instead of Eqs. (41)-(42)."""
    psi = state.phi
    for _ in range(p.S):
        psi = phi_step(psi, g, state.w1, state.w2, state.b1, state.b2, p)
    w1, w2, b1, b2 = w_b_fixed_point(psi, g, state.w1, state.w2, state.b1, state.b2, p, sweeps)
    state.phi, state.w1, state.w2, state.b1, state.b2 = psi, w1, w2, b1, b2


def outer_iteration_inner_tol(state: "State", g, p: Params, tol: float) -> list:
    """One outer iteration of Alg. 1 in place with the inner exit of Sec. 4:
    after each inner step s the relative change ||psi^{s+1} - psi^s|| /
    (||psi^s|| + 1e-6) is formed and the loop stops once it is <= tol, after
    at most p.S steps; then Eqs. (41), (42), (40), (23).  Returns the relative
    changes of the steps taken."""
    psi = state.phi
    rels = []
    for _ in range(p.S):
        nxt = phi_step(psi, g, state.w1, state.w2, state.b1, state.b2, p)
        rels.append(float(np.linalg.norm(nxt - psi) / (np.linalg.norm(psi) + 1e-6)))
        psi = nxt
        if rels[-1] <= tol:
            break
    w1, w2, b1, b2 = w_b_update(psi, g, state.w1, state.w2, state.b1, state.b2, p)
    state.phi, state.w1, state.w2, state.b1, state.b2 = psi, w1, w2, b1, b2
    return rels


def init(phi0):
    """Alg. 1 initialisation: w0 = grad phi0, b0 = 0."""
    phi0 = _f64(phi0)
    w1, w2, b1, b2 = (np.empty_like(phi0) for _ in range(4))
    lib().oc_init(phi0.shape[0], phi0.shape[1], _p(phi0), _p(w1), _p(w2), _p(b1), _p(b2))
    return w1, w2, b1, b2


@dataclasses.dataclass
class State:
    phi: np.ndarray
    w1: np.ndarray
    w2: np.ndarray
    b1: np.ndarray
    b2: np.ndarray

    def copy(self) -> "State":
        return State(*(a.copy() for a in (self.phi, self.w1, self.w2, self.b1, self.b2)))


def initial_state(phi0) -> State:
    phi0 = _f64(phi0).copy()
    return State(phi0, *init(phi0))


def iterate(state: State, g, K: int, p: Params) -> np.ndarray:
    """Alg. 1: K outer iterations in place; returns the relative-change trace."""
    g = _f64(g)
    rel = np.zeros(max(K, 1))
    pc = p.c()
    M, N = state.phi.shape
    lib().oc_iterate(M, N, C.byref(pc), _p(g), _p(state.phi), _p(state.w1), _p(state.w2),
                     _p(state.b1), _p(state.b2), int(K), _p(rel))
    return rel[:K]


def energy(phi, g, p: Params):
    """Discrete energy of Eqs. (7)-(10): (E, E_g, E_a, E_r)."""
    phi, g = _f64(phi), _f64(g)
    out = np.zeros(4)
    pc = p.c()
    lib().oc_energy(phi.shape[0], phi.shape[1], C.byref(pc), _p(phi), _p(g), _p(out))
    return tuple(out)


def mask(phi):
    """Eq. (3): 1 inside (phi < 0)."""
    phi = _f64(phi)
    m = np.empty(phi.shape, dtype=np.uint8)
    lib().oc_mask(phi.shape[0], phi.shape[1], _p(phi), m.ctypes.data_as(C.POINTER(C.c_ubyte)))
    return m


def set_threads(n: int) -> None:
    """Thread count for the OpenMP loops (must be called before the first call)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
