"""Python binding of the C-ABI in include/sr.h (argument marshalling only).

Every function here forwards to the entry point of the same name in libsr.so;
all arithmetic runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current stream.  There is no fallback: if libsr.so is missing
or cannot be loaded, the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsr.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "sr.h")

SR_OK, SR_EINVAL, SR_ENOMEM, SR_ECUDA, SR_ENONFINITE = 0, 1, 2, 3, 4
SR_ENOTCONVERGED, SR_ETIMEOUT, SR_EUNSUPPORTED = 5, 6, 7
KCLASS = {"rowfft": 0, "colsolve": 1, "rowifft": 2, "wb_update": 3, "reduce": 4, "prep": 5,
          "resident": 6}


class SRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sr status {status}: {msg}")
        self.status = status


class sr_params(C.Structure):
    _fields_ = [("alpha", C.c_float), ("beta", C.c_float), ("gamma", C.c_float),
                ("mu", C.c_float), ("tau", C.c_float), ("eps", C.c_float),
                ("band_l", C.c_float), ("d", C.c_float), ("win_radius", C.c_int),
                ("inner_S", C.c_int), ("inner_tol", C.c_float), ("rho", C.c_float),
                ("sigma", C.c_float), ("s_pow", C.c_int), ("check_every", C.c_int)]


class sr_schedule(C.Structure):
    _fields_ = [("row_values_per_thread", C.c_int), ("row_threads", C.c_int),
                ("col_schedule", C.c_int), ("tuned_us", C.c_float)]


_lib = None
_P = C.c_void_p


HEADERS = [HEADER, os.path.join(os.path.dirname(_HERE), "include", "sr_net.h"),
           os.path.join(os.path.dirname(_HERE), "include", "sr3.h")]


def declared_functions() -> list[str]:
    """Names of the functions include/sr.h and include/sr_net.h declare."""
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        text = re.sub(r"#define[^\n]*", "", text)
        names |= set(re.findall(r"\b(sr3?_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def lib() -> C.CDLL:
    """Load libsr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    st = C.c_int
    L.sr_status_string.restype = C.c_char_p
    L.sr_status_string.argtypes = [st]
    L.sr_last_error.restype = C.c_char_p
    L.sr_last_error.argtypes = [_P]
    L.sr_params_default.restype = st
    L.sr_params_default.argtypes = [C.POINTER(sr_params)]
    L.sr_create.restype = st
    L.sr_create.argtypes = [C.c_int, C.c_int, C.POINTER(sr_params), _P, C.POINTER(_P)]
    L.sr_destroy.restype = None
    L.sr_destroy.argtypes = [_P]
    for name, n in [("sr_edge_function", 1), ("sr_set_phi", 1), ("sr_get_phi", 1)]:
        getattr(L, name).restype = st
        getattr(L, name).argtypes = [_P, _P, C.c_int]
    L.sr_mask.restype = st
    L.sr_mask.argtypes = [_P, _P, C.c_int]
    L.sr_iterate.restype = st
    L.sr_iterate.argtypes = [_P, C.c_int, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.sr_get_state.restype = st
    L.sr_get_state.argtypes = [_P] * 6
    L.sr_set_state.restype = st
    L.sr_set_state.argtypes = [_P] * 6
    L.sr_get_g.restype = st
    L.sr_get_g.argtypes = [_P, _P]
    L.sr_set_g.restype = st
    L.sr_set_g.argtypes = [_P, _P]
    L.sr_energy.restype = st
    L.sr_energy.argtypes = [_P] + [C.POINTER(C.c_double)] * 4
    L.sr_repulsion_field.restype = st
    L.sr_repulsion_field.argtypes = [_P] * 6
    L.sr_phi_step.restype = st
    L.sr_phi_step.argtypes = [_P] * 7
    L.sr_fft_solve.restype = st
    L.sr_fft_solve.argtypes = [_P] * 3
    L.sr_w_b_update.restype = st
    L.sr_w_b_update.argtypes = [_P] * 10
    L.sr_w_b_fixed_point.restype = st
    L.sr_w_b_fixed_point.argtypes = [_P] * 6 + [C.c_int] + [_P] * 4
    L.sr_set_w_sweeps.restype = st
    L.sr_set_w_sweeps.argtypes = [_P, C.c_int]
    L.sr_inner_steps.restype = C.c_longlong
    L.sr_inner_steps.argtypes = [_P, C.c_int]
    L.sr_kernel_launches.restype = C.c_longlong
    L.sr_kernel_launches.argtypes = [_P, C.c_int]
    L.sr_profile_enable.restype = st
    L.sr_profile_enable.argtypes = [_P, C.c_int]
    L.sr_profile_overhead.restype = st
    L.sr_profile_overhead.argtypes = [_P, C.POINTER(C.c_double)]
    L.sr_kernel_times.restype = st
    L.sr_kernel_times.argtypes = [_P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    L.sr_get_schedule.restype = st
    L.sr_get_schedule.argtypes = [_P, C.POINTER(sr_schedule)]
    L.sr_set_schedule.restype = st
    L.sr_set_schedule.argtypes = [_P, C.POINTER(sr_schedule)]
    L.sr_phi_step_noalloc.restype = st
    L.sr_phi_step_noalloc.argtypes = [C.c_int, C.c_int, C.POINTER(sr_params)] + [_P] * 7 + [_P]
    L.sr_segment_host.restype = st
    L.sr_segment_host.argtypes = [_P, _P, _P, C.c_int, C.c_double, _P, _P,
                                  C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.sr_group_create.restype = st
    L.sr_group_create.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(_P)]
    L.sr_group_iterate.restype = st
    L.sr_group_iterate.argtypes = [_P, C.c_int]
    L.sr_group_tune.restype = st
    L.sr_group_tune.argtypes = [_P, C.POINTER(C.c_int)]
    L.sr_group_run.restype = st
    L.sr_group_run.argtypes = [_P, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int),
                               C.POINTER(C.c_double)]
    L.sr_group_destroy.restype = None
    L.sr_group_destroy.argtypes = [_P]
    L.sr_set_phi_solver.restype = st
    L.sr_set_phi_solver.argtypes = [_P, C.c_int]
    L.sr_set_resident.restype = st
    L.sr_set_resident.argtypes = [_P, C.c_int]
    L.sr_set_boundary.restype = st
    L.sr_set_boundary.argtypes = [_P, C.c_int]
    L.sr_aos_solve.restype = st
    L.sr_aos_solve.argtypes = [_P, _P, _P]
    L.sr_test_stall_waits.restype = st
    L.sr_test_stall_waits.argtypes = [_P, C.c_longlong]
    L.sr_test_fail_allocations.restype = st
    L.sr_test_fail_allocations.argtypes = [C.c_longlong]
    _lib = L
    return L


def params_default() -> sr_params:
    p = sr_params()
    _check(lib().sr_params_default(C.byref(p)), None)
    return p


def make_params(**kw) -> sr_params:
    """Defaults of sr_params_default with the given fields replaced."""
    p = params_default()
    for k, v in kw.items():
        if k == "R":
            k = "win_radius"
        if k == "S":
            k = "inner_S"
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _check(status: int, ctx) -> int:
    if status in (SR_OK, SR_ENOTCONVERGED):
        return status
    msg = lib().sr_status_string(status).decode()
    # without a context: why the last sr_create of this thread failed
    detail = lib().sr_last_error(ctx.handle if ctx is not None and ctx.handle else None).decode()
    if detail and detail != msg:
        msg += ": " + detail
    raise SRError(status, msg)


class Context:
    """One solver (sr_create ... sr_destroy) for H x W images on the current device."""

    def __init__(self, H: int, W: int, params: sr_params | None = None, stream=None):
        self.H, self.W = int(H), int(W)
        self.params = params if params is not None else params_default()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = _P()
        st = lib().sr_create(self.H, self.W, C.byref(self.params), C.c_void_p(stream.cuda_stream),
                             C.byref(h))
        self.handle = None
        _check(st, None)
        self.handle = h

    # -- helpers
    def _dev(self, t: torch.Tensor, dtype=torch.float32, name="buffer"):
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype:
            raise TypeError(f"{name} must be a {dtype} tensor on {self.device}")
        if not t.is_contiguous() or tuple(t.shape) != (self.H, self.W):
            raise ValueError(f"{name} must be contiguous with shape ({self.H}, {self.W})")
        return C.c_void_p(t.data_ptr())

    def _new(self, dtype=torch.float32):
        return torch.empty((self.H, self.W), dtype=dtype, device=self.device)

    def close(self):
        if self.handle:
            lib().sr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C-ABI mirrors
    def edge_function(self, image: torch.Tensor):
        _check(lib().sr_edge_function(self.handle, self._dev(image, name="image"), self.W), self)

    def set_phi(self, phi0: torch.Tensor):
        _check(lib().sr_set_phi(self.handle, self._dev(phi0, name="phi0"), self.W), self)

    def iterate(self, max_outer: int, tol: float = 0.0, want_rel: bool = False):
        done = C.c_int(0)
        rel = C.c_double(float("nan"))
        st = lib().sr_iterate(self.handle, int(max_outer), float(tol), C.byref(done),
                              C.byref(rel) if (want_rel or tol > 0) else None)
        _check(st, self)
        return done.value, rel.value, st == SR_OK

    def mask(self, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self._new(torch.uint8) if out is None else out
        _check(lib().sr_mask(self.handle, self._dev(out, torch.uint8, "mask"), self.W), self)
        return out

    def get_phi(self, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self._new() if out is None else out
        _check(lib().sr_get_phi(self.handle, self._dev(out, name="phi"), self.W), self)
        return out

    def get_state(self):
        bufs = [self._new() for _ in range(5)]
        _check(lib().sr_get_state(self.handle, *[self._dev(b) for b in bufs]), self)
        return tuple(bufs)

    def set_state(self, phi, w1, w2, b1, b2):
        _check(lib().sr_set_state(self.handle, *[self._dev(b) for b in (phi, w1, w2, b1, b2)]),
               self)

    def get_g(self) -> torch.Tensor:
        out = self._new()
        _check(lib().sr_get_g(self.handle, self._dev(out)), self)
        return out

    def set_g(self, g: torch.Tensor):
        _check(lib().sr_set_g(self.handle, self._dev(g, name="g")), self)

    def energy(self):
        vals = [C.c_double() for _ in range(4)]
        _check(lib().sr_energy(self.handle, *[C.byref(v) for v in vals]), self)
        return tuple(v.value for v in vals)

    def repulsion_field(self, phi, w1, w2):
        v1, v2 = self._new(), self._new()
        _check(lib().sr_repulsion_field(self.handle, *[self._dev(t) for t in (phi, w1, w2, v1, v2)]),
               self)
        return v1, v2

    def phi_step(self, psi, w1, w2, b1, b2, out: torch.Tensor | None = None):
        out = self._new() if out is None else out
        _check(lib().sr_phi_step(self.handle, *[self._dev(t) for t in (psi, w1, w2, b1, b2, out)]),
               self)
        return out

    def fft_solve(self, rhs, out: torch.Tensor | None = None):
        out = self._new() if out is None else out
        _check(lib().sr_fft_solve(self.handle, self._dev(rhs), self._dev(out)), self)
        return out

    def aos_solve(self, rhs, out: torch.Tensor | None = None):
        out = self._new() if out is None else out
        _check(lib().sr_aos_solve(self.handle, self._dev(rhs), self._dev(out)), self)
        return out

    def set_boundary(self, boundary: str):
        """'periodic' (the default reading) or 'neumann' (Eq. (27) literally)."""
        _check(lib().sr_set_boundary(self.handle, {"periodic": 0, "neumann": 1}[boundary]), self)

    def set_resident(self, on: bool = True, cluster: int | None = None):
        """sr_set_resident: outer iterations in one launch with the state in one
        cluster's shared memory (small images); cluster = 8 or 16 asks for
        that many CTAs per image."""
        _check(lib().sr_set_resident(self.handle, (cluster or 1) if on else 0), self)

    def set_phi_solver(self, solver: str):
        """'fft' (Eqs. (31)-(33), default) or 'aos' (Eqs. (19)-(20) form)."""
        _check(lib().sr_set_phi_solver(self.handle, {"fft": 0, "aos": 1}[solver]), self)

    def w_b_update(self, phi1, w1, w2, b1, b2):
        outs = [self._new() for _ in range(4)]
        args = [self._dev(t) for t in (phi1, w1, w2, b1, b2, *outs)]
        _check(lib().sr_w_b_update(self.handle, *args), self)
        return tuple(outs)

    def w_b_fixed_point(self, phi1, w1, w2, b1, b2, sweeps: int):
        outs = [self._new() for _ in range(4)]
        _check(lib().sr_w_b_fixed_point(self.handle, *[self._dev(b) for b in (phi1, w1, w2, b1, b2)],
                                        int(sweeps), *[self._dev(b) for b in outs]), self)
        return tuple(outs)

    def set_w_sweeps(self, sweeps: int):
        _check(lib().sr_set_w_sweeps(self.handle, int(sweeps)), self)

    def get_schedule(self) -> dict:
        sc = sr_schedule()
        _check(lib().sr_get_schedule(self.handle, C.byref(sc)), self)
        return {f: getattr(sc, f) for f, _ in sr_schedule._fields_}

    def set_schedule(self, row_values_per_thread: int, row_threads: int, col_schedule: int):
        sc = sr_schedule(row_values_per_thread, row_threads, col_schedule, 0.0)
        _check(lib().sr_set_schedule(self.handle, C.byref(sc)), self)

    def inner_steps(self, reset: bool = False) -> int:
        return int(lib().sr_inner_steps(self.handle, int(reset)))

    def kernel_launches(self, reset: bool = False) -> int:
        return int(lib().sr_kernel_launches(self.handle, int(reset)))

    def profile_enable(self, on: bool = True):
        _check(lib().sr_profile_enable(self.handle, int(on)), self)

    def profile_overhead_us(self) -> float:
        us = C.c_double()
        _check(lib().sr_profile_overhead(self.handle, C.byref(us)), self)
        return us.value

    def kernel_times(self, kclass) -> tuple[float, int]:
        k = KCLASS[kclass] if isinstance(kclass, str) else int(kclass)
        ms, n = C.c_double(), C.c_longlong()
        _check(lib().sr_kernel_times(self.handle, k, C.byref(ms), C.byref(n)), self)
        return ms.value, n.value

    def segment_host(self, image_host, phi0_host, max_outer: int, tol: float, mask_host,
                     phi_host=None):
        """Host buffers (pinned torch CPU tensors or numpy arrays), see sr_segment_host."""
        def hptr(a, dtype):
            if isinstance(a, torch.Tensor):
                if a.device.type != "cpu" or a.dtype != dtype or not a.is_contiguous() or \
                        a.numel() != self.H * self.W:
                    raise ValueError("host buffer has the wrong type, device or shape")
                return C.c_void_p(a.data_ptr())
            arr = np.asarray(a)
            want = np.float32 if dtype == torch.float32 else np.uint8
            if arr.dtype != want or not arr.flags.c_contiguous or arr.size != self.H * self.W:
                raise ValueError("host buffer has the wrong type or shape")
            return C.c_void_p(arr.ctypes.data)

        done, rel = C.c_int(0), C.c_double(float("nan"))
        st = lib().sr_segment_host(self.handle, hptr(image_host, torch.float32),
                                   hptr(phi0_host, torch.float32), int(max_outer), float(tol),
                                   hptr(mask_host, torch.uint8),
                                   hptr(phi_host, torch.float32) if phi_host is not None else None,
                                   C.byref(done), C.byref(rel))
        _check(st, self)
        return done.value, rel.value


class Group:
    """Many contexts (sizes may differ) iterated by one CUDA graph whose
    branches run concurrently (sr_group_create / sr_group_iterate).  The group
    does not own the contexts; close it before them."""

    def __init__(self, members: list["Context"]):
        self.members = list(members)
        arr = (_P * len(members))(*[m.handle for m in members])
        h = _P()
        st = lib().sr_group_create(arr, len(members), C.byref(h))
        _check(st, members[0] if members else None)
        self.handle = h

    def iterate(self, max_outer: int):
        _check(lib().sr_group_iterate(self.handle, int(max_outer)), self.members[0])

    def tune(self) -> int:
        """sr_group_tune: the lane count chosen by timing."""
        lanes = C.c_int()
        _check(lib().sr_group_tune(self.handle, C.byref(lanes)), self.members[0])
        return lanes.value

    def run(self, max_outer: int, tol: float, check_every: int = 10):
        """sr_group_run: per-member device-side stopping; returns (outer_done,
        rel_change, all_converged)."""
        n = len(self.members)
        done = (C.c_int * n)()
        rel = (C.c_double * n)()
        st = lib().sr_group_run(self.handle, int(max_outer), float(tol), int(check_every), done, rel)
        _check(st, self.members[0])
        return list(done), list(rel), st == SR_OK

    def close(self):
        if getattr(self, "handle", None):
            lib().sr_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def phi_step_noalloc(params: sr_params, g: torch.Tensor, psi: torch.Tensor, w1: torch.Tensor,
                     w2: torch.Tensor, b1: torch.Tensor, b2: torch.Tensor,
                     out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """sr_phi_step_noalloc: one inner phi step without a context and without
    allocating device memory (for callers that cannot allocate; sizes up to
    512 x 512).  Tensors: contiguous float32 (H, W) on the current device."""
    H, W = psi.shape
    for t in (g, psi, w1, w2, b1, b2):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or \
                tuple(t.shape) != (H, W):
            raise ValueError("inputs must be contiguous float32 CUDA tensors of one shape")
    out = torch.empty_like(psi) if out is None else out
    stream = torch.cuda.current_stream() if stream is None else stream
    st = lib().sr_phi_step_noalloc(int(H), int(W), C.byref(params),
                                   *[C.c_void_p(t.data_ptr()) for t in (g, psi, w1, w2, b1, b2, out)],
                                   C.c_void_p(stream.cuda_stream))
    if st == SR_EUNSUPPORTED:
        raise SRError(st, f"{H} x {W} is not a power-of-two size within the 512 x 512 maximum "
                          "of the fixed scratch array")
    _check(st, None)
    return out
