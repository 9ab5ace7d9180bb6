"""Python binding of include/sr3.h, the SR iteration on volumes (argument
marshalling only; the arithmetic runs in libsr.so's kernels, and there is no
fallback)."""
from __future__ import annotations

import ctypes as C

import torch

from .sr import _P, SRError, _check, lib, sr_params

_P3 = _P * 3
_done = False


def lib3() -> C.CDLL:
    global _done
    L = lib()
    if not _done:
        st = C.c_int
        L.sr3_create.restype = st
        L.sr3_create.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(sr_params), _P, C.POINTER(_P)]
        L.sr3_destroy.restype = None
        L.sr3_destroy.argtypes = [_P]
        for name, args in [("sr3_set_g", [_P, _P]), ("sr3_set_phi", [_P, _P]),
                           ("sr3_set_state", [_P, _P, _P3, _P3]),
                           ("sr3_get_state", [_P, _P, _P3, _P3]),
                           ("sr3_iterate", [_P, C.c_int]),
                           ("sr3_window_sum", [_P, _P, _P3, _P3]),
                           ("sr3_fft_solve", [_P, _P, _P]),
                           ("sr3_phi_step", [_P, _P, _P3, _P3, _P]),
                           ("sr3_w_b_update", [_P, _P, _P3, _P3, _P3, _P3])]:
            getattr(L, name).restype = st
            getattr(L, name).argtypes = args
        L.sr3_kernel_launches.restype = C.c_longlong
        L.sr3_kernel_launches.argtypes = [_P]
        _done = True
    return L


class Volume:
    """One solver (sr3_create ... sr3_destroy) for Z x M x N volumes."""

    def __init__(self, Z: int, M: int, N: int, params: sr_params, stream=None):
        self.shape = (int(Z), int(M), int(N))
        self.params = params
        stream = torch.cuda.current_stream() if stream is None else stream
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = _P()
        st = lib3().sr3_create(*self.shape, C.byref(params), C.c_void_p(stream.cuda_stream),
                               C.byref(h))
        self.handle = None
        if st != 0:
            raise SRError(st, lib().sr_status_string(st).decode())
        self.handle = h

    def _p(self, t: torch.Tensor):
        if (not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float32
                or not t.is_contiguous() or tuple(t.shape) != self.shape):
            raise ValueError(f"expected a contiguous float32 {self.shape} tensor on {self.device}")
        return C.c_void_p(t.data_ptr())

    def _p3(self, ts):
        return _P3(*[self._p(t) for t in ts])

    def _new(self, n=None):
        if n is None:
            return torch.empty(self.shape, dtype=torch.float32, device=self.device)
        return [torch.empty(self.shape, dtype=torch.float32, device=self.device) for _ in range(n)]

    def _call(self, name, *args):
        st = getattr(lib3(), name)(self.handle, *args)
        if st != 0:
            raise SRError(st, lib().sr_status_string(st).decode())

    def set_g(self, g):
        self._call("sr3_set_g", self._p(g))

    def set_phi(self, phi0):
        self._call("sr3_set_phi", self._p(phi0))

    def set_state(self, phi, w, b):
        self._call("sr3_set_state", self._p(phi), self._p3(w), self._p3(b))

    def get_state(self):
        phi, w, b = self._new(), self._new(3), self._new(3)
        self._call("sr3_get_state", self._p(phi), self._p3(w), self._p3(b))
        return phi, w, b

    def iterate(self, max_outer: int):
        self._call("sr3_iterate", int(max_outer))

    def window_sum(self, phi, w):
        v = self._new(3)
        self._call("sr3_window_sum", self._p(phi), self._p3(w), self._p3(v))
        return v

    def fft_solve(self, rhs):
        out = self._new()
        self._call("sr3_fft_solve", self._p(rhs), self._p(out))
        return out

    def phi_step(self, psi, w, b):
        out = self._new()
        self._call("sr3_phi_step", self._p(psi), self._p3(w), self._p3(b), self._p(out))
        return out

    def w_b_update(self, phi1, w, b):
        wo, bo = self._new(3), self._new(3)
        self._call("sr3_w_b_update", self._p(phi1), self._p3(w), self._p3(b), self._p3(wo),
                   self._p3(bo))
        return wo, bo

    def kernel_launches(self) -> int:
        return int(lib3().sr3_kernel_launches(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib3().sr3_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Volume", "lib3", "_check"]
