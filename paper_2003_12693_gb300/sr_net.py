"""Python binding of include/sr_net.h, the learned warm start (argument
marshalling only).

Every call forwards to the entry point of the same name in libsr.so; the
network's forward and backward passes, its loss and its optimiser all run in
the library's CUDA kernels.  There is no fallback: without libsr.so the
binding raises.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import sr as _sr

SR_CONV_RELU, SR_CONV_PLAIN, SR_CONV_MASK, SR_CONV_OUT1 = 0, 1, 2, 3
_P = C.c_void_p
_declared = False


def lib() -> C.CDLL:
    global _declared
    L = _sr.lib()
    if _declared:
        return L
    st = C.c_int
    L.sr_net_layer_shape.restype = st
    L.sr_net_layer_shape.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.sr_net_param_count.restype = C.c_longlong
    L.sr_net_param_count.argtypes = []
    L.sr_net_create.restype = st
    L.sr_net_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_float, _P, C.POINTER(_P)]
    L.sr_net_destroy.restype = None
    L.sr_net_destroy.argtypes = [_P]
    L.sr_net_last_error.restype = C.c_char_p
    L.sr_net_last_error.argtypes = [_P]
    for name in ("sr_net_set_params", "sr_net_get_params", "sr_net_get_grads"):
        getattr(L, name).restype = st
        getattr(L, name).argtypes = [_P, _P]
    L.sr_net_forward.restype = st
    L.sr_net_forward.argtypes = [_P, _P, C.c_int, _P]
    L.sr_net_gradients.restype = st
    L.sr_net_gradients.argtypes = [_P, _P, _P, C.c_int, _P]
    L.sr_net_train_step.restype = st
    L.sr_net_train_step.argtypes = [_P, _P, _P, C.c_int, C.c_float, _P]
    L.sr_net_kernel_launches.restype = C.c_longlong
    L.sr_net_kernel_launches.argtypes = [_P, C.c_int]
    L.sr_conv3x3.restype = st
    L.sr_conv3x3.argtypes = [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, C.c_int, C.c_int,
                             _P, _P, C.c_float, _P]
    L.sr_conv3x3_dgrad.restype = st
    L.sr_conv3x3_dgrad.argtypes = [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, C.c_int, C.c_int,
                                   _P, _P, _P]
    L.sr_conv3x3_wgrad.restype = st
    L.sr_conv3x3_wgrad.argtypes = [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_int, _P, _P, _P]
    _declared = True
    return L


def _check(status: int, handle=None):
    if status == _sr.SR_OK:
        return
    L = lib()
    msg = L.sr_status_string(status).decode()
    detail = L.sr_net_last_error(handle).decode()
    raise _sr.SRError(status, msg + (": " + detail if detail else ""))


def layers() -> list[tuple[int, int]]:
    """(Cin, Cout) of the six layers."""
    out = []
    for k in range(6):
        ci, co = C.c_int(), C.c_int()
        _check(lib().sr_net_layer_shape(k, C.byref(ci), C.byref(co)))
        out.append((ci.value, co.value))
    return out


def param_count() -> int:
    return int(lib().sr_net_param_count())


def _ptr(t: torch.Tensor | None, dtype, name: str):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype:
        raise TypeError(f"{name} must be a CUDA {dtype} tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Net:
    """The warm-start network (sr_net_create ... sr_net_destroy)."""

    def __init__(self, H: int, W: int, max_batch: int, phi_clip: float = 4.0, stream=None):
        self.H, self.W, self.max_batch, self.clip = int(H), int(W), int(max_batch), float(phi_clip)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.P = param_count()
        h = _P()
        self.handle = None
        _check(lib().sr_net_create(self.H, self.W, self.max_batch, self.clip,
                                   C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            lib().sr_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _batch(self, t: torch.Tensor, name: str) -> tuple[C.c_void_p, int]:
        if t.dim() != 3 or tuple(t.shape[1:]) != (self.H, self.W):
            raise ValueError(f"{name} must have shape (B, {self.H}, {self.W})")
        return _ptr(t, torch.float32, name), int(t.shape[0])

    def set_params(self, theta: torch.Tensor):
        if theta.numel() != self.P:
            raise ValueError(f"theta must hold {self.P} floats")
        _check(lib().sr_net_set_params(self.handle, _ptr(theta, torch.float32, "theta")),
               self.handle)

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.P, dtype=torch.float32, device="cuda")
        _check(lib().sr_net_get_params(self.handle, _ptr(out, torch.float32, "theta")),
               self.handle)
        return out

    def get_grads(self) -> torch.Tensor:
        out = torch.empty(self.P, dtype=torch.float32, device="cuda")
        _check(lib().sr_net_get_grads(self.handle, _ptr(out, torch.float32, "grad")), self.handle)
        return out

    def forward(self, f: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        pf, B = self._batch(f, "f")
        if out is None:
            out = torch.empty_like(f)
        _check(lib().sr_net_forward(self.handle, pf, B, _ptr(out, torch.float32, "phi0")),
               self.handle)
        return out

    def gradients(self, f: torch.Tensor, phi_star: torch.Tensor,
                  loss: torch.Tensor | None = None):
        pf, B = self._batch(f, "f")
        pp, B2 = self._batch(phi_star, "phi_star")
        if B2 != B:
            raise ValueError("f and phi_star batch sizes differ")
        _check(lib().sr_net_gradients(self.handle, pf, pp, B, _ptr(loss, torch.float64, "loss")),
               self.handle)

    def train_step(self, f: torch.Tensor, phi_star: torch.Tensor, lr: float,
                   loss: torch.Tensor | None = None):
        pf, B = self._batch(f, "f")
        pp, B2 = self._batch(phi_star, "phi_star")
        if B2 != B:
            raise ValueError("f and phi_star batch sizes differ")
        _check(lib().sr_net_train_step(self.handle, pf, pp, B, float(lr),
                                       _ptr(loss, torch.float64, "loss")), self.handle)

    def kernel_launches(self, reset: bool = False) -> int:
        return int(lib().sr_net_kernel_launches(self.handle, int(reset)))


def _bf(t, name):
    return _ptr(t, torch.bfloat16, name)


def conv3x3(x: torch.Tensor, w: torch.Tensor, bias: torch.Tensor | None, mode: int,
            ref: torch.Tensor | None = None, out_scale: float = 1.0) -> torch.Tensor:
    """sr_conv3x3: x [B, H, W, cin] bf16, w [cout, 3, 3, cin] bf16."""
    B, H, W, cin = x.shape
    cout = w.shape[0]
    if mode == SR_CONV_OUT1:
        y = torch.empty((B, H, W), dtype=torch.float32, device=x.device)
    else:
        y = torch.empty((B, H, W, cout), dtype=torch.bfloat16, device=x.device)
    _check(lib().sr_conv3x3(_bf(x, "x"), B, H, W, cin, _bf(w, "w"),
                            _ptr(bias, torch.float32, "bias"), cout, mode, _bf(ref, "ref"),
                            C.c_void_p(y.data_ptr()), float(out_scale), _stream()))
    return y


def conv3x3_dgrad(dy: torch.Tensor, w: torch.Tensor, mode: int = SR_CONV_PLAIN,
                  ref: torch.Tensor | None = None) -> torch.Tensor:
    """sr_conv3x3_dgrad: dy [B, H, W, cout], w [cout, 3, 3, cin] -> dx [B, H, W, cin]."""
    B, H, W, cout = dy.shape
    cin = w.shape[3]
    dx = torch.empty((B, H, W, cin), dtype=torch.bfloat16, device=dy.device)
    _check(lib().sr_conv3x3_dgrad(_bf(dy, "dy"), B, H, W, cout, _bf(w, "w"), cin, mode,
                                  _bf(ref, "ref"), _bf(dx, "dx"), _stream()))
    return dx


def conv3x3_wgrad(dy: torch.Tensor, x: torch.Tensor, cin_real: int | None = None,
                  cout_real: int | None = None):
    """sr_conv3x3_wgrad: returns (dW [cout_real, 3, 3, cin_real], db [cout_real]) float32."""
    B, H, W, cout = dy.shape
    cin = x.shape[3]
    cin_real = cin if cin_real is None else cin_real
    cout_real = cout if cout_real is None else cout_real
    dw = torch.zeros((cout_real, 3, 3, cin_real), dtype=torch.float32, device=dy.device)
    db = torch.zeros(cout_real, dtype=torch.float32, device=dy.device)
    _check(lib().sr_conv3x3_wgrad(_bf(dy, "dy"), _bf(x, "x"), B, H, W, cin, cout, cin_real,
                                  cout_real, _ptr(dw, torch.float32, "dw"),
                                  _ptr(db, torch.float32, "db"), _stream()))
    return dw, db
