"""FP64 CPU oracle of the learned warm start: a 6-layer 3x3 convolutional
encoder-decoder that maps an image f to an initial level set phi0.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product path
never does.  It shares no code with the CUDA path.

The paper initialises phi0 by thresholding (Sec. 5) and has no network; the
network is the warm start that proposes phi0 before the plain Split Bregman
iteration (Alg. 1) finishes the solve.  Everything here is written from the
plain definitions:

* convolution: zero-padded 3x3 cross-correlation, y[b,i,j,o] =
  bias[o] + sum_{ky,kx,c} x[b, i+ky-1, j+kx-1, c] * W[o,ky,kx,c];
* 2x2 average pooling and 2x nearest-neighbour upsampling;
* ReLU after every layer but the last;
* loss 1/(2n) sum (y - t)^2 over the n output pixels, with the target
  t = clip(phi*, -c, c) / c for a converged level set phi*;
* the backward pass is the adjoint of each linear map (not a flipped-kernel
  convolution), so it checks the kernels' own formulation independently;
* Adam (Kingma and Ba, 2015) with bias correction.

Arrays are float64, activations NHWC (batch, rows, columns, channels),
weights (Cout, 3, 3, Cin).
"""
from __future__ import annotations

import numpy as np

# (Cin, Cout) of the six layers; the network's input is the image alone (one
# channel), its output phi0 / c.
LAYERS = [(1, 32), (32, 64), (64, 128), (128, 64), (64, 32), (32, 1)]


def param_shapes(layers=LAYERS):
    """[(W shape, b shape)] per layer; the flat parameter vector holds, layer
    after layer, W in (Cout, 3, 3, Cin) order followed by b."""
    return [((co, 3, 3, ci), (co,)) for ci, co in layers]


def param_count(layers=LAYERS) -> int:
    return sum(co * 9 * ci + co for ci, co in layers)


def unflatten(theta, layers=LAYERS):
    """Split a flat parameter vector into [(W, b)] (views, float64)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, k = [], 0
    for ws, bs in param_shapes(layers):
        nw = int(np.prod(ws))
        out.append((theta[k:k + nw].reshape(ws), theta[k + nw:k + nw + bs[0]]))
        k += nw + bs[0]
    assert k == theta.size, (k, theta.size)
    return out


def flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


# ----------------------------------------------------------------------------
# Layers and their adjoints
# ----------------------------------------------------------------------------
def conv3x3(x, W, b=None):
    """Zero-padded 3x3 cross-correlation, NHWC in and out."""
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, Wd, W.shape[0]))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + Wd, :], W[:, ky, kx, :])
    if b is not None:
        y += b
    return y


def conv3x3_adjoint(dy, W, x_shape):
    """d/dx of <conv3x3(x, W), dy>: the transpose of the linear map x -> conv(x)."""
    B, H, Wd, Cin = x_shape
    dxp = np.zeros((B, H + 2, Wd + 2, Cin))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + Wd, :] += np.einsum("bhwo,oc->bhwc", dy, W[:, ky, kx, :])
    return dxp[:, 1:H + 1, 1:Wd + 1, :]


def conv3x3_wgrad(x, dy):
    """dW[o,ky,kx,c] = sum_{b,i,j} dy[b,i,j,o] x[b,i+ky-1,j+kx-1,c]; db = sum dy."""
    B, H, Wd, Cin = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros((dy.shape[3], 3, 3, Cin))
    for ky in range(3):
        for kx in range(3):
            dW[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dy, xp[:, ky:ky + H, kx:kx + Wd, :])
    return dW, dy.sum(axis=(0, 1, 2))


def avgpool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_adjoint(dy):
    """Each input pixel receives a quarter of its window's output gradient."""
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) * 0.25


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_adjoint(dy):
    """Sum of the four copies of each input pixel."""
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def relu(z):
    return np.maximum(z, 0.0)


# ----------------------------------------------------------------------------
# The network: conv-ReLU-pool, conv-ReLU-pool, conv-ReLU, conv-ReLU-up,
# conv-ReLU-up, conv
# ----------------------------------------------------------------------------
def forward(params, f):
    """f: (B, H, W) image; returns (y (B, H, W), cache)."""
    x = np.asarray(f, dtype=np.float64)[..., None]
    (W1, b1), (W2, b2), (W3, b3), (W4, b4), (W5, b5), (W6, b6) = params
    a1 = relu(conv3x3(x, W1, b1))
    p1 = avgpool2(a1)
    a2 = relu(conv3x3(p1, W2, b2))
    p2 = avgpool2(a2)
    a3 = relu(conv3x3(p2, W3, b3))
    a4 = relu(conv3x3(a3, W4, b4))
    u4 = up2(a4)
    a5 = relu(conv3x3(u4, W5, b5))
    u5 = up2(a5)
    y = conv3x3(u5, W6, b6)[..., 0]
    cache = dict(x=x, a1=a1, p1=p1, a2=a2, p2=p2, a3=a3, a4=a4, u4=u4, a5=a5, u5=u5)
    return y, cache


def target(phi_star, clip):
    """Regression target of a converged level set: clip(phi*, -c, c) / c."""
    return np.clip(np.asarray(phi_star, dtype=np.float64), -clip, clip) / clip


def loss(y, t):
    return 0.5 * np.mean((y - t) ** 2)


def deltas(params, cache, y, t):
    """Per layer, the pair (layer input, loss gradient at the layer's
    pre-activation output) that its weight gradient contracts, by the
    adjoints of the forward pass in reverse order."""
    (_, _), (W2, _), (W3, _), (W4, _), (W5, _), (W6, _) = params
    c = cache
    d6 = ((y - t) / y.size)[..., None]
    d5 = up2_adjoint(conv3x3_adjoint(d6, W6, c["u5"].shape)) * (c["a5"] > 0)
    d4 = up2_adjoint(conv3x3_adjoint(d5, W5, c["u4"].shape)) * (c["a4"] > 0)
    d3 = conv3x3_adjoint(d4, W4, c["a3"].shape) * (c["a3"] > 0)
    d2 = avgpool2_adjoint(conv3x3_adjoint(d3, W3, c["p2"].shape)) * (c["a2"] > 0)
    d1 = avgpool2_adjoint(conv3x3_adjoint(d2, W2, c["p1"].shape)) * (c["a1"] > 0)
    return [(c["x"], d1), (c["p1"], d2), (c["p2"], d3), (c["a3"], d4), (c["u4"], d5),
            (c["u5"], d6)]


def backward(params, cache, y, t):
    """Gradients [(dW, db)] of loss(y, t) with respect to every (W, b)."""
    return [conv3x3_wgrad(x, d) for x, d in deltas(params, cache, y, t)]


def loss_and_grad(theta, f, phi_star, clip, layers=LAYERS):
    """(loss, flat gradient) of the network with flat parameters theta."""
    params = unflatten(theta, layers)
    y, cache = forward(params, f)
    t = target(phi_star, clip)
    return loss(y, t), flatten(backward(params, cache, y, t))


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; step counts from 1.  Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
