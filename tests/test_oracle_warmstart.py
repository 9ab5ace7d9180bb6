"""Pins of the warm-start network oracle against what the mathematics fixes.

Each layer is checked against something other than itself: the convolution
against scipy's 2-D correlation, the adjoints by the inner-product identity
<A x, y> = <x, A^T y> on random vectors, the whole backward pass by central
finite differences of the loss, Adam by its closed-form first step."""
import numpy as np
import pytest
import scipy.signal

from oracle import warmstart as ws
from paper_2003_12693_gb300 import synth

TINY = [(1, 2), (2, 3), (3, 4), (4, 3), (3, 2), (2, 1)]


def test_param_count_and_layout():
    assert ws.param_count() == 185217
    theta = np.arange(ws.param_count(TINY), dtype=float)
    params = ws.unflatten(theta, TINY)
    assert params[0][0].shape == (2, 3, 3, 1) and params[0][1].tolist() == [18.0, 19.0]
    assert np.array_equal(ws.flatten(params), theta)


def test_conv3x3_matches_scipy_correlate2d():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 5, 3))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = ws.conv3x3(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.signal.correlate2d(x[n, :, :, c], W[o, :, :, c], mode="same",
                                                      boundary="fill") for c in range(3))
            assert np.allclose(y[n, :, :, o], ref, atol=1e-12)


def test_conv3x3_identity_and_shift_kernels():
    """The centre tap copies, an off-centre tap shifts with zero fill."""
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 6, 6, 1))
    W = np.zeros((1, 3, 3, 1))
    W[0, 1, 1, 0] = 1.0
    assert np.array_equal(ws.conv3x3(x, W), x)
    W[:] = 0.0
    W[0, 0, 2, 0] = 1.0    # y[i, j] = x[i - 1, j + 1]
    y = ws.conv3x3(x, W)
    assert np.array_equal(y[0, 1:, :-1, 0], x[0, :-1, 1:, 0])
    assert np.all(y[0, 0, :, 0] == 0) and np.all(y[0, :, -1, 0] == 0)


@pytest.mark.parametrize("op", ["conv", "pool", "up"])
def test_adjoint_identity(op):
    rng = np.random.default_rng(2)
    if op == "conv":
        W = rng.normal(size=(3, 3, 3, 2))
        x = rng.normal(size=(2, 6, 8, 2))
        fwd = ws.conv3x3(x, W)
        y = rng.normal(size=fwd.shape)
        adj = ws.conv3x3_adjoint(y, W, x.shape)
    elif op == "pool":
        x = rng.normal(size=(2, 6, 8, 3))
        fwd = ws.avgpool2(x)
        y = rng.normal(size=fwd.shape)
        adj = ws.avgpool2_adjoint(y)
    else:
        x = rng.normal(size=(2, 3, 4, 3))
        fwd = ws.up2(x)
        y = rng.normal(size=fwd.shape)
        adj = ws.up2_adjoint(y)
    assert abs(np.vdot(fwd, y) - np.vdot(x, adj)) < 1e-10 * max(1.0, abs(np.vdot(fwd, y)))


def test_wgrad_is_the_weight_adjoint():
    """<conv(x, W), dy> is linear in W, so its W-gradient is conv3x3_wgrad."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 5, 6, 2))
    dy = rng.normal(size=(2, 5, 6, 3))
    dW, db = ws.conv3x3_wgrad(x, dy)
    for _ in range(5):
        V = rng.normal(size=(3, 3, 3, 2))
        assert abs(np.vdot(ws.conv3x3(x, V), dy) - np.vdot(V, dW)) < 1e-10
    assert np.allclose(db, dy.sum(axis=(0, 1, 2)))


def test_pool_and_up_closed_forms():
    x = np.arange(16.0).reshape(1, 4, 4, 1)
    assert ws.avgpool2(x)[0, :, :, 0].tolist() == [[2.5, 4.5], [10.5, 12.5]]
    u = ws.up2(np.array([[1.0, 2.0]]).reshape(1, 1, 2, 1))
    assert u[0, :, :, 0].tolist() == [[1, 1, 2, 2], [1, 1, 2, 2]]


def test_backward_matches_central_differences():
    """Every parameter of a tiny network against central differences of the
    loss (a dropped ReLU mask, a wrong adjoint or pooling scale fails here)."""
    rng = np.random.default_rng(4)
    theta = synth.net_init(5, TINY)
    theta[-1] = 0.3                      # non-zero last bias
    f = rng.normal(size=(2, 8, 12))
    phi = 3.0 * rng.normal(size=(2, 8, 12))
    L, g = ws.loss_and_grad(theta, f, phi, clip=2.0, layers=TINY)
    h = 1e-6
    num = np.empty_like(theta)
    for k in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        num[k] = (ws.loss_and_grad(tp, f, phi, 2.0, TINY)[0]
                  - ws.loss_and_grad(tm, f, phi, 2.0, TINY)[0]) / (2 * h)
    assert np.abs(num - g).max() <= 1e-6 * np.abs(g).max() + 1e-9
    assert L == pytest.approx(0.5 * np.mean((ws.forward(ws.unflatten(theta, TINY), f)[0]
                                             - np.clip(phi, -2, 2) / 2) ** 2))


def test_target_clip_and_scale():
    t = ws.target(np.array([-10.0, -2.0, 0.0, 1.0, 7.0]), 4.0)
    assert t.tolist() == [-1.0, -0.5, 0.0, 0.25, 1.0]


def test_adam_first_step_closed_form():
    """With m = v = 0 the bias-corrected first step is lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = ws.adam(th, g, np.zeros(50), np.zeros(50), 1, lr=1e-2)
    assert np.allclose(new, th - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps the bias-corrected step at lr g / (|g| + eps)
    th2, m, v = ws.adam(new, g, m, v, 2, lr=1e-2)
    assert np.allclose(th2, new - 1e-2 * g / (np.abs(g) + 1e-8), atol=1e-12)


def test_seeded_network_parameters():
    """He-normal weights per layer (the last layer's scaled by 0.1), zero
    biases, the same vector for the same seed."""
    theta = synth.net_init(9, ws.LAYERS)
    assert theta.size == ws.param_count()
    assert np.array_equal(theta, synth.net_init(9, ws.LAYERS))
    for k, ((W, b), (ci, co)) in enumerate(zip(ws.unflatten(theta), ws.LAYERS)):
        assert np.all(b == 0.0)
        want = np.sqrt(2.0 / (9 * ci)) * (0.1 if k == len(ws.LAYERS) - 1 else 1.0)
        if W.size >= 1000:
            assert W.std() == pytest.approx(want, rel=0.1)


def test_bf16_exact_matches_torch_rounding():
    import torch
    rng = np.random.default_rng(10)
    a = rng.normal(size=20000) * np.exp(rng.normal(size=20000) * 4)
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(synth.bf16_exact(a), ref)
