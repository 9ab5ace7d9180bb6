"""The warm-start network's kernels against the FP64 oracle.

Layer by layer on bf16-representable inputs (so both sides start from the
same values): the tensor-core convolution in each output mode, its input
gradient (the kernel uses flipped transposed weights, the oracle the plain
adjoint), its weight and bias gradients; then the whole network's output and
gradients, Adam's first step, and a short training run.

Tolerances.  A convolution output rounded to bf16 carries a relative error of
at most 2^-9 from the rounding, plus the fp32 accumulation error, at most
K 2^-24 sum |x||w| over its K products; the tests use 2^-8 |ref| +
K 2^-24 conv(|x|, |w|).  Weight gradients stay in fp32: K 2^-24 times the
sum of |dy||x| over the K = B H W pixels.  The whole network rounds every
activation and gradient to bf16 (six layers deep); there the tests bound the
output's relative L2 error by 2e-2 and each gradient block's error by 3e-2
of the norm of its sum of absolute terms."""
import numpy as np
import pytest
import torch

from gpu_common import report
from oracle import warmstart as ws
from paper_2003_12693_gb300 import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def sn():
    from paper_2003_12693_gb300 import sr_net
    return sr_net


def bfdev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16)


def fdev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().float().cpu().numpy().astype(np.float64)


def rand_bf(rng, shape, scale=1.0):
    return synth.bf16_exact(rng.normal(size=shape) * scale)


CONV_SHAPES = [(16, 32), (32, 64), (64, 128), (128, 64), (64, 32), (32, 16), (16, 16), (48, 64)]


@pytest.mark.parametrize("cin,cout", CONV_SHAPES)
@pytest.mark.parametrize("mode", ["relu", "plain"])
def test_conv3x3_forward(cin, cout, mode):
    """M = 2 x 10 x 14 = 280 pixels: three 128-pixel tiles, the last ragged."""
    S = sn()
    rng = np.random.default_rng(cin * 7 + cout)
    x = rand_bf(rng, (2, 10, 14, cin))
    w = rand_bf(rng, (cout, 3, 3, cin), 0.2)
    b = synth.bf16_exact(rng.normal(size=cout))
    m = S.SR_CONV_RELU if mode == "relu" else S.SR_CONV_PLAIN
    y = host(S.conv3x3(bfdev(x), bfdev(w), fdev(b), m))
    ref = ws.conv3x3(x, w, b)
    if mode == "relu":
        ref = np.maximum(ref, 0.0)
    A = ws.conv3x3(np.abs(x), np.abs(w), np.abs(b))
    tol = 2.0 ** -8 * np.abs(ref) + 9 * cin * U * A + 1e-30
    report("net_conv_fwd", cin=cin, cout=cout, mode=mode, max_err=np.abs(y - ref).max())
    assert np.all(np.abs(y - ref) <= tol)


def test_conv3x3_out1_channel0_scaled():
    S = sn()
    rng = np.random.default_rng(3)
    x = rand_bf(rng, (3, 12, 20, 32))
    w = np.zeros((16, 3, 3, 32))
    w[:1] = rand_bf(rng, (1, 3, 3, 32), 0.2)
    b = np.zeros(16)
    b[0] = 0.375
    y = host(S.conv3x3(bfdev(x), bfdev(w), fdev(b), S.SR_CONV_OUT1, out_scale=4.0))
    ref = 4.0 * ws.conv3x3(x, w[:1], b[:1])[..., 0]
    A = 4.0 * ws.conv3x3(np.abs(x), np.abs(w[:1]), np.abs(b[:1]))[..., 0]
    assert y.shape == (3, 12, 20)
    assert np.all(np.abs(y - ref) <= 9 * 32 * U * A * 2 + 1e-6)


@pytest.mark.parametrize("cout,cin", [(16, 32), (32, 64), (64, 128), (128, 64), (64, 32)])
@pytest.mark.parametrize("mask", [False, True])
def test_conv3x3_dgrad_is_the_adjoint(cout, cin, mask):
    S = sn()
    rng = np.random.default_rng(cout * 3 + cin)
    shape = (2, 9, 13, cin)
    dy = rand_bf(rng, (2, 9, 13, cout))
    w = rand_bf(rng, (cout, 3, 3, cin), 0.2)
    ref = ws.conv3x3_adjoint(dy, w, shape)
    A = ws.conv3x3_adjoint(np.abs(dy), np.abs(w), shape)
    if mask:
        a = rand_bf(rng, shape)
        a[a < 0] = 0.0                      # ReLU outputs: zeros and positives
        ref = ref * (a > 0)
        dx = host(S.conv3x3_dgrad(bfdev(dy), bfdev(w), S.SR_CONV_MASK, bfdev(a)))
    else:
        dx = host(S.conv3x3_dgrad(bfdev(dy), bfdev(w)))
    tol = 2.0 ** -8 * np.abs(ref) + 9 * cout * U * A + 1e-30
    report("net_conv_dgrad", cin=cin, cout=cout, mask=mask, max_err=np.abs(dx - ref).max())
    assert np.all(np.abs(dx - ref) <= tol)


@pytest.mark.parametrize("cin,cout,cin_real,cout_real",
                         [(16, 32, 1, 32), (32, 64, 32, 64), (64, 128, 64, 128),
                          (128, 64, 128, 64), (64, 32, 64, 32), (32, 16, 32, 1),
                          (16, 16, 16, 16), (32, 32, 32, 32)])
def test_conv3x3_wgrad(cin, cout, cin_real, cout_real):
    """Pixel slabs of 64 with a ragged last chunk (B H W = 3 x 11 x 17 = 561)."""
    S = sn()
    rng = np.random.default_rng(cin + 5 * cout)
    x = rand_bf(rng, (3, 11, 17, cin))
    dy = rand_bf(rng, (3, 11, 17, cout), 0.5)
    x[..., cin_real:] = 0.0
    dw, db = S.conv3x3_wgrad(bfdev(dy), bfdev(x), cin_real, cout_real)
    dw, db = host(dw), host(db)
    rW, rb = ws.conv3x3_wgrad(x[..., :cin_real], dy[..., :cout_real])
    AW, Ab = ws.conv3x3_wgrad(np.abs(x[..., :cin_real]), np.abs(dy[..., :cout_real]))
    K = 3 * 11 * 17
    report("net_conv_wgrad", cin=cin, cout=cout, max_err=np.abs(dw - rW).max())
    assert dw.shape == rW.shape
    assert np.all(np.abs(dw - rW) <= K * U * AW + 1e-30)
    assert np.all(np.abs(db - rb) <= K * U * Ab + 1e-30)


def test_wgrad_accumulates_into_the_output():
    S = sn()
    rng = np.random.default_rng(9)
    x = rand_bf(rng, (1, 8, 8, 32))
    dy = rand_bf(rng, (1, 8, 8, 32))
    lib = S.lib()
    import ctypes as C
    dw = torch.ones((32, 3, 3, 32), dtype=torch.float32, device="cuda")
    xd, dyd = bfdev(x), bfdev(dy)
    st = lib.sr_conv3x3_wgrad(C.c_void_p(dyd.data_ptr()), C.c_void_p(xd.data_ptr()), 1, 8, 8, 32,
                              32, 32, 32, C.c_void_p(dw.data_ptr()), None,
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    rW, _ = ws.conv3x3_wgrad(x, dy)
    assert np.allclose(host(dw), 1.0 + rW, rtol=1e-5, atol=1e-5)


# ----------------------------------------------------------------------------
# The whole network
# ----------------------------------------------------------------------------
def net_inputs(seed, B, H, W):
    """bf16-exact weights (the kernels' operands) and images, fp32 biases."""
    theta = synth.net_init(seed, ws.LAYERS)
    rng = np.random.default_rng(seed + 1)
    params = ws.unflatten(theta)
    for Wt, b in params:
        Wt[...] = synth.bf16_exact(Wt)
        b[...] = np.asarray(rng.normal(size=b.shape) * 0.05, dtype=np.float32)
    theta = ws.flatten(params)
    f = synth.bf16_exact(rng.uniform(0.0, 1.0, (B, H, W)) + 0.1 * rng.normal(size=(B, H, W)))
    phi = 6.0 * np.sin(np.arange(H)[:, None] / 5.0 + np.arange(W)[None, :] / 7.0) + \
        rng.normal(size=(B, H, W))
    return theta, f, np.asarray(phi, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("B,H,W", [(3, 32, 32), (2, 24, 40), (1, 64, 48)])
def test_net_forward_matches_oracle(B, H, W):
    S = sn()
    theta, f, _ = net_inputs(11 + H, B, H, W)
    net = S.Net(H, W, max_batch=4, phi_clip=4.0)
    net.set_params(fdev(theta))
    phi0 = host(net.forward(fdev(f)))
    y, _ = ws.forward(ws.unflatten(theta), f)
    ref = 4.0 * y
    report("net_forward", shape=f"{B}x{H}x{W}", rel_l2=rel(phi0, ref))
    assert rel(phi0, ref) <= 2e-2
    net.close()


@pytest.mark.parametrize("B,H,W", [(2, 32, 32), (1, 24, 40)])
def test_net_gradients_match_oracle(B, H, W):
    """Each gradient block is a sum over the pixels whose terms carry the
    bf16 roundings of eleven stages (forward and backward); the sums cancel
    (|sum| is about a tenth of sum |.| here), which magnifies their relative
    error.  So the error is bounded against the norm of the sum of absolute
    terms, wgrad(|x|, |delta|), computed by the oracle, and, per block, the
    relative L2 distance to the oracle's gradient is bounded too."""
    S = sn()
    theta, f, phi = net_inputs(23 + W, B, H, W)
    net = S.Net(H, W, max_batch=B, phi_clip=4.0)
    net.set_params(fdev(theta))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.gradients(fdev(f), fdev(phi), loss)
    g = host(net.get_grads())
    params = ws.unflatten(theta)
    y, cache = ws.forward(params, f)
    t = ws.target(phi, 4.0)
    L = ws.loss(y, t)
    assert host(loss)[0] == pytest.approx(L, rel=2e-2)
    k, bad = 0, []
    for li, ((ci, co), (x, d)) in enumerate(zip(ws.LAYERS, ws.deltas(params, cache, y, t))):
        rW, rb = ws.conv3x3_wgrad(x, d)
        aW, ab = ws.conv3x3_wgrad(np.abs(x), np.abs(d))
        for name, r, aa in (("W", rW, aW), ("b", rb, ab)):
            n = r.size
            a = g[k:k + n]
            r, aa = r.ravel(), aa.ravel()
            err = np.linalg.norm(a - r) / np.linalg.norm(aa)
            cos = np.dot(a, r) / max(np.linalg.norm(a) * np.linalg.norm(r), 1e-30)
            report("net_grad", shape=f"{B}x{H}x{W}", layer=li + 1, part=name, rel_l2=rel(a, r),
                   err_vs_abs=err, cos=cos)
            # and per block against the oracle itself: bf16 rounding of eleven
            # stages magnified by the cancellation (|sum| ~ sum|.| / 8) gives
            # up to about 11 % here (measured on GB300); 20 % is the bound, so
            # a dropped or doubled term that carries a fifth of a block fails
            if not (err <= 3e-2 and cos >= 0.99 and rel(a, r) <= 0.2):
                bad.append((li + 1, name, err, cos, rel(a, r)))
            k += n
    assert k == g.size
    assert not bad, bad
    net.close()


def test_adam_first_step_is_lr_sign():
    """From fresh moments the bias-corrected step is lr g / (|g| + eps), g the
    gradient the step itself computed (a property of the kernel's own output)."""
    S = sn()
    theta, f, phi = net_inputs(31, 2, 32, 32)
    net = S.Net(32, 32, max_batch=2)
    net.set_params(fdev(theta))
    th0 = host(net.get_params())
    lr = 1e-3
    net.train_step(fdev(f), fdev(phi), lr=lr)
    th1 = host(net.get_params())
    g = host(net.get_grads())
    step = -lr * g / (np.abs(g) + 1e-8)
    assert np.all(np.abs((th1 - th0) - step) <= 4e-6 * lr + 2.0 ** -22 * np.abs(th0))
    assert np.count_nonzero(g) > 0.5 * g.size
    net.close()


def test_training_lowers_the_loss_on_a_fixed_batch():
    S = sn()
    theta, f, phi = net_inputs(41, 4, 32, 32)
    net = S.Net(32, 32, max_batch=4)
    net.set_params(fdev(theta))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    fd, pd = fdev(f), fdev(phi)
    hist = []
    for _ in range(80):
        net.train_step(fd, pd, lr=2e-3, loss=loss)
        hist.append(host(loss)[0])
    report("net_train_fixed_batch", first=hist[0], last=hist[-1])
    assert np.isfinite(hist).all()
    assert hist[-1] < 0.5 * hist[0]
    # the oracle's loss at the trained parameters agrees with the kernel's
    L, _ = ws.loss_and_grad(host(net.get_params()), synth.bf16_exact(f), phi, 4.0)
    net.gradients(fd, pd, loss)
    assert host(loss)[0] == pytest.approx(L, rel=5e-2)
    net.close()


def test_net_argument_checks():
    S = sn()
    with pytest.raises(S._sr.SRError):
        S.Net(30, 32, 1)
    net = S.Net(32, 32, 2)
    with pytest.raises(ValueError):
        net.forward(torch.zeros((1, 32, 16), device="cuda"))
    with pytest.raises(S._sr.SRError):
        net.forward(torch.zeros((3, 32, 32), device="cuda"))
    net.close()
