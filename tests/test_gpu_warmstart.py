"""What the trained warm-start network gains over the rectangle start.

A short run of the whole learned pipeline on 128 x 128 ellipse scenes: the
plain solver produces (image, phi after 1500 iterations) pairs, the network
trains on them with its own kernels, and on held-out images its phi0 is
compared with the inset-rectangle start of Alg. 1 against the plain solver's
state.  The iteration counts until the mask settles are reported, not
asserted: on these scenes the plain contour keeps creeping for thousands of
iterations."""
import numpy as np
import pytest
import torch

from gpu_common import report
from paper_2003_12693_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12693_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def test_trained_network_starts_closer_than_the_rectangle():
    from paper_2003_12693_gb300 import sr, sr_net, warmstart as wsm
    n, n_train, n_eval, t_ref = 128, 256, 8, 1500
    imgs = np.stack([synth.ellipse_scene(30000 + k, n, n, scale=n / 512.0)
                     for k in range(n_train + n_eval)]).astype(np.float32)
    prm = dict(synth.WORKLOADS["ellipses_512"].params())
    prm.update(rho=1e4, sigma=3.0)
    p = sr.make_params(**prm)
    rect = torch.from_numpy(synth.inset_rect_sdf(n, n).astype(np.float32)).cuda()
    trd = torch.from_numpy(imgs[:n_train]).cuda()
    evd = torch.from_numpy(imgs[n_train:]).cuda()
    phis = wsm.generate_pairs(trd, rect, p, t_ref)
    ref_phi = wsm.generate_pairs(evd, rect, p, t_ref)
    net = sr_net.Net(n, n, max_batch=16, phi_clip=4.0)
    net.set_params(torch.from_numpy(synth.net_init(7, sr_net.layers()).astype(np.float32)).cuda())
    hist = wsm.train(net, trd, phis, 600, 16, 2e-3)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.gradients(evd, ref_phi, loss)
    tgt = torch.clamp(ref_phi, -4.0, 4.0) / 4.0
    rect_loss = 0.5 * torch.mean((torch.clamp(rect, -4.0, 4.0) / 4.0 - tgt) ** 2).item()
    phi0 = net.forward(evd)
    ref_m = [(ref_phi[k] < 0).to(torch.uint8) for k in range(n_eval)]
    iou_net = np.mean([wsm._iou((phi0[k] < 0).to(torch.uint8), ref_m[k]) for k in range(n_eval)])
    iou_rect = np.mean([wsm._iou((rect < 0).to(torch.uint8), m) for m in ref_m])
    thr = int(0.002 * n * n)
    plain = wsm.solve_plain(evd, rect, p, check=100, thr=thr, max_iters=2 * t_ref)
    learned = wsm.solve_batched(evd, phi0, p, check=100, thr=thr, max_iters=2 * t_ref)
    report("warm_start_gain", train_loss_first=hist[0], train_loss_last=float(np.mean(hist[-20:])),
           heldout_loss=loss.item(), rect_loss=rect_loss, start_iou_net=iou_net,
           start_iou_rect=iou_rect, plain_iters=float(np.mean(plain.iters)),
           learned_iters=float(np.mean(learned.iters)), plain_s=plain.seconds,
           learned_batched_s=learned.seconds)
    assert np.mean(hist[-20:]) < 0.5 * hist[0]
    assert loss.item() < rect_loss
    assert iou_net > iou_rect
    net.close()
