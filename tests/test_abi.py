"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point that include/sr.h declares; argument validation happens before
any CUDA call."""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def srmod():
    from paper_2003_12693_gb300 import build, sr
    build.build()
    return sr


def test_library_exports_every_declared_function(srmod):
    names = srmod.declared_functions()
    assert len(names) >= 20
    lib = srmod.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    for core in ("sr_create", "sr_edge_function", "sr_iterate", "sr_mask"):
        assert core in names


def test_params_default_is_fig1_set(srmod):
    p = srmod.params_default()
    assert (p.alpha, p.beta, p.gamma, p.mu, p.tau, p.eps, p.band_l) == \
        pytest.approx((4.0, 0.2, 4.0, 8.0, 0.1, 1.0, 1.0))
    assert p.inner_S == 3 and p.inner_tol == 0.0 and p.s_pow == 2 and p.check_every >= 1


def _create(srmod, H, W, **kw):
    p = srmod.make_params(**kw)
    h = C.c_void_p()
    st = srmod.lib().sr_create(H, W, C.byref(p), None, C.byref(h))
    return st, h


@pytest.mark.parametrize("kw,status", [
    (dict(mu=0.0), 1), (dict(tau=-0.1), 1), (dict(eps=0.0), 1), (dict(alpha=float("nan")), 1),
    (dict(beta=float("inf")), 1), (dict(win_radius=9), 1), (dict(win_radius=-1), 1),
    (dict(inner_S=0), 1), (dict(s_pow=3), 1), (dict(check_every=0), 1), (dict(d=0.0), 1),
    (dict(sigma=11.0), 1), (dict(inner_tol=float("nan")), 1),
])
def test_create_rejects_bad_parameters_before_touching_cuda(srmod, kw, status):
    st, h = _create(srmod, 64, 64, **kw)
    assert st == status and not h.value


@pytest.mark.parametrize("H,W", [(0, 64), (64, -1), (40, 64), (64, 100), (8, 64), (8192, 64),
                                 (592, 64), (64, 1184)])
def test_create_rejects_unsupported_sizes(srmod, H, W):
    st, h = _create(srmod, H, W)
    assert st in (1, 7) and not h.value


def test_null_arguments(srmod):
    L = srmod.lib()
    assert L.sr_create(64, 64, None, None, None) == 1
    assert L.sr_params_default(None) == 1
    assert L.sr_iterate(None, 1, 0.0, None, None) == 1
    assert L.sr_mask(None, None, 64) == 1
    L.sr_destroy(None)
    assert L.sr_status_string(3) == b"CUDA error"
    assert L.sr_last_error(None) == b""


def test_mode_entry_points_reject_null_context(srmod):
    """The mode switches validate their context before any CUDA call."""
    L = srmod.lib()
    for on in (0, 1, 8, 16, 4):
        assert L.sr_set_resident(None, on) == 1
    assert L.sr_set_phi_solver(None, 1) == 1
    assert L.sr_set_boundary(None, 1) == 1


def test_w_sweep_entry_points_reject_null_context(srmod):
    L = srmod.lib()
    assert L.sr_set_w_sweeps(None, 2) == 1
    assert L.sr_w_b_fixed_point(None, None, None, None, None, None, 1, None, None, None, None) == 1


@pytest.fixture(scope="module")
def netmod(srmod):
    from paper_2003_12693_gb300 import sr_net
    sr_net.lib()
    return sr_net


def test_network_layer_table_matches_the_oracle(netmod):
    from oracle import warmstart as ws
    assert netmod.layers() == [tuple(x) for x in ws.LAYERS]
    assert netmod.param_count() == ws.param_count() == 185217
    import ctypes as C
    ci, co = C.c_int(), C.c_int()
    assert netmod.lib().sr_net_layer_shape(6, C.byref(ci), C.byref(co)) == 1
    assert netmod.lib().sr_net_layer_shape(-1, C.byref(ci), C.byref(co)) == 1


@pytest.mark.parametrize("H,W,B,clip", [(30, 32, 1, 4.0), (32, 6, 1, 4.0), (32, 32, 0, 4.0),
                                        (32, 32, 1, 0.0), (32, 32, 1, float("nan")),
                                        (8192, 32, 1, 4.0)])
def test_network_create_rejects_bad_arguments_before_touching_cuda(netmod, H, W, B, clip):
    import ctypes as C
    h = C.c_void_p()
    assert netmod.lib().sr_net_create(H, W, B, clip, None, C.byref(h)) == 1
    assert not h.value
    assert netmod.lib().sr_net_create(32, 32, 1, 4.0, None, None) == 1


def test_network_layer_calls_reject_bad_shapes_before_touching_cuda(netmod):
    import ctypes as C
    L = netmod.lib()
    p = C.c_void_p(16)   # never dereferenced: validation fails first
    # cin not a multiple of 16
    assert L.sr_conv3x3(p, 1, 8, 8, 24, p, p, 32, 0, None, p, 1.0, None) == 1
    # cout not 16, 32 or a multiple of 64
    assert L.sr_conv3x3(p, 1, 8, 8, 32, p, p, 48, 0, None, p, 1.0, None) == 1
    # mask mode without ref, bad mode
    assert L.sr_conv3x3(p, 1, 8, 8, 32, p, p, 32, 2, None, p, 1.0, None) == 1
    assert L.sr_conv3x3(p, 1, 8, 8, 32, p, p, 32, 7, None, p, 1.0, None) == 1
    assert L.sr_conv3x3_dgrad(p, 1, 8, 8, 32, p, 32, 0, None, p, None) == 1   # RELU not allowed
    assert L.sr_conv3x3_wgrad(p, p, 1, 8, 8, 32, 48, 32, 48, p, None, None) == 1
    assert L.sr_conv3x3_wgrad(p, p, 1, 8, 8, 32, 32, 33, 32, p, None, None) == 1
    for name in ("sr_net_set_params", "sr_net_get_params", "sr_net_get_grads"):
        assert getattr(L, name)(None, p) == 1
    assert L.sr_net_forward(None, p, 1, p) == 1
    assert L.sr_net_kernel_launches(None, 0) == -1
    L.sr_net_destroy(None)


def test_failure_hooks_validate_without_a_gpu(srmod):
    L = srmod.lib()
    assert L.sr_test_stall_waits(None, 10) == 1
    assert L.sr_test_fail_allocations(-1) == 0
