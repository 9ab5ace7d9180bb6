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
    (dict(sigma=11.0), 1), (dict(inner_tol=1e-3), 7),
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
