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


def test_td_adjoint_checks_and_storage(gs):
    """gsis_td_adjoint_workspace_bytes: argument checks (GSIS only, uniform
    mesh, reflection-closed quadrature, no pseudo-time, checkpoint_every >= 1)
    and the storage of ceil(nsteps/C) checkpoints plus one C-step segment."""
    mu, eta, w = gs.quadrature_level_symmetric(4)
    dx = np.full(16, 1 / 16)
    ok = gs.default_options()

    def nb(nsteps, C, o=ok, ddx=dx):
        return gs.td_adjoint_workspace_bytes(ddx, dx, mu, eta, w, 0.1, nsteps, C, options=o)

    for bad in (dict(o=gs.default_options(scheme=gs.SCHEME_SI)), dict(o=gs.default_options(beta=1.0)),
                dict(ddx=np.linspace(0.5, 1.5, 16) / 16.0)):
        with pytest.raises(gs.GsisError) as e:
            nb(4, 2, **bad)
        assert e.value.status == gs.GSIS_ERR_ARG
    with pytest.raises(gs.GsisError):
        nb(4, 0)
    KN8 = len(w) * 16 * 16 * 8
    # one more checkpoint or one more segment step costs one intensity array plus per-cell
    # vectors: 7 in a checkpoint (state and the predictor's history), 3 in a step record
    N8 = 16 * 16 * 8
    assert KN8 <= nb(9, 3) - nb(6, 3) < 2 * KN8          # 3 -> 2 checkpoints
    d = nb(12, 6) - nb(12, 4)                            # 2 checkpoints + 6 steps vs 3 + 4
    assert KN8 + (2 * 3 - 7) * N8 <= d < KN8 + 2 * N8    # one array more, one checkpoint's vectors fewer
    assert nb(5, 5) == nb(5, 9)                           # the segment never exceeds the run


def test_td_adjoint_binding_rejects_before_device_use(gs):
    """The binding's argument list matches the C signature: a call with the
    SI scheme returns GSIS_ERR_ARG before any device pointer is touched."""
    mu, eta, w = gs.quadrature_level_symmetric(4)
    a = gs._Args(np.full(8, 0.125), np.full(8, 0.125), mu, eta, w)
    tp = gs.TimeParams(0.1, 1.0, 1.0, 1.0, 3)
    dummy = ctypes.c_void_p(0x1000)   # never dereferenced
    its = (ctypes.c_int * 3)()
    lib = gs._td_adj_load()
    rc = lib.gsis_td_adjoint(ctypes.byref(a.mesh), ctypes.byref(a.quad),
                             ctypes.byref(gs.default_options(scheme=gs.SCHEME_SI)), ctypes.byref(tp), 2,
                             *([dummy] * 14), its, ctypes.c_void_p(256), ctypes.c_size_t(1 << 40), None)
    assert rc == gs.GSIS_ERR_ARG
    rc = lib.gsis_td_adjoint(ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(gs.default_options()),
                             ctypes.byref(tp), 2, *([dummy] * 14), its, None, ctypes.c_size_t(0), None)
    assert rc == gs.GSIS_ERR_WORKSPACE
    tp.predictor = 2   # accepted: the checkpoints carry the predictor's history
    rc = lib.gsis_td_adjoint(ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(gs.default_options()),
                             ctypes.byref(tp), 2, *([dummy] * 14), its, None, ctypes.c_size_t(0), None)
    assert rc == gs.GSIS_ERR_WORKSPACE
    tp.predictor = 3
    rc = lib.gsis_td_adjoint(ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(gs.default_options()),
                             ctypes.byref(tp), 2, *([dummy] * 14), its, None, ctypes.c_size_t(0), None)
    assert rc == gs.GSIS_ERR_ARG and "predictor" in gs.last_error()


def test_td_solve_rejects_predictor_out_of_range(gs):
    """gsis_time_params::predictor is 0, 1 or 2; anything else is
    GSIS_ERR_ARG before any device pointer is touched."""
    mu, eta, w = gs.quadrature_level_symmetric(4)
    a = gs._Args(np.full(8, 0.125), np.full(8, 0.125), mu, eta, w)
    dummy = ctypes.c_void_p(0x1000)   # never dereferenced
    its = (ctypes.c_int * 3)()
    lib = gs._td_load()
    for bad in (-1, 3):
        tp = gs.TimeParams(0.1, 1.0, 1.0, 1.0, 3, bad)
        rc = lib.gsis_td_solve(ctypes.byref(a.mesh), ctypes.byref(a.quad), ctypes.byref(gs.default_options()),
                               ctypes.byref(tp), *([dummy] * 9), its, None, None, ctypes.c_size_t(0), None)
        assert rc == gs.GSIS_ERR_ARG and "predictor" in gs.last_error()


def test_mesh_size_limits(gs):
    """Sides above 2^20 - 1 cells and meshes above 2^30 cells are rejected on
    the host (GSIS_ERR_ARG) before anything is sized or launched; the largest
    side is accepted."""
    mu, eta, w = gs.quadrature_level_symmetric(4)
    big = (1 << 20) - 1
    ok = gs.workspace_bytes(np.full(big, 1.0 / big), np.full(1, 1.0), mu, eta, w)
    assert ok > 0
    for nx, ny in ((big + 1, 1), ((1 << 15) + 1, (1 << 15) + 1)):
        with pytest.raises(gs.GsisError) as e:
            gs.workspace_bytes(np.full(nx, 1.0 / nx), np.full(ny, 1.0 / ny), mu, eta, w)
        assert e.value.status == gs.GSIS_ERR_ARG
