"""gsis_transport_sweep_static: the kinetic step for callers that cannot
allocate device memory (it uses the library's fixed 32 MiB static device
scratch instead of a caller workspace).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def gs():
    import torch
    from paper_2507_03975_gb300 import build, gsis
    build.build()
    gsis.load()
    torch.cuda.set_device(0)
    return gsis


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_sweep_matches_workspace_sweep(gs, prec):
    p = W.random_problem(70, 45, order=6, seed=91)
    opt = gs.default_options(precision=gs.FP64 if prec == "fp64" else gs.FP32_SWEEP)
    assert gs.workspace_bytes(p.dx, p.dy, p.mu, p.eta, p.w, opt) <= 32 * 1024 * 1024
    args = (p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q))
    rng = np.random.Generator(np.random.PCG64(3))
    inflow = _t(p.inflow.reshape(-1))
    for call in range(2):                      # two calls in a row share the static scratch
        rho_in = _t(rng.uniform(0.0, 2.0, p.N))
        ref = gs.transport_sweep(*args, rho_in, inflow, opt)
        got = gs.transport_sweep_static(*args, rho_in, inflow, opt)
        for key in ("rho", "F", "P", "bflux"):
            assert _rel(got[key], ref[key]) < TOL64, (call, key)


def test_static_scratch_rejects_oversized_problem(gs):
    p = W.config_channel()                     # needs ~105 MB of scratch
    opt = gs.default_options()
    assert gs.workspace_bytes(p.dx, p.dy, p.mu, p.eta, p.w, opt) > 32 * 1024 * 1024
    z = _t(np.zeros(p.N))
    with pytest.raises(gs.GsisError) as ei:
        gs.transport_sweep_static(p.dx, p.dy, p.mu, p.eta, p.w, z, z, z, z, None, opt)
    assert ei.value.status == gs.GSIS_ERR_WORKSPACE
    assert "static array" in str(ei.value)


def test_static_scratch_sizes_the_kinetic_step_not_the_solve(gs):
    # gsis_transport_sweep runs first-order upwind without pseudo-time
    # whatever the options ask, so options that enlarge only the full solve's
    # workspace (second-order faces, pseudo-time) must not get a problem
    # rejected: 128x128 S12 needs 29 MiB for the sweep, 40 MiB for the solve
    p = W.random_problem(128, 128, order=12, seed=92)
    opt = gs.default_options(spatial_order=2, beta=10.0)
    plain = gs.default_options()
    assert gs.workspace_bytes(p.dx, p.dy, p.mu, p.eta, p.w, opt) > 32 * 1024 * 1024
    assert gs.workspace_bytes(p.dx, p.dy, p.mu, p.eta, p.w, plain) <= 32 * 1024 * 1024
    args = (p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q))
    rho_in = _t(np.random.Generator(np.random.PCG64(5)).uniform(0.0, 2.0, p.N))
    inflow = _t(p.inflow.reshape(-1))
    for call in range(2):
        ref = gs.transport_sweep(*args, rho_in, inflow, plain)
        got = gs.transport_sweep_static(*args, rho_in, inflow, opt)
        for key in ("rho", "F", "P", "bflux"):
            assert _rel(got[key], ref[key]) < TOL64, (call, key)
