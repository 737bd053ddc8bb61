"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Tolerances: FP64 path 1e-10 relative (max norm, relative
to the oracle field's max), FP32-sweep path 1e-5 relative in the energy
density."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


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


def _inflow(p):
    return None if p.inflow is None else _t(p.inflow.reshape(-1))


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


SWEEP_CASES = [
    ("random_70x45_S6", lambda: W.random_problem(70, 45, order=6, seed=1)),
    ("random_33x97_S8_vacuum", lambda: W.random_problem(33, 97, order=8, seed=2, with_inflow=False)),
    ("uniform_64_S8", lambda: W.config_small()),
    ("one_cell", lambda: W.random_problem(1, 1, order=4, seed=3)),
    ("one_row", lambda: W.random_problem(40, 1, order=4, seed=4)),
    ("one_column", lambda: W.random_problem(1, 40, order=4, seed=5)),
    ("short_rows", lambda: W.random_problem(7, 66, order=6, seed=6)),
    ("ragged_33", lambda: W.random_problem(130, 33, order=4, seed=7)),
    ("thick_thin", lambda: W.channel_problem(64, 8, 2, width=2)),
]


@pytest.mark.parametrize("name,make", SWEEP_CASES, ids=[c[0] for c in SWEEP_CASES])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_transport_sweep_parity(gs, name, make, prec):
    p = make()
    rng = np.random.Generator(np.random.PCG64(17))
    rho_in = rng.uniform(0.0, 3.0, p.N)
    o = oracle.transport_sweep(p, rho_in)
    opt = gs.default_options(precision=gs.FP64 if prec == "fp64" else gs.FP32_SWEEP)
    r = gs.transport_sweep(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q),
                           _t(rho_in), _inflow(p), opt)
    N = p.N
    F = r["F"].cpu().numpy()
    P = r["P"].cpu().numpy()
    tol = TOL64 if prec == "fp64" else TOL32
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < tol
    if prec == "fp64":
        scale = max(np.abs(o["rho"]).max(), 1e-300)
        for got, key in ((F[:N], "Fx"), (F[N:], "Fy"), (P[:N], "Pxx"), (P[N:2 * N], "Pxy"), (P[2 * N:], "Pyy")):
            assert np.abs(got - o[key]).max() / scale < TOL64, key
        assert np.abs(r["bflux"].cpu().numpy() - o["fb"]).max() / scale < TOL64
    else:
        scale = np.abs(o["rho"]).max()
        assert np.abs(F[:N] - o["Fx"]).max() / scale < 1e-4
        assert np.abs(r["bflux"].cpu().numpy() - o["fb"]).max() / scale < 1e-4


def _rotated(p, angle):
    """The same problem with its ordinates rotated about the z axis: a valid
    quadrature (weights and moments kept) without (mu, eta) -> (-mu, eta)
    pairs, so the moments take their plain per-direction sums."""
    import dataclasses
    c, s_ = math.cos(angle), math.sin(angle)
    mu = c * p.mu - s_ * p.eta
    eta = s_ * p.mu + c * p.eta
    return dataclasses.replace(p, mu=mu, eta=eta, inflow=None)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sweep_parity_without_reflection_pairs(gs, prec):
    p = _rotated(W.random_problem(70, 45, order=6, seed=18), 0.1)
    rng = np.random.Generator(np.random.PCG64(19))
    rho_in = rng.uniform(0.0, 3.0, p.N)
    o = oracle.transport_sweep(p, rho_in)
    r = gs.transport_sweep(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), _t(rho_in), None,
                           gs.default_options(precision=gs.FP64 if prec == "fp64" else gs.FP32_SWEEP))
    tol = TOL64 if prec == "fp64" else TOL32
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < tol
    N = p.N
    F = r["F"].cpu().numpy()
    scale = np.abs(o["rho"]).max()
    assert np.abs(F[:N] - o["Fx"]).max() / scale < (TOL64 if prec == "fp64" else 1e-4)
    assert np.abs(F[N:] - o["Fy"]).max() / scale < (TOL64 if prec == "fp64" else 1e-4)


def test_sweep_is_deterministic(gs):
    p = W.random_problem(70, 45, order=6, seed=1)
    rho_in = np.linspace(0, 1, p.N)
    a = gs.transport_sweep(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q),
                           _t(rho_in), _inflow(p))
    b = gs.transport_sweep(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q),
                           _t(rho_in), _inflow(p))
    assert bool((a["rho"] == b["rho"]).all()) and bool((a["F"] == b["F"]).all())


# (320, 300) and larger: no strip plan fits a cluster's shared memory, so
# the tiled solver runs over a cooperative grid of every SM; (513, 290) and
# (257, 600) have odd level sizes, ragged rectangles and sub-tiles
@pytest.mark.parametrize("seed,shape", [(11, (40, 37)), (12, (9, 70)), (13, (1, 5)), (14, (320, 300)),
                                        (15, (513, 290)), (16, (257, 600))])
def test_synthetic_step_parity(gs, seed, shape):
    p = W.random_problem(shape[0], shape[1], order=6, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    rho_m = rng.uniform(0.0, 2.0, p.N)
    sw = oracle.transport_sweep(p, rho_m)
    gx, gy = oracle.alsm_gradient(p, sw["rho"])
    hx, hy = oracle.high_order_terms(p, sw["Fx"], sw["Fy"], gx, gy)
    b = oracle.synthetic_rhs(p, sw["rho"], hx, hy, sw["fb"])
    rho_new = oracle.SyntheticSolver(p).solve(b)
    F = np.concatenate([sw["Fx"], sw["Fy"]])
    opt = gs.default_options(synth_rtol=1e-14, synth_max_iter=3000)
    r = gs.synthetic_step(p.dx, p.dy, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), _t(sw["rho"]), _t(F),
                          _t(sw["fb"]), None, opt)
    hot = r["hot"].cpu().numpy()
    N = p.N
    sh = max(np.abs(hx).max(), np.abs(hy).max())
    assert np.abs(hot[:N] - hx).max() / sh < 1e-12
    assert np.abs(hot[N:] - hy).max() / sh < 1e-12
    assert rel(r["rhs"].cpu().numpy(), b) < 1e-12
    assert rel(r["rho"].cpu().numpy(), rho_new) < TOL64
    assert r["synth_iters"] > 0


def _solve(gs, p, **kw):
    opt = gs.default_options(**kw)
    return gs.solve(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), _inflow(p), opt)


SOLVE_CASES = [
    ("random_40x37_S6", lambda: W.random_problem(40, 37, order=6, seed=21, ratio_range=(0.5, 0.99))),
    ("random_320x300_S4_grid_solver", lambda: W.random_problem(320, 300, order=4, seed=22, ratio_range=(0.5, 0.99))),
    ("uniform_64_S8", lambda: W.config_small()),
    ("channel_64_S8", lambda: W.channel_problem(64, 8, 2, width=2, sigma_bulk=200.0)),
]


@pytest.mark.parametrize("name,make", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
@pytest.mark.parametrize("scheme", ["si", "gsis"])
def test_solve_parity_fixed_iterations(gs, name, make, scheme):
    p = make()
    m = 6
    if scheme == "si":
        o = oracle.si_solve(p, fixed_iters=m)
        r = _solve(gs, p, scheme=gs.SCHEME_SI, fixed_iters=m, max_iter=m)
    else:
        o = oracle.gsis_solve(p, fixed_iters=m)
        r = _solve(gs, p, scheme=gs.SCHEME_GSIS, fixed_iters=m, max_iter=m, synth_rtol=1e-14,
                   synth_max_iter=3000)
    assert r["status"] == gs.GSIS_OK and r["iters"] == m
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < TOL64
    np.testing.assert_allclose(r["history"], o["history"], rtol=1e-8)
    N = p.N
    F = r["F"].cpu().numpy()
    P = r["P"].cpu().numpy()
    s = np.abs(o["rho"]).max()
    assert np.abs(F[:N] - o["Fx"]).max() / s < TOL64
    assert np.abs(P[:N] - o["Pxx"]).max() / s < TOL64
    assert np.abs(P[2 * N:] - o["Pyy"]).max() / s < TOL64


def test_gsis_pseudo_time_parity(gs):
    p = W.channel_problem(64, 8, 2, width=2)          # 2000 / 0.2 jump: needs beta
    m = 8
    o = oracle.gsis_solve(p, fixed_iters=m, beta=10.0)
    r = _solve(gs, p, fixed_iters=m, max_iter=m, beta=10.0, synth_rtol=1e-14, synth_max_iter=3000)
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < TOL64
    np.testing.assert_allclose(r["history"], o["history"], rtol=1e-7)


def test_si_pseudo_time_parity(gs):
    p = W.random_problem(30, 20, order=4, seed=31)
    o = oracle.si_solve(p, fixed_iters=5, cfl_p=0.5, beta=4.0)
    r = _solve(gs, p, scheme=gs.SCHEME_SI, fixed_iters=5, max_iter=5, cfl_p=0.5, beta=4.0)
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < TOL64


def test_fp32_gsis_pseudo_time_parity(gs):
    """FP32 sweeps over the per-ordinate source X = src + shift I^m with the
    diagonal sigma_t + shift as one FP32 array (FP64 synthetic solve), on the
    2000 / 0.2 opacity jump: eight iterations and the converged result
    against the FP64 oracle within the FP32 sweep tolerance."""
    p = W.channel_problem(64, 8, 2, width=2)
    m = 8
    o = oracle.gsis_solve(p, fixed_iters=m, beta=10.0)
    r = _solve(gs, p, precision=gs.FP32_SWEEP, fixed_iters=m, max_iter=m, beta=10.0, synth_rtol=1e-14,
               synth_max_iter=3000)
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < TOL32
    oc = oracle.gsis_solve(p, tol=1e-10, beta=10.0)
    rc = _solve(gs, p, precision=gs.FP32_SWEEP, tol=1e-7, beta=10.0, synth_rtol=1e-13, synth_max_iter=3000,
                stall_window=8)
    assert rel(rc["rho"].cpu().numpy(), oc["rho"]) < TOL32


def test_fp32_si_pseudo_time_parity(gs):
    p = W.random_problem(30, 20, order=4, seed=31)
    o = oracle.si_solve(p, fixed_iters=5, cfl_p=0.5, beta=4.0)
    r = _solve(gs, p, scheme=gs.SCHEME_SI, precision=gs.FP32_SWEEP, fixed_iters=5, max_iter=5, cfl_p=0.5,
               beta=4.0)
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < TOL32


@pytest.mark.parametrize("scheme", ["si", "gsis"])
def test_uniform_square_converged_parity(gs, scheme):
    """The 64x64 S8 workload to Err < 1e-8: same iteration count as the
    oracle and the same result."""
    p = W.config_small()
    if scheme == "si":
        o = oracle.si_solve(p, tol=1e-8)
        r = _solve(gs, p, scheme=gs.SCHEME_SI, tol=1e-8)
    else:
        o = oracle.gsis_solve(p, tol=1e-8)
        r = _solve(gs, p, tol=1e-8, synth_rtol=1e-14, synth_max_iter=3000)
    assert r["status"] == gs.GSIS_OK
    assert r["iters"] == o["iters"]
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < TOL64


def test_fp32_sweep_solve_error(gs):
    """FP32 sweeps with FP64 synthetic solve: energy density within 1e-5 of
    the FP64 oracle after convergence."""
    p = W.config_small()
    o = oracle.gsis_solve(p, tol=1e-10)
    r = _solve(gs, p, precision=gs.FP32_SWEEP, tol=1e-7, synth_rtol=1e-13, synth_max_iter=3000)
    assert r["status"] == gs.GSIS_OK
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < TOL32


@pytest.mark.parametrize("cap", [2, 5])
def test_capped_synthetic_solve_same_fixed_point(gs, cap):
    """Capping the synthetic solve at a few inner iterations per GSIS
    iteration (warm-started) changes the path, not the fixed point: the
    converged result matches the oracle's exactly-solved GSIS."""
    p = W.channel_problem(64, 8, 2, width=2)
    o = oracle.gsis_solve(p, tol=1e-12, beta=10.0)
    r = _solve(gs, p, tol=1e-12, beta=10.0, synth_rtol=1e-12, synth_max_iter=cap)
    assert r["status"] == gs.GSIS_OK
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < 1e-9


def test_channel_full_size_parity(gs):
    """256x256 S12 channel workload with the solver settings of the
    benchmark (GSIS, FP64, local pseudo-time beta = 10): three iterations
    against the oracle, then properties of the converged run."""
    p = W.config_channel()
    m = 3
    o = oracle.gsis_solve(p, fixed_iters=m, beta=10.0)
    r = _solve(gs, p, fixed_iters=m, max_iter=m, beta=10.0, synth_rtol=1e-14, synth_max_iter=3000)
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < TOL64


def test_channel_full_size_sweep_parity(gs):
    p = W.config_channel()
    rng = np.random.Generator(np.random.PCG64(23))
    rho_in = rng.uniform(0.0, 10.0, p.N)
    o = oracle.transport_sweep(p, rho_in)
    for prec, tol in ((gs.FP64, 1e-11), (gs.FP32_SWEEP, TOL32)):
        r = gs.transport_sweep(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q),
                               _t(rho_in), _inflow(p), gs.default_options(precision=prec))
        assert rel(r["rho"].cpu().numpy(), o["rho"]) < tol


def test_si_converged_energy_balance(gs):
    """Property at any size: at the SI fixed point absorption plus net
    outflow equals the source."""
    p = W.random_problem(50, 60, order=6, seed=41, ratio_range=(0.2, 0.9))
    r = _solve(gs, p, scheme=gs.SCHEME_SI, tol=1e-13)
    rho = r["rho"].cpu().numpy()
    sw = gs.transport_sweep(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q),
                            r["rho"], _inflow(p))
    fb = sw["bflux"].cpu().numpy()
    V = (p.dx[None, :] * p.dy[:, None]).ravel()
    A = np.concatenate([p.dy, p.dy, p.dx, p.dx])
    lhs = np.sum(V * p.sigma_a * rho) + np.sum(A * fb)
    assert abs(lhs - np.sum(V * p.q)) < 1e-10 * np.sum(V * p.q)


def test_negative_opacity_rejected_on_device(gs):
    p = W.random_problem(8, 8, order=4, seed=51)
    sa = p.sigma_a.copy()
    sa[5] = -1.0
    with pytest.raises(gs.GsisError) as ei:
        gs.solve(p.dx, p.dy, p.mu, p.eta, p.w, _t(sa), _t(p.sigma_s), _t(p.q), None,
                 gs.default_options(max_iter=3))
    assert ei.value.status == gs.GSIS_ERR_ARG


def test_maxiter_status(gs):
    p = W.config_small()
    r = _solve(gs, p, scheme=gs.SCHEME_SI, tol=1e-12, max_iter=5)
    assert r["status"] == gs.GSIS_ERR_MAXITER and r["iters"] == 5


def test_bounded_wait_reports_timeout_and_context_survives(gs):
    """A device wait bounded far below a sweep's duration gives up: with 8
    bands per ordinate the band above must wait for the band below's first
    results (31 steps away), so a 1 ns bound always runs out.  The call
    returns GSIS_ERR_DEVICE_TIMEOUT and the CUDA context stays usable."""
    p = W.random_problem(64, 256, order=8, seed=61)
    with pytest.raises(gs.GsisError) as ei:
        _solve(gs, p, scheme=gs.SCHEME_SI, fixed_iters=2, max_iter=2, wait_limit_s=1e-9)
    assert ei.value.status == gs.GSIS_ERR_DEVICE_TIMEOUT
    o = oracle.si_solve(p, fixed_iters=2)
    r = _solve(gs, p, scheme=gs.SCHEME_SI, fixed_iters=2, max_iter=2)
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < TOL64


def test_channel_converged_at_benchmark_settings(gs):
    """The 256x256 S12 channel at the benchmark's own solver settings (GSIS,
    FP64, local pseudo-time beta = 10, synthetic solve capped at 2
    warm-started inner iterations) against the oracle's GSIS with the
    synthetic system solved exactly, both converged: the cap changes the
    path, not the fixed point (Sec. 3.1, Eq. (GSIS_update); stopping on Err,
    Eq. (Err_W)).  Run to 1e-12 the two agree to 1e-9; the benchmark's own
    stop at Err < 1e-8 leaves the result within 1e-6 of it."""
    p = W.config_channel()
    o = oracle.gsis_solve(p, tol=1e-12, beta=10.0)
    assert o["converged"]
    tight = _solve(gs, p, tol=1e-12, beta=10.0, max_iter=5000, check_every=16, synth_max_iter=2)
    assert tight["status"] == gs.GSIS_OK
    assert rel(tight["rho"].cpu().numpy(), o["rho"]) < 1e-9
    bench = _solve(gs, p, tol=1e-8, beta=10.0, max_iter=5000, check_every=16, synth_max_iter=2)
    assert bench["status"] == gs.GSIS_OK
    assert rel(bench["rho"].cpu().numpy(), o["rho"]) < 1e-6
