"""GPU time-dependent radiation-material solve (gsis_td_solve) against the
FP64 oracle (oracle/timedep.py) on the same seeded inputs.

Tolerances: FP64, steps converged to 1e-13 with an exact synthetic solve:
1e-9 relative (max norm) in rho and T after several steps; the same
iteration count per step within one.  Fixed inner iterations per step:
1e-10.  FP32 sweeps (FP64 synthetic solve and material update), steps to
1e-6: 1e-5 relative in rho and T.  At the 1024^2 S16 size: a medium in
equilibrium with its walls stays there (1e-5 in FP32 sweeps)."""
import dataclasses
import math

import numpy as np
import pytest

import workloads as W
from oracle import timedep as TD

pytestmark = pytest.mark.gpu


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


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / np.abs(b).max()


def _solve(gs, p, tp, nsteps, rho0, T0, predictor=0, **kw):
    opt = gs.default_options(**kw)
    return gs.td_solve(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), _t(rho0), _t(T0),
                       tp.dt, nsteps, c=tp.c, a=tp.a, cv=tp.cv,
                       inflow=None if p.inflow is None else _t(p.inflow.reshape(-1)), options=opt,
                       predictor=predictor)


def _case(seed, nx=20, ny=16, order=4):
    p = W.random_problem(nx, ny, order=order, seed=seed, ratio_range=(0.2, 0.95))
    rng = np.random.Generator(np.random.PCG64(seed + 50))
    T0 = rng.uniform(0.4, 1.2, p.N)
    rho0 = T0 ** 4 * rng.uniform(0.5, 1.5, p.N)
    return p, rho0, T0


CASES = [
    ("random_20x16_S4", lambda: _case(1), TD.TimeParams(dt=0.05, c=1.0, a=1.0, cv=0.7)),
    ("random_33x40_S6_c3", lambda: _case(2, 33, 40, 6), TD.TimeParams(dt=0.2, c=3.0, a=0.5, cv=2.0)),
    ("channel_64_S4", lambda: (W.channel_td_problem(64, 4, base=64, width=2, sigma_bulk=200.0),
                               np.full(4096, 1e-4), np.full(4096, 0.1)), TD.TimeParams(dt=1e-3 * 16)),
]


@pytest.mark.parametrize("name,make,tp", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("scheme", ["gsis", "si"])
def test_converged_steps_match_oracle(gs, name, make, tp, scheme):
    p, rho0, T0 = make()
    nsteps = 3
    o = TD.run(p, tp, nsteps, rho0, T0, scheme=scheme, tol=1e-13)
    r = _solve(gs, p, tp, nsteps, rho0, T0, scheme=gs.SCHEME_GSIS if scheme == "gsis" else gs.SCHEME_SI,
               tol=1e-13, max_iter=5000, synth_rtol=1e-14, synth_max_iter=3000, check_every=8)
    assert r["status"] == gs.GSIS_OK
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < 1e-9
    assert rel(r["T"].cpu().numpy(), o["T"]) < 1e-9
    assert np.abs(r["step_iters"] - o["iters"]).max() <= 1


@pytest.mark.parametrize("scheme", ["gsis", "si"])
def test_predictor_reaches_the_same_steps_in_fewer_iterations(gs, scheme):
    """Steps started from a linear or quadratic extrapolation of the last
    steps' (rho, T) converge to the oracle's implicit solution (which starts
    every step from the previous one) and take no more iterations in all
    than starting from the previous step."""
    p = W.channel_td_problem(64, 4, base=64, width=2, sigma_bulk=200.0)
    rho0, T0 = np.full(p.N, 1e-4), np.full(p.N, 0.1)
    tp = TD.TimeParams(dt=1e-3 * 16)
    nsteps = 8
    o = TD.run(p, tp, nsteps, rho0, T0, scheme=scheme, tol=1e-13)
    kw = dict(scheme=gs.SCHEME_GSIS if scheme == "gsis" else gs.SCHEME_SI, tol=1e-13, max_iter=5000,
              synth_rtol=1e-14, synth_max_iter=3000, check_every=8)
    total = {}
    for pred in (0, 1, 2):
        r = _solve(gs, p, tp, nsteps, rho0, T0, predictor=pred, **kw)
        assert r["status"] == gs.GSIS_OK
        assert rel(r["rho"].cpu().numpy(), o["rho"]) < 1e-9, pred
        assert rel(r["T"].cpu().numpy(), o["T"]) < 1e-9, pred
        total[pred] = int(r["step_iters"].sum())
    assert abs(total[0] - int(o["iters"].sum())) <= nsteps
    assert total[1] <= total[0] and total[2] <= total[0], total


def test_fixed_inner_iterations_match_oracle(gs):
    """Three GSIS iterations per step, two steps: the iterates themselves
    (not only the converged steps) agree."""
    p, rho0, T0 = _case(3, 24, 18, 6)
    tp = TD.TimeParams(dt=0.1, c=1.0, a=1.0, cv=1.0)
    rho, T, I = rho0.copy(), T0.copy(), TD.isotropic(p, rho0)
    for _ in range(2):
        o = TD.gsis_time_step(p, tp, rho, T, I, fixed_iters=3)
        rho, T, I = o["rho"], o["T"], o["I"]
    r = _solve(gs, p, tp, 2, rho0, T0, fixed_iters=3, max_iter=3, synth_rtol=1e-14, synth_max_iter=3000)
    assert rel(r["rho"].cpu().numpy(), rho) < 1e-10
    assert rel(r["T"].cpu().numpy(), T) < 1e-10


@pytest.mark.parametrize("predictor", [0, 2])
def test_fp32_sweeps_match_oracle(gs, predictor):
    p, rho0, T0 = _case(4, 40, 30, 6)
    tp = TD.TimeParams(dt=0.05)
    o = TD.run(p, tp, 3, rho0, T0, scheme="gsis", tol=1e-12)
    r = _solve(gs, p, tp, 3, rho0, T0, predictor=predictor, precision=gs.FP32_SWEEP, tol=1e-6, max_iter=500,
               synth_rtol=1e-13, synth_max_iter=3000)
    assert r["status"] == gs.GSIS_OK
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < 1e-5
    assert rel(r["T"].cpu().numpy(), o["T"]) < 1e-5


def test_rejects_bad_arguments(gs):
    p, rho0, T0 = _case(5, 8, 8)
    tp = TD.TimeParams(dt=0.1)
    with pytest.raises(gs.GsisError) as e:
        _solve(gs, p, tp, 1, rho0, T0, beta=10.0)
    assert e.value.status == gs.GSIS_ERR_ARG
    with pytest.raises(gs.GsisError) as e:
        _solve(gs, p, TD.TimeParams(dt=-1.0), 1, rho0, T0)
    assert e.value.status == gs.GSIS_ERR_ARG
    bad = T0.copy()
    bad[3] = 0.0
    with pytest.raises(gs.GsisError) as e:
        _solve(gs, p, tp, 1, rho0, bad)
    assert e.value.status == gs.GSIS_ERR_ARG


def test_full_size_equilibrium_is_preserved(gs):
    """1024^2 S16 (the radiation-material workload's mesh and quadrature,
    FP32 sweeps): a medium at T = 0.5 with I = a c T^4/4pi and the same
    intensity entering through every wall stays in equilibrium."""
    p = W.config_timedep()
    T0 = 0.5
    eq = T0 ** 4 / (4 * math.pi)
    p = dataclasses.replace(p, inflow=np.full((p.n_bface, p.K), eq))
    r = _solve(gs, p, TD.TimeParams(dt=1e-3), 2, np.full(p.N, 4 * math.pi * eq), np.full(p.N, T0),
               precision=gs.FP32_SWEEP, tol=1e-6, max_iter=200, synth_max_iter=2)
    assert r["status"] == gs.GSIS_OK
    assert np.abs(r["rho"].cpu().numpy() / (4 * math.pi * eq) - 1).max() < 1e-5
    assert np.abs(r["T"].cpu().numpy() / T0 - 1).max() < 1e-5


@pytest.fixture(scope="module")
def full_size_first_step():
    """The oracle's first backward-Euler step of the headline workload
    (1024^2 S16, the x4 channel, cold start T = 0.1, dt = 1e-3) with two GSIS
    iterations (sparse LU of the synthetic system)."""
    from oracle import gsis as G
    p = W.config_timedep()
    td = W.TIMEDEP
    tp = TD.TimeParams(dt=td["dt"], c=td["c"], a=td["a"], cv=td["cv"])
    T0 = np.full(p.N, td["T0"])
    rho0 = td["a"] * td["c"] * T0 ** 4
    G.use_threads(True)   # the oracle's C sweeps on every host core (the same bits as one thread)
    try:
        o = TD.gsis_time_step(p, tp, rho0, T0, TD.isotropic(p, rho0), fixed_iters=2)
    finally:
        G.use_threads(False)
    return p, tp, rho0, T0, o


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_first_step_matches_oracle(gs, full_size_first_step, prec):
    """The headline workload itself: the first step's two GSIS iterations,
    synthetic system solved to 1e-14, against the oracle's: 1e-9 (FP64
    sweeps), 1e-5 (FP32 sweeps)."""
    p, tp, rho0, T0, o = full_size_first_step
    r = _solve(gs, p, tp, 1, rho0, T0, precision=gs.FP64 if prec == "fp64" else gs.FP32_SWEEP, fixed_iters=2,
               max_iter=2, synth_rtol=1e-14, synth_max_iter=3000)
    tol = 1e-9 if prec == "fp64" else 1e-5
    assert rel(r["rho"].cpu().numpy(), o["rho"]) < tol
    assert rel(r["T"].cpu().numpy(), o["T"]) < tol
