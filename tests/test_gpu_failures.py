"""Failure detection on the GPU, each case made on the host side and
faulting nothing: an iteration that diverges, one that stalls, and (in the
time-dependent solve) steps that stall at the FP32 floor.  Every call returns
its status code and the CUDA context keeps working.

* Divergence: Sec. 6.2.2 states that the steady synthetic iteration without
  pseudo-time is unstable at a strong opacity jump.  On the 64^2 thick / thin
  channel (bulk sigma_t 2000, channel 0.2) the oracle's rho grows ~3.5x per
  iteration; the FP32 inner synthetic solve leaves its range after ~70
  iterations, the solver then stops and poisons its solution, and Err(rho)
  turns non-finite: GSIS_ERR_DIVERGED.
* Stall: FP32 sweeps cannot reach Err < 1e-15 (their floor is near 1e-8);
  with a stall window the solve ends with GSIS_ERR_STALLED at that floor.
"""
import numpy as np
import pytest

import oracle
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


def _solve(gs, p, **kw):
    return gs.solve(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q),
                    None if p.inflow is None else _t(p.inflow.reshape(-1)), gs.default_options(**kw))


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _context_still_works(gs):
    p = W.random_problem(20, 17, order=4, seed=5)
    r = _solve(gs, p, fixed_iters=3, max_iter=3, synth_rtol=1e-14, synth_max_iter=3000)
    assert _rel(r["rho"].cpu().numpy(), oracle.gsis_solve(p, fixed_iters=3)["rho"]) < 1e-10


@pytest.mark.parametrize("cap", [0, 2])
def test_unstable_gsis_reports_diverged(gs, cap):
    p = W.channel_problem(64, 4, 2, width=2)
    kw = {"synth_max_iter": cap} if cap else {"synth_rtol": 1e-12, "synth_max_iter": 3000}
    r = _solve(gs, p, tol=1e-8, max_iter=1000, check_every=8, **kw)
    assert r["status"] == gs.GSIS_ERR_DIVERGED
    assert r["iters"] < 400
    assert not np.isfinite(r["err"]) or r["err"] > 1e6
    _context_still_works(gs)


def test_steady_channel_without_pseudo_time_reports_diverged(gs):
    """The 256^2 S12 channel workload at its benchmark settings (synthetic
    solve capped at 2 inner iterations) but without the local pseudo-time it
    needs (reading R14): an oscillating mode grows until the solve reports
    GSIS_ERR_DIVERGED (~70 iterations)."""
    p = W.config_channel()
    r = _solve(gs, p, tol=1e-8, max_iter=2000, check_every=16, synth_max_iter=2)
    assert r["status"] == gs.GSIS_ERR_DIVERGED
    assert r["iters"] < 500
    _context_still_works(gs)


def test_fp32_floor_reports_stalled(gs):
    p = W.config_small()
    r = _solve(gs, p, precision=gs.FP32_SWEEP, tol=1e-15, max_iter=3000, check_every=4, stall_window=5,
               synth_rtol=1e-13, synth_max_iter=3000)
    assert r["status"] == gs.GSIS_ERR_STALLED
    assert r["iters"] < 3000
    assert 1e-13 < r["err"] < 1e-6
    # the stalled iterate is still the FP32 form of the converged answer
    assert _rel(r["rho"].cpu().numpy(), oracle.gsis_solve(p, tol=1e-10)["rho"]) < 1e-5
    _context_still_works(gs)


def test_time_dependent_steps_stall_at_fp32_floor_and_run_goes_on(gs):
    p = W.random_problem(30, 26, order=4, seed=8, ratio_range=(0.2, 0.95))
    rng = np.random.Generator(np.random.PCG64(58))
    T0 = rng.uniform(0.4, 1.2, p.N)
    rho0 = T0 ** 4
    tp = TD.TimeParams(dt=0.05)
    nsteps = 3
    o = TD.run(p, tp, nsteps, rho0, T0, scheme="gsis", tol=1e-12)
    opt = gs.default_options(precision=gs.FP32_SWEEP, tol=1e-15, max_iter=2000, check_every=2, stall_window=4,
                             synth_rtol=1e-13, synth_max_iter=3000)
    r = gs.td_solve(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), _t(rho0), _t(T0), tp.dt,
                    nsteps, inflow=_t(p.inflow.reshape(-1)), options=opt)
    assert r["status"] == gs.GSIS_ERR_STALLED
    assert (r["step_iters"] > 0).all() and (r["step_iters"] < 2000).all()   # every step ran, each ended
    assert np.isfinite(r["step_err"]).all() and r["step_err"].max() < 1e-6
    assert _rel(r["rho"].cpu().numpy(), o["rho"]) < 1e-5
    assert _rel(r["T"].cpu().numpy(), o["T"]) < 1e-5
    _context_still_works(gs)


def test_grid_barrier_timeout_reports_and_next_call_recovers(gs):
    """The synthetic solve over the whole grid (a 513 x 290 mesh: more cells
    than one cluster holds) with its barrier waits bounded at 1 ns: CTAs that
    arrive before the last one give up, the call reports
    GSIS_ERR_DEVICE_TIMEOUT, and the next call (whose status reset clears the
    barrier word) gives the oracle's answer."""
    p = W.random_problem(513, 290, order=4, seed=71)
    rng = np.random.Generator(np.random.PCG64(71))
    rho_m = rng.uniform(0.0, 2.0, p.N)
    sw = oracle.transport_sweep(p, rho_m)
    gx, gy = oracle.alsm_gradient(p, sw["rho"])
    hx, hy = oracle.high_order_terms(p, sw["Fx"], sw["Fy"], gx, gy)
    b = oracle.synthetic_rhs(p, sw["rho"], hx, hy, sw["fb"])
    rho_new = oracle.SyntheticSolver(p).solve(b)
    F = np.concatenate([sw["Fx"], sw["Fy"]])
    args = (p.dx, p.dy, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), _t(sw["rho"]), _t(F), _t(sw["fb"]), None)
    with pytest.raises(gs.GsisError) as ei:
        gs.synthetic_step(*args, gs.default_options(synth_rtol=1e-14, synth_max_iter=3000, wait_limit_s=1e-9))
    assert ei.value.status == gs.GSIS_ERR_DEVICE_TIMEOUT
    for _ in range(2):
        r = gs.synthetic_step(*args, gs.default_options(synth_rtol=1e-14, synth_max_iter=3000))
        assert _rel(r["rho"].cpu().numpy(), rho_new) < 1e-10
