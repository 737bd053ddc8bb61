"""GPU adjoint of a time-dependent GSIS run (gsis_td_adjoint) against the
oracle's step-by-step adjoint (oracle/td_adjoint.py) on the same seeded
inputs, its independence of the checkpoint interval, and central
differences of GPU forward runs at the full 1024^2 S16 workload size.

Tolerances (max norm relative to the largest component of each gradient):
FP64 sweeps, forward steps and adjoint iterations converged to 1e-13 with
an exact synthetic solve: 1e-8 against the oracle (the final state 1e-9).
FP32 sweeps (FP64 synthetic solve, material update and gradient terms),
steps and adjoint iterations to 1e-6: 2e-3.  Checkpoint intervals 1, 2 and
the whole run: bit-identical (the recomputation repeats the same kernels on
the same data).  Full size, FP64 sweeps, steps to 1e-10: the directional
derivative along a random perturbation of sigma_a equals the central
difference of two forward runs (h = 1e-4) within 1e-4."""
import numpy as np
import pytest

import workloads as W
from oracle import td_adjoint as OTA
from oracle import timedep as TD

pytestmark = pytest.mark.gpu

TOL64 = 1e-8
TOL32 = 2e-3


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
    a, b = np.asarray(a), np.asarray(b)
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


CASES = [
    # name, problem, time parameters, steps
    ("random_24x20_S4", lambda: W.random_problem(24, 20, order=4, seed=21, nonuniform=False,
                                                 log10_range=(-0.5, 1.0), ratio_range=(0.2, 0.8)),
     TD.TimeParams(dt=0.05, c=1.0, a=1.0, cv=0.7), 3),
    ("ragged_40x37_S6_vacuum", lambda: W.random_problem(40, 37, order=6, seed=22, nonuniform=False,
                                                        log10_range=(-0.5, 1.5), ratio_range=(0.3, 0.9),
                                                        with_inflow=False),
     TD.TimeParams(dt=0.5, c=2.0, a=0.5, cv=2.0), 2),
]


def _state(p, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.0, 0.5, p.N), rng.uniform(0.6, 1.4, p.N), rng.uniform(0.0, 1.0, p.N),
            rng.uniform(0.0, 1.0, p.N))


def _opts(gs, prec, tol):
    if prec == "fp64":
        return gs.default_options(tol=tol, synth_rtol=1e-14, synth_max_iter=3000, precision=gs.FP64, check_every=4)
    return gs.default_options(tol=tol, synth_rtol=1e-14, synth_max_iter=3000, precision=gs.FP32_SWEEP,
                              check_every=4, max_iter=400)


def _gpu(gs, p, tp, nsteps, rho0, T0, g_rho, g_T, opt, C=None, predictor=0):
    return gs.td_adjoint(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), _t(rho0), _t(T0),
                         tp.dt, nsteps, dJ_drho=_t(g_rho), dJ_dT=_t(g_T), checkpoint_every=C, c=tp.c, a=tp.a,
                         cv=tp.cv, inflow=None if p.inflow is None else _t(p.inflow.reshape(-1)), options=opt,
                         predictor=predictor)


@pytest.fixture(scope="module")
def oracle_results():
    out = {}
    for name, make, tp, nsteps in CASES:
        p = make()
        rho0, T0, g_rho, g_T = _state(p, 7)
        out[name] = OTA.gradient(p, tp, nsteps, rho0, T0, g_rho, g_T, tol=1e-13, adj_tol=1e-14)
    return out


@pytest.mark.parametrize("name,make,tp,nsteps", CASES, ids=[c[0] for c in CASES])
def test_gradient_matches_oracle_fp64(gs, oracle_results, name, make, tp, nsteps):
    p = make()
    rho0, T0, g_rho, g_T = _state(p, 7)
    o = oracle_results[name]
    r = _gpu(gs, p, tp, nsteps, rho0, T0, g_rho, g_T, _opts(gs, "fp64", 1e-13), C=2)
    assert r["status"] == gs.GSIS_OK
    assert _rel(r["rho"].cpu().numpy(), o["recs"][-1]["rho"]) < 1e-9
    assert _rel(r["T"].cpu().numpy(), o["recs"][-1]["T"]) < 1e-9
    for k in ("grad_sa", "grad_ss"):
        key = "grad_sigma_a" if k == "grad_sa" else "grad_sigma_s"
        assert _rel(r[key].cpu().numpy(), o[k]) < TOL64, k
    assert _rel(r["grad_rho0"].cpu().numpy(), o["grad_rho0"]) < TOL64
    assert _rel(r["grad_T0"].cpu().numpy(), o["grad_T0"]) < TOL64
    assert np.all(r["adj_iters"] > 0)


def test_gradient_fp32_sweeps(gs, oracle_results):
    name, make, tp, nsteps = CASES[0]
    p = make()
    rho0, T0, g_rho, g_T = _state(p, 7)
    o = oracle_results[name]
    r = _gpu(gs, p, tp, nsteps, rho0, T0, g_rho, g_T, _opts(gs, "fp32", 1e-6), C=2)
    assert r["status"] == gs.GSIS_OK
    assert _rel(r["grad_sigma_a"].cpu().numpy(), o["grad_sa"]) < TOL32
    assert _rel(r["grad_sigma_s"].cpu().numpy(), o["grad_ss"]) < TOL32
    assert _rel(r["grad_rho0"].cpu().numpy(), o["grad_rho0"]) < TOL32
    assert _rel(r["grad_T0"].cpu().numpy(), o["grad_T0"]) < TOL32


def test_checkpoint_interval_does_not_change_the_gradient(gs):
    name, make, tp, _ = CASES[0]
    p = make()
    rho0, T0, g_rho, g_T = _state(p, 8)
    opt = _opts(gs, "fp64", 1e-12)
    runs = [_gpu(gs, p, tp, 5, rho0, T0, g_rho, g_T, opt, C=C) for C in (1, 2, 5)]
    for r in runs[1:]:
        for k in ("grad_sigma_a", "grad_sigma_s", "grad_rho0", "grad_T0", "rho", "T"):
            assert np.array_equal(r[k].cpu().numpy(), runs[0][k].cpu().numpy()), k
        assert np.array_equal(r["adj_iters"], runs[0]["adj_iters"])


def test_predictor_run_gradient_matches_oracle_for_every_checkpoint_interval(gs, oracle_results):
    """The adjoint of a run whose steps start from the quadratic predictor:
    the checkpoints carry the predictor's history, so the recomputed steps
    repeat the forward run bit for bit whatever the interval, and the
    converged steps (hence the gradient) equal the oracle's, whose steps
    start from the previous one."""
    name, make, tp, nsteps = CASES[0]
    p = make()
    rho0, T0, g_rho, g_T = _state(p, 7)
    o = oracle_results[name]
    opt = _opts(gs, "fp64", 1e-13)
    runs = [_gpu(gs, p, tp, nsteps, rho0, T0, g_rho, g_T, opt, C=C, predictor=2) for C in (1, 2, nsteps)]
    r = runs[0]
    assert r["status"] == gs.GSIS_OK
    assert _rel(r["rho"].cpu().numpy(), o["recs"][-1]["rho"]) < 1e-9
    for k, key in (("grad_sa", "grad_sigma_a"), ("grad_ss", "grad_sigma_s"), ("grad_rho0", "grad_rho0"),
                   ("grad_T0", "grad_T0")):
        assert _rel(r[key].cpu().numpy(), o[k]) < TOL64, k
    for q in runs[1:]:
        for k in ("grad_sigma_a", "grad_sigma_s", "grad_rho0", "grad_T0", "rho", "T"):
            assert np.array_equal(q[k].cpu().numpy(), r[k].cpu().numpy()), k


def test_full_size_directional_derivative(gs):
    """1024^2 S16 channel, cold start, two steps of dt = 1e-3, FP64 sweeps:
    J = the sum of rho after the two steps over the channel cells next to
    the left wall."""
    import torch
    p = W.config_timedep()
    td = W.TIMEDEP
    tp = TD.TimeParams(dt=td["dt"], c=td["c"], a=td["a"], cv=td["cv"])
    nsteps = 2
    T0 = np.full(p.N, td["T0"])
    rho0 = td["a"] * td["c"] * T0 ** 4
    g_rho = np.zeros(p.N)
    mask = (p.sigma_a + p.sigma_s) < 1.0
    cols = np.arange(p.N) % p.nx
    g_rho[mask & (cols < 64)] = 1.0
    opt = gs.default_options(tol=1e-10, synth_rtol=1e-12, synth_max_iter=400, precision=gs.FP64, check_every=4)
    r = _gpu(gs, p, tp, nsteps, rho0, T0, g_rho, np.zeros(p.N), opt)
    assert r["status"] == gs.GSIS_OK
    ga = r["grad_sigma_a"].cpu().numpy()
    assert np.all(np.isfinite(ga)) and np.abs(ga).max() > 0
    rng = np.random.default_rng(9)
    delta = rng.uniform(0.0, 1.0, p.N) * p.sigma_a
    h = 1e-4
    Js = []
    for sgn in (1.0, -1.0):
        f = gs.td_solve(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a + sgn * h * delta), _t(p.sigma_s), _t(p.q),
                        _t(rho0), _t(T0), tp.dt, nsteps, c=tp.c, a=tp.a, cv=tp.cv,
                        inflow=_t(p.inflow.reshape(-1)), options=opt)
        assert f["status"] == gs.GSIS_OK
        Js.append(float(torch.dot(f["rho"], _t(g_rho)).item()))
    fd = (Js[0] - Js[1]) / (2 * h)
    ad = float(ga @ delta)
    assert abs(fd - ad) <= 1e-4 * abs(ad), (fd, ad)
    del r


def test_unconverged_forward_step_reports_maxiter(gs):
    """A forward step that cannot reach the tolerance within max_iter stops
    the call with GSIS_ERR_MAXITER (a status, not an exception)."""
    name, make, tp, _ = CASES[0]
    p = make()
    rho0, T0, g_rho, g_T = _state(p, 9)
    opt = gs.default_options(tol=1e-15, max_iter=2, check_every=1, synth_rtol=1e-14, synth_max_iter=3000,
                             precision=gs.FP64)
    r = _gpu(gs, p, tp, 2, rho0, T0, g_rho, g_T, opt, C=1)
    assert r["status"] == gs.GSIS_ERR_MAXITER
