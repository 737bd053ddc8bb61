"""Batched solve (gsis_solve_batch, gsis_batch_autotune) through the C ABI.

Every problem of a batch goes through the iteration of the single-problem
gsis_solve, so with the synthetic solver on gsis_solve's cluster size
(synth_cells_per_cta = 0) its rho, F, iteration count and Err must equal the
single solve's bit for bit, whatever the sweep order and placement.  Other
cluster sizes change only the rounding order of the synthetic solve's sums:
those runs are checked against the FP64 oracle (1e-10 relative after a fixed
number of iterations with an exact synthetic solve, as the single-problem
parity tests)."""
import numpy as np
import pytest

import oracle
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


def _dev(p):
    return dict(dx=p.dx, dy=p.dy, mu=p.mu, eta=p.eta, w=p.w, sigma_a=_t(p.sigma_a), sigma_s=_t(p.sigma_s),
                q=_t(p.q), inflow=None if p.inflow is None else _t(p.inflow.reshape(-1)))


def _single(gs, d, opt):
    return gs.solve(d["dx"], d["dy"], d["mu"], d["eta"], d["w"], d["sigma_a"], d["sigma_s"], d["q"], d["inflow"],
                    opt, want_P=False)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _mixed():
    # uneven sizes and orders; ragged bands; problems too small for the strip
    # solver (their synthetic solve is launched on its own); one cell, one row,
    # one column; inflow on some, vacuum on others
    return [
        W.random_problem(16, 12, order=4, seed=1),
        W.random_problem(40, 33, order=6, seed=2, with_inflow=False),
        W.random_problem(7, 66, order=4, seed=3),
        W.random_problem(70, 45, order=8, seed=4),
        W.random_problem(33, 97, order=6, seed=5, nonuniform=False),
        W.random_problem(1, 1, order=4, seed=6),
        W.random_problem(37, 1, order=6, seed=7),     # one row
        W.random_problem(1, 45, order=4, seed=8),     # one column
        W.channel_problem(64, 8, 2, width=2, sigma_bulk=200.0),
    ]


def _opts(gs, prec="fp64", scheme="gsis", **kw):
    base = dict(scheme=gs.SCHEME_GSIS if scheme == "gsis" else gs.SCHEME_SI,
                precision=gs.FP64 if prec == "fp64" else gs.FP32_SWEEP, tol=1e-9, max_iter=3000,
                synth_rtol=1e-12, synth_max_iter=20, beta=10.0, check_every=4)
    base.update(kw)
    return gs.default_options(**base)


def _assert_same(gs, batch_res, singles):
    import torch
    for i, (b, s) in enumerate(zip(batch_res, singles)):
        assert b["status"] == s["status"], i
        assert b["iters"] == s["iters"], (i, b["iters"], s["iters"])
        assert b["err"] == s["err"], i
        assert torch.equal(b["rho"], s["rho"]), i
        assert torch.equal(b["F"], s["F"]), i


@pytest.mark.parametrize("prec,scheme", [("fp64", "gsis"), ("fp32", "gsis"), ("fp64", "si")])
def test_batch_equals_single_solves(gs, prec, scheme):
    probs = [_dev(p) for p in _mixed()]
    kw = {"tol": 1e-6, "stall_window": 4} if prec == "fp32" else {}
    if scheme == "si":
        kw = {"max_iter": 300}
    opt = _opts(gs, prec, scheme, **kw)
    singles = [_single(gs, d, opt) for d in probs]
    assert any(s["iters"] != singles[0]["iters"] for s in singles)   # problems stop at different iterations
    for order in (gs.ORDER_PROBLEM, gs.ORDER_BAND, gs.ORDER_LONGEST, gs.ORDER_BAND_LONGEST):
        for dyn in (0, 1):
            t = gs.default_batch_tuning(sweep_order=order, sweep_dynamic=dyn, synth_cells_per_cta=0)
            r = gs.solve_batch(probs, opt, tuning=t)
            _assert_same(gs, r["results"], singles)


@pytest.mark.parametrize("cells_per_cta", [64, 4096, 1 << 20])
def test_batch_cluster_sizes_oracle_parity(gs, cells_per_cta):
    """Strip solver on 16, mixed, or 2-CTA clusters (the groups run
    concurrently): six GSIS iterations with an exact synthetic solve against
    the oracle."""
    ps = _mixed()
    m = 6
    opt = _opts(gs, fixed_iters=m, max_iter=m, beta=0.0, synth_rtol=1e-14, synth_max_iter=3000)
    t = gs.default_batch_tuning(synth_cells_per_cta=cells_per_cta)
    r = gs.solve_batch([_dev(p) for p in ps], opt, tuning=t)
    assert r["status"] == gs.GSIS_OK
    for p, res in zip(ps, r["results"]):
        o = oracle.gsis_solve(p, fixed_iters=m)
        assert res["iters"] == m
        assert rel(res["rho"].cpu().numpy(), o["rho"]) < TOL64, p.name
        N = p.N
        assert np.abs(res["F"].cpu().numpy()[:N] - o["Fx"]).max() / np.abs(o["rho"]).max() < TOL64


def test_batch_si_pseudo_time_oracle_parity(gs):
    ps = [W.random_problem(30, 20, order=4, seed=31), W.random_problem(12, 41, order=6, seed=32)]
    opt = _opts(gs, scheme="si", fixed_iters=5, max_iter=5, cfl_p=0.5, beta=4.0)
    r = gs.solve_batch([_dev(p) for p in ps], opt)
    for p, res in zip(ps, r["results"]):
        o = oracle.si_solve(p, fixed_iters=5, cfl_p=0.5, beta=4.0)
        assert rel(res["rho"].cpu().numpy(), o["rho"]) < TOL64


def test_batch_per_problem_status(gs):
    """One problem that cannot reach the tolerance within max_iter stops with
    GSIS_ERR_MAXITER while the others converge; the call reports it."""
    slow = W.homogeneous(32, 32, 4, sigma_t=50.0, ratio=0.9999)
    fast = W.random_problem(20, 20, order=4, seed=8, ratio_range=(0.1, 0.3))
    probs = [_dev(fast), _dev(slow)]
    opt = _opts(gs, scheme="si", tol=1e-10, max_iter=40, beta=0.0)
    singles = [_single(gs, d, opt) for d in probs]
    r = gs.solve_batch(probs, opt)
    assert r["status"] == gs.GSIS_ERR_MAXITER
    assert [x["status"] for x in r["results"]] == [gs.GSIS_OK, gs.GSIS_ERR_MAXITER]
    _assert_same(gs, r["results"], singles)


def test_batch_rejects_bad_arguments(gs):
    p = _dev(W.random_problem(8, 8, order=4, seed=9))
    bad = dict(p, sigma_a=_t(-np.ones(64)))
    with pytest.raises(gs.GsisError) as e:
        gs.solve_batch([p, bad], _opts(gs, max_iter=3))
    assert e.value.status == gs.GSIS_ERR_ARG
    with pytest.raises(gs.GsisError) as e:
        gs.solve_batch([p], _opts(gs), tuning=gs.default_batch_tuning(sweep_order=7))
    assert e.value.status == gs.GSIS_ERR_ARG


def test_autotune_choice_is_remembered(gs):
    probs = [_dev(p) for p in _mixed()]
    opt = _opts(gs)
    a = gs.batch_autotune(probs, opt, trial_iters=2)
    t = a["tuning"]
    assert 0 <= t.sweep_order <= 3 and t.sweep_dynamic in (0, 1) and t.synth_cells_per_cta in (0, 4096, 16384)
    assert a["ms_per_iter"] > 0 and a["class_ms"]["sweep"] > 0 and a["class_ms"]["synth"] > 0
    r1 = gs.solve_batch(probs, opt)                # tuning=None: the remembered choice
    r2 = gs.solve_batch(probs, opt, tuning=t)
    _assert_same(gs, r1["results"], r2["results"])


def test_batch_workload_full_size(gs):
    """The 64-problem batch (sides 32-256, S8-S16, sigma_t in [1e-2, 1e4]) in
    its benchmark configuration (FP32 sweeps, GSIS with beta = 10, capped
    synthetic solve): every problem converges; sampled problems (the three
    smallest and three largest) equal their single-problem solves bit for
    bit, under the default tuning and under the autotuner's."""
    ps = W.config_batch()
    probs = [_dev(p) for p in ps]
    opt = _opts(gs, "fp32", tol=1e-6, synth_max_iter=2, stall_window=8, check_every=8)
    r = gs.solve_batch(probs, opt, tuning=gs.default_batch_tuning())
    assert r["status"] == gs.GSIS_OK, [x["status"] for x in r["results"]]
    order = np.argsort([p.N * p.K for p in ps])
    sample = list(order[:3]) + list(order[-3:])
    singles = [_single(gs, probs[i], opt) for i in sample]
    _assert_same(gs, [r["results"][i] for i in sample], singles)
    a = gs.batch_autotune(probs, opt, trial_iters=2, workspace=r["workspace"])
    if a["tuning"].synth_cells_per_cta == 0:
        r2 = gs.solve_batch(probs, opt, tuning=a["tuning"], workspace=r["workspace"])
        _assert_same(gs, [r2["results"][i] for i in sample], singles)
