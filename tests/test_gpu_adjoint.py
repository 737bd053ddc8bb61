"""GPU adjoint (gsis_adjoint and the autograd wrapper) against the oracle's
adjoint gradient and against central differences of GPU forward solves.

Tolerances (max norm relative to the largest gradient component): FP64
transposed sweeps 1e-8 against the oracle; FP32 transposed sweeps (the
reduced-precision form, FP64 synthetic solve) 1e-3.  Central differences
with h = 1e-6 and 1e-4 relative: 1e-5 relative plus the noise of two forward
solves, 1e-13 |J| / h, plus 1e-8 of the largest component."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA

pytestmark = pytest.mark.gpu

TOL_ORACLE64 = 1e-8
TOL_ORACLE32 = 1e-3


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


def _opts(gs, prec="fp64", tol=1e-13):
    if prec == "fp64":
        return gs.default_options(tol=tol, synth_rtol=1e-14, synth_max_iter=3000, precision=gs.FP64)
    # FP32 sweeps: Err has a floor near 1e-7; stop there (stall window) instead of the FP64 tolerance
    return gs.default_options(tol=max(tol, 1e-6), synth_rtol=1e-14, synth_max_iter=3000, precision=gs.FP32_SWEEP,
                              max_iter=400, stall_window=4)


def _forward(gs, p, opt):
    r = gs.solve(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), _inflow(p), opt,
                 want_P=False)
    return r["rho"]


def _adjoint(gs, p, rho, g, opt):
    return gs.adjoint(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), rho, _t(g),
                      inflow=_inflow(p), options=opt)


def _small():
    # uniform mesh, heterogeneous opacities and sources, inflow on every wall
    return W.random_problem(16, 12, order=4, seed=11, nonuniform=False, log10_range=(0.0, 1.0),
                            ratio_range=(0.5, 0.9))


def _detector(p, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    g = np.zeros(p.N)
    g[rng.choice(p.N, n, replace=False)] = 1.0
    return g


def _rel(a, b):
    s = np.abs(b).max()
    return np.abs(np.asarray(a) - b).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_gradient_matches_oracle(gs, prec):
    p = _small()
    g = _detector(p, 5, 1)
    _, rho_o = OA.functional(p, g)
    ga_o, gs_o, info = OA.gradient(p, rho_o, g)
    opt = _opts(gs, prec)
    rho = _forward(gs, p, opt)
    out = _adjoint(gs, p, rho, g, opt)
    tol = TOL_ORACLE64 if prec == "fp64" else TOL_ORACLE32
    ea = _rel(out["grad_sigma_a"].cpu().numpy(), ga_o)
    es = _rel(out["grad_sigma_s"].cpu().numpy(), gs_o)
    assert ea < tol and es < tol, (ea, es)
    # the transposed iteration converges like GSIS
    if prec == "fp64":
        assert out["iters"] <= 3 * info["iters"] + 5


def test_adjoint_c3_central_differences_and_oracle(gs):
    # 64x64 uniform, S8, sigma_t = 10, ratio 0.99, q = 1, vacuum; J = sum of rho over
    # 16 seed-3 detector cells; central differences on 32 seed-3 cells
    p = W.config_small()
    g = _detector(p, 16, 3)
    rng = np.random.Generator(np.random.PCG64(3))
    fd_cells = rng.choice(p.N, 32, replace=False)
    opt = _opts(gs, "fp64", tol=1e-14)
    rho = _forward(gs, p, opt)
    out = _adjoint(gs, p, rho, g, opt)
    ga, gsg = out["grad_sigma_a"].cpu().numpy(), out["grad_sigma_s"].cpu().numpy()
    scale = max(np.abs(ga).max(), np.abs(gsg).max())

    def J(pp):
        return float(np.dot(g, _forward(gs, pp, opt).cpu().numpy()))

    J0 = J(p)
    # central differences: h = 1e-6 relative (the configuration's step), where the
    # noise of two solves accurate to ~1e-13 relative, 1e-13 |J| / h, dominates for
    # the small sigma_a = 0.1; and h = 1e-4 relative, where that noise is 100x
    # smaller and the O(h^2) truncation still ~1e-8 relative
    for c in fd_cells:
        for which, grad in (("sigma_a", ga), ("sigma_s", gsg)):
            base = getattr(p, which)
            for rel_h in (1e-6, 1e-4):
                h = rel_h * base[c]
                up, dn = base.copy(), base.copy()
                up[c] += h
                dn[c] -= h
                fd = (J(dataclasses.replace(p, **{which: up})) - J(dataclasses.replace(p, **{which: dn}))) / (2 * h)
                tol = 1e-5 * abs(fd) + 1e-13 * abs(J0) / h + 1e-8 * scale
                assert abs(fd - grad[c]) <= tol, (int(c), which, rel_h, fd, grad[c])
    # every cell against the oracle's adjoint gradient (FP64 and the FP32-sweep form)
    _, rho_o = OA.functional(p, g)
    ga_o, gs_o, _ = OA.gradient(p, rho_o, g)
    assert _rel(ga, ga_o) < TOL_ORACLE64 and _rel(gsg, gs_o) < TOL_ORACLE64
    opt32 = _opts(gs, "fp32")
    out32 = _adjoint(gs, p, _forward(gs, p, opt32), g, opt32)
    e32 = max(_rel(out32["grad_sigma_a"].cpu().numpy(), ga_o), _rel(out32["grad_sigma_s"].cpu().numpy(), gs_o))
    assert e32 < TOL_ORACLE32, e32


def test_autograd_function(gs):
    import torch
    p = _small()
    g = _detector(p, 5, 2)
    opt = _opts(gs, "fp64")
    sa = _t(p.sigma_a).requires_grad_(True)
    ss = _t(p.sigma_s).requires_grad_(True)
    rho = gs.solve_differentiable(p.dx, p.dy, p.mu, p.eta, p.w, sa, ss, _t(p.q), inflow=_inflow(p), options=opt)
    loss = torch.sum(rho * _t(g))
    loss.backward()
    out = _adjoint(gs, p, rho.detach(), g, opt)
    assert torch.equal(sa.grad, out["grad_sigma_a"]) and torch.equal(ss.grad, out["grad_sigma_s"])
    # a nonlinear functional: gradient of sum(rho^2) = adjoint with dJ/drho = 2 rho
    sa.grad = None
    ss.grad = None
    rho = gs.solve_differentiable(p.dx, p.dy, p.mu, p.eta, p.w, sa, ss, _t(p.q), inflow=_inflow(p), options=opt)
    torch.sum(rho * rho).backward()
    out2 = gs.adjoint(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), rho.detach(),
                      2.0 * rho.detach(), inflow=_inflow(p), options=opt)
    assert torch.equal(sa.grad, out2["grad_sigma_a"])


def test_adjoint_rejects_what_it_does_not_cover(gs):
    p = _small()
    g = _t(np.ones(p.N))
    rho = _t(np.ones(p.N))
    cases = [
        (dataclasses.replace(p, dx=W.random_problem(16, 12, order=4, seed=1).dx), _opts(gs)),   # non-uniform
        (p, gs.default_options(scheme=gs.SCHEME_SI)),
        (p, gs.default_options(beta=10.0)),
    ]
    for pp, opt in cases:
        with pytest.raises(gs.GsisError) as e:
            gs.adjoint(pp.dx, pp.dy, pp.mu, pp.eta, pp.w, _t(pp.sigma_a), _t(pp.sigma_s), _t(pp.q), rho, g,
                       inflow=_inflow(pp), options=opt)
        assert e.value.status == gs.GSIS_ERR_ARG
