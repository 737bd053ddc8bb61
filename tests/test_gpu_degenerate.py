"""GPU solves on the method's degenerate inputs against the oracle: a single
cell, one row of cells (one 32-row band with a single live row) and one
column (every band row one cell wide), by SI and GSIS, with and without the
local pseudo-time; and the zero problem (no source, vacuum walls): rho = 0
exactly, Err defined as 0, converged at the first iteration.

Tolerance: 1e-10 relative (max norm) in rho after four iterations (exact
synthetic solve), as for the other FP64 fixed-iteration parity tests."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W

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


CASES = [
    ("one_cell_S4", lambda: W.random_problem(1, 1, order=4, seed=71)),
    ("one_row_37x1_S6", lambda: W.random_problem(37, 1, order=6, seed=72)),
    ("one_column_1x45_S4", lambda: W.random_problem(1, 45, order=4, seed=73)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("scheme", ["si", "gsis"])
@pytest.mark.parametrize("beta", [0.0, 10.0])
def test_degenerate_meshes_match_oracle(gs, name, make, scheme, beta):
    p = make()
    m = 4
    ref = oracle.gsis_solve if scheme == "gsis" else oracle.si_solve
    o = ref(p, fixed_iters=m, beta=beta)
    opt = gs.default_options(scheme=gs.SCHEME_GSIS if scheme == "gsis" else gs.SCHEME_SI, fixed_iters=m,
                             max_iter=m, beta=beta, synth_rtol=1e-14, synth_max_iter=3000)
    r = gs.solve(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q),
                 _t(p.inflow.reshape(-1)), opt)
    assert r["status"] == gs.GSIS_OK and r["iters"] == m
    rho = r["rho"].cpu().numpy()
    assert np.abs(rho - o["rho"]).max() / np.abs(o["rho"]).max() < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_zero_problem(gs, prec):
    p = W.random_problem(20, 17, order=4, seed=74, with_inflow=False)
    p = dataclasses.replace(p, q=np.zeros(p.N))
    opt = gs.default_options(precision=gs.FP64 if prec == "fp64" else gs.FP32_SWEEP, beta=10.0)
    r = gs.solve(p.dx, p.dy, p.mu, p.eta, p.w, _t(p.sigma_a), _t(p.sigma_s), _t(p.q), None, opt)
    assert r["status"] == gs.GSIS_OK and r["iters"] == 1 and r["err"] == 0.0
    assert not r["rho"].any() and not r["F"].any()
