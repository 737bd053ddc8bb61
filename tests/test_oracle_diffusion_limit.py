"""Asymptotic-preserving pin (Sec. 3.3 and Appendix A): with sigma_s = 1/eps,
sigma_a = 0, q = eps and vacuum walls, the transport solution tends to the
diffusion solution rho = 3 u(x, y), -Laplace(u) = 1, u = 0 on the walls.
GSIS on a fixed coarse mesh recovers it independently of eps, converging at
first order in the cell size; plain UW1 source iteration does not."""
import math

import numpy as np

import oracle
import workloads as W


def u_series(x, y, terms=199):
    """Double sine series of the unit-square Poisson problem -Laplace(u) = 1."""
    u = np.zeros_like(x)
    for m in range(1, terms + 1, 2):
        for n in range(1, terms + 1, 2):
            u += 16.0 / (math.pi ** 4 * m * n * (m * m + n * n)) * np.sin(m * math.pi * x) * np.sin(n * math.pi * y)
    return u


def _problem(n, eps, order=4):
    return W.homogeneous(n, n, order, 1.0 / eps, 1.0, eps)


def _exact(n):
    xc = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(xc, xc)
    return 3.0 * u_series(X, Y).ravel()


def test_gsis_recovers_diffusion_limit_first_order():
    errs = {}
    for n in (16, 32):
        ex = _exact(n)
        for eps in (1e-4, 1e-5):
            r = oracle.gsis_solve(_problem(n, eps), tol=1e-10, max_iter=2000)
            assert r["converged"] and r["iters"] < 60
            errs[(n, eps)] = np.abs(r["rho"] - ex).max() / ex.max()
    for n in (16, 32):
        assert abs(errs[(n, 1e-4)] - errs[(n, 1e-5)]) < 2e-3      # eps-independent
    ratio = errs[(16, 1e-4)] / errs[(32, 1e-4)]
    assert 1.8 < ratio < 2.2, errs                               # first order in dx
    assert errs[(32, 1e-4)] < 0.08


def test_uw1_source_iteration_misses_diffusion_limit():
    n, eps = 16, 1e-4
    ex = _exact(n)
    r = oracle.si_solve(_problem(n, eps), tol=1e-10, max_iter=400)
    assert not r["converged"]
    assert np.abs(r["rho"] - ex).max() / ex.max() > 0.5


def _gsis_with_half(p, **kw):
    last = {}
    r = oracle.gsis_solve(p, callback=lambda m, rho, sw, e: last.update(half=sw["rho"].copy()), **kw)
    return r, last.get("half")


def test_gsis_reaches_its_discrete_limit_at_first_order_in_eps():
    """On a fixed mesh the GSIS fixed point converges to a discrete limit as
    eps -> 0 at first order in eps, and becomes kinetically consistent
    (rho* - rho*_{1/2} = O(eps)), the asymptotic-preserving property of
    Sec. 3.3: differences shrink tenfold per decade of eps."""
    n = 16
    rho, gap = {}, {}
    for eps in (1e-4, 1e-5, 1e-6):
        r, half = _gsis_with_half(_problem(n, eps), tol=1e-10, max_iter=200)
        assert r["converged"]
        rho[eps] = r["rho"]
        gap[eps] = np.abs(r["rho"] - half).max() / np.abs(r["rho"]).max()
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    d1, d2 = rel(rho[1e-4], rho[1e-5]), rel(rho[1e-5], rho[1e-6])
    assert d1 < 1e-3 and 8.0 < d1 / d2 < 12.0
    assert gap[1e-4] < 5e-4 and 8.0 < gap[1e-4] / gap[1e-5] < 12.0 and 8.0 < gap[1e-5] / gap[1e-6] < 12.0


def test_diffusion_limit_does_not_depend_on_the_boundary_increment_coefficient(monkeypatch):
    """The synthetic boundary flux is the kinetic one plus beta (rho - rho_{1/2})
    (Eq. (macro_bc_delta_flux)); at the fixed point beta multiplies
    rho* - rho*_{1/2} = O(eps), so in the diffusion limit the result is the
    same with a different beta (a planted 1/2 for the 1/4), while dropping the
    1/4 (no outflow term in the synthetic boundary operator) makes the
    iteration diverge."""
    from oracle import gsis as G
    eps = 1e-6
    base = oracle.gsis_solve(_problem(16, eps), tol=1e-10, max_iter=200)["rho"]
    orig = G.boundary_beta
    monkeypatch.setattr(G, "boundary_beta", lambda s, d, n: orig(s, d, n) + 0.25)
    half = oracle.gsis_solve(_problem(16, eps), tol=1e-10, max_iter=200)
    assert half["converged"]
    assert np.abs(half["rho"] - base).max() / np.abs(base).max() < 2e-5
    monkeypatch.setattr(G, "boundary_beta", lambda s, d, n: orig(s, d, n) - 0.25)
    with np.errstate(all="ignore"):
        zero = oracle.gsis_solve(_problem(16, eps), tol=1e-10, max_iter=200)
    assert not zero["converged"]
