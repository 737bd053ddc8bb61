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
