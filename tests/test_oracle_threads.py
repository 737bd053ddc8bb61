"""The -fopenmp build of the oracle's C sweeps (only used to time the oracle
on all host cores) computes the same numbers as the plain build: the
ordinates are independent, and every moment and boundary-flux sum runs over
the ordinates in index order in both builds."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA
from oracle import gsis as G
from oracle import uw2 as OU


@pytest.fixture
def both():
    def run(fn):
        G.use_threads(False)
        a = fn()
        G.use_threads(True)
        try:
            b = fn()
        finally:
            G.use_threads(False)
        return a, b
    return run


def _same(a, b):
    if isinstance(a, dict):
        keys = [k for k in a if isinstance(a[k], np.ndarray)]
        assert keys
        for k in keys:
            assert np.array_equal(a[k], b[k]), k
    else:
        assert np.array_equal(a, b)


def test_threaded_build_uses_several_threads():
    G.use_threads(True)
    try:
        assert G.threads() >= 1
    finally:
        G.use_threads(False)
    assert G.threads() == 1


@pytest.mark.parametrize("beta", [0.0, 3.0])
def test_gsis_iterations_equal(both, beta):
    p = W.random_problem(40, 33, order=6, seed=5)
    _same(*both(lambda: G.gsis_solve(p, fixed_iters=4, beta=beta)))


def test_si_iterations_equal(both):
    p = W.random_problem(17, 29, order=4, seed=6, with_inflow=False)
    _same(*both(lambda: G.si_solve(p, fixed_iters=5)))


def test_transposed_sweep_equal(both):
    p = W.random_problem(21, 14, order=4, seed=7, nonuniform=False)
    psi = np.random.default_rng(8).standard_normal((p.K, p.N))
    _same(*both(lambda: OA.transposed_sweep(p, psi)))


def test_increment_sweep_equal(both):
    p = W.random_problem(19, 23, order=6, seed=9)
    R = np.random.default_rng(10).standard_normal((p.K, p.N))
    shift = np.random.default_rng(11).uniform(0.0, 2.0, p.N)
    _same(*both(lambda: OU.increment(p, R, shift)))
