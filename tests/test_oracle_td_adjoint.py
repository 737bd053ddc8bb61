"""Pins of the time-dependent adjoint oracle (oracle/td_adjoint.py): the
gradient of J = g_rho . rho^N + g_T . T^N with respect to sigma_a, sigma_s
(per cell) and the initial state rho^0, T^0 equals central finite
differences of full forward runs of the time-dependent oracle (h = 1e-6
relative, every step converged to Err < 1e-13).  The problems are far from
radiative equilibrium (T^0 in [0.6, 1.4], rho^0 in [0, 0.5]) so that every
term of the step adjoint (kinetic, synthetic, material coupling, the carry
between steps) carries weight, on non-uniform meshes with heterogeneous
opacities and wall inflow or vacuum."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import td_adjoint as TA
from oracle import timedep as TD

CASES = [
    # (seed, order, time parameters, steps, inflow)
    (11, 4, TD.TimeParams(dt=0.05, c=1.0, a=1.0, cv=0.7), 3, True),
    (12, 6, TD.TimeParams(dt=0.5, c=2.0, a=0.5, cv=2.0), 2, False),
]


def _case(seed, order, with_inflow):
    p = W.random_problem(5, 4, order=order, seed=seed, log10_range=(-0.5, 1.0), ratio_range=(0.2, 0.8),
                         with_inflow=with_inflow)
    rng = np.random.default_rng(seed + 50)
    rho0 = rng.uniform(0.0, 0.5, p.N)
    T0 = rng.uniform(0.6, 1.4, p.N)
    g_rho = rng.uniform(0.0, 1.0, p.N)
    g_T = rng.uniform(0.0, 1.0, p.N)
    return p, rho0, T0, g_rho, g_T


@pytest.mark.parametrize("seed,order,tp,nsteps,inflow", CASES)
def test_gradient_matches_central_differences(seed, order, tp, nsteps, inflow):
    p, rho0, T0, g_rho, g_T = _case(seed, order, inflow)
    g = TA.gradient(p, tp, nsteps, rho0, T0, g_rho, g_T)

    def J(pp=p, r0=rho0, t0=T0):
        return TA.functional(pp, tp, nsteps, r0, t0, g_rho, g_T)

    cells = [0, 9, p.N - 1]
    for name, key in (("sigma_a", "grad_sa"), ("sigma_s", "grad_ss")):
        v = getattr(p, name)
        scale = np.abs(g[key]).max()
        for c in cells:
            h = 1e-6 * v[c]
            vp, vm = v.copy(), v.copy()
            vp[c] += h
            vm[c] -= h
            fd = (J(dataclasses.replace(p, **{name: vp})) - J(dataclasses.replace(p, **{name: vm}))) / (2 * h)
            assert abs(fd - g[key][c]) <= 2e-6 * scale, (name, c, fd, g[key][c])
    for arg, key, arr in (("r0", "grad_rho0", rho0), ("t0", "grad_T0", T0)):
        scale = np.abs(g[key]).max()
        for c in cells:
            h = 1e-6 * max(abs(arr[c]), 0.1)
            ap, am = arr.copy(), arr.copy()
            ap[c] += h
            am[c] -= h
            fd = (J(**{arg: ap}) - J(**{arg: am})) / (2 * h)
            assert abs(fd - g[key][c]) <= 2e-6 * scale, (key, c, fd, g[key][c])


def test_single_step_zero_target_gives_zero_gradient():
    """J = 0 (g = 0): every adjoint and gradient vanishes exactly."""
    p, rho0, T0, _, _ = _case(13, 4, True)
    tp = TD.TimeParams(dt=0.1)
    z = np.zeros(p.N)
    g = TA.gradient(p, tp, 1, rho0, T0, z, z)
    for k in ("grad_sa", "grad_ss", "grad_rho0", "grad_T0"):
        assert np.all(g[k] == 0.0)
