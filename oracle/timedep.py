"""FP64 oracle of the time-dependent gray radiation-material problem
(backward Euler in time) on the 2D Cartesian mesh, by source iteration with
the Fleck-Cummings linearisation and by GSIS with the coupled rho-T
synthetic system.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy/scipy in
float64 on top of the steady oracle's kinetic step (oracle/gsis.py,
oracle/sweep.c) and synthetic operator.

Problem (Sec. 2.1, Eqs. (RTE_g), (Tm_g)): emission phi = a c T^4,
  (1/c) dI/dt + Omega.grad I = sigma_a (phi/4pi - I) + sigma_s (rho/4pi - I) + q/4pi,
  C_v dT/dt = sigma_a (rho - phi).
Backward Euler from t^n to t^{n+1} = t^n + dt (Sec. 4.1, Eq. (RTE_d)).

Kinetic step of inner iteration m (Eqs. (RTE_g_semi), (RTE_d_res)), the
exact first-order upwind solve of
  (1/(c dt) + sigma_t) I^{m+1/2} + upwind = S + I^n/(c dt),
with the shift 1/(c dt) on the diagonal and the stored I^n on the right.

SI (Sec. 2.2, Eqs. (Tm_semi_linear), (RTE_SI), (arti_sigmaT), (SI_update)):
Fleck-Cummings linearisation about T^n, kappa = 4 a c (T^n)^3, Fleck factor
f = (C_v/dt) / (C_v/dt + kappa sigma_a), mu = 1 - f:
  S = ((sigma_s + mu sigma_a) rho^m + f sigma_a phi^n + q) / 4pi,
  rho^{m+1} = rho^{m+1/2};  at the end of the step
  phi^{n+1} = (1 - f) rho^{n+1} + f phi^n,
  T^{n+1} = (phi^{n+1} + 3 phi^n) / kappa   (phi = kappa T - 3 phi^n).

GSIS (Sec. 3.1, Eqs. (GSIS_HoT), (GSIS_dse), (GSIS_update); Sec. 4.2,
Eqs. (MSE_d), (Tm_d), (MSE_d1), (MSE_d2), (elem_mtx_M)):
  S = (sigma_s rho^m + sigma_a phi(T^m) + q) / 4pi;  sweep -> rho^{m+1/2},
  F^{m+1/2}, boundary flux;  HoT as in the steady scheme;
  the macroscopic system
    V (rho - rho^n)/(c dt) + sum_faces A F.n = V [sigma_a (phi(T) - rho) + q],
    C_v (T - T^n)/dt = sigma_a (rho - phi(T)),
  one Newton step about T^m per GSIS iteration, with T eliminated cell by
  cell: kappa_m = 4 a c (T^m)^3, D2 = C_v/dt + kappa_m sigma_a,
  f_m = (C_v/dt)/D2, and
    [D_steady + diag(V (1/(c dt) + f_m sigma_a - sigma_a))] rho^{m+1}
        = b_steady with q -> q + rho^n/(c dt) + f_m sigma_a (phi^m + kappa_m (T^n - T^m)),
    T^{m+1} = T^n + sigma_a (rho^{m+1} - phi^m + kappa_m (T^m - T^n)) / D2,
    I^{m+1} = I^{m+1/2} + (rho^{m+1} - rho^{m+1/2}) / 4pi.
  At the fixed point the linearisation is exact: the step's result is the
  fully implicit discrete solution (Eqs. (RTE_d), (MSE_d), (Tm_d)).

Readings:
  * the printed mu = a c T^3 dt sigma_a / (C_v + a c T^3 dt sigma_a) lacks
    the factor 4 that Eq. (Tm_semi_linear) gives; the derivation is followed
    (mu = 1 - f with kappa = 4 a c T^3);
  * the GSIS macroscopic system keeps the rho-T coupling in the Newton step
    (T eliminated into the diagonal) rather than the paper's block-Jacobi
    sub-iteration (Eqs. (MSE_d1), (MSE_d2) without the coupling term); both
    converge to the solution of Eqs. (MSE_d), (Tm_d);
  * the diffusion coefficient of the synthetic equation is 1/(3 sigma_t)
    with the plain sigma_t (Eqs. (GSIS_HoT), (GSIS_dse));
  * no pseudo-time in the time-dependent form (the paper switches it off
    except in one steady test);
  * the initial intensity is isotropic, I^0 = rho^0 / 4pi.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import gsis as G


@dataclasses.dataclass(frozen=True)
class TimeParams:
    dt: float           # time step
    c: float = 1.0      # speed of light
    a: float = 1.0      # radiation constant
    cv: float = 1.0     # volumetric heat capacity C_v


def emission(T, tp: TimeParams):
    """phi = a c T^4."""
    return tp.a * tp.c * np.asarray(T, dtype=np.float64) ** 4


def kinetic_step(prob, tp: TimeParams, rho, source_q, I_n):
    """(1/(c dt) + sigma_t) I + upwind = (sigma_s rho + source_q)/4pi + I^n/(c dt):
    the steady kinetic step with the diagonal shift 1/(c dt) and the stored
    intensity I^n ([K, N]) on the right-hand side."""
    p = dataclasses.replace(prob, q=np.asarray(source_q, dtype=np.float64))
    shift = np.full(prob.N, 1.0 / (tp.c * tp.dt))
    return G.transport_sweep(p, rho, keep_intensity=True, shift=shift, I_prev=I_n)


def isotropic(prob, rho):
    return np.repeat((np.asarray(rho, dtype=np.float64) / (4.0 * math.pi))[None, :], prob.K, axis=0)


def si_time_step(prob, tp: TimeParams, rho_n, T_n, I_n, tol=1e-8, max_iter=100000):
    """One backward-Euler step by SI with the Fleck-Cummings linearisation."""
    V = G.cell_volumes(prob)
    sa = prob.sigma_a
    kappa = 4.0 * tp.a * tp.c * T_n ** 3
    f = (tp.cv / tp.dt) / (tp.cv / tp.dt + kappa * sa)
    mu = 1.0 - f
    phi_n = emission(T_n, tp)
    rho = rho_n.copy()
    hist = []
    for m in range(max_iter):
        sw = kinetic_step(prob, tp, rho, mu * sa * rho + f * sa * phi_n + prob.q, I_n)
        new = sw["rho"]
        e = G.err_w(new, rho, V)
        hist.append(e)
        rho = new.copy()
        if e < tol or not np.isfinite(e):
            break
    phi = (1.0 - f) * rho + f * phi_n
    T = (phi + 3.0 * phi_n) / kappa
    return dict(rho=rho, T=T, I=sw["I"], fb=sw["fb"], Fx=sw["Fx"], Fy=sw["Fy"], iters=len(hist),
                history=np.array(hist))


def gsis_time_step(prob, tp: TimeParams, rho_n, T_n, I_n, tol=1e-8, max_iter=10000, fixed_iters=0):
    """One backward-Euler step by GSIS with the Newton-eliminated rho-T
    synthetic system (one Newton step per GSIS iteration)."""
    V = G.cell_volumes(prob)
    sa = prob.sigma_a
    D0 = G.synthetic_matrix(prob)
    rho, T = rho_n.copy(), T_n.copy()
    hist = []
    n = fixed_iters if fixed_iters else max_iter
    for m in range(n):
        phi = emission(T, tp)
        sw = kinetic_step(prob, tp, rho, sa * phi + prob.q, I_n)
        gx, gy = G.alsm_gradient(prob, sw["rho"])
        hx, hy = G.high_order_terms(prob, sw["Fx"], sw["Fy"], gx, gy)
        kappa = 4.0 * tp.a * tp.c * T ** 3
        D2 = tp.cv / tp.dt + kappa * sa
        f = (tp.cv / tp.dt) / D2
        q_eff = prob.q + rho_n / (tp.c * tp.dt) + f * sa * (phi + kappa * (T_n - T))
        b = G.synthetic_rhs(dataclasses.replace(prob, q=q_eff), sw["rho"], hx, hy, sw["fb"])
        D = (D0 + sp.diags(V * (1.0 / (tp.c * tp.dt) + f * sa - sa))).tocsc()
        rho_new = spla.spsolve(D, b)
        T_new = T_n + sa * (rho_new - phi + kappa * (T - T_n)) / D2
        I_new = sw["I"] + ((rho_new - sw["rho"]) / (4.0 * math.pi))[None, :]
        e = G.err_w(rho_new, rho, V)
        hist.append(e)
        rho, T = rho_new, T_new
        if (not fixed_iters and e < tol) or not np.isfinite(e):
            break
    return dict(rho=rho, T=T, I=I_new, fb=sw["fb"], Fx=sw["Fx"], Fy=sw["Fy"], rho_half=sw["rho"],
                iters=len(hist), history=np.array(hist))


def run(prob, tp: TimeParams, nsteps, rho0, T0, scheme="gsis", tol=1e-8, max_iter=10000, callback=None):
    """nsteps backward-Euler steps from rho^0, T^0 (I^0 = rho^0/4pi); returns the
    final state and each step's inner iteration count."""
    rho = np.array(rho0, dtype=np.float64)
    T = np.array(T0, dtype=np.float64)
    I = isotropic(prob, rho)
    iters = []
    step = gsis_time_step if scheme == "gsis" else si_time_step
    out = None
    for n in range(nsteps):
        out = step(prob, tp, rho, T, I, tol=tol, max_iter=max_iter)
        rho, T, I = out["rho"], out["T"], out["I"]
        iters.append(out["iters"])
        if callback is not None:
            callback(n, out)
    return dict(rho=rho, T=T, I=I, iters=np.array(iters), last=out)
