"""FP64 oracle of the adjoint (reverse-mode) derivative of a time-dependent
GSIS run (backward Euler, radiation-material coupling) with respect to the
per-cell opacities and the initial state.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy/scipy in
float64 on top of the time-dependent oracle (oracle/timedep.py) and the
steady adjoint's transposed steps (oracle/adjoint.py); the explicit
sigma-derivatives of the steady terms are taken by PyTorch CPU autograd of
the forward formulas (oracle/adjoint.py), a library primitive used as a step.

Step n (t^n -> t^{n+1}, Sec. 4.1, Eq. (RTE_d); Sec. 4.2, Eqs. (MSE_d),
(Tm_d)) maps the state x^n = (I^n, rho^n, T^n) to x^{n+1}.  The converged
GSIS step (oracle/timedep.gsis_time_step) is the fixed point y = (I^h, rho,
T) of
  R1_k = A_k I^h_k - s(rho, T) - I^n_k/(c dt)                       = 0,
         A_k = the first-order upwind operator with 1/(c dt) + sigma_t on
         the diagonal, s = (sigma_s rho + sigma_a phi(T) + q)/4pi,
  R2   = D_t rho - b(I^h; q + rho^n/(c dt)) - V sigma_a phi(T)       = 0,
         D_t = D_steady + diag(V/(c dt)), b the synthetic right-hand side
         with the HoT of the moments of I^h (Eqs. (GSIS_HoT), (Fij_d),
         (macro_bc_delta_flux)),
  R3   = C_v (T - T^n)/dt - sigma_a (rho - phi(T))                   = 0,
with phi = a c T^4, and x^{n+1} = (I^h + (rho - sum_k w_k I^h_k)/4pi, rho, T)
(Eq. (GSIS_update)).  (At the fixed point the Newton-eliminated synthetic
system of the forward iteration reduces to R2 with R3.)

For J = g_rho . rho^N + g_T . T^N the adjoint of step n, with multipliers
(phi_k, nu, tau) of (R1, R2, R3) and the adjoints (I', rho', T') of x^{n+1},
solves J_y^T (phi, nu, tau) = y_bar with
  y_bar_I,k = I'_k - w_k sum_j I'_j / 4pi,
  y_bar_rho = rho' + sum_j I'_j / 4pi,        y_bar_T = T';
eliminating tau (kappa = 4 a c T^3, D2 = C_v/dt + kappa sigma_a,
f = (C_v/dt)/D2) leaves
  A_k^T phi_k = y_bar_I,k + (db/dI^h_k)^T nu,
  D' nu = y_bar_rho + sigma_a y_bar_T / D2 + ((sigma_s + (1 - f) sigma_a)/4pi) sum_k phi_k,
  D' = D_steady + diag(V (1/(c dt) + f sigma_a - sigma_a))   (the forward's
       Newton-eliminated operator at the fixed point, symmetric),
  tau = (y_bar_T + (sigma_a kappa/4pi) sum_k phi_k + V sigma_a kappa nu) / D2,
solved here, like the steady adjoint, by the transposed GSIS iteration on
lam = D' nu.  The adjoints of x^n are I_bar_k = phi_k/(c dt),
rho_bar = V nu/(c dt), T_bar = tau C_v/dt, and the step adds to dJ/dsigma the
explicit derivative of -(phi, nu, tau).R at fixed (y, x^n):
  the steady terms of the kinetic and synthetic residuals (oracle/adjoint.py),
  + (phi(T)/4pi) sum_k phi_k + V nu phi(T) + tau (rho - phi(T))   (sigma_a only).
With I^0 = rho^0/4pi, dJ/drho^0 = rho_bar^0 + sum_k I_bar^0_k/4pi and
dJ/dT^0 = T_bar^0.  Every step follows this statement in this order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import adjoint as A
from . import gsis as G
from . import timedep as TD


def forward(prob, tp, nsteps, rho0, T0, tol=1e-13, max_iter=10000):
    """The GSIS run of oracle/timedep.run, keeping every step's fixed point:
    a list of dicts with the step's input (rho_n, T_n) and its I^h
    (= I^{n+1} - (rho - rho^{m+1/2})/4pi), rho^{m+1/2}, F, F_b, rho, T."""
    rho = np.array(rho0, dtype=np.float64)
    T = np.array(T0, dtype=np.float64)
    I = TD.isotropic(prob, rho)
    recs = []
    for n in range(nsteps):
        o = TD.gsis_time_step(prob, tp, rho, T, I, tol=tol, max_iter=max_iter)
        I_h = o["I"] - ((o["rho"] - o["rho_half"]) / (4.0 * math.pi))[None, :]
        recs.append(dict(rho_n=rho, T_n=T, I_h=I_h, rho_half=o["rho_half"], Fx=o["Fx"], Fy=o["Fy"], fb=o["fb"],
                         rho=o["rho"], T=o["T"], iters=o["iters"]))
        rho, T, I = o["rho"], o["T"], o["I"]
    return recs


def functional(prob, tp, nsteps, rho0, T0, g_rho, g_T, tol=1e-13):
    r = TD.run(prob, tp, nsteps, rho0, T0, scheme="gsis", tol=tol)
    return float(np.dot(g_rho, r["rho"]) + np.dot(g_T, r["T"]))


def step_operator(prob, tp, T):
    """kappa, D2, f and D' at the temperature T of a step's fixed point."""
    V = G.cell_volumes(prob)
    sa = prob.sigma_a
    kappa = 4.0 * tp.a * tp.c * T ** 3
    D2 = tp.cv / tp.dt + kappa * sa
    f = (tp.cv / tp.dt) / D2
    D = (G.synthetic_matrix(prob) + sp.diags(V * (1.0 / (tp.c * tp.dt) + f * sa - sa))).tocsc()
    return kappa, D2, f, D


def step_adjoint(prob, tp, rec, I_bar, rho_bar, T_bar, tol=1e-14, max_iter=2000):
    """Adjoint of one step at its fixed point rec, given the adjoints
    (I_bar [K, N], rho_bar, T_bar) of its output state.  Returns phi, nu,
    tau, the adjoint iteration count and the step's explicit gradient terms."""
    V = G.cell_volumes(prob)
    sa, ss = prob.sigma_a, prob.sigma_s
    inv_cdt = 1.0 / (tp.c * tp.dt)
    # adjoint of the output map x^{n+1}(y)
    sI = I_bar.sum(0)
    y_I = I_bar - prob.w[:, None] * (sI / (4.0 * math.pi))[None, :]
    y_rho = rho_bar + sI / (4.0 * math.pi)
    y_T = T_bar
    # the transposed step with T eliminated
    kappa, D2, f, D = step_operator(prob, tp, rec["T"])
    lu = spla.splu(D)
    sig_eff = ss + (1.0 - f) * sa
    c0 = y_rho + sa * y_T / D2
    p_shift = dataclasses.replace(prob, sigma_a=sa + inv_cdt)   # diagonal 1/(c dt) + sigma_t

    def transposed(lam):
        nu = lu.solve(lam)
        psi = A.moments_transpose(prob, *A.rhs_transpose(prob, nu)) + y_I
        phi = A.transposed_sweep(p_shift, psi)
        return nu, phi

    lam = c0.copy()
    it = 0
    for it in range(1, max_iter + 1):
        _, phi = transposed(lam)
        new = c0 + sig_eff * phi.sum(0) / (4.0 * math.pi)
        err = G.err_w(new, lam, V)
        lam = new
        if err < tol:
            break
    nu, phi = transposed(lam)
    sphi = phi.sum(0)
    tau = (y_T + sa * kappa * sphi / (4.0 * math.pi) + V * sa * kappa * nu) / D2
    # explicit sigma terms: the steady kinetic and synthetic ones at this
    # step's (I^h, rho^{m+1/2}, rho) ...
    import torch

    sw = dict(rho=rec["rho_half"], Fx=rec["Fx"], Fy=rec["Fy"], fb=rec["fb"], I=rec["I_h"])
    terms = A._torch_terms(prob, rec["rho"], sw, nu, phi)
    tsa = torch.tensor(sa, dtype=torch.float64, requires_grad=True)
    tss = torch.tensor(ss, dtype=torch.float64, requires_grad=True)
    L, _, _ = terms(tsa, tss)
    L.backward()
    g_sa = tsa.grad.numpy().copy()
    g_ss = tss.grad.numpy().copy()
    # ... plus the emission in the kinetic source and the synthetic balance,
    # and the material equation
    emis = tp.a * tp.c * rec["T"] ** 4
    g_sa += emis * sphi / (4.0 * math.pi) + V * nu * emis + tau * (rec["rho"] - emis)
    return dict(phi=phi, nu=nu, tau=tau, iters=it, grad_sa=g_sa, grad_ss=g_ss)


def gradient(prob, tp, nsteps, rho0, T0, g_rho, g_T, tol=1e-13, adj_tol=1e-14, recs=None):
    """dJ/dsigma_a, dJ/dsigma_s, dJ/drho^0, dJ/dT^0 of J = g_rho . rho^N +
    g_T . T^N by the adjoint of every step, last to first."""
    if recs is None:
        recs = forward(prob, tp, nsteps, rho0, T0, tol=tol)
    V = G.cell_volumes(prob)
    inv_cdt = 1.0 / (tp.c * tp.dt)
    I_bar = np.zeros((prob.K, prob.N))
    rho_bar = np.array(g_rho, dtype=np.float64)
    T_bar = np.array(g_T, dtype=np.float64)
    g_sa = np.zeros(prob.N)
    g_ss = np.zeros(prob.N)
    iters = []
    for rec in reversed(recs):
        a = step_adjoint(prob, tp, rec, I_bar, rho_bar, T_bar, tol=adj_tol)
        g_sa += a["grad_sa"]
        g_ss += a["grad_ss"]
        I_bar = a["phi"] * inv_cdt
        rho_bar = V * a["nu"] * inv_cdt
        T_bar = a["tau"] * tp.cv / tp.dt
        iters.append(a["iters"])
    g_rho0 = rho_bar + I_bar.sum(0) / (4.0 * math.pi)
    return dict(grad_sa=g_sa, grad_ss=g_ss, grad_rho0=g_rho0, grad_T0=T_bar, adj_iters=iters[::-1], recs=recs)
