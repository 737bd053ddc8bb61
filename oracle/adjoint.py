"""FP64 oracle of the adjoint (reverse-mode) derivative of the GSIS solution
with respect to the per-cell opacities sigma_a, sigma_s.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): plain numpy/scipy in
float64, the transposed sweep is the plain C loop in sweep.c, and the
explicit sigma-derivatives are taken by PyTorch CPU autograd of the same
formulas the forward oracle evaluates (a library primitive used as one step).

The converged steady GSIS solution rho* (Sec. 3.1) solves, together with the
intensities I_k of the kinetic step taken at rho*,

    A_k(sigma) I_k = s(sigma, rho*),  s = (sigma_s rho + q)/4pi   (Eqs. (RTE_d), (RTE_SI))
    D(sigma) rho*  = b(sigma; rho_1/2, F, F_b)                     (Eqs. (MSE_d1), (Fij_d),
                                                                   (macro_bc_delta_flux))

with (rho_1/2, F, F_b) the moments and boundary flux of the I_k (Eqs.
(def_rho), (def_F)).  For a functional J = g . rho* the Lagrangian

    L = g.rho + sum_k phi_k . (s - A_k I_k) + nu . (b - D rho)

is stationary in (I, rho) exactly when

    A_k^T phi_k = psi_k(nu) = (db/dI_k)^T nu,
    D nu = g + (sigma_s / 4pi) sum_k phi_k,

and then dJ/dsigma = dL/dsigma taken at fixed (I, rho*, phi, nu).  With
lam = D nu the second equation reads lam = M^T lam + g, M the linear part of
one GSIS iteration (D symmetric): the adjoint is the transposed GSIS
iteration and converges at the same rate.  Functions follow these steps in
this order; no step is blocked, fused or reordered.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import gsis as G

def _clib():
    return G._clib()


def transposed_sweep(prob, psi):
    """phi_k = A_k^{-T} psi_k for every ordinate (psi, phi: [K, N])."""
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    assert psi.shape == (prob.K, prob.N)
    phi = np.zeros_like(psi)
    c = np.ascontiguousarray
    _clib().oracle_sweep_transposed(prob.nx, prob.ny, G._ptr(c(prob.dx)), G._ptr(c(prob.dy)), prob.K,
                                    G._ptr(c(prob.mu)), G._ptr(c(prob.eta)), G._ptr(c(prob.sigma_t)),
                                    G._ptr(psi), G._ptr(phi))
    return phi


def forward_intensities(prob, rho):
    """I_k = A_k^{-1} s(rho) for every ordinate (the kinetic step at rho), plus
    its moments and boundary flux."""
    return G.transport_sweep(prob, rho, keep_intensity=True)


def alsm_transpose(prob, hx, hy):
    """Transpose of the (linear) ALSM gradient operator of gsis.alsm_gradient:
    G_i = P_i sum_j d_ij (U_j - U_i) with P_i the pseudo-inverse of the 2x2
    normal matrix, so L^T h puts +(P_i d_ij).h_i on U_j and -(P_i d_ij).h_i
    on U_i for every ordered neighbour pair (i, j)."""
    sig = prob.sigma_t
    g = G.geometry(prob)
    N = prob.N
    M = np.zeros((N, 2, 2))
    pairs = []
    for (i, j, rl, rr) in ((g.a, g.b, g.rL, g.rR), (g.b, g.a, g.rR, g.rL)):
        d = -rl + (sig[j] / sig[i])[:, None] * rr
        np.add.at(M, i, d[:, :, None] * d[:, None, :])
        pairs.append((i, j, d))
    Pinv = np.linalg.pinv(M)
    h = np.stack([hx, hy], 1)
    u = np.zeros(N)
    for (i, j, d) in pairs:
        pd = np.einsum("nij,nj->ni", Pinv[i], d)      # P_i d_ij
        t = np.sum(pd * h[i], 1)
        np.add.at(u, j, t)
        np.add.at(u, i, -t)
    return u


def rhs_transpose(prob, nu):
    """(db/d(rho_1/2, F_x, F_y, F_b))^T nu for the right-hand side of
    gsis.synthetic_rhs with HoT = F + grad(rho_1/2)/(3 sigma_t)."""
    g = G.geometry(prob)
    N = prob.N
    # face fluxes: b_a -= A (HoT_a + HoT_b)/2 . n, b_b += the same
    w = g.A * 0.5 * (nu[g.b] - nu[g.a])
    hx = np.zeros(N)
    hy = np.zeros(N)
    for c in (g.a, g.b):
        np.add.at(hx, c, w * g.n[:, 0])
        np.add.at(hy, c, w * g.n[:, 1])
    # boundary: b_c -= A (F_b - beta rho_1/2_c)
    beta = G.boundary_beta(prob.sigma_t[g.bc], g.bd, g.bn)
    fbb = np.zeros(prob.n_bface)
    fbb[g.bf] = -g.bA * nu[g.bc]
    rb = np.zeros(N)
    np.add.at(rb, g.bc, g.bA * beta * nu[g.bc])
    # HoT = F + G(rho_1/2)/(3 sigma_t)
    s3 = 3.0 * prob.sigma_t
    rb += alsm_transpose(prob, hx / s3, hy / s3)
    return rb, hx.copy(), hy.copy(), fbb


def moments_transpose(prob, rb, Fxb, Fyb, fbb):
    """psi_k = (d(rho_1/2, F, F_b)/dI_k)^T (rb, Fxb, Fyb, fbb): the moments give
    w_k (rb + mu_k Fxb + eta_k Fyb); an outgoing boundary face f of cell c
    (Omega_k . n_f >= 0, the forward sweep's convention) adds w_k (Omega_k.n_f) fbb_f."""
    K, N = prob.K, prob.N
    g = G.geometry(prob)
    psi = prob.w[:, None] * (rb[None, :] + prob.mu[:, None] * Fxb[None, :] + prob.eta[:, None] * Fyb[None, :])
    on = prob.mu[:, None] * g.bn[None, :, 0] + prob.eta[:, None] * g.bn[None, :, 1]   # [K, nbf]
    add = np.where(on >= 0.0, prob.w[:, None] * on * fbb[None, g.bf], 0.0)
    for k in range(K):
        np.add.at(psi[k], g.bc, add[k])
    return psi


def map_transpose(prob, lam, solver):
    """M^T lam = (sigma_s/4pi) sum_k A_k^{-T} psi_k(D^{-1} lam); returns it with nu, phi."""
    nu = solver.solve(lam)
    rb, Fxb, Fyb, fbb = rhs_transpose(prob, nu)
    phi = transposed_sweep(prob, moments_transpose(prob, rb, Fxb, Fyb, fbb))
    return prob.sigma_s * phi.sum(0) / (4.0 * math.pi), nu, phi


def map_linear(prob, drho, solver):
    """M drho: one GSIS iteration (gsis.gsis_iteration) with q = 0 and vacuum
    walls, i.e. the linear part of the affine iteration map."""
    p0 = dataclasses.replace(prob, q=np.zeros(prob.N), inflow=None)
    rho_new, _ = G.gsis_iteration(p0, drho, solver)
    return rho_new


def adjoint_solve(prob, g, tol=1e-14, max_iter=2000, solver=None):
    """lam = M^T lam + g by fixed-point iteration from lam = g, stopped when
    Err(lam) (Eq. (Err_W) applied to lam) < tol; returns lam, nu = D^{-1} lam,
    phi = the transposed sweeps at nu, and the iteration count."""
    solver = solver or G.SyntheticSolver(prob)
    V = G.cell_volumes(prob)
    lam = np.array(g, dtype=np.float64)
    for it in range(1, max_iter + 1):
        mt, _, _ = map_transpose(prob, lam, solver)
        new = g + mt
        err = G.err_w(new, lam, V)
        lam = new
        if err < tol:
            break
    _, nu, phi = map_transpose(prob, lam, solver)
    return lam, nu, phi, it


# ---------------------------------------------------------------- explicit sigma terms (torch, CPU, float64)

def _torch_terms(prob, rho_star, sw, nu, phi):
    """The explicit part of the Lagrangian as a differentiable function of
    (sigma_a, sigma_s), written with the forward oracle's formulas."""
    import torch

    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64)
    g = G.geometry(prob)
    V = T(G.cell_volumes(prob))
    q = T(prob.q)
    rho = T(rho_star)
    rho_h, Fx, Fy, fb = T(sw["rho"]), T(sw["Fx"]), T(sw["Fy"]), T(sw["fb"])
    I = T(sw["I"])
    phi_t, nu_t = T(phi), T(nu)
    a, b_, n, A = torch.as_tensor(g.a), torch.as_tensor(g.b), T(g.n), T(g.A)
    rL, rR = T(g.rL), T(g.rR)
    bc, bn, bA, bd, bf = torch.as_tensor(g.bc), T(g.bn), T(g.bA), T(g.bd), torch.as_tensor(g.bf)

    def terms(sa, ss):
        st = sa + ss
        # kinetic residual s - A_k I_k: only sigma_t on the diagonal depends on sigma
        s = (ss * rho + q) / (4.0 * math.pi)
        kin = torch.sum(phi_t * (s[None, :] - st[None, :] * I))
        # ALSM gradient (gsis.alsm_gradient) and HoT (gsis.high_order_terms)
        M = torch.zeros((prob.N, 2, 2), dtype=torch.float64)
        rhs = torch.zeros((prob.N, 2), dtype=torch.float64)
        for (i, j, rl, rr) in ((a, b_, rL, rR), (b_, a, rR, rL)):
            d = -rl + (st[j] / st[i])[:, None] * rr
            M = M.index_add(0, i, d[:, :, None] * d[:, None, :])
            rhs = rhs.index_add(0, i, d * (rho_h[j] - rho_h[i])[:, None])
        Gr = torch.einsum("nij,nj->ni", torch.linalg.pinv(M), rhs)
        hx = Fx + Gr[:, 0] / (3.0 * st)
        hy = Fy + Gr[:, 1] / (3.0 * st)
        # right-hand side (gsis.synthetic_rhs)
        bvec = V * q
        flux = A * 0.5 * ((hx[a] + hx[b_]) * n[:, 0] + (hy[a] + hy[b_]) * n[:, 1])
        bvec = bvec.index_add(0, a, -flux).index_add(0, b_, flux)
        beta = torch.sum(bd * bn, -1) / (3.0 * st[bc] * torch.sum(bd * bd, -1)) + 0.25
        bvec = bvec.index_add(0, bc, -bA * (fb[bf] - beta * rho_h[bc]))
        # D rho* (gsis.synthetic_matrix)
        vv = st[a][:, None] * rL - st[b_][:, None] * rR
        gam = A * (-torch.sum(vv * n, -1) / (3.0 * torch.sum(vv * vv, -1)))
        diag = V * sa
        diag = diag.index_add(0, a, gam).index_add(0, b_, gam).index_add(0, bc, bA * beta)
        Drho = diag * rho
        Drho = Drho.index_add(0, a, -gam * rho[b_]).index_add(0, b_, -gam * rho[a])
        syn = torch.sum(nu_t * (bvec - Drho))
        return kin + syn, bvec, Drho

    return terms


def gradient(prob, rho_star, g, tol=1e-14, max_iter=2000):
    """dJ/dsigma_a, dJ/dsigma_s of J = g . rho* at the converged GSIS solution
    rho* (steady, no pseudo-time): adjoint solve, then the explicit derivative
    of the Lagrangian.  Returns (grad_sa, grad_ss, info)."""
    import torch

    solver = G.SyntheticSolver(prob)
    sw = forward_intensities(prob, rho_star)
    lam, nu, phi, iters = adjoint_solve(prob, g, tol=tol, max_iter=max_iter, solver=solver)
    terms = _torch_terms(prob, rho_star, sw, nu, phi)
    sa = torch.tensor(prob.sigma_a, dtype=torch.float64, requires_grad=True)
    ss = torch.tensor(prob.sigma_s, dtype=torch.float64, requires_grad=True)
    L, _, _ = terms(sa, ss)
    L.backward()
    return sa.grad.numpy().copy(), ss.grad.numpy().copy(), {"lam": lam, "nu": nu, "phi": phi, "iters": iters,
                                                              "I": sw["I"]}


def functional(prob, g, tol=1e-14, max_iter=10000):
    """J = g . rho* with rho* the oracle's converged GSIS solution."""
    r = G.gsis_solve(prob, tol=tol, max_iter=max_iter)
    return float(np.dot(g, r["rho"])), r["rho"]
