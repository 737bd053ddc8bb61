"""FP64 oracle of the second-order upwind (UW2) kinetic step in the paper's
delta form, and of SI / GSIS built on it (steady).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  numpy on top of the
steady oracle (oracle/gsis.py) and the plain C increment solve
`oracle_sweep_delta` (oracle/sweep.c).

Kinetic step (Sec. 4.1):
  * per ordinate k, the cell gradient of I^m_k by the adaptive least-squares
    method (Sec. 5.2, Eqs. (shifted_j), (new_vector), (LSF_mdf); interior
    neighbours only, as for rho);
  * the Barth-Jespersen limiter psi_i,k: with U_max / U_min the extremes of
    I^m over the cell and its face neighbours and Delta_f = grad I . (x_f - x_i)
    the unlimited change to face f, psi = min over the four faces of
    min(1, (U_max - I_i)/Delta_f) (Delta_f > 0), min(1, (U_min - I_i)/Delta_f)
    (Delta_f < 0), 1 (Delta_f = 0);
  * face values I_i + psi grad I . (x_f - x_i) (Eq. (Ii,k)), taken from the
    upwind side (Eq. (Iij)); incoming boundary faces take the inflow;
  * residual per unit volume (Eq. (RTE_d_res), steady):
    r = S - sigma_t I_i - (1/V) sum_f A_f (Omega.n_f) I_f,  S = (sigma_s rho^m + q)/4pi;
  * increment: the first-order upwind system with the (pseudo-time shifted)
    diagonal (Eqs. (RTE_d_increment), (delta_Iij), (RTE_d_mtx),
    (elem_main_shifted)), dI = 0 on inflow faces; I^{m+1/2} = I^m + dI;
  * moments of I^{m+1/2}; the boundary kinetic flux uses the reconstructed
    outgoing face values of I^{m+1/2} (Sec. 4.4, Eq. (micro_bc)).
SI: rho^{m+1} = rho^{m+1/2}.  GSIS: the steady synthetic step of
oracle/gsis.py, then I^{m+1} = I^{m+1/2} + (rho^{m+1} - rho^{m+1/2})/4pi
(Eq. (GSIS_update)).  Initial I^0 = 0, rho^0 = 0.

Readings: the gradient of I uses the same adaptive
least squares as rho; the limiter's neighbourhood is the interior face
neighbours; incoming boundary faces take the prescribed inflow (no
reconstruction); psi is applied to both gradient components.  Besides the
paper's Barth-Jespersen limiter, "none" (unlimited reconstruction) and
"zero" (first order) are offered: the limiter's non-smooth switching at
smooth extrema slows the iteration markedly in the diffusion limit.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import gsis as G

def _clib():
    return G._clib()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Stencil:
    """Per-cell data of the gradient and reconstruction (built once)."""

    def __init__(self, prob, adaptive=True):
        nx, ny = prob.nx, prob.ny
        N = prob.N
        sig = prob.sigma_t
        g = G.geometry(prob)
        M = np.zeros((N, 2, 2))
        self.pairs = []   # (i, j, d): rows of the least-squares system of cell i
        for (i, j, rl, rr) in ((g.a, g.b, g.rL, g.rR), (g.b, g.a, g.rR, g.rL)):
            ratio = sig[j] / sig[i] if adaptive else np.ones(i.size)
            d = -rl + ratio[:, None] * rr
            np.add.at(M, i, d[:, :, None] * d[:, None, :])
            self.pairs.append((i, j, d))
        self.Minv = np.linalg.pinv(M)
        jj, ii = np.divmod(np.arange(N), nx)
        self.hx = prob.dx[ii]
        self.hy = prob.dy[jj]
        # face neighbours W E S N (-1 outside)
        self.nb = np.stack([np.where(ii > 0, np.arange(N) - 1, -1), np.where(ii < nx - 1, np.arange(N) + 1, -1),
                            np.where(jj > 0, np.arange(N) - nx, -1), np.where(jj < ny - 1, np.arange(N) + nx, -1)])
        self.ii, self.jj = ii, jj


def limited_gradient(prob, U, st: Stencil, limiter="bj"):
    """Limited gradient (psi grad U) of every row of U ([K, N] or [N]):
    limiter "bj" (Barth-Jespersen, the paper's), "none" (psi = 1) or "zero"
    (psi = 0: first-order upwind)."""
    U = np.atleast_2d(U)
    rhs = np.zeros(U.shape + (2,))
    for (i, j, d) in st.pairs:
        np.add.at(rhs, (slice(None), i), d[None, :, :] * (U[:, j] - U[:, i])[:, :, None])
    grad = np.einsum("nij,knj->kni", st.Minv, rhs)
    gx, gy = grad[..., 0], grad[..., 1]
    if limiter == "zero":
        return 0.0 * gx, 0.0 * gy
    if limiter == "none":
        return gx, gy
    Umax = U.copy()
    Umin = U.copy()
    for f in range(4):
        nb = st.nb[f]
        ok = nb >= 0
        Umax[:, ok] = np.maximum(Umax[:, ok], U[:, nb[ok]])
        Umin[:, ok] = np.minimum(Umin[:, ok], U[:, nb[ok]])
    psi = np.ones_like(U)
    for delta in (-0.5 * st.hx * gx, 0.5 * st.hx * gx, -0.5 * st.hy * gy, 0.5 * st.hy * gy):   # W E S N
        with np.errstate(divide="ignore", invalid="ignore"):
            phi = np.where(delta > 0, np.minimum(1.0, (Umax - U) / delta),
                           np.where(delta < 0, np.minimum(1.0, (Umin - U) / delta), 1.0))
        psi = np.minimum(psi, phi)
    return psi * gx, psi * gy


def face_values(prob, U, st: Stencil, limiter="bj"):
    """Reconstructed values of every cell at its W, E, S, N faces ([4, K, N])."""
    U = np.atleast_2d(U)
    lx, ly = limited_gradient(prob, U, st, limiter)
    return np.stack([U - 0.5 * st.hx * lx, U + 0.5 * st.hx * lx, U - 0.5 * st.hy * ly, U + 0.5 * st.hy * ly])


def residual(prob, S, I, st: Stencil, limiter="bj"):
    """UW2 residual per unit volume, [K, N]; S is [N] (isotropic) or [K, N]."""
    K, N = prob.K, prob.N
    nx, ny = prob.nx, prob.ny
    fv = face_values(prob, I, st, limiter)
    S = np.broadcast_to(np.asarray(S, dtype=np.float64), (K, N))
    r = S - prob.sigma_t[None, :] * I
    inflow = prob.inflow
    ii, jj = st.ii, st.jj
    # boundary face index of each cell's W E S N face (when on the boundary)
    bf = [jj, ny + jj, 2 * ny + ii, 2 * ny + nx + ii]
    opp = [1, 0, 3, 2]
    for f, (h, sgn) in enumerate(((st.hx, -1.0), (st.hx, 1.0), (st.hy, -1.0), (st.hy, 1.0))):
        for k in range(K):
            on = sgn * (prob.mu[k] if f < 2 else prob.eta[k])
            nb = st.nb[f]
            if on >= 0.0:
                val = fv[f, k]
            else:
                val = np.where(nb >= 0, fv[opp[f], k, np.maximum(nb, 0)],
                               inflow[bf[f], k] if inflow is not None else 0.0)
            r[k] -= on / h * val
    return r


def boundary_flux(prob, I, st: Stencil, limiter="bj"):
    """sum_k w_k (Omega_k . n) I_face,k on every boundary face: reconstructed
    outgoing values, inflow on incoming ones."""
    nx, ny = prob.nx, prob.ny
    fv = face_values(prob, I, st, limiter)
    fb = np.zeros(prob.n_bface)
    for k in range(prob.K):
        for f in range(prob.n_bface):
            if f < ny: c, on, side = nx * f, -prob.mu[k], 0
            elif f < 2 * ny: c, on, side = nx - 1 + nx * (f - ny), prob.mu[k], 1
            elif f < 2 * ny + nx: c, on, side = f - 2 * ny, -prob.eta[k], 2
            else: c, on, side = (f - 2 * ny - nx) + nx * (ny - 1), prob.eta[k], 3
            val = fv[side, k, c] if on >= 0.0 else (prob.inflow[f, k] if prob.inflow is not None else 0.0)
            fb[f] += prob.w[k] * on * val
    return fb


def increment(prob, R, shift=None):
    """dI of the first-order upwind increment system (oracle_sweep_delta)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    dI = np.zeros_like(R)
    sh = None if shift is None else np.ascontiguousarray(shift, dtype=np.float64)
    _clib().oracle_sweep_delta(prob.nx, prob.ny, _ptr(np.ascontiguousarray(prob.dx)),
                               _ptr(np.ascontiguousarray(prob.dy)), prob.K, _ptr(np.ascontiguousarray(prob.mu)),
                               _ptr(np.ascontiguousarray(prob.eta)), _ptr(np.ascontiguousarray(prob.sigma_t)),
                               _ptr(sh), _ptr(R), _ptr(dI))
    return dI


def kinetic_step(prob, rho, I_m, st: Stencil, shift=None, limiter="bj", S=None):
    """One UW2 kinetic step from I^m with source S = (sigma_s rho + q)/4pi
    (or the given S, [N] or [K, N]); returns the moments of I^{m+1/2}, the
    boundary flux and I^{m+1/2}."""
    if S is None:
        S = G.angular_source(prob, rho)
    R = residual(prob, S, I_m, st, limiter)
    I = I_m + increment(prob, R, shift)
    w = prob.w[:, None]
    out = {"I": I, "R": R,
           "rho": np.sum(w * I, 0), "Fx": np.sum(w * prob.mu[:, None] * I, 0),
           "Fy": np.sum(w * prob.eta[:, None] * I, 0),
           "Pxx": np.sum(w * (prob.mu ** 2)[:, None] * I, 0), "Pxy": np.sum(w * (prob.mu * prob.eta)[:, None] * I, 0),
           "Pyy": np.sum(w * (prob.eta ** 2)[:, None] * I, 0),
           "fb": boundary_flux(prob, I, st, limiter)}
    return out


def solve(prob, scheme="gsis", tol=1e-8, max_iter=10000, fixed_iters=0, cfl_p=0.0, beta=0.0, limiter="bj"):
    """SI or GSIS with the UW2 kinetic step, from rho^0 = 0, I^0 = 0."""
    st = Stencil(prob)
    V = G.cell_volumes(prob)
    shift = G.pseudo_time_shift(prob, cfl_p, beta) if (cfl_p > 0.0 or beta > 0.0) else None
    solver = G.SyntheticSolver(prob) if scheme == "gsis" else None
    rho = np.zeros(prob.N)
    I = np.zeros((prob.K, prob.N))
    hist = []
    n = fixed_iters if fixed_iters else max_iter
    sw = None
    converged = False
    for m in range(n):
        sw = kinetic_step(prob, rho, I, st, shift, limiter)
        if scheme == "gsis":
            gx, gy = G.alsm_gradient(prob, sw["rho"])
            hx, hy = G.high_order_terms(prob, sw["Fx"], sw["Fy"], gx, gy)
            b = G.synthetic_rhs(prob, sw["rho"], hx, hy, sw["fb"])
            new = solver.solve(b)
            I = sw["I"] + ((new - sw["rho"]) / (4.0 * math.pi))[None, :]
        else:
            new = sw["rho"].copy()
            I = sw["I"]
        e = G.err_w(new, rho, V)
        hist.append(e)
        rho = new
        if not fixed_iters and e < tol:
            converged = True
            break
        if not np.isfinite(e):
            break
    out = G._finish(prob, rho, sw, scheme)
    out.update(iters=len(hist), err=hist[-1], history=np.array(hist), converged=converged, I=I)
    return out
