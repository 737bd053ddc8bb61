"""FP64 oracle of source iteration (SI) and the general synthetic iterative
scheme (GSIS) for the steady gray RTE on a 2D Cartesian finite-volume mesh.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy/scipy in
float64; the transport sweep is the plain C loop in sweep.c.  Every step
follows the paper's statement of it, in the paper's order:

  SI   (Sec. 2.2, Eqs. (RTE_SI), (SI_update)):
       S = (sigma_s rho^m + q)/4pi; sweep -> rho^{m+1/2}; rho^{m+1} = rho^{m+1/2}.
  GSIS (Sec. 3.1, Eqs. (GSIS_HoT), (GSIS_M0), (dse_iter), (GSIS_update);
        Sec. 4.2, Eqs. (MSE_d), (Fij_d), (Gamma_ij_def), (elem_mtx_M);
        Sec. 4.4, Eqs. (macro_bc_delta_flux), (macro_bc_delta_flux2);
        Sec. 5, Eqs. (shifted_j), (new_vector), (LSF_mdf), (Gamma_ij_com2)):
       sweep -> rho^{m+1/2}, F^{m+1/2}, boundary flux F_iw^init;
       g = ALSM gradient of rho^{m+1/2};  HoT = F^{m+1/2} + g/(3 sigma_t);
       solve the finite-volume synthetic equation for rho^{m+1}.
  Err  (Sec. 6, Eq. (Err_W)).

Readings where the paper is silent or ambiguous:
  * steady state: 1/(c dt) = 0, hatted cross sections equal the plain ones;
  * diffusion part of the face flux is the compact two-point flux
    Gamma_ij (rho_i - rho_j) (Eq. (Gamma_ij_def)), which Appendix A states is
    the central-difference scheme for cell centres; the high-order part is the
    face average of cell-centred HoT (Eq. (Fij_d));
  * boundary flux of the synthetic equation = kinetic flux of the last sweep
    plus [ (x_iw - x_i)/(3 sigma_t |x_iw - x_i|^2) + n/4 ] (rho_i - rho_i^{m+1/2});
  * ALSM uses interior neighbours only;
  * initial guess rho^0 = 0;
  * synthetic system solved exactly (sparse direct LU) instead of the paper's
    LU-SGS/SOR sub-iterations, which converge to the same solution.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import build as _build

_libs = {}
_threaded = False


def use_threads(on: bool) -> None:
    """Selects, for later calls, the -fopenmp build of the C sweeps (the
    ordinates on all host cores; every sum in the same order, so the same
    results).  Only for timing the oracle; the default is the plain build."""
    global _threaded
    _threaded = bool(on)


def threads() -> int:
    """Host threads the selected C sweep library runs on."""
    return int(_clib().oracle_threads())


def _clib():
    lib = _libs.get(_threaded)
    if lib is None:
        lib = ctypes.CDLL(_build.build(threads=_threaded))
        P = ctypes.POINTER(ctypes.c_double)
        lib.oracle_sweep.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P, P,
                                     P, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_sweep.restype = ctypes.c_int
        lib.oracle_sweep_transposed.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, P]
        lib.oracle_sweep_transposed.restype = ctypes.c_int
        lib.oracle_sweep_delta.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, P, P]
        lib.oracle_sweep_delta.restype = ctypes.c_int
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        _libs[_threaded] = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def cell_volumes(prob):
    return (prob.dx[None, :] * prob.dy[:, None]).reshape(-1)


def angular_source(prob, rho):
    """Isotropic angular source of one source iteration (Eq. (RTE_SI), steady):
    S_i = (sigma_s,i rho_i + q_i) / (4 pi)."""
    return (prob.sigma_s * rho + prob.q) / (4.0 * math.pi)


def transport_sweep(prob, rho, keep_intensity=False, shift=None, I_prev=None):
    """Kinetic step (Sec. 4.1): exact first-order-upwind solve for every
    ordinate with source S(rho); returns the moments of I^{m+1/2} and the
    kinetic net flux F_iw . n on every boundary face (Sec. 4.4).
    With `shift` (per-cell pseudo-time diagonal, Sec. 4.3) the step is the
    delta form about I_prev = I^m ([K, N])."""
    N, K, nbf = prob.N, prob.K, prob.n_bface
    if shift is not None:
        shift = np.ascontiguousarray(shift, dtype=np.float64)
        I_prev = np.ascontiguousarray(I_prev, dtype=np.float64)
        assert I_prev.shape == (K, N)
    S = np.ascontiguousarray(angular_source(prob, np.asarray(rho, dtype=np.float64)))
    sig_t = np.ascontiguousarray(prob.sigma_t)
    out = {n: np.zeros(N) for n in ("rho", "Fx", "Fy", "Pxx", "Pxy", "Pyy")}
    out["fb"] = np.zeros(nbf)
    I = np.zeros((K, N)) if keep_intensity else None
    inflow = None if prob.inflow is None else np.ascontiguousarray(prob.inflow, dtype=np.float64)
    rc = _clib().oracle_sweep(
        prob.nx, prob.ny, _ptr(np.ascontiguousarray(prob.dx)), _ptr(np.ascontiguousarray(prob.dy)),
        K, _ptr(np.ascontiguousarray(prob.mu)), _ptr(np.ascontiguousarray(prob.eta)),
        _ptr(np.ascontiguousarray(prob.w)), _ptr(sig_t), _ptr(S), _ptr(inflow), _ptr(shift),
        _ptr(I_prev if shift is not None else None), _ptr(I),
        _ptr(out["rho"]), _ptr(out["Fx"]), _ptr(out["Fy"]), _ptr(out["Pxx"]), _ptr(out["Pxy"]),
        _ptr(out["Pyy"]), _ptr(out["fb"]))
    if rc != 0:
        raise MemoryError("oracle sweep allocation failed")
    if keep_intensity:
        out["I"] = I
    return out


def _centres(prob):
    xc = np.cumsum(prob.dx) - 0.5 * prob.dx
    yc = np.cumsum(prob.dy) - 0.5 * prob.dy
    return xc, yc


class Geometry:
    """Faces of the Cartesian mesh as arrays (built once per problem).

    Interior faces (i -> j): cell indices a, b, unit normal n_ij (from a to b),
    area A, r^L (face centre -> centre of a), r^R (face centre -> centre of b).
    Boundary faces: cell, outward normal, area, x_iw - x_i, face number
    (W j, E ny+j, S 2ny+i, N 2ny+nx+i).
    """

    def __init__(self, prob):
        nx, ny = prob.nx, prob.ny
        xc, yc = _centres(prob)
        xf = np.concatenate([[0.0], np.cumsum(prob.dx)])
        yf = np.concatenate([[0.0], np.cumsum(prob.dy)])
        I, J = np.meshgrid(np.arange(nx - 1), np.arange(ny), indexing="xy")
        I, J = I.ravel(), J.ravel()
        fcx = np.stack([xf[I + 1], yc[J]], 1)
        ax = dict(a=I + nx * J, b=I + 1 + nx * J, n=np.tile([1.0, 0.0], (I.size, 1)), A=prob.dy[J],
                  rL=np.stack([xc[I], yc[J]], 1) - fcx, rR=np.stack([xc[I + 1], yc[J]], 1) - fcx)
        I, J = np.meshgrid(np.arange(nx), np.arange(ny - 1), indexing="xy")
        I, J = I.ravel(), J.ravel()
        fcy = np.stack([xc[I], yf[J + 1]], 1)
        ay = dict(a=I + nx * J, b=I + nx * (J + 1), n=np.tile([0.0, 1.0], (I.size, 1)), A=prob.dx[I],
                  rL=np.stack([xc[I], yc[J]], 1) - fcy, rR=np.stack([xc[I], yc[J + 1]], 1) - fcy)
        for key in ax:
            setattr(self, key, np.concatenate([ax[key], ay[key]]))
        j, i = np.arange(ny), np.arange(nx)
        z_j, z_i = np.zeros(ny), np.zeros(nx)
        self.bc = np.concatenate([nx * j, nx - 1 + nx * j, i, i + nx * (ny - 1)])
        self.bn = np.concatenate([np.stack([-1 + z_j, z_j], 1), np.stack([1 + z_j, z_j], 1),
                                  np.stack([z_i, -1 + z_i], 1), np.stack([z_i, 1 + z_i], 1)])
        self.bA = np.concatenate([prob.dy, prob.dy, prob.dx, prob.dx])
        self.bd = np.concatenate([np.stack([-0.5 * prob.dx[0] + z_j, z_j], 1),
                                  np.stack([0.5 * prob.dx[nx - 1] + z_j, z_j], 1),
                                  np.stack([z_i, -0.5 * prob.dy[0] + z_i], 1),
                                  np.stack([z_i, 0.5 * prob.dy[ny - 1] + z_i], 1)])
        self.bf = np.arange(2 * (nx + ny))


_GEOM = {}


def geometry(prob):
    key = id(prob)
    g = _GEOM.get(key)
    if g is None or g[0] is not prob:
        g = (prob, Geometry(prob))
        _GEOM.clear()
        _GEOM[key] = g
    return g[1]


def face_lists(prob):
    return geometry(prob)


def alsm_gradient(prob, U, adaptive=True):
    """Adaptive least-squares gradient (Sec. 5.2, Eqs. (shifted_j),
    (new_vector), (LSF_mdf)).  For cell i and each interior neighbour j the
    neighbour centre is moved along r^R_ij to x'_j = x_ij + (sigma_j/sigma_i)
    r^R_ij; the gradient minimises sum_j [G.(x'_j - x_i) - (U_j - U_i)]^2,
    i.e. solves the 2x2 normal equations of Eq. (LSM_mtx) with x'_j
    (minimum-norm solution where they are singular).
    adaptive=False gives the classic least-squares gradient (Eq. (LSF)).
    """
    sig = prob.sigma_t
    g = geometry(prob)
    N = prob.N
    M = np.zeros((N, 2, 2))
    rhs = np.zeros((N, 2))
    for (i, j, rl, rr) in ((g.a, g.b, g.rL, g.rR), (g.b, g.a, g.rR, g.rL)):
        ratio = sig[j] / sig[i] if adaptive else np.ones(i.size)
        d = -rl + ratio[:, None] * rr            # x'_j - x_i = (x_ij - x_i) + ratio r^R
        np.add.at(M, i, d[:, :, None] * d[:, None, :])
        np.add.at(rhs, i, d * (U[j] - U[i])[:, None])
    G = np.einsum("nij,nj->ni", np.linalg.pinv(M), rhs)
    return G[:, 0].copy(), G[:, 1].copy()


def high_order_terms(prob, Fx, Fy, gx, gy):
    """HoT_F = F^{m+1/2} + grad(rho^{m+1/2}) / (3 sigma_t)  (Eq. (GSIS_HoT))."""
    s3 = 3.0 * prob.sigma_t
    return Fx + gx / s3, Fy + gy / s3


def pseudo_time_shift(prob, cfl_p=0.0, beta=0.0):
    """Per-cell diagonal shift of the kinetic system (Sec. 4.3):
    1/(c dt_p,i) = 1/(CFL_p dx_ref,i)                            (Eq. (cfl_pse))
    1/(c tau_p,i) = max_j |sigma_i r^L_ij - sigma_j r^R_ij| / (beta dx_ref,i)
                                                                   (Eq. (tau_pse))
    with dx_ref,i = min(dx_i, dy_i); a control <= 0 switches its term off."""
    ref = np.minimum(prob.dx[None, :], prob.dy[:, None]).reshape(-1)
    shift = np.zeros(prob.N)
    if cfl_p > 0.0:
        shift += 1.0 / (cfl_p * ref)
    if beta > 0.0:
        g = geometry(prob)
        sig = prob.sigma_t
        v = sig[g.a][:, None] * g.rL - sig[g.b][:, None] * g.rR
        thick = np.sqrt(np.sum(v * v, -1))            # |sigma_i r^L - sigma_j r^R|, same seen from j
        m = np.zeros(prob.N)
        np.maximum.at(m, g.a, thick)
        np.maximum.at(m, g.b, thick)
        shift += m / (beta * ref)
    return shift


def gamma_coefficient(sig_i, sig_j, rL, rR, n):
    """Gamma_ij = -(sigma_i r^L - sigma_j r^R).n / (3 |sigma_i r^L - sigma_j r^R|^2)
    (Eq. (Gamma_ij_com2)); vectorised over faces (arrays of shape [F] and [F,2])."""
    v = np.asarray(sig_i)[..., None] * rL - np.asarray(sig_j)[..., None] * rR
    return -np.sum(v * n, -1) / (3.0 * np.sum(v * v, -1))


def boundary_beta(sig_i, dvec, n):
    """Normal component of the boundary-flux increment per unit drho
    (Eq. (macro_bc_delta_flux)): [ (x_iw - x_i)/(3 sigma_t |x_iw - x_i|^2) + n/4 ] . n."""
    return np.sum(dvec * n, -1) / (3.0 * np.asarray(sig_i) * np.sum(dvec * dvec, -1)) + 0.25


def synthetic_matrix(prob):
    """Finite-volume synthetic operator (Eqs. (MSE_d1), (elem_mtx_M), steady,
    multiplied by V_i):  D_ii = V_i sigma_a,i + sum_int A Gamma + sum_bnd A beta,
    D_ij = -A Gamma."""
    sig = prob.sigma_t
    g = geometry(prob)
    diag = cell_volumes(prob) * prob.sigma_a
    gam = g.A * gamma_coefficient(sig[g.a], sig[g.b], g.rL, g.rR, g.n)
    np.add.at(diag, g.a, gam)
    np.add.at(diag, g.b, gam)
    np.add.at(diag, g.bc, g.bA * boundary_beta(sig[g.bc], g.bd, g.bn))
    N = prob.N
    rows = np.concatenate([g.a, g.b, np.arange(N)])
    cols = np.concatenate([g.b, g.a, np.arange(N)])
    vals = np.concatenate([-gam, -gam, diag])
    return sp.csc_matrix((vals, (rows, cols)), shape=(N, N))


def synthetic_rhs(prob, rho_half, HoTx, HoTy, fb):
    """Right-hand side of the synthetic equation (times V_i):
    b_i = V_i q_i - sum_int A (HoT_i + HoT_j)/2 . n_ij
          - sum_bnd A [ F_iw^init . n - beta rho_i^{m+1/2} ]."""
    g = geometry(prob)
    b = cell_volumes(prob) * prob.q
    flux = g.A * 0.5 * ((HoTx[g.a] + HoTx[g.b]) * g.n[:, 0] + (HoTy[g.a] + HoTy[g.b]) * g.n[:, 1])
    np.add.at(b, g.a, -flux)
    np.add.at(b, g.b, flux)
    sig = prob.sigma_t
    beta = boundary_beta(sig[g.bc], g.bd, g.bn)
    np.add.at(b, g.bc, -g.bA * (fb[g.bf] - beta * rho_half[g.bc]))
    return b


class SyntheticSolver:
    """Exact solve of the synthetic system (sparse LU of D, factored once)."""

    def __init__(self, prob):
        self.D = synthetic_matrix(prob)
        self.lu = spla.splu(self.D)

    def solve(self, b):
        return self.lu.solve(b)


def err_w(new, old, V):
    """Err(W^m) = sqrt( sum (W^m - W^{m-1})^2 V / sum (W^m)^2 V )  (Eq. (Err_W))."""
    den = float(np.sum(new * new * V))
    num = float(np.sum((new - old) ** 2 * V))
    if den == 0.0:
        return 0.0 if num == 0.0 else math.inf
    return math.sqrt(num / den)


def si_iteration(prob, rho, shift=None, I=None):
    """One SI iteration: returns rho^{m+1} and the sweep moments
    (with a pseudo-time shift, I^{m+1} = I^{m+1/2} is returned in sw["I"])."""
    sw = transport_sweep(prob, rho, keep_intensity=shift is not None, shift=shift, I_prev=I)
    return sw["rho"].copy(), sw


def gsis_iteration(prob, rho, solver, adaptive=True, shift=None, I=None):
    """One GSIS iteration (kinetic step, then synthetic step).  With a
    pseudo-time shift the stored intensity is corrected isotropically,
    I^{m+1} = I^{m+1/2} + (rho^{m+1} - rho^{m+1/2})/4pi (Eq. (GSIS_update)),
    and returned in sw["I"]."""
    sw = transport_sweep(prob, rho, keep_intensity=shift is not None, shift=shift, I_prev=I)
    gx, gy = alsm_gradient(prob, sw["rho"], adaptive=adaptive)
    hx, hy = high_order_terms(prob, sw["Fx"], sw["Fy"], gx, gy)
    b = synthetic_rhs(prob, sw["rho"], hx, hy, sw["fb"])
    rho_new = solver.solve(b)
    if shift is not None:
        sw["I"] = sw["I"] + ((rho_new - sw["rho"]) / (4.0 * math.pi))[None, :]
    sw.update(gx=gx, gy=gy, HoTx=hx, HoTy=hy, b=b)
    return rho_new, sw


def _finish(prob, rho, sw, scheme):
    """Moments of I^{m+1}: for GSIS the isotropic correction (Eq. (GSIS_update))
    adds (rho^{m+1} - rho^{m+1/2})/3 to P_xx and P_yy and leaves F unchanged."""
    out = {"rho": rho, "Fx": sw["Fx"], "Fy": sw["Fy"], "Pxx": sw["Pxx"].copy(),
           "Pxy": sw["Pxy"], "Pyy": sw["Pyy"].copy(), "fb": sw["fb"]}
    if scheme == "gsis":
        d = (rho - sw["rho"]) / 3.0
        out["Pxx"] += d
        out["Pyy"] += d
    return out


def _run(prob, scheme, tol, max_iter, fixed_iters, rho0, adaptive, cfl_p, beta, callback):
    V = cell_volumes(prob)
    rho = np.zeros(prob.N) if rho0 is None else np.array(rho0, dtype=np.float64)
    solver = SyntheticSolver(prob) if scheme == "gsis" else None
    use_pt = cfl_p > 0.0 or beta > 0.0
    shift = pseudo_time_shift(prob, cfl_p, beta) if use_pt else None
    I = np.zeros((prob.K, prob.N)) if use_pt else None          # I^0 = 0
    if use_pt and rho0 is not None:
        I[:] = (rho / (4.0 * math.pi))[None, :]
    hist = []
    sw = None
    n = fixed_iters if fixed_iters else max_iter
    converged = False
    for m in range(n):
        if scheme == "gsis":
            new, sw = gsis_iteration(prob, rho, solver, adaptive, shift, I)
        else:
            new, sw = si_iteration(prob, rho, shift, I)
        if use_pt:
            I = sw["I"]
        e = err_w(new, rho, V)
        hist.append(e)
        rho = new
        if callback is not None:
            callback(m, rho, sw, e)
        if not fixed_iters and e < tol:
            converged = True
            break
        if not np.isfinite(e):
            break
    out = _finish(prob, rho, sw, scheme)
    out.update(iters=len(hist), err=hist[-1], history=np.array(hist), converged=converged)
    return out


def si_solve(prob, tol=1e-8, max_iter=100000, fixed_iters=0, rho0=None, cfl_p=0.0, beta=0.0,
             callback=None):
    """Source iteration until Err(rho) < tol (or exactly fixed_iters iterations)."""
    return _run(prob, "si", tol, max_iter, fixed_iters, rho0, True, cfl_p, beta, callback)


def gsis_solve(prob, tol=1e-8, max_iter=10000, fixed_iters=0, rho0=None, adaptive=True,
               cfl_p=0.0, beta=0.0, callback=None):
    """GSIS until Err(rho) < tol (or exactly fixed_iters iterations);
    cfl_p / beta > 0 switch on the pseudo-time shifts of Sec. 4.3."""
    return _run(prob, "gsis", tol, max_iter, fixed_iters, rho0, adaptive, cfl_p, beta, callback)
