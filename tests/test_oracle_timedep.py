"""Pins of the time-dependent oracle (oracle/timedep.py).

* Brute force on tiny meshes: the fully implicit backward-Euler step of the
  first-order upwind discrete ordinates equations (Sec. 4.1, Eq. (RTE_d)
  with psi = 0) coupled to the material equation (Eq. (Tm_d)), assembled
  here face by face as one dense system and solved by Newton on T.  GSIS
  converges to it on a single cell: there the synthetic balance (no interior
  faces) forces rho^{m+1/2} = rho^{m+1} at the fixed point.  With interior
  faces GSIS's fixed point differs from it by the gap between the compact
  two-point diffusion flux and the face-averaged least-squares gradient
  (the steady scheme's own property).  The Fleck-Cummings linearised system
  (Eqs. (Tm_semi_linear), (RTE_SI)), assembled the same way, must equal the
  converged SI step on any mesh.
* Equilibrium: a medium at T with I = a c T^4 / 4pi everywhere and the same
  intensity entering through every wall stays there.
* Energy: for a converged GSIS step, sum V [(rho^{n+1} - rho^n)/c + C_v
  (T^{n+1} - T^n)] / dt + sum_bnd A F.n = sum V q with the synthetic
  equation's boundary flux A [F_iw.n + beta (rho - rho^{m+1/2})] (Eq.
  (macro_bc_delta_flux)); for a converged SI step with the kinetic flux.
* dt -> infinity: the step reaches radiative equilibrium, the steady problem
  with all absorption turned into scattering, and T = (rho/(a c))^(1/4).
"""
import dataclasses
import math

import numpy as np
import pytest
import scipy.optimize as so

import oracle
import workloads as W
from oracle import timedep as TD


def _upwind_operator(p, tp):
    """Dense matrix M and vector r with M I = r + (emission/scattering terms
    added by the caller): rows (k, cell), V (1/(c dt) + sigma_t) I_kc +
    sum_faces A (Omega.n) I_face, inflow moved to the right-hand side."""
    nx, ny, K = p.nx, p.ny, p.K
    N = nx * ny
    M = np.zeros((K * N, K * N))
    r = np.zeros(K * N)
    st = p.sigma_a + p.sigma_s
    for k in range(K):
        mu, eta = p.mu[k], p.eta[k]
        for j in range(ny):
            for i in range(nx):
                c = i + nx * j
                row = k * N + c
                V = p.dx[i] * p.dy[j]
                M[row, row] += V * (1.0 / (tp.c * tp.dt) + st[c])
                # faces: (normal x, normal y, area, neighbour or None, boundary face index)
                faces = [(1.0, 0.0, p.dy[j], (i + 1, j) if i + 1 < nx else None, ny + j),
                         (-1.0, 0.0, p.dy[j], (i - 1, j) if i > 0 else None, j),
                         (0.0, 1.0, p.dx[i], (i, j + 1) if j + 1 < ny else None, 2 * ny + nx + i),
                         (0.0, -1.0, p.dx[i], (i, j - 1) if j > 0 else None, 2 * ny + i)]
                for nxf, nyf, A, nb, bf in faces:
                    on = mu * nxf + eta * nyf
                    if on >= 0.0:
                        M[row, row] += A * on
                    elif nb is not None:
                        M[row, k * N + nb[0] + nx * nb[1]] += A * on
                    elif p.inflow is not None:
                        r[row] -= A * on * p.inflow[bf, k]
    return M, r


def _moment_rows(p):
    N, K = p.N, p.K
    R = np.zeros((N, K * N))
    for k in range(K):
        R[np.arange(N), k * N + np.arange(N)] = p.w[k]
    return R


def brute_force_implicit(p, tp, I_n, T_n):
    N, K = p.N, p.K
    V = (p.dx[None, :] * p.dy[:, None]).reshape(-1)
    M, r = _upwind_operator(p, tp)
    R = _moment_rows(p)
    rep = lambda v: np.tile(v, K)   # per-cell vector for every (k, cell) row
    # scattering: - V sigma_s rho / 4pi on the left
    A = M - (rep(V * p.sigma_s / (4 * math.pi))[:, None] * np.tile(R, (K, 1)))
    base = r + rep(V) * (I_n.reshape(-1) / (tp.c * tp.dt)) + rep(V * p.q / (4 * math.pi))

    def intensities(T):
        phi = tp.a * tp.c * T ** 4
        return np.linalg.solve(A, base + rep(V * p.sigma_a * phi / (4 * math.pi)))

    def material(T):
        rho = R @ intensities(T)
        return tp.cv * (T - T_n) / tp.dt - p.sigma_a * (rho - tp.a * tp.c * T ** 4)

    T = so.fsolve(material, T_n.copy(), xtol=1e-13)
    I = intensities(T)
    return R @ I, T


def brute_force_fleck(p, tp, I_n, T_n):
    N, K = p.N, p.K
    V = (p.dx[None, :] * p.dy[:, None]).reshape(-1)
    M, r = _upwind_operator(p, tp)
    R = _moment_rows(p)
    rep = lambda v: np.tile(v, K)
    kappa = 4 * tp.a * tp.c * T_n ** 3
    f = (tp.cv / tp.dt) / (tp.cv / tp.dt + kappa * p.sigma_a)
    phi_n = tp.a * tp.c * T_n ** 4
    # emission phi = (1 - f) rho + f phi^n acts as extra scattering (1 - f) sigma_a
    A = M - (rep(V * (p.sigma_s + (1 - f) * p.sigma_a) / (4 * math.pi))[:, None] * np.tile(R, (K, 1)))
    rhs = r + rep(V) * (I_n.reshape(-1) / (tp.c * tp.dt)) + rep(V * (p.q + f * p.sigma_a * phi_n) / (4 * math.pi))
    rho = R @ np.linalg.solve(A, rhs)
    phi = (1 - f) * rho + f * phi_n
    return rho, (phi + 3 * phi_n) / kappa


def _tiny(seed, nx=3, ny=2, order=4):
    p = W.random_problem(nx, ny, order=order, seed=seed, log10_range=(-0.5, 1.5), ratio_range=(0.2, 0.8))
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    I_n = rng.uniform(0.1, 1.0, (p.K, p.N))
    T_n = rng.uniform(0.5, 1.5, p.N)
    return p, I_n, T_n


@pytest.mark.parametrize("seed,order,tp", [(1, 4, TD.TimeParams(dt=0.05, c=1.0, a=1.0, cv=0.7)),
                                           (2, 6, TD.TimeParams(dt=0.3, c=3.0, a=0.5, cv=2.0)),
                                           (9, 8, TD.TimeParams(dt=2.0, c=1.0, a=2.0, cv=0.3))])
def test_gsis_step_equals_brute_force_implicit_one_cell(seed, order, tp):
    p, I_n, T_n = _tiny(seed, nx=1, ny=1, order=order)
    rho_n = I_n.T @ p.w
    o = TD.gsis_time_step(p, tp, rho_n, T_n, I_n, tol=1e-14, max_iter=200)
    rho_b, T_b = brute_force_implicit(p, tp, I_n, T_n)
    assert np.abs(o["rho"] - rho_b).max() < 1e-10 * np.abs(rho_b).max()
    assert np.abs(o["T"] - T_b).max() < 1e-10 * np.abs(T_b).max()


@pytest.mark.parametrize("seed,tp", [(3, TD.TimeParams(dt=0.05, c=1.0, a=1.0, cv=0.7)),
                                     (4, TD.TimeParams(dt=0.3, c=3.0, a=0.5, cv=2.0))])
def test_si_step_equals_brute_force_fleck(seed, tp):
    p, I_n, T_n = _tiny(seed)
    rho_n = I_n.T @ p.w
    o = TD.si_time_step(p, tp, rho_n, T_n, I_n, tol=1e-14, max_iter=2000)
    rho_b, T_b = brute_force_fleck(p, tp, I_n, T_n)
    assert np.abs(o["rho"] - rho_b).max() < 1e-10 * np.abs(rho_b).max()
    assert np.abs(o["T"] - T_b).max() < 1e-10 * np.abs(T_b).max()


def test_fleck_and_implicit_differ():
    # the Fleck-Cummings step is a linearisation: it must not coincide with
    # the fully implicit step when T changes (guards against both pins
    # collapsing onto one system)
    tp = TD.TimeParams(dt=0.3, c=1.0, a=1.0, cv=0.5)
    p, I_n, T_n = _tiny(5)
    rho_i, T_i = brute_force_implicit(p, tp, I_n, T_n)
    rho_f, T_f = brute_force_fleck(p, tp, I_n, T_n)
    assert np.abs(T_i - T_f).max() > 1e-6


@pytest.mark.parametrize("scheme", ["gsis", "si"])
def test_equilibrium_is_preserved(scheme):
    T0, tp = 0.8, TD.TimeParams(dt=0.1, c=2.0, a=0.7, cv=1.3)
    p = W.random_problem(9, 7, order=6, seed=6, ratio_range=(0.2, 0.9))
    eq = tp.a * tp.c * T0 ** 4 / (4 * math.pi)
    p = dataclasses.replace(p, q=np.zeros(p.N), inflow=np.full((p.n_bface, p.K), eq))
    rho0 = np.full(p.N, 4 * math.pi * eq)
    out = TD.run(p, tp, 2, rho0, np.full(p.N, T0), scheme=scheme, tol=1e-13)
    assert np.abs(out["rho"] / rho0 - 1).max() < 1e-11
    assert np.abs(out["T"] / T0 - 1).max() < 1e-11


@pytest.mark.parametrize("scheme", ["gsis", "si"])
def test_energy_conservation_of_a_converged_step(scheme):
    tp = TD.TimeParams(dt=0.02, c=1.0, a=1.0, cv=1.0)
    p = W.random_problem(14, 11, order=6, seed=7, ratio_range=(0.3, 0.95))
    rng = np.random.Generator(np.random.PCG64(7))
    T_n = rng.uniform(0.3, 1.2, p.N)
    rho_n = tp.a * tp.c * T_n ** 4 * rng.uniform(0.5, 1.5, p.N)
    I_n = TD.isotropic(p, rho_n)
    V = (p.dx[None, :] * p.dy[:, None]).reshape(-1)
    A = np.concatenate([p.dy, p.dy, p.dx, p.dx])
    if scheme == "gsis":
        o = TD.gsis_time_step(p, tp, rho_n, T_n, I_n, tol=1e-14)
        # boundary flux of the synthetic equation: A [F_iw.n + beta (rho_i - rho_i^{m+1/2})]
        g = oracle.geometry(p)
        beta = oracle.boundary_beta(p.sigma_t[g.bc], g.bd, g.bn)
        bflux = np.sum(g.bA * (o["fb"][g.bf] + beta * (o["rho"][g.bc] - o["rho_half"][g.bc])))
        # rho^n + I^n correction: the step's rho is the synthetic solution
    else:
        o = TD.si_time_step(p, tp, rho_n, T_n, I_n, tol=1e-14)
        # the kinetic flux of the converged step; the Fleck-Cummings material
        # update conserves C_v dT against sigma_a (rho - phi) with the linearised phi
        bflux = np.sum(A * o["fb"])
    lhs = np.sum(V * ((o["rho"] - rho_n) / tp.c + tp.cv * (o["T"] - T_n))) / tp.dt + bflux
    rhs = np.sum(V * p.q)
    scale = np.sum(V * np.abs(o["rho"] - rho_n)) / (tp.c * tp.dt) + abs(rhs) + abs(bflux)
    assert abs(lhs - rhs) < 1e-9 * scale


def test_long_step_reaches_radiative_equilibrium():
    tp = TD.TimeParams(dt=1e12, c=1.0, a=1.0, cv=1.0)
    p = W.random_problem(10, 8, order=4, seed=8, ratio_range=(0.3, 0.9), with_inflow=False)
    rng = np.random.Generator(np.random.PCG64(8))
    T_n = rng.uniform(0.5, 1.0, p.N)
    rho_n = T_n ** 4
    o = TD.gsis_time_step(p, tp, rho_n, T_n, TD.isotropic(p, rho_n), tol=1e-13)
    steady = dataclasses.replace(p, sigma_a=np.zeros(p.N), sigma_s=p.sigma_a + p.sigma_s)
    s = oracle.gsis_solve(steady, tol=1e-13)
    assert np.abs(o["rho"] - s["rho"]).max() < 1e-8 * np.abs(s["rho"]).max()
    assert np.abs(o["T"] - (s["rho"] / (tp.a * tp.c)) ** 0.25).max() < 1e-8


def test_gsis_step_intensity_carries_the_corrected_density():
    # Eq. (GSIS_update): I^{n+1} = I^{m+1/2} + (rho^{m+1} - rho^{m+1/2})/4pi, so the
    # zeroth moment of the intensity handed to the next step is rho^{n+1}
    tp = TD.TimeParams(dt=0.05)
    p = W.random_problem(12, 9, order=6, seed=10, ratio_range=(0.3, 0.9))
    rng = np.random.Generator(np.random.PCG64(10))
    T_n = rng.uniform(0.5, 1.0, p.N)
    rho_n = T_n ** 4
    o = TD.gsis_time_step(p, tp, rho_n, T_n, TD.isotropic(p, rho_n), fixed_iters=3)
    assert np.abs(o["rho_half"] - o["rho"]).max() > 1e-8 * np.abs(o["rho"]).max()   # the correction is not trivial
    np.testing.assert_allclose(o["I"].T @ p.w, o["rho"], rtol=1e-13, atol=1e-14 * np.abs(o["rho"]).max())
