"""Pins of the FP64 oracle against what the paper and the mathematics fix:
closed forms, conservation, brute force on tiny meshes, symmetry, and the
algebraic properties of the adaptive least-squares gradient and of the
synthetic operator.  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import workloads as W
from oracle import gsis as G

FOURPI = 4.0 * math.pi


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("order", [4, 6, 8, 10, 12, 14, 16])
def test_level_symmetric_moments(order):
    """Sum w = 4pi, odd moments vanish, second moments 4pi/3, fourth 4pi/5,
    mixed fourth 4pi/15 (exact sphere integrals)."""
    mu, eta, w = W.level_symmetric_2d(order)
    assert len(mu) == order * (order + 2) // 2
    assert np.all(w > 0) and np.all(mu ** 2 + eta ** 2 < 1.0)
    tol = 1e-13
    assert abs(w.sum() - FOURPI) < tol
    for f in (mu, eta, mu * eta, mu ** 3, mu * eta ** 2):
        assert abs((w * f).sum()) < tol
    assert abs((w * mu ** 2).sum() - FOURPI / 3) < tol
    assert abs((w * eta ** 2).sum() - FOURPI / 3) < tol
    assert abs((w * mu ** 4).sum() - FOURPI / 5) < tol
    assert abs((w * mu ** 2 * eta ** 2).sum() - FOURPI / 15) < tol


# ---------------------------------------------------------- helper problems
def _uniform_medium(nx=7, ny=5, order=4, sa=0.3, ss=1.7, q=2.0, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    mu, eta, w = W.level_symmetric_2d(order)
    dx = rng.uniform(0.5, 1.5, nx); dx /= dx.sum()
    dy = rng.uniform(0.5, 1.5, ny); dy /= dy.sum()
    N = nx * ny
    inflow = np.full((2 * (nx + ny), len(mu)), q / (FOURPI * sa))
    return W.Problem("inf", nx, ny, dx, dy, mu, eta, w, np.full(N, sa), np.full(N, ss),
                     np.full(N, q), inflow)


def test_infinite_medium_single_sweep_is_fixed_point():
    """Equilibrium inflow q/(4 pi sigma_a): I = q/(4 pi sigma_a) solves every
    cell equation, so one sweep from rho = q/sigma_a returns it exactly,
    F = 0, P = rho/3 on the diagonal, zero net boundary flux."""
    p = _uniform_medium()
    rho = np.full(p.N, 2.0 / 0.3)
    sw = oracle.transport_sweep(p, rho)
    assert np.allclose(sw["rho"], rho, rtol=1e-13, atol=0)
    assert np.abs(sw["Fx"]).max() < 1e-13 and np.abs(sw["Fy"]).max() < 1e-13
    assert np.allclose(sw["Pxx"], rho / 3, rtol=1e-13) and np.allclose(sw["Pyy"], rho / 3, rtol=1e-13)
    assert np.abs(sw["Pxy"]).max() < 1e-13
    assert np.abs(sw["fb"]).max() < 1e-12


@pytest.mark.parametrize("scheme", ["si", "gsis"])
def test_infinite_medium_converges_to_equilibrium(scheme):
    p = _uniform_medium()
    solve = oracle.si_solve if scheme == "si" else oracle.gsis_solve
    r = solve(p, tol=1e-14, max_iter=5000)
    assert r["converged"]
    assert np.allclose(r["rho"], 2.0 / 0.3, rtol=1e-12, atol=0)
    assert np.abs(r["Fx"]).max() < 1e-11


def test_infinite_medium_gsis_hot_vanishes():
    p = _uniform_medium()
    rho = np.full(p.N, 2.0 / 0.3)
    solver = G.SyntheticSolver(p)
    new, sw = G.gsis_iteration(p, rho, solver)
    assert np.allclose(new, rho, rtol=1e-12)
    assert np.abs(sw["HoTx"]).max() < 1e-12 and np.abs(sw["HoTy"]).max() < 1e-12


# ------------------------------------------------------- pure absorber
def _absorber(nx, ny, axis, seed=3, order=6):
    """sigma_s = q = 0; unit inflow through the W (axis 0) or S (axis 1) wall;
    the two side walls carry the exact discrete 1D profile, so the discrete
    solution is invariant along the other axis."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu, eta, w = W.level_symmetric_2d(order)
    dx = rng.uniform(0.5, 1.5, nx); dx /= dx.sum()
    dy = rng.uniform(0.5, 1.5, ny); dy /= dy.sum()
    n_along = nx if axis == 0 else ny
    sig_line = 10.0 ** rng.uniform(-0.5, 1.5, n_along)      # varies along the beam
    if axis == 0:
        sig = np.tile(sig_line, ny)
        cos, h = mu, dx
    else:
        sig = np.repeat(sig_line, nx)
        cos, h = eta, dy
    K = len(mu)
    prof = np.zeros((n_along, K))   # exact UW1 profile: I_i = I_{i-1} (c/h_i)/(sigma_i + c/h_i)
    for k in range(K):
        if cos[k] <= 0:
            continue
        I = 1.0
        for i in range(n_along):
            a = cos[k] / h[i]
            I = I * a / (sig_line[i] + a)
            prof[i, k] = I
    inflow = np.zeros((2 * (nx + ny), K))
    if axis == 0:
        inflow[0:ny, :] = 1.0
        inflow[2 * ny:2 * ny + nx, :] = prof          # S wall
        inflow[2 * ny + nx:, :] = prof                # N wall
    else:
        inflow[2 * ny:2 * ny + nx, :] = 1.0
        inflow[0:ny, :] = prof                        # W wall
        inflow[ny:2 * ny, :] = prof                   # E wall
    N = nx * ny
    p = W.Problem("abs", nx, ny, dx, dy, mu, eta, w, sig.copy(), np.zeros(N), np.zeros(N), inflow)
    return p, prof


@pytest.mark.parametrize("axis", [0, 1])
def test_pure_absorber_discrete_closed_form(axis):
    nx, ny = (17, 6) if axis == 0 else (6, 17)
    p, prof = _absorber(nx, ny, axis)
    sw = oracle.transport_sweep(p, np.zeros(p.N), keep_intensity=True)
    I = sw["I"].reshape(p.K, ny, nx)
    expect = prof.T[:, None, :] if axis == 0 else prof.T[:, :, None]
    np.testing.assert_allclose(I, np.broadcast_to(expect, I.shape), rtol=1e-13, atol=1e-300)
    rho_line = prof @ p.w
    rho = sw["rho"].reshape(ny, nx)
    np.testing.assert_allclose(rho, np.broadcast_to(rho_line[None, :] if axis == 0 else rho_line[:, None],
                                                    rho.shape), rtol=1e-13)


def test_pure_absorber_first_order_to_exponential():
    """As dx -> 0 the upwind profile tends to exp(-sigma x / mu) at first order."""
    mu1 = 0.35
    errs = []
    for n in (50, 100, 200, 400):
        dx = 1.0 / n
        mu, eta, w = np.array([mu1, -mu1]), np.array([0.2, 0.2]), np.array([2 * math.pi, 2 * math.pi])
        inflow = np.zeros((2 * (n + 1), 2))
        inflow[0, :] = 1.0
        N = n
        sig = np.full(N, 2.0)
        p = W.Problem("beam", n, 1, np.full(n, dx), np.array([1.0]), mu, eta, w, sig, np.zeros(N),
                      np.zeros(N), inflow)
        # top/bottom: the single row sees its own profile through S for eta>0
        prof = (mu1 / dx / (2.0 + mu1 / dx)) ** np.arange(1, n + 1)
        p.inflow[2:2 + n, 0] = prof
        sw = oracle.transport_sweep(p, np.zeros(N), keep_intensity=True)
        xo = (np.arange(n) + 1) * dx          # outflow face of each cell
        errs.append(np.abs(sw["I"][0] - np.exp(-2.0 * xo / mu1)).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(0.9 < o < 1.1 for o in orders), orders


# ------------------------------------------------------- energy balance
def test_sweep_energy_balance_exact():
    """Telescoping UW1 fluxes: sum V sigma_t rho^{1/2} + sum_bnd A F.n
    = sum V (sigma_s rho^m + q) for ANY rho^m (one sweep)."""
    p = W.random_problem(9, 7, order=6, seed=11)
    rng = np.random.Generator(np.random.PCG64(5))
    rho_m = rng.uniform(0, 3, p.N)
    sw = oracle.transport_sweep(p, rho_m)
    V = G.cell_volumes(p)
    g = G.geometry(p)
    lhs = np.sum(V * p.sigma_t * sw["rho"]) + np.sum(g.bA * sw["fb"][g.bf])
    rhs = np.sum(V * (p.sigma_s * rho_m + p.q))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_gsis_synthetic_balance_exact():
    """Synthetic step conserves energy: interior face terms cancel, so
    sum V sigma_a rho^{m+1} + sum_bnd A [F_iw.n + beta (rho^{m+1} - rho^{m+1/2})]
    = sum V q."""
    p = W.random_problem(9, 7, order=6, seed=12)
    rng = np.random.Generator(np.random.PCG64(6))
    rho_m = rng.uniform(0, 3, p.N)
    solver = G.SyntheticSolver(p)
    new, sw = G.gsis_iteration(p, rho_m, solver)
    V = G.cell_volumes(p)
    g = G.geometry(p)
    beta = G.boundary_beta(p.sigma_t[g.bc], g.bd, g.bn)
    lhs = np.sum(V * p.sigma_a * new) + np.sum(g.bA * (sw["fb"][g.bf] + beta * (new[g.bc] - sw["rho"][g.bc])))
    rhs = np.sum(V * p.q)
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)


def test_si_converged_global_balance():
    p = W.random_problem(10, 8, order=4, seed=13, ratio_range=(0.3, 0.8))
    r = oracle.si_solve(p, tol=1e-14, max_iter=5000)
    V = G.cell_volumes(p)
    g = G.geometry(p)
    lhs = np.sum(V * p.sigma_a * r["rho"]) + np.sum(g.bA * r["fb"][g.bf])
    assert abs(lhs - np.sum(V * p.q)) < 1e-11 * np.sum(V * p.q)


# ------------------------------------------------------- brute force
def _dense_transport(p):
    """The full discrete steady RTE (every ordinate, every cell) as one dense
    linear system, written from the finite-volume statement with upwind faces
    and isotropic scattering; solved by LU."""
    nx, ny, K, N = p.nx, p.ny, p.K, p.N
    A = np.zeros((K * N, K * N))
    b = np.zeros(K * N)
    st = p.sigma_t
    for k in range(K):
        for j in range(ny):
            for i in range(nx):
                c = i + nx * j
                r = k * N + c
                V = p.dx[i] * p.dy[j]
                A[r, r] += st[c]
                b[r] += p.q[c] / FOURPI
                for kk in range(K):
                    A[r, kk * N + c] -= p.sigma_s[c] * p.w[kk] / FOURPI
                # (Omega . A, neighbour cell or None, boundary face number)
                faces = [(-p.mu[k] * p.dy[j], c - 1 if i > 0 else None, j),
                         (p.mu[k] * p.dy[j], c + 1 if i < nx - 1 else None, ny + j),
                         (-p.eta[k] * p.dx[i], c - nx if j > 0 else None, 2 * ny + i),
                         (p.eta[k] * p.dx[i], c + nx if j < ny - 1 else None, 2 * ny + nx + i)]
                for oa, nb, bf in faces:
                    if oa >= 0:
                        A[r, r] += oa / V
                    else:
                        if nb is not None:
                            A[r, k * N + nb] += oa / V
                        elif p.inflow is not None:
                            b[r] -= oa / V * p.inflow[bf, k]
    I = sla.solve(A, b).reshape(K, N)
    return p.w @ I


@pytest.mark.parametrize("shape,order,seed", [((4, 4), 4, 21), ((5, 3), 6, 22), ((3, 6), 4, 23)])
def test_si_fixed_point_equals_dense_transport_solve(shape, order, seed):
    p = W.random_problem(shape[0], shape[1], order=order, seed=seed, ratio_range=(0.2, 0.9))
    rho_dense = _dense_transport(p)
    r = oracle.si_solve(p, tol=1e-15, max_iter=20000)
    np.testing.assert_allclose(r["rho"], rho_dense, rtol=1e-12, atol=0)


@pytest.mark.parametrize("beta", [0.0, 10.0])
def test_gsis_fixed_point_equals_dense_affine_solve(beta):
    """The GSIS map is affine in its state (rho, and I with pseudo-time);
    build it column by column and solve (I - A) x = Phi(0) densely."""
    p = W.random_problem(4, 4, order=4, seed=31, ratio_range=(0.5, 0.95))
    solver = G.SyntheticSolver(p)
    N, K = p.N, p.K
    if beta == 0.0:
        def phi(x):
            return G.gsis_iteration(p, x, solver)[0]
        n = N
    else:
        shift = G.pseudo_time_shift(p, 0.0, beta)

        def phi(x):
            rho, I = x[:N], x[N:].reshape(K, N)
            new, sw = G.gsis_iteration(p, rho, solver, True, shift, I)
            return np.concatenate([new, sw["I"].ravel()])
        n = N + N * K
    f0 = phi(np.zeros(n))
    A = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n); e[c] = 1.0
        A[:, c] = phi(e) - f0
    x = sla.solve(np.eye(n) - A, f0)
    r = oracle.gsis_solve(p, tol=1e-15, max_iter=5000, beta=beta)
    np.testing.assert_allclose(r["rho"], x[:N], rtol=1e-11, atol=0)


# ------------------------------------------------------- symmetry
def test_uniform_square_symmetry():
    p = W.config_small()
    for solve in (oracle.si_solve, oracle.gsis_solve):
        r = solve(p, tol=1e-12)["rho"].reshape(64, 64)
        s = np.abs(r).max()
        assert np.abs(r - r.T).max() < 1e-12 * s
        assert np.abs(r - r[:, ::-1]).max() < 1e-12 * s
        assert np.abs(r - r[::-1, :]).max() < 1e-12 * s


# ------------------------------------------------------- ALSM / Gamma
def _mesh_problem(nx, ny, sig, seed=41):
    rng = np.random.Generator(np.random.PCG64(seed))
    mu, eta, w = W.level_symmetric_2d(4)
    dx = rng.uniform(0.5, 1.5, nx); dx /= dx.sum()
    dy = rng.uniform(0.5, 1.5, ny); dy /= dy.sum()
    N = nx * ny
    return W.Problem("m", nx, ny, dx, dy, mu, eta, w, 0.1 * sig, 0.9 * sig, np.ones(N), None)


def test_alsm_uniform_sigma_exact_for_linear_fields():
    p = _mesh_problem(7, 6, np.full(42, 3.0))
    xc, yc = G._centres(p)
    X, Y = np.meshgrid(xc, yc)
    U = (1.5 + 2.0 * X - 0.7 * Y).ravel()
    for adaptive in (True, False):
        gx, gy = oracle.alsm_gradient(p, U, adaptive=adaptive)
        np.testing.assert_allclose(gx, 2.0, rtol=1e-12)
        np.testing.assert_allclose(gy, -0.7, rtol=1e-12)


def test_classic_lsq_is_central_difference_on_uniform_mesh():
    nx = ny = 6
    mu, eta, w = W.level_symmetric_2d(4)
    p = W.Problem("u", nx, ny, np.full(nx, 1 / nx), np.full(ny, 1 / ny), mu, eta, w,
                  np.full(36, 0.1), np.full(36, 1.0), np.ones(36), None)
    rng = np.random.Generator(np.random.PCG64(4))
    U = rng.uniform(0, 1, 36)
    gx, gy = oracle.alsm_gradient(p, U, adaptive=False)
    Ug = U.reshape(ny, nx)
    cx = (Ug[:, 2:] - Ug[:, :-2]) / (2 / nx)
    cy = (Ug[2:, :] - Ug[:-2, :]) / (2 / ny)
    np.testing.assert_allclose(gx.reshape(ny, nx)[:, 1:-1], cx, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gy.reshape(ny, nx)[1:-1, :], cy, rtol=1e-12, atol=1e-12)


def _flux_continuous_profile(p, sig_col, C=0.37, cy=0.25):
    """Piecewise-linear U(x) + cy*y with slope s_i = C sigma_i in column i, so
    the diffusion flux -s/(3 sigma) = -C/3 is continuous across every face."""
    s = C * sig_col
    Ux = np.zeros(p.nx)
    for i in range(1, p.nx):
        Ux[i] = Ux[i - 1] + 0.5 * (s[i - 1] * p.dx[i - 1] + s[i] * p.dx[i])
    _, yc = G._centres(p)
    return (Ux[None, :] + cy * yc[:, None]).ravel(), s


def test_alsm_exact_for_flux_continuous_profiles():
    """At opacity jumps the shifted points (Eq. (shifted_j)) make the gradient
    of a flux-continuous piecewise-linear field exact in every cell, while
    the classic least-squares gradient is not."""
    nx, ny = 9, 5
    rng = np.random.Generator(np.random.PCG64(8))
    sig_col = 10.0 ** rng.uniform(-2, 3, nx)
    p = _mesh_problem(nx, ny, np.tile(sig_col, ny))
    U, s = _flux_continuous_profile(p, sig_col)
    gx, gy = oracle.alsm_gradient(p, U)
    np.testing.assert_allclose(gx.reshape(ny, nx), np.broadcast_to(s, (ny, nx)), rtol=1e-10)
    np.testing.assert_allclose(gy, 0.25, rtol=1e-10)
    gx0, _ = oracle.alsm_gradient(p, U, adaptive=False)
    assert np.abs(gx0.reshape(ny, nx) - s).max() > 1e-2 * np.abs(s).max()


def test_gamma_is_harmonic_face_opacity_and_exact_flux():
    """Gamma_ij (Eq. (Gamma_ij_com2)) equals 1/(3 sigma_{i+1/2} (x_{i+1}-x_i))
    with the equivalent face opacity of Eq. (face_coe_harmonic), and the
    two-point flux Gamma (U_i - U_j) reproduces the exact diffusion flux of a
    flux-continuous profile."""
    nx, ny = 8, 4
    rng = np.random.Generator(np.random.PCG64(9))
    sig_col = 10.0 ** rng.uniform(-2, 3, nx)
    p = _mesh_problem(nx, ny, np.tile(sig_col, ny))
    g = G.geometry(p)
    sig = p.sigma_t
    gam = G.gamma_coefficient(sig[g.a], sig[g.b], g.rL, g.rR, g.n)
    xc, yc = G._centres(p)
    xface = g.n[:, 0] == 1.0
    ia, ib = g.a % nx, g.b % nx
    ja, jb = g.a // nx, g.b // nx
    hx_a, hx_b = p.dx[ia], p.dx[ib]
    sig_f = (sig[g.a] * hx_a + sig[g.b] * hx_b) / (hx_a + hx_b)
    np.testing.assert_allclose(gam[xface], 1.0 / (3 * sig_f * (xc[ib] - xc[ia]))[xface], rtol=1e-13)
    hy_a, hy_b = p.dy[ja], p.dy[jb]
    sig_fy = (sig[g.a] * hy_a + sig[g.b] * hy_b) / (hy_a + hy_b)
    np.testing.assert_allclose(gam[~xface], 1.0 / (3 * sig_fy * (yc[jb] - yc[ja]))[~xface], rtol=1e-13)
    U, s = _flux_continuous_profile(p, sig_col, C=0.37, cy=0.0)
    flux = gam * (U[g.a] - U[g.b])
    np.testing.assert_allclose(flux[xface], -0.37 / 3.0, rtol=1e-12)


def test_alsm_face_value_matches_flux_equality():
    """Reconstructing from a one-neighbour cell with the ALSM slope gives the
    face value fixed by equal diffusion fluxes on both sides of the face
    (Eq. (face_coe_harmonic_diffusion_flux_eq))."""
    mu, eta, w = W.level_symmetric_2d(4)
    dx = np.array([0.3, 0.7])
    sig = np.array([2.0, 450.0])
    p = W.Problem("2", 2, 1, dx, np.array([1.0]), mu, eta, w, 0.1 * sig, 0.9 * sig, np.ones(2), None)
    U = np.array([1.0, 0.2])
    gx, _ = oracle.alsm_gradient(p, U)
    face_from_0 = U[0] + gx[0] * dx[0] / 2
    face_from_1 = U[1] - gx[1] * dx[1] / 2
    # (U_f - U_0)/(sigma_0 dx_0/2) = (U_1 - U_f)/(sigma_1 dx_1/2)
    a, b = sig[0] * dx[0] / 2, sig[1] * dx[1] / 2
    Uf = (b * U[0] + a * U[1]) / (a + b)
    assert abs(face_from_0 - Uf) < 1e-14 and abs(face_from_1 - Uf) < 1e-14


def test_boundary_beta_cartesian():
    p = _mesh_problem(5, 4, np.linspace(1.0, 40.0, 20))
    g = G.geometry(p)
    beta = G.boundary_beta(p.sigma_t[g.bc], g.bd, g.bn)
    h = np.where(np.abs(g.bn[:, 0]) == 1.0, p.dx[g.bc % 5], p.dy[g.bc // 5])
    np.testing.assert_allclose(beta, 2.0 / (3.0 * p.sigma_t[g.bc] * h) + 0.25, rtol=1e-14)


def test_synthetic_matrix_spd_and_row_sums():
    p = W.random_problem(7, 6, order=4, seed=51)
    D = G.synthetic_matrix(p).toarray()
    assert np.abs(D - D.T).max() < 1e-14 * np.abs(D).max()
    np.linalg.cholesky(D)
    g = G.geometry(p)
    beta = G.boundary_beta(p.sigma_t[g.bc], g.bd, g.bn)
    rs = G.cell_volumes(p) * p.sigma_a
    np.add.at(rs, g.bc, g.bA * beta)
    np.testing.assert_allclose(D.sum(1), rs, rtol=1e-10, atol=1e-12 * np.abs(D).max())


# ------------------------------------------------------- pseudo-time
def test_pseudo_time_shift_formula():
    mu, eta, w = W.level_symmetric_2d(4)
    dx = np.array([0.1, 0.2, 0.3])
    sig = np.array([1.0, 100.0, 10.0])
    p = W.Problem("3", 3, 1, dx, np.array([0.5]), mu, eta, w, 0.5 * sig, 0.5 * sig, np.ones(3), None)
    s = G.pseudo_time_shift(p, cfl_p=0.5, beta=4.0)
    t01 = (1.0 * 0.05 + 100.0 * 0.1)
    t12 = (100.0 * 0.1 + 10.0 * 0.15)
    expect = np.array([1 / (0.5 * 0.1) + t01 / (4 * 0.1),
                       1 / (0.5 * 0.2) + max(t01, t12) / (4 * 0.2),
                       1 / (0.5 * 0.3) + t12 / (4 * 0.3)])
    np.testing.assert_allclose(s, expect, rtol=1e-14)


def test_delta_form_equals_shifted_direct_solve():
    """With an isotropic I^m = c/4pi the delta-form step solves
    (L + s) I = S + s c/4pi, i.e. the direct sweep with sigma_a + s and q + s c."""
    p = W.random_problem(8, 6, order=6, seed=61)
    rng = np.random.Generator(np.random.PCG64(7))
    s = rng.uniform(0, 50, p.N)
    c = rng.uniform(0, 2, p.N)
    rho = rng.uniform(0, 2, p.N)
    I_prev = np.tile(c / FOURPI, (p.K, 1))
    a = oracle.transport_sweep(p, rho, shift=s, I_prev=I_prev)
    p2 = W.Problem("m", p.nx, p.ny, p.dx, p.dy, p.mu, p.eta, p.w, p.sigma_a + s, p.sigma_s,
                   p.q + s * c, p.inflow)
    b = oracle.transport_sweep(p2, rho)
    for key in ("rho", "Fx", "Fy", "Pxy", "fb"):
        np.testing.assert_allclose(a[key], b[key], rtol=1e-11, atol=1e-13)


def test_gsis_outputs_are_moments_of_corrected_intensity():
    """F and P of the GSIS result are the moments of
    I^{m+1} = I^{m+1/2} + (rho^{m+1} - rho^{m+1/2})/4pi (Eq. (GSIS_update))."""
    p = W.random_problem(6, 5, order=6, seed=71)
    r = oracle.gsis_solve(p, fixed_iters=3)
    r2 = oracle.gsis_solve(p, fixed_iters=2)
    sw = oracle.transport_sweep(p, r2["rho"], keep_intensity=True)
    I1 = sw["I"] + ((r["rho"] - sw["rho"]) / FOURPI)[None, :]
    np.testing.assert_allclose(r["Pxx"], (p.w * p.mu ** 2) @ I1, rtol=1e-12)
    np.testing.assert_allclose(r["Pyy"], (p.w * p.eta ** 2) @ I1, rtol=1e-12)
    np.testing.assert_allclose(r["Fx"], (p.w * p.mu) @ I1, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(p.w @ I1, r["rho"], rtol=1e-12)


def test_err_definition():
    V = np.array([1.0, 2.0, 0.5])
    new = np.array([1.0, 2.0, 4.0])
    old = np.array([1.0, 1.0, 2.0])
    num = (0 + 1 * 2 + 4 * 0.5)
    den = (1 + 8 + 8)
    assert abs(G.err_w(new, old, V) - math.sqrt(num / den)) < 1e-15
