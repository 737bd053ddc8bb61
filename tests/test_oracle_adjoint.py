"""Pins of the oracle's adjoint (oracle/adjoint.py) against the forward oracle:
each transposed step satisfies the dot-product identity <L^T y, x> = <y, L x>
with the forward step it transposes, the explicit sigma terms re-evaluate the
forward formulas, and the gradient of J = g . rho* matches central finite
differences of full forward solves (h = 1e-6 relative)."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as A
from oracle import gsis as G


@pytest.fixture(scope="module")
def het():
    # non-uniform mesh, heterogeneous opacities and sources, inflow on every wall
    return W.random_problem(7, 5, order=4, seed=3)


def test_transposed_sweep_dot_product_per_direction(het):
    rng = np.random.default_rng(0)
    S = rng.random(het.N)
    p0 = dataclasses.replace(het, q=4 * np.pi * S, sigma_s=np.zeros(het.N), sigma_a=het.sigma_t.copy(),
                             inflow=None)
    I = G.transport_sweep(p0, np.zeros(het.N), keep_intensity=True)["I"]   # I_k = A_k^{-1} S
    psi = rng.standard_normal((het.K, het.N))
    phi = A.transposed_sweep(p0, psi)
    lhs = np.einsum("kn,kn->k", psi, I)
    rhs = phi @ S
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=0)


def test_rhs_transpose_dot_product(het):
    rng = np.random.default_rng(1)
    nu = rng.standard_normal(het.N)
    x = [rng.standard_normal(het.N) for _ in range(3)] + [rng.standard_normal(het.n_bface)]
    pq = dataclasses.replace(het, q=np.zeros(het.N))      # linear part of b
    gx, gy = G.alsm_gradient(pq, x[0])
    hx, hy = G.high_order_terms(pq, x[1], x[2], gx, gy)
    b = G.synthetic_rhs(pq, x[0], hx, hy, x[3])
    t = A.rhs_transpose(het, nu)
    assert abs(nu @ b - sum(ti @ xi for ti, xi in zip(t, x))) <= 1e-12 * abs(nu @ b)


def test_moments_transpose_dot_product(het):
    rng = np.random.default_rng(2)
    p0 = dataclasses.replace(het, inflow=None)
    sw = G.transport_sweep(p0, rng.random(het.N), keep_intensity=True)
    y = [rng.standard_normal(het.N) for _ in range(3)] + [rng.standard_normal(het.n_bface)]
    psi = A.moments_transpose(p0, *y)
    lhs = float(np.sum(psi * sw["I"]))
    rhs = y[0] @ sw["rho"] + y[1] @ sw["Fx"] + y[2] @ sw["Fy"] + y[3] @ sw["fb"]
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gsis_map_transpose_dot_product(het):
    rng = np.random.default_rng(3)
    solver = G.SyntheticSolver(het)
    lam, d = rng.standard_normal(het.N), rng.standard_normal(het.N)
    mt, _, _ = A.map_transpose(het, lam, solver)
    md = A.map_linear(het, d, solver)
    assert abs(mt @ d - lam @ md) <= 1e-12 * abs(lam @ md)


def test_explicit_terms_reproduce_forward_formulas(het):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    rho = rng.random(het.N)
    sw = G.transport_sweep(het, rho, keep_intensity=True)
    terms = A._torch_terms(het, rho, sw, np.zeros(het.N), np.zeros((het.K, het.N)))
    _, bvec, Drho = terms(torch.tensor(het.sigma_a), torch.tensor(het.sigma_s))
    gx, gy = G.alsm_gradient(het, sw["rho"])
    hx, hy = G.high_order_terms(het, sw["Fx"], sw["Fy"], gx, gy)
    b = G.synthetic_rhs(het, sw["rho"], hx, hy, sw["fb"])
    np.testing.assert_allclose(bvec.numpy(), b, rtol=1e-13, atol=1e-13 * np.abs(b).max())
    Dr = G.synthetic_matrix(het) @ rho
    np.testing.assert_allclose(Drho.numpy(), Dr, rtol=1e-13, atol=1e-13 * np.abs(Dr).max())


def test_adjoint_iteration_converges_like_gsis(het):
    # lam = M^T lam + g; M^T has the spectrum of M, so the count is of the order of GSIS's
    g = np.zeros(het.N)
    g[[3, 11]] = 1.0
    lam, nu, phi, iters = A.adjoint_solve(het, g, tol=1e-13)
    fwd = G.gsis_solve(het, tol=1e-13)
    assert iters <= 3 * fwd["iters"] + 5
    # fixed point: lam = M^T lam + g
    mt, _, _ = A.map_transpose(het, lam, G.SyntheticSolver(het))
    np.testing.assert_allclose(mt + g, lam, rtol=1e-11, atol=1e-11 * np.abs(lam).max())


def test_gradient_matches_central_differences():
    pytest.importorskip("torch")
    p = W.random_problem(8, 6, order=4, seed=5, log10_range=(0.0, 1.0), ratio_range=(0.5, 0.9))
    rng = np.random.default_rng(1)
    det = rng.choice(p.N, 3, replace=False)
    g = np.zeros(p.N)
    g[det] = 1.0
    _, rho = A.functional(p, g)
    ga, gs, _ = A.gradient(p, rho, g)
    scale = max(np.abs(ga).max(), np.abs(gs).max())
    # corner, opposite corner, west wall, a detector cell, interior cells
    for c in (0, p.N - 1, 8, int(det[0]), 20, 27):
        for which, grad in (("sigma_a", ga), ("sigma_s", gs)):
            base = getattr(p, which)
            h = 1e-6 * base[c]
            vals = []
            for sgn in (1.0, -1.0):
                arr = base.copy()
                arr[c] += sgn * h
                vals.append(A.functional(dataclasses.replace(p, **{which: arr}), g)[0])
            fd = (vals[0] - vals[1]) / (2.0 * h)
            assert abs(fd - grad[c]) <= 1e-5 * abs(fd) + 1e-8 * scale, (c, which, fd, grad[c])
