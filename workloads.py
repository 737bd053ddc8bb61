"""Seeded synthetic problem data for the steady gray RTE, shared by the oracle,
the tests and the benchmark.

This module holds problem *data* only: mesh spacings, discrete-ordinate sets,
per-cell opacities and sources, and boundary inflow.  It performs no step of
the solution method (no sweep, no moment, no gradient, no synthetic solve).

Conventions (they are also the C-ABI conventions of ``include/gsis.h``):

* cells are row-major, cell ``c = i + nx*j`` with ``i`` along x;
* boundary faces are numbered W (``j``), E (``ny + j``), S (``2*ny + i``),
  N (``2*ny + nx + i``); ``inflow`` is ``[n_bface, K]``, the intensity that
  enters the domain through that face in direction ``k`` (read only where the
  direction points into the domain);
* ``q`` is the angle-integrated volumetric source, so the angular source of
  the transport equation is ``q / (4*pi)`` (the right-hand side ``4*pi*Q`` of
  the linearised synthetic equation, Sec. 3.2, Eq. (dse_iter)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# First direction cosine of the classic level-symmetric LQ_n sets; the rest of
# each set follows from the level-symmetric constraint and moment matching.
# For S4 (one weight class) mu_1 is the exact root that integrates mu^4
# exactly: with t = mu_1^2, 2 t^2 + (1 - 2 t)^2 = 3/5, i.e. 6 t^2 - 4 t + 0.4 = 0.
LS_MU1 = {
    4: math.sqrt((4.0 - math.sqrt(6.4)) / 12.0), 6: 0.2666355, 8: 0.2182179, 10: 0.1893213,
    12: 0.1672126, 14: 0.1519859, 16: 0.1389568,
}


def _double_factorial(k: int) -> int:
    r = 1
    while k > 1:
        r *= k
        k -= 2
    return r


def level_symmetric_octant(order: int):
    """Points and weights of one octant of the level-symmetric S_order set.

    Cosines: mu_i^2 = mu_1^2 + (i-1) * 2 (1 - 3 mu_1^2) / (order - 2).
    Points: (mu_a, mu_b, mu_c) with a + b + c = order/2 + 2.  Points that are
    permutations of each other share one weight; the class weights are the
    least-squares solution of the even moment conditions
    sum w mux^2a muy^2b muz^2c = (2a-1)!!(2b-1)!!(2c-1)!!/(2(a+b+c)+1)!!
    for a + b + c < order/2 (octant weights sum to 1).  For order <= 16 the
    system is consistent and all weights are positive.
    """
    if order not in LS_MU1:
        raise ValueError(f"level-symmetric order {order} not supported")
    n = order // 2
    mu1 = LS_MU1[order]
    step = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (order - 2) if order > 2 else 0.0
    lev = np.sqrt(mu1 * mu1 + step * np.arange(n))
    pts, cls = [], []
    for a in range(1, n + 1):
        for b in range(1, n + 1):
            c = n + 2 - a - b
            if 1 <= c <= n:
                pts.append((lev[a - 1], lev[b - 1], lev[c - 1]))
                cls.append(tuple(sorted((a, b, c))))
    ucls = sorted(set(cls))
    ci = np.array([ucls.index(c) for c in cls])
    P = np.array(pts)
    rows, rhs = [], []
    for a in range(n):
        for b in range(n - a):
            for c in range(n - a - b):
                row = np.zeros(len(ucls))
                np.add.at(row, ci, P[:, 0] ** (2 * a) * P[:, 1] ** (2 * b) * P[:, 2] ** (2 * c))
                rows.append(row)
                rhs.append(_double_factorial(2 * a - 1) * _double_factorial(2 * b - 1)
                           * _double_factorial(2 * c - 1) / _double_factorial(2 * (a + b + c) + 1))
    wc = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
    return P, wc[ci]


def level_symmetric_2d(order: int):
    """2D discrete-ordinate set from the level-symmetric S_order set.

    The xi > 0 hemisphere is kept and its weights doubled (the 2D problem is
    symmetric in z), so sum(w) = 4*pi.  Returns (mu, eta, w), K = order(order+2)/2,
    grouped by quadrant in the order (+,+), (-,+), (+,-), (-,-).
    """
    P, wo = level_symmetric_octant(order)
    mu, eta, w = [], [], []
    for sx, sy in ((1, 1), (-1, 1), (1, -1), (-1, -1)):
        mu.append(sx * P[:, 0])
        eta.append(sy * P[:, 1])
        w.append(wo * (4.0 * math.pi / 8.0) * 2.0)
    return np.concatenate(mu), np.concatenate(eta), np.concatenate(w)


@dataclasses.dataclass
class Problem:
    """One steady gray-RTE problem on a 2D Cartesian mesh (all float64)."""
    name: str
    nx: int
    ny: int
    dx: np.ndarray          # [nx] cell widths
    dy: np.ndarray          # [ny] cell heights
    mu: np.ndarray          # [K] x direction cosines
    eta: np.ndarray         # [K] y direction cosines
    w: np.ndarray           # [K] weights, sum = 4 pi
    sigma_a: np.ndarray     # [N]
    sigma_s: np.ndarray     # [N]
    q: np.ndarray           # [N] angle-integrated source
    inflow: np.ndarray | None = None   # [n_bface, K] or None (vacuum)

    @property
    def N(self) -> int:
        return self.nx * self.ny

    @property
    def K(self) -> int:
        return int(self.mu.shape[0])

    @property
    def n_bface(self) -> int:
        return 2 * (self.nx + self.ny)

    @property
    def sigma_t(self) -> np.ndarray:
        return self.sigma_a + self.sigma_s


def uniform_mesh(n: int, length: float = 1.0) -> np.ndarray:
    return np.full(n, length / n)


def isotropic_inflow(nx: int, ny: int, mu, eta, walls: dict) -> np.ndarray:
    """Inflow array with a constant intensity per wall, e.g. {"W": 1.0}."""
    K = len(mu)
    inflow = np.zeros((2 * (nx + ny), K))
    sl = {"W": slice(0, ny), "E": slice(ny, 2 * ny),
          "S": slice(2 * ny, 2 * ny + nx), "N": slice(2 * ny + nx, 2 * (nx + ny))}
    for wall, val in walls.items():
        inflow[sl[wall], :] = val
    return inflow


def homogeneous(nx=64, ny=None, order=8, sigma_t=10.0, ratio=0.99, q=1.0,
                inflow_walls=None, name=None) -> Problem:
    """Uniform medium on the unit square (the 64x64, S8, sigma_t=10,
    scattering ratio 0.99, q=1, vacuum workload by default)."""
    ny = nx if ny is None else ny
    mu, eta, w = level_symmetric_2d(order)
    N = nx * ny
    sig_s = np.full(N, sigma_t * ratio)
    sig_a = np.full(N, sigma_t) - sig_s
    inflow = None if not inflow_walls else isotropic_inflow(nx, ny, mu, eta, inflow_walls)
    return Problem(name or f"homogeneous_{nx}x{ny}_S{order}", nx, ny, uniform_mesh(nx),
                   uniform_mesh(ny), mu, eta, w, sig_a, sig_s, np.full(N, float(q)), inflow)


def channel_mask(n: int, seed: int = 2, width: int = 8) -> np.ndarray:
    """Boolean [n, n] mask (index [j, i]) of a bent channel crossing the domain
    from the left wall, drawn with numpy's PCG64 seeded generator.

    The centreline starts at the left wall at a height drawn from
    U[n/4, 3n/4]; it then alternates horizontal runs of length U[n/8, 3n/8]
    and vertical jogs of +-U[n/32, n/8], clamped to [n/32, n - n/16], until
    it reaches the right wall.  The channel is `width` cells wide around it.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    s = n / 256.0
    lo, hi = int(round(8 * s)), int(round(240 * s))
    half = width // 2
    mask = np.zeros((n, n), dtype=bool)
    x = 0
    y = int(rng.integers(int(64 * s), int(192 * s) + 1))
    while x < n:
        run = int(rng.integers(int(32 * s), int(96 * s) + 1))
        x1 = min(n - 1, x + run)
        mask[max(0, y - half):min(n, y + half), x:x1 + 1] = True
        x = x1
        if x >= n - 1:
            break
        jog = int(rng.integers(int(8 * s), int(32 * s) + 1)) * (1 if rng.random() < 0.5 else -1)
        y1 = int(np.clip(y + jog, lo, hi))
        ya, yb = min(y, y1), max(y, y1)
        mask[max(0, ya - half):min(n, yb + half), max(0, x - half):min(n, x + half)] = True
        y = y1
    return mask


def channel_problem(n=256, order=12, seed=2, width=8, sigma_bulk=2000.0, sigma_channel=0.2,
                    ratio=0.999, name=None) -> Problem:
    """Thick medium with a thin bent channel (the 256x256, S12 multiscale
    workload by default): bulk sigma_t=2000, channel sigma_t=0.2, both with
    scattering ratio 0.999, isotropic unit intensity entering through the
    left wall, vacuum elsewhere, no volumetric source."""
    mu, eta, w = level_symmetric_2d(order)
    m = channel_mask(n, seed, width).reshape(-1)
    sig_t = np.where(m, sigma_channel, sigma_bulk)
    sig_s = ratio * sig_t
    sig_a = sig_t - sig_s
    inflow = isotropic_inflow(n, n, mu, eta, {"W": 1.0})
    return Problem(name or f"channel_{n}x{n}_S{order}_seed{seed}", n, n, uniform_mesh(n),
                   uniform_mesh(n), mu, eta, w, sig_a, sig_s, np.zeros(n * n), inflow)


def random_problem(nx, ny, order=4, seed=0, log10_range=(-1.0, 2.0), ratio_range=(0.3, 0.99),
                   nonuniform=True, with_inflow=True, name=None) -> Problem:
    """Heterogeneous problem for parity checks: random non-uniform spacings,
    log-uniform per-cell sigma_t, uniform scattering ratios, random sources
    and random inflow on every wall (PCG64 seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu, eta, w = level_symmetric_2d(order)
    N = nx * ny
    if nonuniform:
        dx = rng.uniform(0.5, 1.5, nx); dx /= dx.sum()
        dy = rng.uniform(0.5, 1.5, ny); dy /= dy.sum()
    else:
        dx, dy = uniform_mesh(nx), uniform_mesh(ny)
    sig_t = 10.0 ** rng.uniform(*log10_range, N)
    ratio = rng.uniform(*ratio_range, N)
    sig_s = ratio * sig_t
    sig_a = sig_t - sig_s
    q = rng.uniform(0.0, 2.0, N)
    inflow = rng.uniform(0.0, 1.0, (2 * (nx + ny), len(mu))) if with_inflow else None
    return Problem(name or f"random_{nx}x{ny}_S{order}_seed{seed}", nx, ny, dx, dy, mu, eta, w,
                   sig_a, sig_s, q, inflow)


def config_small() -> Problem:
    """64x64 cells, S8 (40 directions), sigma_t=10, ratio 0.99, q=1, vacuum."""
    return homogeneous(64, 64, 8, 10.0, 0.99, 1.0, name="uniform_64x64_S8")


def config_channel() -> Problem:
    """256x256 cells, S12 (84 directions), 2000 / 0.2 channel, seed 2."""
    return channel_problem(256, 12, 2, name="channel_256x256_S12")


def smooth_field(n: int, rng: np.random.Generator, modes: int = 16, kmax: int = 4) -> np.ndarray:
    """Unit-variance smooth random field on the n x n cell centres of the unit
    square: sum of `modes` Fourier modes with integer wave vectors
    0 < |k| <= kmax and uniform random phases, scaled by sqrt(2/modes) (each
    cosine has variance 1/2 over a uniform phase)."""
    ks = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(-kmax, kmax + 1)
          if 0 < kx * kx + ky * ky <= kmax * kmax]
    pick = rng.choice(len(ks), modes, replace=False)
    phase = rng.uniform(0.0, 2.0 * math.pi, modes)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")   # X varies along i (x), Y along j
    g = np.zeros((n, n))
    for m, idx in enumerate(pick):
        kx, ky = ks[idx]
        g += np.cos(2.0 * math.pi * (kx * X + ky * Y) + phase[m])
    return (g * math.sqrt(2.0 / modes)).reshape(-1)


def batch_problems(n: int = 64, seed: int = 4, side_range=(32, 256), orders=(8, 10, 12, 14, 16),
                   log10_lo: float = -2.0, log10_span: float = 6.0, ratio_range=(0.5, 0.9999)) -> list:
    """Independent square problems of uneven size for the batched solve.
    Side = round(s0 * (s1/s0)^u), u ~ U[0,1] (log-uniform in [s0, s1]); order
    uniform over `orders`; log10 sigma_t = log10_lo + log10_span * Phi(g) with
    g a unit-variance smooth field (Phi the standard normal CDF, so the
    marginal of sigma_t is log-uniform); one scattering ratio per problem,
    uniform in ratio_range; q = 1; vacuum walls; uniform mesh on the unit
    square (PCG64 seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s0, s1 = side_range
    out = []
    for p in range(n):
        side = int(round(s0 * (s1 / s0) ** rng.uniform()))
        order = int(orders[rng.integers(len(orders))])
        g = smooth_field(side, rng)
        phi = 0.5 * (1.0 + np.vectorize(math.erf)(g / math.sqrt(2.0)))
        sig_t = 10.0 ** (log10_lo + log10_span * phi)
        ratio = rng.uniform(*ratio_range)
        mu, eta, w = level_symmetric_2d(order)
        sig_s = ratio * sig_t
        sig_a = sig_t - sig_s
        out.append(Problem(f"batch{seed}_{p}_{side}x{side}_S{order}", side, side, uniform_mesh(side),
                           uniform_mesh(side), mu, eta, w, sig_a, sig_s, np.ones(side * side), None))
    return out


def config_batch() -> list:
    """64 problems, seed 4: sides 32-256 log-uniform, S8-S16, sigma_t
    log-uniform in [1e-2, 1e4] on smooth fields, ratio U[0.5, 0.9999], q = 1,
    vacuum."""
    return batch_problems()


def channel_td_problem(n: int = 1024, order: int = 16, seed: int = 2, base: int = 256, width: int = 8,
                       sigma_bulk: float = 2000.0, sigma_channel: float = 0.2, ratio: float = 0.999,
                       name=None) -> Problem:
    """The 256x256 channel geometry scaled by n/base: the base mask (`width`
    cells wide, seed 2) with every cell replaced by an (n/base)^2 block (a 32-cell
    wide channel at n = 1024); bulk sigma_t = 2000, channel sigma_t = 0.2,
    scattering ratio 0.999, isotropic unit intensity entering through the
    left wall, vacuum elsewhere, q = 0; uniform mesh on the unit square."""
    f = n // base
    if f < 1 or f * base != n:
        raise ValueError("n must be a multiple of base")
    m = np.kron(channel_mask(base, seed, width), np.ones((f, f), dtype=bool)).reshape(-1)
    mu, eta, w = level_symmetric_2d(order)
    sig_t = np.where(m, sigma_channel, sigma_bulk)
    sig_s = ratio * sig_t
    inflow = isotropic_inflow(n, n, mu, eta, {"W": 1.0})
    return Problem(name or f"channel_td_{n}x{n}_S{order}_seed{seed}", n, n, uniform_mesh(n), uniform_mesh(n),
                   mu, eta, w, sig_t - sig_s, sig_s, np.zeros(n * n), inflow)


# time stepping of the radiation-material workload: backward Euler, dt = 1e-3,
# 100 steps, c = a = C_v = 1, cold start T^0 = 0.1 with rho^0 = a c (T^0)^4
TIMEDEP = dict(dt=1e-3, nsteps=100, c=1.0, a=1.0, cv=1.0, T0=0.1)


def config_timedep() -> Problem:
    """1024x1024 cells, S16 (144 directions), the channel scaled x4."""
    return channel_td_problem()
