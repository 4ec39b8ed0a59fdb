"""Plain FP64 oracle for the UQ layer: samples, quadrature, gPC basis, projection, statistics.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by the
CPU-baseline legs of ``bench.py``; nothing in the product package imports it.  Written
to be read against arXiv 2508.13867 line by line, not to be fast; it shares no code
with the CUDA library.

Paper passages followed:
  * Sec. 4.1, Eq. meanMCS and Eq. varMCS: Monte Carlo mean and variance (1/(N-1));
    Algorithm 1 uses 1/N instead, exposed here as ``ddof``.
  * Sec. 4.2, Eq. gPC, Eq. coef_integral, Eq. coef_discrete: orthonormal basis
    (gamma_k = 1) and the discrete projection c_k = sum_j a_j M(Z_j) Phi_k(Z_j).
  * Eq. gpc_mean and Eq. gpc_std: mean = c_0, variance = sum of the squared
    non-constant coefficients (the upper summation limit in the paper is garbled;
    read as all K-1 non-constant terms).
  * Sec. 6.2-6.3 (sampling strategies and quadrature rules): tensor-product
    Gauss-Legendre collocation and seeded Monte Carlo draws from a joint
    distribution of independent uniforms (Sec. 8.3 code sample ``joint``).

Readings where the paper is silent (all listed in the design notes): tensor grids are
lexicographic with the last dimension fastest; the total-degree basis is ordered by
degree, then by exponent tuples in descending lexicographic order; Monte Carlo draws
use Philox4x32-10 (Salmon et al., SC'11) with key = seed and counter = (sample index
low, high, dimension, 0), u = ((x1 << 32 | x0) >> 11) * 2^-53.
"""
from __future__ import annotations

import math
from itertools import product

import numpy as np

# --------------------------------------------------------------------------------------
# Gauss-Legendre quadrature (textbook Newton iteration on P_n)
# --------------------------------------------------------------------------------------


def legendre_p_and_derivative(n: int, x: float) -> tuple[float, float]:
    """P_n(x) and P_n'(x) by the three-term recurrence (k+1)P_{k+1} = (2k+1)xP_k - kP_{k-1}."""
    p_prev, p = 1.0, x
    if n == 0:
        return 1.0, 0.0
    for k in range(1, n):
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    # P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1)
    dp = n * (x * p - p_prev) / (x * x - 1.0)
    return p, dp


def gauss_legendre(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre rule on [-1, 1]: nodes ascending, weights summing to 2."""
    if n < 1:
        raise ValueError("n must be >= 1")
    nodes = np.empty(n)
    weights = np.empty(n)
    for j in range(n):
        x = math.cos(math.pi * (j + 0.75) / (n + 0.5))
        for _ in range(100):
            p, dp = legendre_p_and_derivative(n, x)
            dx = p / dp
            x -= dx
            if abs(dx) < 1e-16:
                break
        _, dp = legendre_p_and_derivative(n, x)
        nodes[j] = x
        weights[j] = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(nodes)
    return nodes[order], weights[order]


# --------------------------------------------------------------------------------------
# Distributions and sample sets
# --------------------------------------------------------------------------------------


def map_uniform(xi: np.ndarray, a: float, b: float) -> np.ndarray:
    """Affine map of reference points xi in [-1, 1] onto [a, b]."""
    return 0.5 * (a + b) + 0.5 * (b - a) * xi


def tensor_grid(pts_per_dim: list[int], bounds: list[tuple[float, float]]):
    """Tensor-product Gauss-Legendre collocation set for independent uniforms.

    Returns (Z [S x d] physical nodes, XI [S x d] reference nodes, a [S] weights of the
    uniform probability measure, summing to 1).  Last dimension varies fastest.
    """
    rules = [gauss_legendre(n) for n in pts_per_dim]
    d = len(rules)
    rows_xi, rows_a = [], []
    for idx in product(*[range(n) for n in pts_per_dim]):
        rows_xi.append([rules[k][0][idx[k]] for k in range(d)])
        w = 1.0
        for k in range(d):
            w *= 0.5 * rules[k][1][idx[k]]
        rows_a.append(w)
    xi = np.array(rows_xi, dtype=np.float64).reshape(-1, d)
    a = np.array(rows_a, dtype=np.float64)
    z = np.column_stack([map_uniform(xi[:, k], *bounds[k]) for k in range(d)])
    return z, xi, a


MASK32 = 0xFFFFFFFF
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr: tuple[int, int, int, int], key: tuple[int, int]) -> tuple[int, int, int, int]:
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11), on Python integers."""
    x0, x1, x2, x3 = (c & MASK32 for c in ctr)
    k0, k1 = (k & MASK32 for k in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * x0
        p1 = PHILOX_M1 * x2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return x0, x1, x2, x3


def mc_uniform01(n: int, d: int, seed: int) -> np.ndarray:
    """[n x d] uniforms in [0, 1) from Philox4x32-10, counter = (s lo, s hi, dim, 0), key = seed."""
    out = np.empty((n, d))
    key = (seed & MASK32, (seed >> 32) & MASK32)
    for s in range(n):
        for k in range(d):
            x0, x1, _, _ = philox4x32_10((s & MASK32, (s >> 32) & MASK32, k, 0), key)
            out[s, k] = ((x1 << 32 | x0) >> 11) * 2.0 ** -53
    return out


def mc_samples(n: int, bounds: list[tuple[float, float]], seed: int):
    """Seeded Monte Carlo draws from independent uniforms: (Z [n x d], XI [n x d])."""
    u = mc_uniform01(n, len(bounds), seed)
    z = np.column_stack([a + (b - a) * u[:, k] for k, (a, b) in enumerate(bounds)])
    return z, 2.0 * u - 1.0


# --------------------------------------------------------------------------------------
# Orthonormal Legendre chaos
# --------------------------------------------------------------------------------------


def multi_indices(d: int, order: int, kind: str = "total") -> np.ndarray:
    """Exponent set: total degree (|alpha| <= order) or tensor (max alpha <= order).

    Ordered by |alpha|, then by alpha in descending lexicographic order.
    """
    cand = [a for a in product(range(order + 1), repeat=d)
            if (sum(a) <= order if kind == "total" else max(a) <= order)]
    cand.sort(key=lambda a: (sum(a), tuple(-x for x in a)))
    return np.array(cand, dtype=np.int64).reshape(-1, d)


def phi_1d(n: int, xi: np.ndarray) -> np.ndarray:
    """Orthonormal Legendre polynomial sqrt(2n+1) P_n(xi) w.r.t. the uniform law on [-1, 1]."""
    xi = np.asarray(xi, dtype=np.float64)
    p_prev = np.ones_like(xi)
    if n == 0:
        return p_prev
    p = xi.copy()
    for k in range(1, n):
        p_prev, p = p, ((2 * k + 1) * xi * p - k * p_prev) / (k + 1)
    return math.sqrt(2 * n + 1) * p


def basis_matrix(alpha: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Phi[k, s] = prod_d phi_{alpha[k, d]}(xi[s, d])."""
    K, d = alpha.shape
    out = np.ones((K, xi.shape[0]))
    for k in range(K):
        for j in range(d):
            out[k] *= phi_1d(int(alpha[k, j]), xi[:, j])
    return out


def weight_matrix(alpha: np.ndarray, xi: np.ndarray, a: np.ndarray) -> np.ndarray:
    """W[k, s] = a_s Phi_k(xi_s): Eq. coef_discrete written as a matrix (gamma_k = 1)."""
    return basis_matrix(alpha, xi) * a[None, :]


def gpc_coefficients(alpha, xi, a, m: np.ndarray) -> np.ndarray:
    """c[k, f] = sum_s a_s Phi_k(xi_s) M[s, f] (Eq. coef_discrete)."""
    return weight_matrix(alpha, xi, a) @ np.asarray(m, dtype=np.float64)


def gpc_mean_var(c: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Eq. gpc_mean / Eq. gpc_std: mean = c_0, var = sum_{k >= 1} c_k^2."""
    return c[0].copy(), (c[1:] ** 2).sum(axis=0)


def mc_mean_var(m: np.ndarray, ddof: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Eq. meanMCS and Eq. varMCS (ddof = 1); Algorithm 1's 1/N form is ddof = 0."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    mean = m.sum(axis=0) / n
    var = ((m - mean[None, :]) ** 2).sum(axis=0) / (n - ddof)
    return mean, var


def relative_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 over all entries."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# --------------------------------------------------------------------------------------
# Closed forms used as pins
# --------------------------------------------------------------------------------------


def tgv_k_analytic(nu, k: float, t: float):
    """Normalised kinetic energy of the TGV for u0 = u_ref: K(t) = exp(-2t/t_d), t_d = 1/(2 nu k^2)."""
    return np.exp(-4.0 * np.asarray(nu, dtype=np.float64) * k * k * t)


def tgv_mean_k_uniform_nu(a: float, b: float, k: float, t: float) -> float:
    """E[K(t)] for nu ~ U(a, b): (e^{-ca} - e^{-cb}) / (c (b - a)), c = 4 k^2 t."""
    c = 4.0 * k * k * t
    return (math.exp(-c * a) - math.exp(-c * b)) / (c * (b - a))


def tgv_second_moment_k_uniform_nu(a: float, b: float, k: float, t: float) -> float:
    """E[K(t)^2] for nu ~ U(a, b): the same integral with rate 2c."""
    c = 8.0 * k * k * t
    return (math.exp(-c * a) - math.exp(-c * b)) / (c * (b - a))


def unit_converter(n: int, ma: float, re: float) -> dict:
    """Lattice parameters of the 4-D TGV set-up (Sec. 8.3, Table of simulation parameters).

    Domain length 2 pi resolved by n nodes: dx = 2 pi / (n - 1); dt = (Ma / sqrt 3) dx
    (lattice velocity = Ma c_s with c_s = 1/sqrt 3 in lattice units and unit physical
    velocity); physical nu = 1 / Re; tau = 3 nu dt / dx^2 + 1/2.
    """
    dx = 2.0 * math.pi / (n - 1)
    dt = ma / math.sqrt(3.0) * dx
    nu = 1.0 / re
    tau = 3.0 * nu * dt / (dx * dx) + 0.5
    return {"dx": dx, "dt": dt, "tau": tau, "nu_lattice": nu * dt / (dx * dx)}


# --------------------------------------------------------------------------------------
# Sparse grids and quasi Monte Carlo (Sec. 4.1 QMC, Sec. 6.3 Clenshaw-Curtis and Smolyak)
# --------------------------------------------------------------------------------------


def clenshaw_curtis(m: int) -> tuple[np.ndarray, np.ndarray]:
    """m-point Clenshaw-Curtis rule on [-1, 1]: nodes cos(pi j/(m-1)) ascending, weights summing
    to 2 (explicit cosine-sum weights, Trefethen SIAM Rev. 2008, Eq. 2.2 family)."""
    if m == 1:
        return np.array([0.0]), np.array([2.0])
    n = m - 1
    theta = np.pi * np.arange(m) / n
    w = np.empty(m)
    for j in range(m):
        s = 0.0
        for k in range(1, n // 2 + 1):
            b = 1.0 if 2 * k == n else 2.0
            s += b / (4.0 * k * k - 1.0) * math.cos(2.0 * k * theta[j])
        c = 1.0 if j in (0, n) else 2.0
        w[j] = c / n * (1.0 - s)
    x = np.cos(theta)
    order = np.argsort(x)
    return x[order], w[order]


def cc_points(level: int) -> int:
    """Nested Clenshaw-Curtis sizes: 1 point at level 1, 2^(l-1) + 1 after."""
    return 1 if level == 1 else 2 ** (level - 1) + 1


def smolyak_cc(d: int, level: int):
    """Smolyak sparse grid on [-1, 1]^d from nested Clenshaw-Curtis rules (combination form):
    A(q, d) = sum_{q-d+1 <= |i| <= q} (-1)^(q-|i|) C(d-1, q-|i|) U^{i_1} x ... x U^{i_d},
    q = d + level, i_j >= 1.  Nested nodes are merged by their index on the finest 1-D grid.
    Returns (XI [S x d], weights [S] of the uniform probability measure)."""
    q = d + level
    finest = cc_points(level + 1)
    acc: dict = {}
    for idx in product(range(1, level + 2), repeat=d):
        s = sum(idx)
        if s < q - d + 1 or s > q:
            continue
        coef = (-1) ** (q - s) * math.comb(d - 1, q - s)
        rules = [clenshaw_curtis(cc_points(i)) for i in idx]
        for pts in product(*[range(len(r[0])) for r in rules]):
            key = []
            w = float(coef)
            for dim, (i, j) in enumerate(zip(idx, pts)):
                m = cc_points(i)
                key.append((finest - 1) // 2 if m == 1 else j * ((finest - 1) // (m - 1)))
                w *= 0.5 * rules[dim][1][j]
            key = tuple(key)
            acc[key] = acc.get(key, 0.0) + w
    keys = sorted(acc)
    xf, _ = clenshaw_curtis(finest)
    xi = np.array([[xf[k] for k in key] for key in keys]).reshape(-1, d)
    a = np.array([acc[k] for k in keys])
    return xi, a


def radical_inverse(i: int, base: int) -> float:
    """Van der Corput radical inverse of i in the given base."""
    f, r = 1.0, 0.0
    while i > 0:
        f /= base
        r += f * (i % base)
        i //= base
    return r


FIRST_PRIMES = [2, 3, 5, 7, 11, 13, 17, 19]


def halton(n: int, d: int, skip: int = 1) -> np.ndarray:
    """[n x d] Halton points in [0, 1): point s has coordinate k = radical inverse of s + skip
    in the k-th prime base."""
    return np.array([[radical_inverse(s + skip, FIRST_PRIMES[k]) for k in range(d)] for s in range(n)]).reshape(n, d)


def wasserstein1(a, b) -> float:
    """1-Wasserstein distance of two empirical distributions on the real line (equal weights per
    value): the integral of |F_a - F_b| over x, evaluated exactly on the merged sorted values
    (Sec. 8.3, W1 of statistical solutions of |u|)."""
    a = np.sort(np.asarray(a, dtype=np.float64).ravel())
    b = np.sort(np.asarray(b, dtype=np.float64).ravel())
    allv = np.concatenate([a, b])
    allv.sort(kind="mergesort")
    deltas = np.diff(allv)
    fa = np.searchsorted(a, allv[:-1], side="right") / a.size
    fb = np.searchsorted(b, allv[:-1], side="right") / b.size
    return float(np.sum(np.abs(fa - fb) * deltas))
