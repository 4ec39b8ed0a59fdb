"""Pins of the FP64 UQ oracle (oracle/uq.py) against closed forms, published vectors and
mathematics that do not depend on the oracle itself.  CPU only."""
import math
import os
from itertools import product

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import uq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]


def _expr(s):
    return eval(s, {"sqrt": math.sqrt, "__builtins__": {}})  # closed forms of the fixture only


def test_gauss_legendre_5_closed_form():
    x, w = uq.gauss_legendre(5)
    rows = [r.split("|") for r in _rows("gauss_legendre_5.txt")]
    for j, (xe, we, xt, wt) in enumerate(rows):
        assert x[j] == pytest.approx(_expr(xe), abs=2e-16)
        assert w[j] == pytest.approx(_expr(we), abs=2e-16)
        assert x[j] == pytest.approx(float(xt), abs=1e-15)
        assert w[j] == pytest.approx(float(wt), abs=1e-15)


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = uq.gauss_legendre(n)
    assert np.all(np.diff(x) > 0) and abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs((w * x ** k).sum() - exact) < 2e-14, k
    # the rule is not exact at degree 2n (its error constant is non-zero)
    k = 2 * n
    assert abs((w * x ** k).sum() - 2.0 / (k + 1)) > 1e-11


def test_tensor_grid_order_and_weights():
    bounds = [(0.02, 0.06), (0.008, 0.012)]
    z, xi, a = uq.tensor_grid([3, 2], bounds)
    x3, w3 = uq.gauss_legendre(3)
    x2, w2 = uq.gauss_legendre(2)
    assert z.shape == (6, 2) and abs(a.sum() - 1.0) < 1e-15
    # last dimension fastest
    assert np.allclose(xi[:, 1], np.tile(x2, 3)) and np.allclose(xi[:, 0], np.repeat(x3, 2))
    assert np.allclose(a, np.outer(w3 / 2, w2 / 2).ravel(), rtol=0, atol=1e-16)
    assert np.allclose(z[:, 0], 0.04 + 0.02 * xi[:, 0]) and np.allclose(z[:, 1], 0.01 + 0.002 * xi[:, 1])


def test_multi_index_total_degree_order_and_count():
    al = uq.multi_indices(2, 2)
    assert al.tolist() == [[0, 0], [1, 0], [0, 1], [2, 0], [1, 1], [0, 2]]
    assert len(uq.multi_indices(4, 4)) == math.comb(8, 4) == 70
    assert len(uq.multi_indices(1, 8)) == 9
    assert len(uq.multi_indices(3, 2, "tensor")) == 27


@pytest.mark.parametrize("n", range(0, 9))
def test_phi_matches_library_legendre(n):
    xi = np.linspace(-1, 1, 17)
    assert np.allclose(uq.phi_1d(n, xi), math.sqrt(2 * n + 1) * eval_legendre(n, xi), rtol=0, atol=1e-13)


def test_discrete_orthonormality_5pow4_total_degree_4():
    """Sum_s a_s Phi_k Phi_l = delta_kl: per-dimension degree <= 8 <= 2*5-1 = 9."""
    b = [(0.02, 0.06), (0.008, 0.012), (-0.1, 0.1), (-0.1, 0.1)]
    _, xi, a = uq.tensor_grid([5] * 4, b)
    al = uq.multi_indices(4, 4)
    phi = uq.basis_matrix(al, xi)
    gram = (phi * a[None, :]) @ phi.T
    assert np.abs(gram - np.eye(len(al))).max() < 1e-13


def test_projection_reproduces_polynomials():
    """A QoI that is a polynomial in the basis span is reproduced exactly (Eq. coef_discrete)."""
    rng = np.random.default_rng(7)
    _, xi, a = uq.tensor_grid([4, 4, 4], [(-1, 1)] * 3)
    al = uq.multi_indices(3, 3)
    c_true = rng.normal(size=(len(al), 5))
    m = uq.basis_matrix(al, xi).T @ c_true          # M[s, f]
    c = uq.gpc_coefficients(al, xi, a, m)
    assert np.abs(c - c_true).max() < 1e-12
    mean, var = uq.gpc_mean_var(c)
    assert np.allclose(mean, c_true[0], atol=1e-12)
    assert np.allclose(var, (c_true[1:] ** 2).sum(0), rtol=1e-12)


def test_gpc_stats_against_closed_form_tgv_energy():
    """cfg-1 form: nu ~ U(0.02, 0.06), K(t) = exp(-4 nu k^2 t); 5-point rule vs closed forms."""
    k, t = 2 * math.pi / 64, 1000.0
    z, xi, a = uq.tensor_grid([5], [(0.02, 0.06)])
    kval = uq.tgv_k_analytic(z[:, 0], k, t)[:, None]
    c = uq.gpc_coefficients(uq.multi_indices(1, 4), xi, a, kval)
    mean, var = uq.gpc_mean_var(c)
    ek = uq.tgv_mean_k_uniform_nu(0.02, 0.06, k, t)
    ek2 = uq.tgv_second_moment_k_uniform_nu(0.02, 0.06, k, t)
    # Gauss rule error for exp(-c nu) at n = 5: (c h)^10 / ... is ~1e-9 relative here
    assert abs(mean[0] - ek) / ek < 1e-8
    assert abs(var[0] - (ek2 - ek * ek)) / (ek2 - ek * ek) < 1e-4
    # the degree-4 coefficients match a 64-point reference projection of the analytic
    # function within the aliasing bound of the 5-point rule: products Phi_k Phi_j with
    # k + j >= 10 are not integrated exactly, |Phi_j| <= sqrt(2j + 1) on [-1, 1]
    z64, xi64, a64 = uq.tensor_grid([64], [(0.02, 0.06)])
    c64 = uq.gpc_coefficients(uq.multi_indices(1, 14), xi64, a64,
                              uq.tgv_k_analytic(z64[:, 0], k, t)[:, None])[:, 0]
    for kk in range(5):
        bound = sum(abs(c64[j]) * math.sqrt((2 * kk + 1) * (2 * j + 1)) for j in range(10 - kk, 15))
        assert abs(c[kk, 0] - c64[kk]) <= bound + 1e-15, kk


def test_philox_known_answers():
    for r in _rows("philox4x32_10_kat.txt"):
        v = [int(h, 16) for h in r.split()]
        assert uq.philox4x32_10(tuple(v[0:4]), tuple(v[4:6])) == tuple(v[6:10])


def test_mc_moments_equal_numpy():
    rng = np.random.default_rng(3)
    m = rng.normal(size=(257, 11)) * 3 + 1
    mean, var = uq.mc_mean_var(m, ddof=1)
    assert np.allclose(mean, m.mean(0), rtol=0, atol=1e-15 * 10)
    assert np.allclose(var, m.var(0, ddof=1), rtol=1e-14)
    _, var0 = uq.mc_mean_var(m, ddof=0)
    assert np.allclose(var0, m.var(0, ddof=0), rtol=1e-14)


def test_mc_uniforms_range_and_determinism():
    u1 = uq.mc_uniform01(512, 4, 123456)
    u2 = uq.mc_uniform01(512, 4, 123456)
    assert np.array_equal(u1, u2) and u1.min() >= 0.0 and u1.max() < 1.0
    assert not np.array_equal(u1, uq.mc_uniform01(512, 4, 123457))
    assert abs(u1.mean() - 0.5) < 0.02
    z, xi = uq.mc_samples(512, [(0.02, 0.06)] * 4, 123456)
    assert z.min() >= 0.02 and z.max() < 0.06 and np.allclose(xi, 2 * u1 - 1)


def test_mc_error_rate_half():
    """MC error of E[exp(-c nu)] shrinks like N^-1/2 (Sec. 4.1), averaged over 32 seeds."""
    k, t = 2 * math.pi / 64, 1000.0
    exact = uq.tgv_mean_k_uniform_nu(0.02, 0.06, k, t)
    ns = np.array([16, 64, 256, 1024])
    errs = []
    for n in ns:
        e = []
        for seed in range(32):
            z, _ = uq.mc_samples(int(n), [(0.02, 0.06)], 1000 + seed)
            mean, _ = uq.mc_mean_var(uq.tgv_k_analytic(z, k, t))
            e.append((mean[0] - exact) ** 2)
        errs.append(math.sqrt(np.mean(e)))
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert -0.6 < slope < -0.4, slope


def test_unit_converter_matches_paper_table():
    """Every printed entry is reproduced to one unit in its last (6th) decimal.  The table
    mixes rounding and truncation (2 pi / 7 = 0.8975979 is printed 0.897598, 2 pi / 127 =
    0.0494739 is printed 0.049473), so the pin is |computed - printed| <= 1e-6."""
    for r in _rows("tgv4d_simulation_parameters.txt"):
        n, ma, re, tau, dx, dt = [float(v) for v in r.split("|")]
        p = uq.unit_converter(int(n), ma, re)
        assert abs(p["tau"] - tau) <= 1e-6 + 1e-12
        assert abs(p["dx"] - dx) <= 1e-6 + 1e-12
        assert abs(p["dt"] - dt) <= 1e-6 + 1e-12


def test_relative_l2():
    assert uq.relative_l2([1.0, 2.0], [1.0, 2.0]) == 0.0
    assert uq.relative_l2([3.0, 4.0], [0.0, 4.0]) == pytest.approx(0.75)


def test_clenshaw_curtis_rules():
    for m in (1, 3, 5, 9, 17):
        x, w = uq.clenshaw_curtis(m)
        assert abs(w.sum() - 2.0) < 1e-14 and np.all(np.diff(x) > 0) if m > 1 else w[0] == 2.0
        deg = m if m % 2 == 1 else m - 1  # symmetric rule with m nodes is exact to degree m (m odd)
        for k in range(deg + 1):
            exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
            assert abs((w * x ** k).sum() - exact) < 1e-14, (m, k)
    x, w = uq.clenshaw_curtis(3)
    assert np.allclose(x, [-1, 0, 1]) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3])  # Simpson's rule


def _uniform_moment(alpha):
    return math.prod(1.0 / (a + 1) if a % 2 == 0 else 0.0 for a in alpha)


@pytest.mark.parametrize("d,level", [(1, 3), (2, 2), (3, 2), (4, 3)])
def test_smolyak_exact_to_total_degree_2k_plus_1(d, level):
    """Smolyak A(d + k, d) over nested Clenshaw-Curtis rules integrates every polynomial of total
    degree <= 2k + 1 exactly (Novak and Ritter 1996) and is not exact at degree 2k + 2."""
    xi, a = uq.smolyak_cc(d, level)
    assert abs(a.sum() - 1.0) < 1e-14
    top = 2 * level + 1
    for alpha in product(range(top + 1), repeat=d):
        if sum(alpha) > top:
            continue
        val = (a * np.prod(xi ** np.array(alpha)[None, :], axis=1)).sum()
        assert abs(val - _uniform_moment(alpha)) < 1e-13, alpha
    if d > 1:  # in one dimension the grid is a single Clenshaw-Curtis rule, exact beyond 2k + 1
        worst = max(abs((a * np.prod(xi ** np.array(al)[None, :], axis=1)).sum() - _uniform_moment(al))
                    for al in product(range(top + 2), repeat=d) if sum(al) == top + 1)
        assert worst > 1e-8


def test_smolyak_point_counts_and_the_papers_grid():
    assert [len(uq.smolyak_cc(4, k)[1]) for k in range(0, 5)] == [1, 9, 41, 137, 401]
    for r in _rows("smolyak_tgv4d_points.txt"):
        d, level, pts = (int(v) for v in r.split("|"))
        assert len(uq.smolyak_cc(d, level)[1]) == pts
    # a level-3 grid supports the order-3 basis: products of degree <= 6 <= 7 are integrated exactly
    xi, a = uq.smolyak_cc(4, 3)
    phi = uq.basis_matrix(uq.multi_indices(4, 3), xi)
    assert np.abs((phi * a[None, :]) @ phi.T - np.eye(phi.shape[0])).max() < 1e-12


def test_halton_radical_inverse_and_rate():
    assert [uq.radical_inverse(i, 2) for i in range(1, 8)] == [0.5, 0.25, 0.75, 0.125, 0.625, 0.375, 0.875]
    assert np.allclose([uq.radical_inverse(i, 3) for i in range(1, 5)], [1 / 3, 2 / 3, 1 / 9, 4 / 9])
    h = uq.halton(5, 3)
    assert np.allclose(h[0], [0.5, 1 / 3, 0.2]) and np.all((h >= 0) & (h < 1))
    # QMC error of a smooth 2-D integral decays close to N^-1 (Sec. 4.1), clearly faster than MC
    f = lambda u: np.exp(-(u[:, 0] + 0.5 * u[:, 1]))  # noqa: E731
    exact = (1 - math.exp(-1)) * (1 - math.exp(-0.5)) / 0.5
    ns = np.array([64, 256, 1024, 4096])
    errs = [abs(f(uq.halton(int(n), 2)).mean() - exact) for n in ns]
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert slope < -0.8, slope


def test_wasserstein1_exact_cases_and_library_cross_check():
    from scipy.stats import wasserstein_distance

    assert uq.wasserstein1([0.0, 1.0], [0.0, 1.0]) == 0.0
    assert uq.wasserstein1([0.0], [1.0]) == 1.0
    rng = np.random.default_rng(4)
    a = rng.normal(size=500)
    assert abs(uq.wasserstein1(a, a + 0.3) - 0.3) < 1e-12          # pure shift
    b = rng.exponential(size=333)
    assert abs(uq.wasserstein1(a, b) - wasserstein_distance(a, b)) < 1e-12
    assert abs(uq.wasserstein1(a, b) - uq.wasserstein1(b, a)) < 1e-12
