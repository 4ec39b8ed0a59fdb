"""Pins of the FP64 C LBM oracle (oracle/lbm_oracle.c) against closed forms, conservation
laws, symmetry and convergence orders.  CPU only; each case runs in seconds."""
import math

import numpy as np
import pytest

from oracle import lbm, uq


def _tgv(n, steps, nu=0.04, u0=0.01, **kw):
    return lbm.Case(lbm.TGV, n, n, steps, nu, u0, u_ref=kw.pop("u_ref", u0), **kw)


def test_rest_state_stays_at_rest():
    r = lbm.run([_tgv(16, 50, u0=0.0, u_ref=1.0)])[0]
    assert np.all(r.u == 0.0) and np.all(r.v == 0.0)
    assert np.allclose(r.rho, 1.0, rtol=0, atol=1e-15)


def test_tgv_conserves_mass_and_momentum():
    """Periodic BGK: sum f and sum c f are collision invariants and streaming permutes f."""
    c = _tgv(32, 1000, amp2=0.001, amp3=-0.0007)
    r = lbm.run([c])[0]
    assert abs(r.mass - 32 * 32) / (32 * 32) < 1e-13
    # initial momentum is zero by symmetry of the sine modes
    assert abs(r.mom_x) < 1e-13 * 32 * 32 and abs(r.mom_y) < 1e-13 * 32 * 32


def test_tgv_initial_energy_is_one():
    """sum sin^2(kx) cos^2(ky) = N^2/4 on the lattice, so K(0) = 1 when u0 = u_ref."""
    r = lbm.run([_tgv(64, 0, qoi_every=1)])[0]
    # u = (sum c f) / rho recovers u0 ~ 1e-2 from O(1) populations: ~1e-14 relative rounding
    assert abs(r.series[0] - 1.0) < 1e-12 and abs(r.k_final - 1.0) < 1e-12


def test_tgv_decay_matches_closed_form():
    """K(t) = exp(-4 nu k^2 t) (Sec. 8.2, t_d = 1 / (nu (kx^2 + ky^2))) within the O(dx^2) error."""
    n, nu = 64, 0.04
    r = lbm.run([_tgv(n, 1000, nu=nu, qoi_every=100)])[0]
    k = 2 * math.pi / n
    ref = uq.tgv_k_analytic(nu, k, np.arange(0, 1001, 100))
    assert np.all(np.abs(r.series - ref) / ref < 5e-3)
    # the per-sample velocity field decays as exp(-2 nu k^2 t) with the initial shape
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    dec = math.exp(-2 * nu * k * k * 1000)
    ua = 0.01 * np.sin(k * x) * np.cos(k * y) * dec
    va = -0.01 * np.cos(k * x) * np.sin(k * y) * dec
    err = uq.relative_l2(np.stack([r.u, r.v]), np.stack([ua, va]))
    assert err < 3e-3


def test_tgv_second_order_under_diffusive_refinement():
    """N = 16/32/64 at fixed tau, u0 ~ 1/N, T ~ N^2: L2 error of u falls as N^-2."""
    errs = []
    ns = [16, 32, 64]
    for n in ns:
        steps = int(60 * (n / 16) ** 2)
        u0 = 0.04 * 16 / n
        r = lbm.run([_tgv(n, steps, nu=0.05, u0=u0)])[0]
        k = 2 * math.pi / n
        x = np.arange(n)[None, :]
        y = np.arange(n)[:, None]
        dec = math.exp(-2 * 0.05 * k * k * steps)
        ua = u0 * np.sin(k * x) * np.cos(k * y) * dec
        va = -u0 * np.cos(k * x) * np.sin(k * y) * dec
        errs.append(uq.relative_l2(np.stack([r.u, r.v]), np.stack([ua, va])))
    order = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert 1.85 < order < 2.15, (errs, order)


def _channel(h, nu=0.1, **kw):
    u = 0.02 * 10 / h
    return lbm.Case(lbm.CHANNEL, 4 * h, h, int(6 * h * h / nu), nu, u, u_ref=0.0, **kw)


def test_channel_poiseuille_profile_second_order():
    """Walls (halfway bounce-back) + velocity inlet + pressure outlet: the developed profile is
    the inlet parabola 4 u_max y (H - y) / H^2 (Sec. 8.1 inflow), to second order in H."""
    errs = []
    for h in (10, 20):
        c = _channel(h)
        r = lbm.run([c])[0]
        y = np.arange(h) + 0.5
        ua = 4 * 1.5 * c.u0 * y * (h - y) / h ** 2
        prof = r.u[:, 2 * h]
        errs.append(np.linalg.norm(prof - ua) / np.linalg.norm(ua))
        assert np.abs(r.v[:, 2 * h]).max() < 1e-4 * c.u0   # no cross-flow in the developed part
    assert errs[0] < 0.03
    order = math.log(errs[0] / errs[1], 2)
    assert 1.8 < order < 2.2, (errs, order)


def test_interpolated_inlet_outlet_poiseuille():
    """Interpolated (finite-difference) inlet and pressure outlet on the end columns (Sec. 8.1,
    Latt et al. 2008): the developed profile is the inlet parabola to second order in H, the
    column next to the inlet already carries it (the boundary populations hold the right
    non-equilibrium part: a wrong sign, a missing or halved shear term makes that column and the
    cross-flow an order of magnitude worse), and the outflow balances the inflow."""
    mids = []
    for h, col_tol, v_tol in ((10, 2.5e-3, 1e-4), (20, 5e-4, 2.5e-5)):
        c = _channel(h, inout_bc=lbm.INTERPOLATED)
        r = lbm.run([c])[0]
        y = np.arange(h) + 0.5
        ua = 4 * 1.5 * c.u0 * y * (h - y) / h ** 2
        err = lambda x: np.linalg.norm(r.u[:, x] - ua) / np.linalg.norm(ua)  # noqa: E731
        assert err(0) < 1e-12                      # the inlet column carries the imposed velocity
        assert err(1) < col_tol, err(1)
        assert np.abs(r.v).max() < v_tol, np.abs(r.v).max()
        qin, qout = (r.rho[:, 0] * r.u[:, 0]).sum(), (r.rho[:, -1] * r.u[:, -1]).sum()
        assert abs(qout / qin - 1) < 5e-3
        assert np.abs(r.rho[:, -1] - 1).max() < 1e-12   # pressure outlet: rho = 1 on the column
        mids.append(err(2 * h))
    order = math.log(mids[0] / mids[1], 2)
    assert mids[0] < 0.03 and 1.8 < order < 2.2, (mids, order)


def test_channel_without_obstacle_has_no_force():
    r = lbm.run([_channel(10)])[0]
    assert r.cd == 0.0 and r.cl == 0.0


def _cyl(nd, steps, cy=None, **kw):
    dx = 0.1 / nd
    nx, ny = round(2.2 / dx), round(0.41 / dx)
    u = 0.04
    return lbm.Case(lbm.CHANNEL, nx, ny, steps, u * nd / 20.0, u, u_ref=0.0, cyl_cx=0.2 / dx,
                    cyl_cy=(0.2 / dx) if cy is None else cy, cyl_r=0.05 / dx,
                    ramp_steps=kw.pop("ramp", 0), **kw)


def test_obstacle_mask_is_staircase_circle():
    c = _cyl(20, 1)
    m = lbm.obstacle_mask(c).astype(bool)
    yy, xx = np.mgrid[0:c.ny, 0:c.nx]
    inside = ((xx + 0.5 - 40.0) ** 2 + (yy + 0.5 - 40.0) ** 2) < 100.0
    assert np.array_equal(m, inside)
    # a 20-node-diameter disc covers close to pi r^2 = 314 nodes
    assert abs(m.sum() - math.pi * 100) < 20


@pytest.mark.parametrize("bc,inout", [(lbm.HALFWAY, lbm.FACE), (lbm.BOUZIDI, lbm.FACE),
                                       (lbm.BOUZIDI, lbm.INTERPOLATED)])
def test_symmetric_obstacle_gives_mirror_flow_and_no_lift(bc, inout):
    """Obstacle centred in the channel: the y -> H - y mirror maps the flow onto itself, so
    v is odd, u and rho are even, and the lift vanishes to round-off."""
    nd = 10
    c = _cyl(nd, 1500, cy=0.205 / (0.1 / nd), qoi_every=100, obstacle_bc=bc, inout_bc=inout)
    r = lbm.run([c])[0]
    assert np.allclose(r.u, r.u[::-1, :], rtol=0, atol=1e-14)
    assert np.allclose(r.v, -r.v[::-1, :], rtol=0, atol=1e-14)
    assert np.allclose(r.rho, r.rho[::-1, :], rtol=0, atol=1e-13)
    assert abs(r.cl) < 1e-10 and r.cd > 0.0


def _golden_rows(name):
    return [[v.strip() for v in r.split("|")] for r in open(__file__.replace("test_oracle_lbm.py", "golden/" + name))
            if r.strip() and not r.startswith("#")]


@pytest.mark.slow
def test_cylinder_drag_loose_anchor_and_bouzidi_against_the_benchmark():
    """Steady nominal drag at 10 nodes per diameter.  Halfway bounce-back on the staircase: within
    10% of the paper's deterministic value at n_x = 20 (Sec. 8.1, table of C_D statistics), a
    loose anchor since the paper's boundary schemes differ.  Bouzidi interpolated bounce-back (the
    paper's obstacle scheme): within 3% of the Schaefer-Turek 2D-1 reference interval, the set-up
    this channel reproduces, and at most half the staircase's error there (an interpolated wall
    removes the staircase's first-order geometry error)."""
    cd_paper = float([r for r in _golden_rows("cylinder_table1.txt") if r[0] == "deterministic"][0][1])
    st = {r[0]: (float(r[1]), float(r[2])) for r in _golden_rows("schafer_turek_2d1.txt")}
    cd_ref = 0.5 * sum(st["c_D"])
    cases = [_cyl(10, 40000, qoi_every=100, steady_tol=1e-7, ramp=1000, obstacle_bc=bc)
             for bc in (lbm.HALFWAY, lbm.BOUZIDI)]
    cases.append(_cyl(10, 40000, qoi_every=100, steady_tol=1e-7, ramp=1000, obstacle_bc=lbm.BOUZIDI,
                      inout_bc=lbm.INTERPOLATED))
    half, bz, bzi = lbm.run(cases)
    # the paper's own boundary set (Bouzidi + interpolated inlet/outlet): a loose anchor within 5%
    # of its deterministic value (the end columns and the outlet's nodal pressure differ in
    # detail; C_D is within 1e-4 of its steady value at the step cap)
    assert abs(bzi.cd - cd_paper) / cd_paper < 0.05, bzi.cd
    assert half.steps_run < 40000 and bz.steps_run < 40000    # reached the steady-state criterion
    assert abs(half.cd - cd_paper) / cd_paper < 0.10, half.cd
    assert abs(half.cl) < 0.05 * half.cd                       # small lift from the 0.2 vs 0.205 offset
    err_half, err_bz = abs(half.cd - cd_ref) / cd_ref, abs(bz.cd - cd_ref) / cd_ref
    assert err_bz < 0.03 and err_bz < 0.5 * err_half, (bz.cd, half.cd)
    assert 0.0 < bz.cl < 2.0 * st["c_L"][1]


def test_bouzidi_link_fractions_are_the_circle_crossings():
    """Every link from a fluid node into the obstacle gets the fraction q in (0, 1) at which the
    segment from the node centre along c_i crosses the circle, found here independently by
    bisection on the sign of |P + s c_i - C|^2 - r^2."""
    c = _cyl(10, 1)
    m = lbm.obstacle_mask(c).astype(bool)
    n_links = 0
    for y in range(c.ny):
        for x in range(c.nx):
            if m[y, x]:
                continue
            for i, (ex, ey) in enumerate(((1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)), 1):
                if not (0 <= y + ey < c.ny and 0 <= x + ex < c.nx) or not m[y + ey, x + ex]:
                    continue
                n_links += 1
                q = lbm.link_fraction(c, x, y, i)
                g = lambda s: (x + 0.5 + s * ex - c.cyl_cx) ** 2 + (y + 0.5 + s * ey - c.cyl_cy) ** 2 - c.cyl_r ** 2  # noqa: E731
                lo, hi = 0.0, 1.0
                for _ in range(60):
                    mid = 0.5 * (lo + hi)
                    lo, hi = (mid, hi) if g(mid) > 0 else (lo, mid)
                assert 0.0 < q < 1.0 and abs(q - 0.5 * (lo + hi)) < 1e-12, (x, y, i, q)
    assert n_links > 4 * 10  # a 10-node diameter circle has tens of boundary links


def test_bouzidi_keeps_a_fluid_at_rest():
    """With no inflow (a ramp far longer than the run) every rule returns weighted averages of
    equal rest populations, so the fluid stays at rest to round-off and the obstacle feels no
    force (each lattice line through the closed obstacle enters it once along c_i and once along
    its opposite, so sum c_i w_i over the links cancels)."""
    for inout in (lbm.FACE, lbm.INTERPOLATED):
        r = lbm.run([_cyl(6, 200, qoi_every=50, ramp=10 ** 12, obstacle_bc=lbm.BOUZIDI, inout_bc=inout)])[0]
        assert np.abs(r.u).max() < 1e-13 and np.abs(r.v).max() < 1e-13   # round-off over 200 steps
        assert abs(r.cd) < 1e-10 and abs(r.cl) < 1e-10                     # F ~ 1e-14 times 2/(u0^2 D)


def test_perturbed_tgv_without_perturbation_is_a_tiled_shifted_tgv():
    """Sec. 8.3 initial field with zeta = 0 on N nodes is the Sec. 8.2 field on N/2 nodes, tiled
    2 x 2 and shifted by N/8 (-cos a sin b = sin(a - pi/2) cos(b - pi/2), and the pressure
    -(cos 4x + cos 4y)/4 maps onto +(cos 2kx + cos 2ky)/4); BGK streaming is translation-covariant,
    so the evolved fields agree to round-off."""
    n, steps, nu, u0 = 32, 150, 0.03, 0.04
    a = lbm.run([lbm.Case(lbm.TGV_PERTURBED, n, n, steps, nu, u0, u_ref=u0)])[0]
    b = lbm.run([lbm.Case(lbm.TGV, n // 2, n // 2, steps, nu, u0, u_ref=u0)])[0]
    s = n // 8
    bu = np.roll(np.roll(np.tile(b.u, (2, 2)), s, axis=0), s, axis=1)
    bv = np.roll(np.roll(np.tile(b.v, (2, 2)), s, axis=0), s, axis=1)
    assert np.abs(a.u - bu).max() < 1e-14 and np.abs(a.v - bv).max() < 1e-14
    assert abs(a.k_final - b.k_final) < 1e-13


@pytest.mark.parametrize("which,linear", [(0, 0.0), (1, 0.0), (2, 0.0), (3, -0.125)])
def test_perturbed_tgv_initial_energy_closed_form(which, linear):
    """K(0) u_ref^2 = u0^2 + c u0 zeta + zeta^2/64 for a single perturbation amplitude zeta_ij,
    from the lattice sums of products of sin/cos(2x), sin/cos(4x) (N > 8): only the cos-cos
    mode (i = j = 1) correlates with the base field, giving c = -1/8."""
    n, u0, z = 32, 0.04, 0.02
    pert = [0.0] * 4
    pert[which] = z
    r = lbm.run([lbm.Case(lbm.TGV_PERTURBED, n, n, 0, 0.03, u0, u_ref=1.0, pert=tuple(pert))])[0]
    assert abs(r.k_final - (u0 * u0 + linear * u0 * z + z * z / 64)) < 1e-15


def test_perturbed_tgv_conserves_mass():
    r = lbm.run([lbm.Case(lbm.TGV_PERTURBED, 24, 24, 300, 0.02, 0.05, u_ref=0.05,
                          pert=(0.01, -0.02, 0.015, 0.005))])[0]
    # initial mass: sum of 1 + 3p with p quadratic in U; compare with the state after 300 steps
    r0 = lbm.run([lbm.Case(lbm.TGV_PERTURBED, 24, 24, 0, 0.02, 0.05, u_ref=0.05,
                           pert=(0.01, -0.02, 0.015, 0.005))])[0]
    assert abs(r.mass - r0.mass) < 1e-12 * r0.mass
