"""Synthetic workloads: the case descriptions and seeded random inputs shared by the tests, the
benchmark and the oracle runs.  This module holds no arithmetic of the method itself (no
quadrature, no lattice Boltzmann, no projection): only parameters, sizes and seeded draws.

Workloads (lattice units; tau = 3 nu + 1/2):
  * tgv64_gpc:  Taylor-Green vortex 64 x 64, nu ~ U(0.02, 0.06), u0 = 0.01, 5 Gauss-Legendre
    points, total degree 4, 1000 steps, FP64 (the plain small case).
  * tgv256_gpc4d: Taylor-Green vortex 256 x 256 with 4-D uncertainty (nu ~ U(0.02, 0.06),
    u0 ~ U(0.008, 0.012), zeta2, zeta3 ~ U(-0.1, 0.1) scaling the 2k and 3k modes by u0),
    5^4 = 625 tensor Gauss-Legendre samples, total degree 4 (70 terms), 2000 steps, FP32.
  * tgv512_mc4d: the same 4-D set-up at 512 x 512 with 4096 seeded Monte Carlo samples.
  * cylinder: channel 2.2 x 0.41 with a D = 0.1 cylinder at (0.2, 0.2), nd nodes per diameter,
    mean inflow u ~ U(0.9, 1.1) x 0.04 at nu = 0.04 nd / 20 (Re 18..22), 9 Gauss-Legendre
    samples, degree 8, run to steady state.
  * uneven: 256 TGV samples of random size in {128, 256, 512}^2 with per-sample nu and step
    counts, plus 64 cylinder samples at 20..40 nodes per diameter.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

TGV, CHANNEL, TGV_PERTURBED = 0, 1, 2
U_REF = 0.01  # normaliser of the kinetic energy K(t)


@dataclass
class SampleSpec:
    """One deterministic run, mirroring the fields of ``uqlb_sample``."""
    kind: int
    nx: int
    ny: int
    steps: int
    nu: float
    u0: float
    amp2: float = 0.0
    amp3: float = 0.0
    u_ref: float = U_REF
    cyl_cx: float = 0.0
    cyl_cy: float = 0.0
    cyl_r: float = 0.0
    ramp_steps: int = 0
    steady_tol: float = 0.0
    steady_checks: int = 1
    pert: tuple = (0.0, 0.0, 0.0, 0.0)
    obstacle_bc: int = 0    # channel obstacle: 0 halfway bounce-back, 1 Bouzidi
    inout_bc: int = 0       # channel inlet/outlet: 0 at the end faces, 1 interpolated on the end columns


@dataclass
class Workload:
    name: str
    base: SampleSpec
    bounds: list            # uniform input bounds, one (a, b) per dimension
    params: list            # parameter driven by each dimension: "nu", "u0", "zeta2", "zeta3"
    method: str             # "gpc", "mc" or "qmc"
    pts_per_dim: int = 5    # Gauss-Legendre points per input, or the Smolyak level
    quad: str = "gl"        # "gl" (tensor Gauss-Legendre) or "smolyak" (Clenshaw-Curtis sparse grid)
    order: int = 4
    n_mc: int = 0
    seed: int = 123456      # the seed of the paper's Monte Carlo example
    storage: str = "f32"
    qoi_every: int = 0
    extra: dict = field(default_factory=dict)


def tgv(n: int, steps: int, nu: float = 0.04, u0: float = U_REF, amp2: float = 0.0, amp3: float = 0.0) -> SampleSpec:
    return SampleSpec(TGV, n, n, steps, nu, u0, amp2, amp3)


OBSTACLE_BC = {"halfway": 0, "bouzidi": 1}
INOUT_BC = {"face": 0, "interpolated": 1}


def channel(nd: int, u_mean: float = 0.04, steps: int = 200000, steady_tol: float = 1e-8,
            ramp: bool = True, re: float = 20.0, obstacle: bool = True, bc: str = "halfway",
            inout: str = "face") -> SampleSpec:
    """Channel 2.2 x 0.41 (D = 0.1) resolved with nd nodes per diameter (ny = floor(4.1 nd));
    nu from Re at the nominal lattice velocity 0.04; bc: obstacle scheme, "halfway" bounce-back
    on the staircase or "bouzidi" interpolated bounce-back; inout: inlet/outlet scheme, "face"
    (moving-wall inlet, anti-bounce-back outlet) or "interpolated" (on the end columns)."""
    nx, ny = 22 * nd, (41 * nd) // 10
    nu = 0.04 * nd / re
    r = 0.5 * nd if obstacle else 0.0
    return SampleSpec(CHANNEL, nx, ny, steps, nu, u_mean, u_ref=0.0, cyl_cx=2.0 * nd, cyl_cy=2.0 * nd, cyl_r=r,
                      ramp_steps=(2000 * nd) // 20 if ramp else 0, steady_tol=steady_tol,
                      obstacle_bc=OBSTACLE_BC[bc], inout_bc=INOUT_BC[inout])


TGV4D_BOUNDS = [(0.02, 0.06), (0.008, 0.012), (-0.1, 0.1), (-0.1, 0.1)]
TGV4D_PARAMS = ["nu", "u0", "zeta2", "zeta3"]


def tgv64_gpc(steps: int = 1000) -> Workload:
    return Workload("tgv64_gpc", tgv(64, steps), [(0.02, 0.06)], ["nu"], "gpc", pts_per_dim=5, order=4,
                    storage="f64")


def tgv256_gpc4d(n: int = 256, steps: int = 2000, pts: int = 5, storage: str = "f32") -> Workload:
    return Workload("tgv256_gpc4d", tgv(n, steps), TGV4D_BOUNDS, TGV4D_PARAMS, "gpc", pts_per_dim=pts, order=4,
                    storage=storage)


def tgv_smolyak4d(n: int = 256, steps: int = 2000, level: int = 3, order: int = 3, storage: str = "f32") -> Workload:
    """The 4-D set-up on the Clenshaw-Curtis Smolyak grid (level 3: 137 samples, order-3 basis)."""
    return Workload("tgv_smolyak4d", tgv(n, steps), TGV4D_BOUNDS, TGV4D_PARAMS, "gpc", pts_per_dim=level,
                    order=order, quad="smolyak", storage=storage)


def tgv512_mc4d(n: int = 512, steps: int = 2000, n_mc: int = 4096, storage: str = "f32") -> Workload:
    return Workload("tgv512_mc4d", tgv(n, steps), TGV4D_BOUNDS, TGV4D_PARAMS, "mc", n_mc=n_mc, storage=storage)


def cylinder_gpc(nd: int = 20, pts: int = 9, order: int = 8, steps: int = 200000, steady_tol: float = 1e-8,
                 storage: str = "f32", steady_checks: int = 0, bc: str = "halfway", inout: str = "face") -> Workload:
    """Steady state: the relative change of C_D over 100 steps stays below steady_tol.  FP32 resolves
    C_D to ~1e-7, so below that tolerance it must hold at 5 consecutive checks (FP64: one)."""
    base = channel(nd, steps=steps, steady_tol=steady_tol, bc=bc, inout=inout)
    base.steady_checks = steady_checks or (1 if storage == "f64" else 5)
    return Workload("cylinder_gpc", base, [(0.9 * 0.04, 1.1 * 0.04)], ["u0"], "gpc", pts_per_dim=pts,
                    order=order, storage=storage, qoi_every=100)


def cylinder_uq(nd: int = 20, method: str = "gpc", n: int = 11, order: int = 5, spread: float = 0.2,
                steps: int = 200000, steady_tol: float = 1e-8, storage: str = "f64", seed: int = 123456,
                bc: str = "halfway", inout: str = "face") -> Workload:
    """The Sec. 8.1 method comparison: mean inflow U ~ U((1 - spread) U_nom, (1 + spread) U_nom) at
    fixed viscosity (the paper's +-20 %), U_nom = 0.04.  method "gpc": n Gauss-Legendre points and
    a degree-`order` expansion (the paper's reference uses 11 points, order 5); "mc" / "qmc": n
    Philox draws / Halton points.  Steady state as in cylinder_gpc."""
    base = channel(nd, steps=steps, steady_tol=steady_tol, bc=bc, inout=inout)
    base.steady_checks = 1 if storage == "f64" else 5
    bounds = [((1.0 - spread) * 0.04, (1.0 + spread) * 0.04)]
    if method == "gpc":
        return Workload("cylinder_uq", base, bounds, ["u0"], "gpc", pts_per_dim=n, order=order, storage=storage,
                        qoi_every=100)
    return Workload("cylinder_uq", base, bounds, ["u0"], method, n_mc=n, seed=seed, storage=storage, qoi_every=100)


def uneven_batch(seed: int = 2508, n_tgv: int = 256, n_cyl: int = 64) -> list[SampleSpec]:
    """Heterogeneous batch: TGV samples of random size and viscosity whose step counts give equal
    decay, T = clamp(round(1000 (0.04 / nu) (n / 256)^2), 500, 4000), plus channel samples."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_tgv):
        n = int(rng.choice([128, 256, 512]))
        nu = float(rng.uniform(0.02, 0.06))
        steps = int(min(max(round(1000 * (0.04 / nu) * (n / 256) ** 2), 500), 4000))
        out.append(tgv(n, steps, nu=nu))
    for _ in range(n_cyl):
        nd = int(rng.integers(20, 41))
        u = float(rng.uniform(0.9, 1.1) * 0.04)
        s = channel(nd, u_mean=u, steps=4000, steady_tol=0.0)
        out.append(s)
    return out


def random_fields(n_samples: int, n_fields: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded stand-in field matrix M[S x F] for projection/statistics tests."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n_samples, n_fields)) * 0.01 + 0.1).astype(dtype)


def with_steps(w: Workload, steps: int) -> Workload:
    return replace(w, base=replace(w.base, steps=steps))


# The paper's own four-dimensional perturbed Taylor-Green set-up (Sec. 8.3): resolutions n with
# Ma = 1.6 / n and Re = 40 n (its table of simulation parameters), T_max = 100, four amplitudes
# zeta_ij ~ U(-0.025, 0.025) in units of u0 = 1.  The periodic lattice has n - 1 nodes per side
# (dx = 2 pi / (n - 1) spans the period once); the lattice values come from uqlb_unit_converter.
PERT4D_BOUNDS = [(-0.025, 0.025)] * 4
PERT4D_PARAMS = ["pert00", "pert01", "pert10", "pert11"]


def tgv_paper4d_params(n: int) -> tuple[float, float]:
    """(Ma, Re) of resolution n in the paper's table."""
    return 1.6 / n, 40.0 * n


def tgv_paper4d(n: int, tau: float, u_lattice: float, steps: int, sampling: str = "mc", n_samples: int = 0,
                level: int = 3, order: int = 3, seed: int = 123456, storage: str = "f32") -> Workload:
    """The Sec. 8.3 set-up at resolution n; tau, the lattice velocity and the step count come from
    the unit converter (lattice viscosity (tau - 1/2) / 3).  sampling = "mc": N Monte Carlo draws
    with N = n by default (the table of simulation parameters lets N grow with n, and the study's
    convergence order is that of MCS); "smolyak": the Clenshaw-Curtis sparse grid of `level`
    (137 points at level 3)."""
    base = SampleSpec(TGV_PERTURBED, n - 1, n - 1, steps, (tau - 0.5) / 3.0, u_lattice, u_ref=u_lattice)
    if sampling == "smolyak":
        return Workload("tgv_paper4d", base, PERT4D_BOUNDS, PERT4D_PARAMS, "gpc", pts_per_dim=level, order=order,
                        quad="smolyak", storage=storage)
    return Workload("tgv_paper4d", base, PERT4D_BOUNDS, PERT4D_PARAMS, "mc", n_mc=n_samples or n, seed=seed,
                    storage=storage)
