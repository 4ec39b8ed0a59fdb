"""Shared test helpers: convert workload specs for the oracle and compare results."""
import numpy as np

from oracle import lbm as olbm


def oracle_case(spec, qoi_every=0):
    return olbm.Case(spec.kind, spec.nx, spec.ny, spec.steps, spec.nu, spec.u0, amp2=spec.amp2, amp3=spec.amp3,
                     u_ref=spec.u_ref, cyl_cx=spec.cyl_cx, cyl_cy=spec.cyl_cy, cyl_r=spec.cyl_r,
                     ramp_steps=spec.ramp_steps, qoi_every=qoi_every, steady_tol=spec.steady_tol,
                     pert=tuple(spec.pert), obstacle_bc=spec.obstacle_bc, inout_bc=spec.inout_bc)


def oracle_row(r):
    """The oracle's result laid out like a field row [u, v, K]."""
    return np.concatenate([r.u.ravel(), r.v.ravel(), [r.k_final]])


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
