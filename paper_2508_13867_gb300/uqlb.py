"""Thin ctypes binding of libuqlb.so (include/uqlb.h): same names, argument marshalling only.

Every function raises ``UqlbError`` when the C call returns a non-zero status.  Device
pointers are plain integers (e.g. ``tensor.data_ptr()``); streams are ``cudaStream_t``
handles as integers (e.g. ``torch.cuda.current_stream().cuda_stream``) or None.
There is no fallback: if the library has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

c_int32, c_int64, c_double, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                  ctypes.c_void_p, ctypes.c_size_t)

# enums of include/uqlb.h
UQLB_OK, UQLB_ERR_ARG, UQLB_ERR_OOM, UQLB_ERR_CUDA, UQLB_ERR_TIMEOUT, UQLB_ERR_UNSTABLE, UQLB_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6
UQLB_DIST_UNIFORM = 0
UQLB_BASIS_TOTAL, UQLB_BASIS_TENSOR = 0, 1
UQLB_QUAD_GAUSS_LEGENDRE_TENSOR, UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK = 0, 1
UQLB_METHOD_NONE, UQLB_METHOD_MC, UQLB_METHOD_GPC = 0, 1, 2
UQLB_CASE_TGV, UQLB_CASE_CHANNEL, UQLB_CASE_TGV_PERTURBED = 0, 1, 2
UQLB_OBSTACLE_HALFWAY, UQLB_OBSTACLE_BOUZIDI = 0, 1
UQLB_INOUT_FACE, UQLB_INOUT_INTERPOLATED = 0, 1
UQLB_SCHEME_AUTO, UQLB_SCHEME_ONE_STEP, UQLB_SCHEME_TWO_STEP = 0, 1, 2
UQLB_SCHEME_TWO_STEP_TILES, UQLB_SCHEME_TWO_STEP_STRIPS, UQLB_SCHEME_GROUPED = 3, 4, 5
UQLB_SCHEME_THREE_STEP_STRIPS, UQLB_SCHEME_CLUSTER = 6, 7
(UQLB_PARAM_NU, UQLB_PARAM_U0, UQLB_PARAM_ZETA2, UQLB_PARAM_ZETA3, UQLB_PARAM_PERT00, UQLB_PARAM_PERT01,
 UQLB_PARAM_PERT10, UQLB_PARAM_PERT11) = range(8)
UQLB_F64, UQLB_F32, UQLB_F16, UQLB_BF16, UQLB_FX16 = 0, 1, 2, 3, 4
UQLB_ROUND_AUTO, UQLB_ROUND_NEAREST, UQLB_ROUND_STOCHASTIC = 0, 1, 2
UQLB_MODE_GRAPH, UQLB_MODE_PERSISTENT, UQLB_MODE_PERSISTENT_TEST_TIMEOUT = 0, 1, 2
(UQLB_QOI_K, UQLB_QOI_MASS, UQLB_QOI_MOMX, UQLB_QOI_MOMY, UQLB_QOI_CD, UQLB_QOI_CL, UQLB_QOI_STEPS,
 UQLB_QOI_STATUS, UQLB_QOI_COLS) = range(9)


class UqlbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"uqlb status {status}: {message}")
        self.status = status


class uqlb_dist(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("reserved", c_int32), ("a", c_double), ("b", c_double)]


class uqlb_sample(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("nx", c_int32), ("ny", c_int32), ("steady_checks", c_int32),
                ("steps", c_int64), ("nu", c_double), ("u0", c_double), ("amp2", c_double),
                ("amp3", c_double), ("u_ref", c_double), ("cyl_cx", c_double), ("cyl_cy", c_double),
                ("cyl_r", c_double), ("ramp_steps", c_int64), ("steady_tol", c_double), ("pert", c_double * 4),
                ("obstacle_bc", c_int32), ("inout_bc", c_int32)]


class uqlb_case(ctypes.Structure):
    _fields_ = [("base", uqlb_sample), ("param_of_dim", c_int32 * 8)]


class uqlb_run_opts(ctypes.Structure):
    _fields_ = [("storage", c_int32), ("fields_dtype", c_int32), ("qoi_every", c_int64),
                ("chunk_steps", c_int32), ("tile_rows", c_int32), ("nodes_per_thread", c_int32),
                ("rounding", c_int32), ("start_step", c_int64), ("mode", c_int32), ("scheme", c_int32),
                ("strip_blocks_per_sm", c_int32), ("strip_stage", c_int32), ("strip_smem_kb", c_int32)]


class uqlb_tune_candidate(ctypes.Structure):
    _fields_ = [("scheme", c_int32), ("tile_rows", c_int32), ("nodes_per_thread", c_int32),
                ("strip_blocks_per_sm", c_int32), ("strip_stage", c_int32), ("strip_smem_kb", c_int32),
                ("ms_per_step", c_double)]


_P = ctypes.POINTER
_SIGNATURES = {
    "uqlb_gauss_legendre": [ctypes.c_int, _P(c_double), _P(c_double)],
    "uqlb_philox4x32_10": [_P(ctypes.c_uint32), _P(ctypes.c_uint32), _P(ctypes.c_uint32)],
    "uqlb_num_multi_indices": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P(c_int64)],
    "uqlb_multi_indices": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P(c_int32)],
    "uqlb_obstacle_mask": [_P(uqlb_sample), _P(ctypes.c_uint8)],
    "uqlb_fx16_quanta": [_P(uqlb_sample), _P(c_double)],
    "uqlb_unit_converter": [ctypes.c_int, c_double, c_double, _P(c_double), _P(c_double), _P(c_double),
                            _P(c_double)],
    "uqlb_mean_host": [_P(c_double), c_int64, _P(c_double)],
    "uqlb_std_host": [_P(c_double), c_int64, ctypes.c_int, _P(c_double)],
    "uqlb_create": [_P(c_void_p), ctypes.c_int],
    "uqlb_destroy": [c_void_p],
    "uqlb_last_error": [c_void_p],
    "uqlb_set_inputs": [c_void_p, ctypes.c_int, _P(uqlb_dist)],
    "uqlb_init_mc": [c_void_p, c_int64, ctypes.c_uint64],
    "uqlb_init_gpc": [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "uqlb_init_qmc": [c_void_p, c_int64, c_int64],
    "uqlb_num_samples": [c_void_p, _P(c_int64)],
    "uqlb_num_terms": [c_void_p, _P(ctypes.c_int)],
    "uqlb_get_samples": [c_void_p, _P(c_double), _P(c_double), _P(c_double)],
    "uqlb_get_weight_matrix": [c_void_p, _P(c_double)],
    "uqlb_batch_workspace_bytes": [_P(uqlb_sample), c_int64, _P(uqlb_run_opts), _P(c_size_t)],
    "uqlb_run_batch": [c_void_p, _P(uqlb_sample), c_int64, _P(uqlb_run_opts), c_void_p, c_size_t, c_void_p,
                       c_int64, c_void_p, c_void_p, c_void_p, c_int64, c_void_p],
    "uqlb_autotune": [c_void_p, _P(uqlb_sample), c_int64, _P(uqlb_run_opts), c_void_p, c_size_t, ctypes.c_int,
                      _P(c_int32), _P(c_int32), _P(c_int32), _P(c_int32), _P(c_double), _P(c_int32), c_void_p],
    "uqlb_autotune_report": [c_void_p, _P(uqlb_tune_candidate), c_int32, _P(c_int32), _P(c_int32)],
    "uqlb_ensemble_samples": [c_void_p, _P(uqlb_case), _P(uqlb_sample)],
    "uqlb_ensemble_workspace_bytes": [c_void_p, _P(uqlb_case), _P(uqlb_run_opts), _P(c_size_t)],
    "uqlb_run_ensemble": [c_void_p, _P(uqlb_case), _P(uqlb_run_opts), c_void_p, c_size_t, c_void_p, c_int64,
                          c_void_p, c_void_p, c_void_p, c_int64, c_void_p],
    "uqlb_plain_workspace_bytes": [_P(uqlb_sample), c_int64, _P(c_size_t)],
    "uqlb_run_plain_f64": [c_void_p, _P(uqlb_sample), c_int64, c_int64, c_void_p, c_size_t, c_void_p, c_int64,
                           c_void_p, c_void_p, c_int64, c_void_p],
    "uqlb_last_loop_time": [c_void_p, _P(c_double), _P(c_int64), _P(c_int64)],
    "uqlb_last_run_geometry": [c_void_p, _P(c_int32), _P(c_int32), _P(c_int32)],
    "uqlb_w1_workspace_bytes": [ctypes.c_int, _P(c_size_t)],
    "uqlb_w1_speed": [c_void_p, c_void_p, ctypes.c_int, c_int64, c_int64, c_int64, c_void_p, ctypes.c_int, c_int64,
                      c_int64, c_int64, ctypes.c_int, c_void_p, c_size_t, _P(c_double), _P(c_double), _P(c_int64),
                      c_void_p],
    "uqlb_post_workspace_bytes": [c_void_p, _P(c_size_t)],
    "uqlb_project_workspace_bytes": [c_void_p, c_int64, _P(c_size_t)],
    "uqlb_last_projection": [c_void_p, _P(ctypes.c_int32)],
    "uqlb_project": [c_void_p, c_void_p, ctypes.c_int, c_int64, c_int64, c_void_p, c_void_p, c_size_t, c_void_p],
    "uqlb_project_noalloc": [c_void_p, c_void_p, ctypes.c_int, c_int64, c_int64, c_void_p, c_void_p],
    "uqlb_get_weight_block": [c_void_p, c_int64, c_int64, _P(c_double)],
    "uqlb_project_block": [c_void_p, c_void_p, ctypes.c_int, c_int64, c_int64, c_int64, c_int64, c_void_p, c_void_p,
                           c_size_t, c_void_p],
    "uqlb_block_moments": [c_void_p, c_void_p, ctypes.c_int, c_int64, c_int64, c_int64, c_void_p, c_void_p,
                           c_void_p],
    "uqlb_stats": [c_void_p, c_void_p, ctypes.c_int, c_int64, c_int64, c_void_p, c_void_p, ctypes.c_int,
                   c_void_p],
    "uqlb_uq_workspace_bytes": [c_void_p, _P(uqlb_case), _P(uqlb_run_opts), _P(c_size_t)],
    "uqlb_run_uq_host": [c_void_p, _P(uqlb_case), _P(uqlb_run_opts), c_void_p, c_size_t, _P(c_double),
                         _P(c_double), _P(c_double), _P(c_double), c_void_p],
}

_lib = None


def header_symbols() -> list[str]:
    """Function names declared in include/uqlb.h."""
    import re

    with open(os.path.join(_build.INCLUDE, "uqlb.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(uqlb_\w+)\s*\(", text, flags=re.M)))


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it was never built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(_build.LIB)
        for name, args in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "uqlb_last_error" else ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, ctx=None) -> None:
    if rc != 0:
        msg = lib().uqlb_last_error(ctx)
        raise UqlbError(rc, msg.decode() if msg else "")


def _dp(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_P(c_double))


def _stream(stream) -> c_void_p:
    return c_void_p(int(stream)) if stream else c_void_p(0)


# ---- host building blocks ---------------------------------------------------------------

def uqlb_gauss_legendre(n: int) -> tuple[np.ndarray, np.ndarray]:
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().uqlb_gauss_legendre(n, _dp(x), _dp(w)))
    return x, w


def uqlb_philox4x32_10(ctr, key) -> tuple[int, int, int, int]:
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    _check(lib().uqlb_philox4x32_10(c, k, o))
    return tuple(int(v) for v in o)


def uqlb_num_multi_indices(dim: int, order: int, basis: int = UQLB_BASIS_TOTAL) -> int:
    k = c_int64()
    _check(lib().uqlb_num_multi_indices(dim, order, basis, ctypes.byref(k)))
    return k.value


def uqlb_multi_indices(dim: int, order: int, basis: int = UQLB_BASIS_TOTAL) -> np.ndarray:
    k = uqlb_num_multi_indices(dim, order, basis)
    a = np.zeros((k, dim), dtype=np.int32)
    _check(lib().uqlb_multi_indices(dim, order, basis, a.ctypes.data_as(_P(c_int32))))
    return a


def uqlb_unit_converter(n: int, ma: float, re: float) -> dict:
    dx, dt, tau, ul = c_double(), c_double(), c_double(), c_double()
    _check(lib().uqlb_unit_converter(n, ma, re, ctypes.byref(dx), ctypes.byref(dt), ctypes.byref(tau),
                                     ctypes.byref(ul)))
    return {"dx": dx.value, "dt": dt.value, "tau": tau.value, "u_lattice": ul.value}


def uqlb_fx16_quanta(sample: uqlb_sample) -> np.ndarray:
    q = np.zeros(3)
    _check(lib().uqlb_fx16_quanta(ctypes.byref(sample), _dp(q)))
    return q


def uqlb_obstacle_mask(sample: uqlb_sample) -> np.ndarray:
    m = np.zeros((sample.ny, sample.nx), dtype=np.uint8)
    _check(lib().uqlb_obstacle_mask(ctypes.byref(sample), m.ctypes.data_as(_P(ctypes.c_uint8))))
    return m


def uqlb_mean_host(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = c_double()
    _check(lib().uqlb_mean_host(_dp(v), v.size, ctypes.byref(out)))
    return out.value


def uqlb_std_host(v, ddof: int = 1) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = c_double()
    _check(lib().uqlb_std_host(_dp(v), v.size, ddof, ctypes.byref(out)))
    return out.value


# ---- UQ manager ---------------------------------------------------------------------------

def uqlb_create(cuda_device: int = 0) -> c_void_p:
    h = c_void_p()
    _check(lib().uqlb_create(ctypes.byref(h), cuda_device))
    return h


def uqlb_destroy(ctx) -> None:
    _check(lib().uqlb_destroy(ctx))


def uqlb_last_error(ctx=None) -> str:
    msg = lib().uqlb_last_error(ctx)
    return msg.decode() if msg else ""


def uqlb_set_inputs(ctx, bounds) -> None:
    arr = (uqlb_dist * len(bounds))(*[uqlb_dist(UQLB_DIST_UNIFORM, 0, float(a), float(b)) for a, b in bounds])
    _check(lib().uqlb_set_inputs(ctx, len(bounds), arr), ctx)


def uqlb_init_mc(ctx, n: int, seed: int) -> None:
    _check(lib().uqlb_init_mc(ctx, n, seed), ctx)


def uqlb_init_qmc(ctx, n: int, skip: int = 1) -> None:
    _check(lib().uqlb_init_qmc(ctx, n, skip), ctx)


def uqlb_init_gpc(ctx, order: int, pts_per_dim: int, basis: int = UQLB_BASIS_TOTAL,
                  quad: int = UQLB_QUAD_GAUSS_LEGENDRE_TENSOR) -> None:
    _check(lib().uqlb_init_gpc(ctx, order, pts_per_dim, basis, quad), ctx)


def uqlb_num_samples(ctx) -> int:
    n = c_int64()
    _check(lib().uqlb_num_samples(ctx, ctypes.byref(n)), ctx)
    return n.value


def uqlb_num_terms(ctx) -> int:
    k = ctypes.c_int()
    _check(lib().uqlb_num_terms(ctx, ctypes.byref(k)), ctx)
    return k.value


def uqlb_get_samples(ctx, dim: int):
    n = uqlb_num_samples(ctx)
    z, xi, a = np.zeros((n, dim)), np.zeros((n, dim)), np.zeros(n)
    _check(lib().uqlb_get_samples(ctx, _dp(z), _dp(xi), _dp(a)), ctx)
    return z, xi, a


def uqlb_get_weight_matrix(ctx) -> np.ndarray:
    w = np.zeros((uqlb_num_terms(ctx), uqlb_num_samples(ctx)))
    _check(lib().uqlb_get_weight_matrix(ctx, _dp(w)), ctx)
    return w


def uqlb_get_weight_block(ctx, s0: int, count: int) -> np.ndarray:
    w = np.zeros((uqlb_num_terms(ctx), count))
    _check(lib().uqlb_get_weight_block(ctx, s0, count, _dp(w)), ctx)
    return w


# ---- runs -------------------------------------------------------------------------------

def _samples_array(samples):
    return (uqlb_sample * len(samples))(*samples)


def uqlb_batch_workspace_bytes(samples, opts: uqlb_run_opts) -> int:
    b = c_size_t()
    _check(lib().uqlb_batch_workspace_bytes(_samples_array(samples), len(samples), ctypes.byref(opts),
                                            ctypes.byref(b)))
    return b.value


def uqlb_run_batch(ctx, samples, opts: uqlb_run_opts, workspace_dev: int, workspace_bytes: int,
                   fields_dev: int = 0, fields_ld: int = 0, qoi_dev: int = 0, series_dev: int = 0,
                   series_cl_dev: int = 0, series_ld: int = 0, stream=None) -> None:
    _check(lib().uqlb_run_batch(ctx, _samples_array(samples), len(samples), ctypes.byref(opts),
                                c_void_p(workspace_dev), workspace_bytes, c_void_p(fields_dev or None),
                                fields_ld, c_void_p(qoi_dev or None), c_void_p(series_dev or None),
                                c_void_p(series_cl_dev or None), series_ld, _stream(stream)), ctx)


def uqlb_autotune(ctx, samples, opts: uqlb_run_opts, workspace_dev: int, workspace_bytes: int,
                  trial_steps: int = 16, stream=None) -> dict:
    """Time every compiled tile geometry on this batch; returns the choice and the table."""
    r, q, nt = c_int32(), c_int32(), c_int32()
    rows, npts, ms = (c_int32 * 16)(), (c_int32 * 16)(), (c_double * 16)()
    _check(lib().uqlb_autotune(ctx, _samples_array(samples), len(samples), ctypes.byref(opts),
                               c_void_p(workspace_dev), workspace_bytes, trial_steps, ctypes.byref(r),
                               ctypes.byref(q), rows, npts, ms, ctypes.byref(nt), _stream(stream)), ctx)
    return {"tile_rows": r.value, "nodes_per_thread": q.value,
            "tried": [(rows[i], npts[i], ms[i]) for i in range(nt.value)]}


def uqlb_autotune_report(ctx) -> dict:
    """The candidates of the context's last autotune (strip knobs included) and the chosen index."""
    n, chosen = c_int32(), c_int32()
    _check(lib().uqlb_autotune_report(ctx, None, 0, ctypes.byref(n), ctypes.byref(chosen)), ctx)
    out = (uqlb_tune_candidate * max(n.value, 1))()
    _check(lib().uqlb_autotune_report(ctx, out, n.value, ctypes.byref(n), ctypes.byref(chosen)), ctx)
    names = [f for f, _ in uqlb_tune_candidate._fields_]
    return {"chosen": chosen.value, "candidates": [{k: getattr(out[i], k) for k in names} for i in range(n.value)]}


def uqlb_ensemble_samples(ctx, case: uqlb_case) -> list:
    n = uqlb_num_samples(ctx)
    out = (uqlb_sample * n)()
    _check(lib().uqlb_ensemble_samples(ctx, ctypes.byref(case), out), ctx)
    return list(out)


def uqlb_ensemble_workspace_bytes(ctx, case: uqlb_case, opts: uqlb_run_opts) -> int:
    b = c_size_t()
    _check(lib().uqlb_ensemble_workspace_bytes(ctx, ctypes.byref(case), ctypes.byref(opts), ctypes.byref(b)), ctx)
    return b.value


def uqlb_run_ensemble(ctx, case: uqlb_case, opts: uqlb_run_opts, workspace_dev: int, workspace_bytes: int,
                      fields_dev: int = 0, fields_ld: int = 0, qoi_dev: int = 0, series_dev: int = 0,
                      series_cl_dev: int = 0, series_ld: int = 0, stream=None) -> None:
    _check(lib().uqlb_run_ensemble(ctx, ctypes.byref(case), ctypes.byref(opts), c_void_p(workspace_dev),
                                   workspace_bytes, c_void_p(fields_dev or None), fields_ld,
                                   c_void_p(qoi_dev or None), c_void_p(series_dev or None),
                                   c_void_p(series_cl_dev or None), series_ld, _stream(stream)), ctx)


def uqlb_plain_workspace_bytes(samples) -> int:
    b = c_size_t()
    _check(lib().uqlb_plain_workspace_bytes(_samples_array(samples), len(samples), ctypes.byref(b)))
    return b.value


def uqlb_run_plain_f64(ctx, samples, qoi_every: int, workspace_dev: int, workspace_bytes: int,
                       fields_dev: int = 0, fields_ld: int = 0, qoi_dev: int = 0, series_dev: int = 0,
                       series_ld: int = 0, stream=None) -> None:
    _check(lib().uqlb_run_plain_f64(ctx, _samples_array(samples), len(samples), qoi_every,
                                    c_void_p(workspace_dev), workspace_bytes, c_void_p(fields_dev or None),
                                    fields_ld, c_void_p(qoi_dev or None), c_void_p(series_dev or None),
                                    series_ld, _stream(stream)), ctx)


def uqlb_last_loop_time(ctx) -> tuple[float, int, int]:
    """(milliseconds of the last run's time loop, its steps, kernels the run launched)."""
    ms, st, la = c_double(), c_int64(), c_int64()
    _check(lib().uqlb_last_loop_time(ctx, ctypes.byref(ms), ctypes.byref(st), ctypes.byref(la)), ctx)
    return ms.value, st.value, la.value


def uqlb_last_run_geometry(ctx) -> tuple[int, int, int]:
    """(scheme, tile_rows, nodes_per_thread) of the last run on this context; scheme is the kernel
    that ran: UQLB_SCHEME_ONE_STEP, _TWO_STEP_TILES, _TWO_STEP_STRIPS or _GROUPED (a batch of unlike
    samples run as groups; the tile geometry is then the first group's)."""
    sc, tr, q = c_int32(), c_int32(), c_int32()
    _check(lib().uqlb_last_run_geometry(ctx, ctypes.byref(sc), ctypes.byref(tr), ctypes.byref(q)), ctx)
    return sc.value, tr.value, q.value


def uqlb_w1_workspace_bytes(bins: int) -> int:
    b = c_size_t()
    _check(lib().uqlb_w1_workspace_bytes(bins, ctypes.byref(b)))
    return b.value


def uqlb_w1_speed(ctx, a_dev: int, dtype_a: int, s_a: int, nodes_a: int, ld_a: int, b_dev: int, dtype_b: int,
                  s_b: int, nodes_b: int, ld_b: int, bins: int, workspace_dev: int, workspace_bytes: int,
                  stream=None) -> tuple[float, float, tuple[int, int]]:
    """(W1 distance of the finite speeds, its error bound = one bin width, non-finite counts)."""
    out, bound, nf = c_double(), c_double(), (c_int64 * 2)()
    _check(lib().uqlb_w1_speed(ctx, c_void_p(a_dev), dtype_a, s_a, nodes_a, ld_a, c_void_p(b_dev), dtype_b, s_b,
                               nodes_b, ld_b, bins, c_void_p(workspace_dev), workspace_bytes, ctypes.byref(out),
                               ctypes.byref(bound), nf, _stream(stream)), ctx)
    return out.value, bound.value, (nf[0], nf[1])


def uqlb_post_workspace_bytes(ctx) -> int:
    b = c_size_t()
    _check(lib().uqlb_post_workspace_bytes(ctx, ctypes.byref(b)), ctx)
    return b.value


def uqlb_project_workspace_bytes(ctx, n_fields: int) -> int:
    b = c_size_t()
    _check(lib().uqlb_project_workspace_bytes(ctx, n_fields, ctypes.byref(b)), ctx)
    return b.value


def uqlb_last_projection(ctx) -> int:
    k = ctypes.c_int32()
    _check(lib().uqlb_last_projection(ctx, ctypes.byref(k)), ctx)
    return k.value


def uqlb_project(ctx, m_dev: int, dtype: int, n_fields: int, m_ld: int, coeffs_dev: int, workspace_dev: int,
                 workspace_bytes: int, stream=None) -> None:
    _check(lib().uqlb_project(ctx, c_void_p(m_dev), dtype, n_fields, m_ld, c_void_p(coeffs_dev),
                              c_void_p(workspace_dev), workspace_bytes, _stream(stream)), ctx)


def uqlb_project_block(ctx, m_dev: int, dtype: int, n_fields: int, m_ld: int, s0: int, count: int, coeffs_dev: int,
                       workspace_dev: int, workspace_bytes: int, stream=None) -> None:
    _check(lib().uqlb_project_block(ctx, c_void_p(m_dev), dtype, n_fields, m_ld, s0, count, c_void_p(coeffs_dev),
                                    c_void_p(workspace_dev), workspace_bytes, _stream(stream)), ctx)


def uqlb_block_moments(ctx, m_dev: int, dtype: int, n_rows: int, n_fields: int, m_ld: int, mean_dev: int,
                       m2_dev: int, stream=None) -> None:
    _check(lib().uqlb_block_moments(ctx, c_void_p(m_dev), dtype, n_rows, n_fields, m_ld, c_void_p(mean_dev),
                                    c_void_p(m2_dev), _stream(stream)), ctx)


def uqlb_project_noalloc(ctx, m_dev: int, dtype: int, n_fields: int, m_ld: int, coeffs_dev: int,
                         stream=None) -> None:
    _check(lib().uqlb_project_noalloc(ctx, c_void_p(m_dev), dtype, n_fields, m_ld, c_void_p(coeffs_dev),
                                      _stream(stream)), ctx)


def uqlb_stats(ctx, in_dev: int, dtype: int, n_fields: int, m_ld: int, mean_dev: int, var_dev: int,
               ddof: int = 1, stream=None) -> None:
    _check(lib().uqlb_stats(ctx, c_void_p(in_dev), dtype, n_fields, m_ld, c_void_p(mean_dev or None),
                            c_void_p(var_dev or None), ddof, _stream(stream)), ctx)


def uqlb_uq_workspace_bytes(ctx, case: uqlb_case, opts: uqlb_run_opts) -> int:
    b = c_size_t()
    _check(lib().uqlb_uq_workspace_bytes(ctx, ctypes.byref(case), ctypes.byref(opts), ctypes.byref(b)), ctx)
    return b.value


def uqlb_run_uq_host(ctx, case: uqlb_case, opts: uqlb_run_opts, workspace_dev: int, workspace_bytes: int,
                     mean_host: np.ndarray, var_host: np.ndarray, coeffs_host: np.ndarray | None = None,
                     qoi_host: np.ndarray | None = None, stream=None) -> None:
    for a in (mean_host, var_host, coeffs_host, qoi_host):
        if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous):
            raise ValueError("host outputs must be C-contiguous float64 arrays")
    _check(lib().uqlb_run_uq_host(ctx, ctypes.byref(case), ctypes.byref(opts), c_void_p(workspace_dev),
                                  workspace_bytes, _dp(mean_host), _dp(var_host), _dp(coeffs_host),
                                  _dp(qoi_host), _stream(stream)), ctx)
