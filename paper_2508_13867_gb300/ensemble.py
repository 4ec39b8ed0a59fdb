"""Torch-backed convenience layer over the C ABI: device memory comes from torch tensors, work
runs on torch's current CUDA stream, and every step of the computation happens inside
libuqlb.so.  Nothing here computes: it sizes buffers, builds the C structs and calls ``uqlb``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import uqlb as U
from .workloads import SampleSpec, Workload

STORAGE = {"f64": U.UQLB_F64, "f32": U.UQLB_F32, "f16": U.UQLB_F16, "bf16": U.UQLB_BF16, "fx16": U.UQLB_FX16}
PARAMS = {"nu": U.UQLB_PARAM_NU, "u0": U.UQLB_PARAM_U0, "zeta2": U.UQLB_PARAM_ZETA2, "zeta3": U.UQLB_PARAM_ZETA3,
          "pert00": U.UQLB_PARAM_PERT00, "pert01": U.UQLB_PARAM_PERT01, "pert10": U.UQLB_PARAM_PERT10,
          "pert11": U.UQLB_PARAM_PERT11}


def sample_struct(s: SampleSpec) -> U.uqlb_sample:
    return U.uqlb_sample(s.kind, s.nx, s.ny, s.steady_checks, s.steps, s.nu, s.u0, s.amp2, s.amp3, s.u_ref,
                         s.cyl_cx, s.cyl_cy, s.cyl_r, s.ramp_steps, s.steady_tol, (U.c_double * 4)(*s.pert),
                         s.obstacle_bc, s.inout_bc)


def case_struct(w: Workload) -> U.uqlb_case:
    c = U.uqlb_case()
    c.base = sample_struct(w.base)
    for i, p in enumerate(w.params):
        c.param_of_dim[i] = PARAMS[p]
    return c


ROUNDING = {"auto": U.UQLB_ROUND_AUTO, "nearest": U.UQLB_ROUND_NEAREST, "stochastic": U.UQLB_ROUND_STOCHASTIC}
MODES = {"graph": U.UQLB_MODE_GRAPH, "persistent": U.UQLB_MODE_PERSISTENT,
         "persistent_test_timeout": U.UQLB_MODE_PERSISTENT_TEST_TIMEOUT}


SCHEMES = {"auto": U.UQLB_SCHEME_AUTO, "one_step": U.UQLB_SCHEME_ONE_STEP, "two_step": U.UQLB_SCHEME_TWO_STEP,
           "two_step_tiles": U.UQLB_SCHEME_TWO_STEP_TILES, "two_step_strips": U.UQLB_SCHEME_TWO_STEP_STRIPS,
           "three_step_strips": U.UQLB_SCHEME_THREE_STEP_STRIPS, "cluster": U.UQLB_SCHEME_CLUSTER}


def opts_struct(storage: str = "f32", fields_dtype: str = "f32", qoi_every: int = 0, chunk_steps: int = 0,
                tile_rows: int = 0, nodes_per_thread: int = 0, rounding: str = "auto",
                start_step: int = 0, mode: str = "graph", scheme: str = "auto", strip_blocks_per_sm: int = 0,
                strip_stage: int = 0, strip_smem_kb: int = 0) -> U.uqlb_run_opts:
    return U.uqlb_run_opts(STORAGE[storage], STORAGE[fields_dtype], qoi_every, chunk_steps, tile_rows,
                           nodes_per_thread, ROUNDING[rounding], start_step, MODES[mode], SCHEMES[scheme],
                           strip_blocks_per_sm, strip_stage, strip_smem_kb)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _torch_dtype(code: int):
    return torch.float64 if code == U.UQLB_F64 else torch.float32


class Ensemble:
    """The UQ manager of one device: inputs, sample set, runs, projection and statistics."""

    def __init__(self, device: int = 0):
        self.device = device
        self.ctx = U.uqlb_create(device)
        self.dim = 0
        self._ws = None

    def close(self):
        if self.ctx is not None:
            U.uqlb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- sampling ---------------------------------------------------------------------
    def set_inputs(self, bounds):
        U.uqlb_set_inputs(self.ctx, bounds)
        self.dim = len(bounds)

    def init_mc(self, n: int, seed: int):
        U.uqlb_init_mc(self.ctx, n, seed)

    def init_gpc(self, order: int, pts_per_dim: int, basis: int = U.UQLB_BASIS_TOTAL,
                 quad: int = U.UQLB_QUAD_GAUSS_LEGENDRE_TENSOR):
        U.uqlb_init_gpc(self.ctx, order, pts_per_dim, basis, quad)

    def init_qmc(self, n: int, skip: int = 1):
        U.uqlb_init_qmc(self.ctx, n, skip)

    def setup(self, w: Workload):
        self.set_inputs(w.bounds)
        if w.method == "gpc":
            quad = U.UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK if w.quad == "smolyak" else U.UQLB_QUAD_GAUSS_LEGENDRE_TENSOR
            self.init_gpc(w.order, w.pts_per_dim, quad=quad)
        elif w.method == "qmc":
            self.init_qmc(w.n_mc)
        else:
            self.init_mc(w.n_mc, w.seed)

    def samples(self):
        return U.uqlb_get_samples(self.ctx, self.dim)

    @property
    def num_samples(self) -> int:
        return U.uqlb_num_samples(self.ctx)

    @property
    def num_terms(self) -> int:
        return U.uqlb_num_terms(self.ctx)

    def ensemble_samples(self, w: Workload) -> list:
        return U.uqlb_ensemble_samples(self.ctx, case_struct(w))

    # ---- device memory ------------------------------------------------------------------
    def workspace(self, nbytes: int) -> torch.Tensor:
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = None
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=f"cuda:{self.device}")
        return self._ws

    # ---- runs -------------------------------------------------------------------------
    def run_batch(self, samples, storage: str = "f32", fields_dtype: str = "f32", qoi_every: int = 0,
                  fields: bool = True, series: bool = False, chunk_steps: int = 0, tile_rows: int = 0,
                  nodes_per_thread: int = 0, rounding: str = "auto", start_step: int = 0, mode: str = "graph",
                  scheme: str = "auto", out: dict | None = None, strip: tuple = (0, 0, 0)) -> dict:
        """Run the given uqlb_sample structs; returns torch tensors (fields M, qoi, series).  With
        start_step > 0 the run continues the state left by the previous call (same samples).  strip:
        the three-step strips' (blocks per SM, staging option, shared-memory KB), 0 = tuned/default."""
        opts = opts_struct(storage, fields_dtype, qoi_every, chunk_steps, tile_rows, nodes_per_thread, rounding,
                           start_step, mode, scheme, *strip)
        nbytes = U.uqlb_batch_workspace_bytes(samples, opts)
        ws = self.workspace(nbytes)
        n = len(samples)
        dev = f"cuda:{self.device}"
        res = out if out is not None else {}
        F = 2 * samples[0].nx * samples[0].ny + 1
        if fields and "fields" not in res:
            res["fields"] = torch.empty((n, F), dtype=_torch_dtype(opts.fields_dtype), device=dev)
        if "qoi" not in res:
            res["qoi"] = torch.full((n, U.UQLB_QOI_COLS), float("nan"), dtype=torch.float64, device=dev)
        ld = 0
        if series and qoi_every > 0:
            ld = max(int(s.steps) for s in samples) // qoi_every + 1
            if "series" not in res:
                res["series"] = torch.full((n, ld), float("nan"), dtype=torch.float64, device=dev)
                res["series_cl"] = torch.full((n, ld), float("nan"), dtype=torch.float64, device=dev)
        U.uqlb_run_batch(self.ctx, samples, opts, ws.data_ptr(), ws.numel(),
                         res["fields"].data_ptr() if fields else 0, F if fields else 0, res["qoi"].data_ptr(),
                         res["series"].data_ptr() if ld else 0, res["series_cl"].data_ptr() if ld else 0, ld,
                         _stream())
        return res

    def autotune(self, samples, storage: str = "f32", trial_steps: int = 16, scheme: str = "auto") -> dict:
        opts = opts_struct(storage, "f32", 0, scheme=scheme)
        ws = self.workspace(U.uqlb_batch_workspace_bytes(samples, opts))
        res = U.uqlb_autotune(self.ctx, samples, opts, ws.data_ptr(), ws.numel(), trial_steps, _stream())
        res.update(U.uqlb_autotune_report(self.ctx))
        return res

    def w1_speed(self, a: torch.Tensor, nodes_a: int, b: torch.Tensor, nodes_b: int, bins: int = 1 << 20):
        """W1 distance between the speed distributions of two field sets (and its error bound)."""
        nb = U.uqlb_w1_workspace_bytes(bins)
        ws = torch.empty(nb, dtype=torch.uint8, device=a.device)
        code = lambda t: U.UQLB_F64 if t.dtype == torch.float64 else U.UQLB_F32  # noqa: E731
        return U.uqlb_w1_speed(self.ctx, a.data_ptr(), code(a), a.shape[0], nodes_a, a.stride(0), b.data_ptr(),
                               code(b), b.shape[0], nodes_b, b.stride(0), bins, ws.data_ptr(), nb, _stream())

    def run_plain_f64(self, samples, qoi_every: int = 0, series: bool = False, fields: bool = True) -> dict:
        nbytes = U.uqlb_plain_workspace_bytes(samples)
        ws = self.workspace(nbytes)
        n = len(samples)
        dev = f"cuda:{self.device}"
        F = 2 * samples[0].nx * samples[0].ny + 1
        res = {"qoi": torch.full((n, U.UQLB_QOI_COLS), float("nan"), dtype=torch.float64, device=dev)}
        if fields:
            res["fields"] = torch.empty((n, F), dtype=torch.float64, device=dev)
        ld = 0
        if series and qoi_every > 0:
            ld = max(int(s.steps) for s in samples) // qoi_every + 1
            res["series"] = torch.full((n, ld), float("nan"), dtype=torch.float64, device=dev)
        U.uqlb_run_plain_f64(self.ctx, samples, qoi_every, ws.data_ptr(), ws.numel(),
                             res["fields"].data_ptr() if fields else 0, F if fields else 0, res["qoi"].data_ptr(),
                             res["series"].data_ptr() if ld else 0, ld, _stream())
        return res

    # ---- postprocessing ---------------------------------------------------------------
    def project(self, m: torch.Tensor, coeffs: torch.Tensor | None = None) -> torch.Tensor:
        """gPC coefficients of the rows of m (the workspace of the library's fastest contraction)."""
        dtype = U.UQLB_F64 if m.dtype == torch.float64 else U.UQLB_F32
        F = m.shape[1]
        if coeffs is None:
            coeffs = torch.empty((self.num_terms, F), dtype=torch.float64, device=m.device)
        wsb = U.uqlb_project_workspace_bytes(self.ctx, F)
        if not hasattr(self, "_post") or self._post.numel() < wsb:
            self._post = torch.empty(max(wsb, 256), dtype=torch.uint8, device=m.device)
        U.uqlb_project(self.ctx, m.data_ptr(), dtype, F, m.stride(0), coeffs.data_ptr(), self._post.data_ptr(),
                       wsb, _stream())
        return coeffs

    def project_block(self, m: torch.Tensor, s0: int, coeffs: torch.Tensor | None = None) -> torch.Tensor:
        """Partial coefficients of the sample block s0 .. s0 + len(m) - 1 (rows of m)."""
        dtype = U.UQLB_F64 if m.dtype == torch.float64 else U.UQLB_F32
        F = m.shape[1]
        if coeffs is None:
            coeffs = torch.empty((self.num_terms, F), dtype=torch.float64, device=m.device)
        wsb = U.uqlb_post_workspace_bytes(self.ctx)
        if not hasattr(self, "_post") or self._post.numel() < wsb:
            self._post = torch.empty(max(wsb, 256), dtype=torch.uint8, device=m.device)
        U.uqlb_project_block(self.ctx, m.data_ptr(), dtype, F, m.stride(0), s0, m.shape[0], coeffs.data_ptr(),
                             self._post.data_ptr(), self._post.numel(), _stream())
        return coeffs

    def block_moments(self, m: torch.Tensor):
        """(rows, mean, sum of squared deviations) of the rows of m, for merging sample blocks."""
        dtype = U.UQLB_F64 if m.dtype == torch.float64 else U.UQLB_F32
        F = m.shape[1]
        mean = torch.empty(F, dtype=torch.float64, device=m.device)
        m2 = torch.empty(F, dtype=torch.float64, device=m.device)
        U.uqlb_block_moments(self.ctx, m.data_ptr(), dtype, m.shape[0], F, m.stride(0), mean.data_ptr(), m2.data_ptr(),
                             _stream())
        return m.shape[0], mean, m2

    def stats(self, x: torch.Tensor, ddof: int = 1):
        """gPC context: x = coefficients [K x F]; MC context: x = fields M [S x F]."""
        dtype = U.UQLB_F64 if x.dtype == torch.float64 else U.UQLB_F32
        F = x.shape[1]
        mean = torch.empty(F, dtype=torch.float64, device=x.device)
        var = torch.empty(F, dtype=torch.float64, device=x.device)
        U.uqlb_stats(self.ctx, x.data_ptr(), dtype, F, x.stride(0), mean.data_ptr(), var.data_ptr(), ddof, _stream())
        return mean, var

    def run_uq_host(self, w: Workload, fields_dtype: str = "f32", coeffs: bool = False, qoi: bool = False):
        """Algorithm 1 end to end through host buffers (one C call); returns numpy arrays."""
        case = case_struct(w)
        opts = opts_struct(w.storage, fields_dtype, w.qoi_every)
        nbytes = U.uqlb_uq_workspace_bytes(self.ctx, case, opts)
        ws = self.workspace(nbytes)
        F = 2 * w.base.nx * w.base.ny + 1
        mean, var = np.zeros(F), np.zeros(F)
        c = np.zeros((self.num_terms, F)) if coeffs and self.num_terms > 0 else None
        q = np.zeros((self.num_samples, U.UQLB_QOI_COLS)) if qoi else None
        U.uqlb_run_uq_host(self.ctx, case, opts, ws.data_ptr(), ws.numel(), mean, var, c, q, _stream())
        return mean, var, c, q
