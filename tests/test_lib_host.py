"""CPU-side checks of libuqlb.so: it loads, exports every symbol of include/uqlb.h, and its host
logic (quadrature, Philox, chaos basis, sample sets, weight matrix, masks, ensemble mapping,
argument checking) matches the oracle.  No device work is launched here."""
import ctypes
from dataclasses import replace
import math

import numpy as np
import pytest

from oracle import lbm as olbm
from oracle import uq as ouq
from paper_2508_13867_gb300 import build as lib_build
from paper_2508_13867_gb300 import uqlb as U
from paper_2508_13867_gb300 import workloads as W
from paper_2508_13867_gb300.ensemble import case_struct, sample_struct


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib_build.build()


def test_library_exports_every_header_symbol():
    names = U.header_symbols()
    assert len(names) >= 25
    L = U.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(U._SIGNATURES), "binding and header disagree"


def test_binding_constants_match_header_enums():
    """Every UQLB_* enumerator of the header has the same value in the Python binding."""
    import re
    from pathlib import Path

    text = Path(__file__).resolve().parents[1].joinpath("include", "uqlb.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    found = 0
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for name, value in re.findall(r"(UQLB_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            assert hasattr(U, name), name
            assert getattr(U, name) == int(value), name
            found += 1
    assert found >= 30


def test_struct_sizes_match_header_layout():
    assert ctypes.sizeof(U.uqlb_dist) == 24
    assert ctypes.sizeof(U.uqlb_sample) == 144
    assert ctypes.sizeof(U.uqlb_case) == 176
    assert ctypes.sizeof(U.uqlb_run_opts) == 64
    assert ctypes.sizeof(U.uqlb_tune_candidate) == 32


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 17, 33, 64])
def test_gauss_legendre_matches_oracle(n):
    x, w = U.uqlb_gauss_legendre(n)
    xo, wo = ouq.gauss_legendre(n)
    assert np.abs(x - xo).max() <= 4e-16 and np.abs(w - wo).max() <= 4e-16


def test_philox_matches_oracle_and_published_vectors():
    rng = np.random.default_rng(11)
    for _ in range(200):
        ctr = tuple(int(v) for v in rng.integers(0, 2 ** 32, 4))
        key = tuple(int(v) for v in rng.integers(0, 2 ** 32, 2))
        assert U.uqlb_philox4x32_10(ctr, key) == ouq.philox4x32_10(ctr, key)
    assert U.uqlb_philox4x32_10((0, 0, 0, 0), (0, 0)) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)


@pytest.mark.parametrize("dim,order,basis", [(1, 8, 0), (2, 3, 0), (4, 4, 0), (3, 2, 1), (8, 2, 0)])
def test_multi_indices_match_oracle(dim, order, basis):
    a = U.uqlb_multi_indices(dim, order, basis)
    assert np.array_equal(a, ouq.multi_indices(dim, order, "total" if basis == 0 else "tensor"))


def test_gpc_sample_set_and_weight_matrix_match_oracle():
    ctx = U.uqlb_create(0)
    try:
        U.uqlb_set_inputs(ctx, W.TGV4D_BOUNDS)
        U.uqlb_init_gpc(ctx, 4, 5)
        z, xi, a = U.uqlb_get_samples(ctx, 4)
        zo, xio, ao = ouq.tensor_grid([5] * 4, W.TGV4D_BOUNDS)
        assert np.abs(z - zo).max() < 1e-17 + 1e-15 * np.abs(zo).max()
        assert np.abs(xi - xio).max() <= 4e-16 and np.abs(a - ao).max() <= 1e-17
        assert U.uqlb_num_terms(ctx) == 70 and U.uqlb_num_samples(ctx) == 625
        wm = U.uqlb_get_weight_matrix(ctx)
        wo = ouq.weight_matrix(ouq.multi_indices(4, 4), xio, ao)
        assert np.abs(wm - wo).max() < 1e-15
    finally:
        U.uqlb_destroy(ctx)


def test_projection_workspace_selects_the_contraction():
    """The projection's workspace query (no device work): a tensor Gauss-Legendre grid of at most 16
    points per input gets the sum-factorization buffers, which grow with the field count (the
    intermediate tensors of rows x fields FP64 values: for 5^4 points and total degree 4, 625 and 375
    rows; for 16^2 points and degree 2, 16 x 3); Smolyak grids, tensor grids of 17 points and Monte
    Carlo sets keep the dense workspace or have none."""
    ctx = U.uqlb_create(0)
    try:
        U.uqlb_set_inputs(ctx, W.TGV4D_BOUNDS)
        U.uqlb_init_gpc(ctx, 4, 5)
        dense = U.uqlb_post_workspace_bytes(ctx)
        assert dense >= 70 * 625 * 8
        small, big = U.uqlb_project_workspace_bytes(ctx, 32), U.uqlb_project_workspace_bytes(ctx, 32 * 1000)
        assert (625 + 375) * 32 * 8 <= small < (625 + 375) * 32 * 8 + 4096
        assert (625 + 375) * 32000 * 8 <= big < (625 + 375) * 32000 * 8 + 4096
        U.uqlb_init_gpc(ctx, 2, 3, 0, U.UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK)
        assert U.uqlb_project_workspace_bytes(ctx, 32000) == U.uqlb_post_workspace_bytes(ctx)
        U.uqlb_set_inputs(ctx, [(0.0, 1.0), (1.0, 2.0)])
        U.uqlb_init_gpc(ctx, 2, 17)
        assert U.uqlb_project_workspace_bytes(ctx, 32000) == U.uqlb_post_workspace_bytes(ctx)
        U.uqlb_init_gpc(ctx, 2, 16)  # one intermediate tensor of 16 x 3 rows
        assert 48 * 32000 * 8 <= U.uqlb_project_workspace_bytes(ctx, 32000) < 48 * 32000 * 8 + 4096
        U.uqlb_init_mc(ctx, 100, 1)
        with pytest.raises(U.UqlbError):
            U.uqlb_project_workspace_bytes(ctx, 32)
    finally:
        U.uqlb_destroy(ctx)


def test_mc_sample_set_matches_oracle_bit_for_bit():
    ctx = U.uqlb_create(0)
    try:
        U.uqlb_set_inputs(ctx, W.TGV4D_BOUNDS)
        U.uqlb_init_mc(ctx, 300, 123456)
        z, xi, a = U.uqlb_get_samples(ctx, 4)
        zo, xio = ouq.mc_samples(300, W.TGV4D_BOUNDS, 123456)
        assert np.array_equal(z, zo) and np.array_equal(xi, xio)
        assert np.allclose(a, 1 / 300, rtol=0, atol=0)
        assert U.uqlb_num_terms(ctx) == 0
    finally:
        U.uqlb_destroy(ctx)


def test_ensemble_mapping_of_inputs_to_parameters():
    ctx = U.uqlb_create(0)
    try:
        w = W.tgv256_gpc4d(n=32, steps=10, pts=2)
        U.uqlb_set_inputs(ctx, w.bounds)
        U.uqlb_init_gpc(ctx, 1, 2)
        smp = U.uqlb_ensemble_samples(ctx, case_struct(w))
        z, _, _ = U.uqlb_get_samples(ctx, 4)
        for s, zz in zip(smp, z):
            assert s.nu == zz[0] and s.u0 == zz[1]
            assert s.amp2 == zz[2] * zz[1] and s.amp3 == zz[3] * zz[1]
            assert (s.nx, s.ny, s.steps) == (32, 32, 10)
    finally:
        U.uqlb_destroy(ctx)


@pytest.mark.parametrize("nd", [10, 20, 40])
def test_obstacle_mask_matches_oracle(nd):
    spec = W.channel(nd)
    m = U.uqlb_obstacle_mask(sample_struct(spec))
    mo = olbm.obstacle_mask(olbm.Case(olbm.CHANNEL, spec.nx, spec.ny, 1, spec.nu, spec.u0, u_ref=0.0,
                                      cyl_cx=spec.cyl_cx, cyl_cy=spec.cyl_cy, cyl_r=spec.cyl_r))
    assert np.array_equal(m, mo)


def test_host_mean_std_match_numpy():
    v = np.random.default_rng(5).normal(size=101)
    assert U.uqlb_mean_host(v) == pytest.approx(v.mean(), rel=1e-15)
    assert U.uqlb_std_host(v, 1) == pytest.approx(v.std(ddof=1), rel=1e-14)
    assert U.uqlb_std_host(v, 0) == pytest.approx(v.std(ddof=0), rel=1e-14)


def test_argument_errors_return_status_codes():
    with pytest.raises(U.UqlbError) as e:
        U.uqlb_gauss_legendre(0)
    assert e.value.status == U.UQLB_ERR_ARG
    ctx = U.uqlb_create(0)
    try:
        with pytest.raises(U.UqlbError) as e:
            U.uqlb_init_gpc(ctx, 2, 3)
        assert e.value.status == U.UQLB_ERR_STATE
        with pytest.raises(U.UqlbError) as e:
            U.uqlb_set_inputs(ctx, [(1.0, 0.5)])
        assert e.value.status == U.UQLB_ERR_ARG and "a < b" in U.uqlb_last_error(ctx)
        U.uqlb_set_inputs(ctx, [(0.02, 0.06)])
        U.uqlb_init_mc(ctx, 4, 1)
        with pytest.raises(U.UqlbError) as e:
            U.uqlb_get_weight_matrix(ctx)
        assert e.value.status == U.UQLB_ERR_STATE
    finally:
        U.uqlb_destroy(ctx)
    bad = sample_struct(W.tgv(1, 10))
    with pytest.raises(U.UqlbError):
        U.uqlb_batch_workspace_bytes([bad], U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0))
    with pytest.raises(U.UqlbError):
        U.uqlb_batch_workspace_bytes([sample_struct(W.tgv(16, 10))], U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 3, 1, 0, 0, 0, 0))


def test_workspace_bytes_cover_the_arena():
    """One lattice for the one-step scheme, two for the two-step scheme (the default for periodic
    FP32, FP16 and BF16 batches)."""
    s = [sample_struct(W.tgv(256, 10)) for _ in range(3)]
    for storage, eb in ((U.UQLB_F64, 8), (U.UQLB_F32, 4), (U.UQLB_F16, 2), (U.UQLB_BF16, 2), (U.UQLB_FX16, 2)):
        arena = 3 * 9 * 256 * 256 * eb
        lattices = 2 if storage != U.UQLB_F64 else 1
        b = U.uqlb_batch_workspace_bytes(s, U.uqlb_run_opts(storage, U.UQLB_F32, 0, 0, 0))
        assert lattices * arena <= b < lattices * arena + 2 ** 20
        one = U.uqlb_run_opts(storage, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, U.UQLB_SCHEME_ONE_STEP)
        assert arena <= U.uqlb_batch_workspace_bytes(s, one) < arena + 2 ** 20
        two = U.uqlb_run_opts(storage, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, U.UQLB_SCHEME_TWO_STEP)
        assert 2 * arena <= U.uqlb_batch_workspace_bytes(s, two) < 2 * arena + 2 ** 20
    # rows are padded to 128 bytes: 100 FP32 columns take a 128-column pitch
    b = U.uqlb_batch_workspace_bytes([sample_struct(W.tgv(100, 10))], U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0))
    assert b >= 9 * 128 * 100 * 4
    assert U.uqlb_plain_workspace_bytes(s) >= 2 * 9 * 256 * 256 * 8


@pytest.mark.parametrize("d,level", [(1, 3), (2, 2), (4, 3), (3, 4)])
def test_smolyak_grid_and_weights_match_oracle(d, level):
    bounds = W.TGV4D_BOUNDS[:d] if d <= 4 else None
    ctx = U.uqlb_create(0)
    try:
        U.uqlb_set_inputs(ctx, bounds)
        U.uqlb_init_gpc(ctx, level, level, U.UQLB_BASIS_TOTAL, U.UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK)
        z, xi, a = U.uqlb_get_samples(ctx, d)
        xo, ao = ouq.smolyak_cc(d, level)
        assert xi.shape == xo.shape and np.abs(xi - xo).max() < 1e-15
        assert np.abs(a - ao).max() < 1e-15
        zo = np.column_stack([ouq.map_uniform(xo[:, k], *bounds[k]) for k in range(d)])
        assert np.abs(z - zo).max() < 1e-15
        wm = U.uqlb_get_weight_matrix(ctx)
        assert np.abs(wm - ouq.weight_matrix(ouq.multi_indices(d, level), xo, ao)).max() < 1e-14
    finally:
        U.uqlb_destroy(ctx)


def test_halton_sample_set_matches_oracle_bit_for_bit():
    ctx = U.uqlb_create(0)
    try:
        U.uqlb_set_inputs(ctx, W.TGV4D_BOUNDS)
        U.uqlb_init_qmc(ctx, 500, 1)
        z, xi, a = U.uqlb_get_samples(ctx, 4)
        u = ouq.halton(500, 4, skip=1)
        assert np.array_equal(xi, 2.0 * u - 1.0)
        assert np.array_equal(z, np.column_stack([lo + (hi - lo) * u[:, k] for k, (lo, hi) in enumerate(W.TGV4D_BOUNDS)]))
        assert np.allclose(a, 1 / 500, rtol=0, atol=0)
        with pytest.raises(U.UqlbError):
            U.uqlb_init_gpc(ctx, 2, 7, U.UQLB_BASIS_TOTAL, U.UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK)
    finally:
        U.uqlb_destroy(ctx)


def test_unit_converter_matches_oracle_and_paper_table():
    for n, ma, re in [(8, 0.2, 320), (64, 0.025, 2560), (256, 0.00625, 10240)]:
        a = U.uqlb_unit_converter(n, ma, re)
        b = ouq.unit_converter(n, ma, re)
        for key in ("dx", "dt", "tau"):
            assert abs(a[key] - b[key]) <= 1e-15 * abs(b[key])
        assert abs(a["u_lattice"] - ma / math.sqrt(3)) < 1e-15


def test_perturbation_parameters_map_to_the_sample():
    ctx = U.uqlb_create(0)
    try:
        p = U.uqlb_unit_converter(32, 1.6 / 32, 40 * 32)
        w = W.tgv_paper4d(32, p["tau"], p["u_lattice"], 100, sampling="smolyak", level=1, order=1)
        U.uqlb_set_inputs(ctx, w.bounds)
        U.uqlb_init_gpc(ctx, 1, 1, U.UQLB_BASIS_TOTAL, U.UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK)
        smp = U.uqlb_ensemble_samples(ctx, case_struct(w))
        z, _, _ = U.uqlb_get_samples(ctx, 4)
        assert len(smp) == 9
        for s, zz in zip(smp, z):
            assert s.kind == U.UQLB_CASE_TGV_PERTURBED and (s.nx, s.ny) == (31, 31)
            assert list(s.pert) == [v * p["u_lattice"] for v in zz]
    finally:
        U.uqlb_destroy(ctx)


def test_paper_study_draws_n_monte_carlo_samples_at_resolution_n():
    ctx = U.uqlb_create(0)
    try:
        for n in (8, 32):
            p = U.uqlb_unit_converter(n, 1.6 / n, 40 * n)
            w = W.tgv_paper4d(n, p["tau"], p["u_lattice"], 10)
            assert w.method == "mc" and w.n_mc == n
            U.uqlb_set_inputs(ctx, w.bounds)
            U.uqlb_init_mc(ctx, w.n_mc, w.seed)
            smp = U.uqlb_ensemble_samples(ctx, case_struct(w))
            z, _, _ = U.uqlb_get_samples(ctx, 4)
            zr, _ = ouq.mc_samples(n, w.bounds, w.seed)
            assert len(smp) == n and np.array_equal(z, zr)
            assert all(abs(v) <= 0.025 * p["u_lattice"] for s in smp for v in s.pert)
    finally:
        U.uqlb_destroy(ctx)


def test_cylinder_method_comparison_samples_are_nested_and_in_the_inflow_range():
    """MC and QMC sets of size N are prefixes of the largest set (one batch serves every N), and
    every sample's mean inflow lies in the +-20 % range of the comparison."""
    ctx = U.uqlb_create(0)
    try:
        lo, hi = 0.8 * 0.04, 1.2 * 0.04
        for method in ("mc", "qmc", "gpc"):
            w = W.cylinder_uq(20, method=method, n=40 if method != "gpc" else 11)
            assert w.bounds == [(lo, hi)]
            U.uqlb_set_inputs(ctx, w.bounds)
            if method == "mc":
                U.uqlb_init_mc(ctx, 40, w.seed)
            elif method == "qmc":
                U.uqlb_init_qmc(ctx, 40, 1)
            else:
                U.uqlb_init_gpc(ctx, 5, 11, U.UQLB_BASIS_TOTAL, U.UQLB_QUAD_GAUSS_LEGENDRE_TENSOR)
            big = U.uqlb_ensemble_samples(ctx, case_struct(w))
            assert all(lo <= s.u0 <= hi and s.kind == U.UQLB_CASE_CHANNEL for s in big)
            if method == "gpc":
                continue
            if method == "mc":
                U.uqlb_init_mc(ctx, 10, w.seed)
            else:
                U.uqlb_init_qmc(ctx, 10, 1)
            small = U.uqlb_ensemble_samples(ctx, case_struct(w))
            assert [s.u0 for s in small] == [s.u0 for s in big[:10]]
    finally:
        U.uqlb_destroy(ctx)


def test_scheme_selection_and_its_limits():
    tgv = [sample_struct(W.tgv(64, 10))]
    chan = [sample_struct(W.channel(5, steps=10, steady_tol=0.0))]
    two = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, U.UQLB_MODE_GRAPH, U.UQLB_SCHEME_TWO_STEP)
    for smp, opts in ((chan, two),
                      (tgv, U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, U.UQLB_MODE_PERSISTENT,
                                            U.UQLB_SCHEME_TWO_STEP)),
                      (tgv, U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 2, 1, 0, 0, 0, U.UQLB_SCHEME_TWO_STEP)),
                      (tgv, U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, 9))):
        with pytest.raises(U.UqlbError) as e:
            U.uqlb_batch_workspace_bytes(smp, opts)
        assert e.value.status == U.UQLB_ERR_ARG
    # the row-strip kernel: FP32/FP16/BF16, one width, up to 2048 (FP32: 1600; rows padded to 64 columns)
    strips = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, U.UQLB_SCHEME_TWO_STEP_STRIPS)
    bf16_strips = U.uqlb_run_opts(U.UQLB_BF16, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, U.UQLB_SCHEME_TWO_STEP_STRIPS)
    tiles = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, U.UQLB_SCHEME_TWO_STEP_TILES)
    f64_strips = U.uqlb_run_opts(U.UQLB_F64, U.UQLB_F64, 0, 0, 0, 0, 0, 0, 0, U.UQLB_SCHEME_TWO_STEP_STRIPS)
    for smp, opts in (([sample_struct(W.tgv(4096, 10))], strips), ([sample_struct(W.tgv(1601, 10))], strips),
                      ([sample_struct(W.tgv(1664, 10))], strips), ([sample_struct(W.tgv(2049, 10))], bf16_strips),
                      ([sample_struct(W.tgv(64, 10)), sample_struct(W.tgv(128, 10))], strips), (tgv, f64_strips),
                      (chan, strips), (chan, tiles)):
        with pytest.raises(U.UqlbError) as e:
            U.uqlb_batch_workspace_bytes(smp, opts)
        assert e.value.status == U.UQLB_ERR_ARG
    for n in (2, 31, 40, 64, 97, 128, 1599, 1600):
        assert U.uqlb_batch_workspace_bytes([sample_struct(W.tgv(n, 10))], strips) >= 2 * 9 * n * n * 4
    assert U.uqlb_batch_workspace_bytes([sample_struct(W.tgv(2048, 10))], bf16_strips) >= 2 * 9 * 2048 * 2048 * 2
    assert U.uqlb_batch_workspace_bytes([sample_struct(W.tgv(40, 10))], tiles) >= 2 * 9 * 40 * 40 * 4
    # auto: channel batches and persistent mode stay one-step (one lattice)
    auto_chan = U.uqlb_batch_workspace_bytes(chan, U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0))
    one_chan = U.uqlb_batch_workspace_bytes(
        chan, U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, U.UQLB_SCHEME_ONE_STEP))
    assert auto_chan == one_chan


def test_strip_launch_shape_options_are_checked():
    """The three-step strips' launch-shape options: blocks per SM 0..32, staging option 0..3 (the
    fixed widths only), shared-memory share 0 or one of the carveout configurations; none of them
    changes the workspace."""
    def opts(bps=0, stage=0, kb=0, scheme=U.UQLB_SCHEME_THREE_STEP_STRIPS):
        return U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, scheme, bps, stage, kb)

    fixed = [sample_struct(W.tgv(256, 10))]
    ragged = [sample_struct(W.tgv(200, 10))]
    base = U.uqlb_batch_workspace_bytes(fixed, opts())
    for bps, stage, kb in ((1, 1, 8), (4, 2, 196), (32, 0, 228), (0, 0, 100), (3, 2, 0), (6, 3, 228)):
        assert U.uqlb_batch_workspace_bytes(fixed, opts(bps, stage, kb)) == base
    assert U.uqlb_batch_workspace_bytes(ragged, opts(2, 0, 164)) > 0
    for smp, o in ((fixed, opts(-1)), (fixed, opts(33)), (fixed, opts(0, 4)), (fixed, opts(0, -1)),
                   (fixed, opts(0, 0, 50)), (fixed, opts(0, 0, 256)), (fixed, opts(0, 0, -8)),
                   (ragged, opts(0, 1)), (ragged, opts(0, 2)), (ragged, opts(0, 3))):
        with pytest.raises(U.UqlbError) as e:
            U.uqlb_batch_workspace_bytes(smp, o)
        assert e.value.status == U.UQLB_ERR_ARG
    # other schemes ignore the strip options (range-checked all the same)
    one = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, U.UQLB_SCHEME_ONE_STEP, 4, 2, 196)
    assert U.uqlb_batch_workspace_bytes(ragged, one) > 0


def test_grouped_batch_workspace_is_the_sum_of_its_groups():
    """Under the auto scheme a batch of unlike samples runs as groups (channel samples one-step,
    periodic samples of each strip width on strips, periodic samples too wide for the strips on
    tiles), each in its own 256-byte aligned slice of the workspace, in that order.  The total is
    the sum of the groups' own workspaces, so a resumed run finds every group where the first run
    left it."""
    tgv64 = [W.tgv(64, 10, nu=0.03), W.tgv(64, 12, nu=0.04)]
    tgv128 = [W.tgv(128, 9, nu=0.05)]
    tgv40 = [W.tgv(40, 11, nu=0.02)]
    chan = [W.channel(5, steps=10, steady_tol=0.0), W.channel(6, steps=8, steady_tol=0.0)]
    mixed = [tgv64[0], chan[0], tgv128[0], tgv40[0], chan[1], tgv64[1]]

    def opts(scheme):
        return U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, U.UQLB_MODE_GRAPH, scheme)

    def ws(specs, scheme):
        return U.uqlb_batch_workspace_bytes([sample_struct(x) for x in specs], opts(scheme))

    align = lambda b: (b + 255) // 256 * 256  # noqa: E731
    parts = [ws(chan, U.UQLB_SCHEME_ONE_STEP), ws(tgv40, U.UQLB_SCHEME_TWO_STEP_STRIPS),
             ws(tgv64, U.UQLB_SCHEME_TWO_STEP_STRIPS), ws(tgv128, U.UQLB_SCHEME_TWO_STEP_STRIPS)]
    assert ws(mixed, U.UQLB_SCHEME_AUTO) == sum(align(b) for b in parts)
    wide = [W.tgv(1700, 3, nu=0.03)]  # wider than the FP32 strips take: tiles
    mixed2 = [wide[0], chan[0], tgv64[0]]
    parts2 = [ws([chan[0]], U.UQLB_SCHEME_ONE_STEP), ws(wide, U.UQLB_SCHEME_TWO_STEP_TILES),
              ws([tgv64[0]], U.UQLB_SCHEME_TWO_STEP_STRIPS)]
    assert ws(mixed2, U.UQLB_SCHEME_AUTO) == sum(align(b) for b in parts2)
    # one group: no split (the batch plans as before)
    assert ws(tgv64, U.UQLB_SCHEME_AUTO) == ws(tgv64, U.UQLB_SCHEME_TWO_STEP_STRIPS)
    assert ws(chan, U.UQLB_SCHEME_AUTO) == ws(chan, U.UQLB_SCHEME_ONE_STEP)
    # FP64 storage and the explicit schemes keep one batch
    f64 = U.uqlb_run_opts(U.UQLB_F64, U.UQLB_F64, 0, 0, 0, 0, 0, 0, U.UQLB_MODE_GRAPH, U.UQLB_SCHEME_AUTO)
    f64_one = U.uqlb_run_opts(U.UQLB_F64, U.UQLB_F64, 0, 0, 0, 0, 0, 0, U.UQLB_MODE_GRAPH, U.UQLB_SCHEME_ONE_STEP)
    smp = [sample_struct(x) for x in mixed]
    assert U.uqlb_batch_workspace_bytes(smp, f64) == U.uqlb_batch_workspace_bytes(smp, f64_one)


def test_interpolated_inlet_outlet_samples_are_checked():
    graph = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 10, 0, 0, 0, 0, 0, U.UQLB_MODE_GRAPH, 0)
    ok = sample_struct(W.channel(5, steps=10, steady_tol=0.0, inout="interpolated"))
    assert U.uqlb_batch_workspace_bytes([ok], graph) > U.uqlb_batch_workspace_bytes(
        [sample_struct(W.channel(5, steps=10, steady_tol=0.0))], graph)  # the boundary buffer
    bad = []
    s = sample_struct(W.channel(5, steps=10, steady_tol=0.0, inout="interpolated"))
    s.cyl_cx = 3.0                      # obstacle reaching into the three inlet columns
    bad.append((s, graph))
    s = sample_struct(W.channel(5, steps=10, steady_tol=0.0, inout="interpolated"))
    s.inout_bc = 5                      # unknown scheme
    bad.append((s, graph))
    bad.append((ok, U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 10, 0, 0, 0, 0, 0, U.UQLB_MODE_PERSISTENT, 0)))
    for smp, opts in bad:
        with pytest.raises(U.UqlbError) as e:
            U.uqlb_batch_workspace_bytes([smp], opts)
        assert e.value.status == U.UQLB_ERR_ARG


def test_bouzidi_samples_are_checked():
    """The obstacle scheme is validated, and Bouzidi batches are refused outside graph mode (the
    force kernel runs between step launches)."""
    s = sample_struct(W.channel(5, steps=10, steady_tol=0.0, bc="bouzidi"))
    graph = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 10, 0, 0, 0, 0, 0, U.UQLB_MODE_GRAPH, 0)
    assert U.uqlb_batch_workspace_bytes([s], graph) > 0
    pers = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 10, 0, 0, 0, 0, 0, U.UQLB_MODE_PERSISTENT, 0)
    with pytest.raises(U.UqlbError) as e:
        U.uqlb_batch_workspace_bytes([s], pers)
    assert e.value.status == U.UQLB_ERR_ARG
    s.obstacle_bc = 7
    with pytest.raises(U.UqlbError) as e:
        U.uqlb_batch_workspace_bytes([s], graph)
    assert e.value.status == U.UQLB_ERR_ARG


def test_untuned_workspace_covers_every_geometry_for_every_entry_point():
    """With geometry 0/0 the batch, ensemble and end-to-end workspace queries all cover every
    compiled tile geometry, since an autotuned run may use any of them."""
    ctx = U.uqlb_create(0)
    try:
        w = W.tgv256_gpc4d(n=96, steps=10, pts=2)
        U.uqlb_set_inputs(ctx, w.bounds)
        U.uqlb_init_gpc(ctx, 1, 2)
        case = case_struct(w)
        smp = U.uqlb_ensemble_samples(ctx, case)
        auto = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, 0)
        ens_b = U.uqlb_ensemble_workspace_bytes(ctx, case, auto)
        assert ens_b == U.uqlb_batch_workspace_bytes(smp, auto)
        assert U.uqlb_uq_workspace_bytes(ctx, case, auto) > ens_b
        for tr, npt in ((4, 4), (8, 2), (8, 4), (16, 2), (16, 4)):  # two-step geometries (auto scheme)
            fixed = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, tr, npt, 0, 0, 0, 0)
            assert U.uqlb_batch_workspace_bytes(smp, fixed) <= ens_b
        one = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, 0, 0, 0, 0, 0, U.UQLB_SCHEME_ONE_STEP)
        one_b = U.uqlb_batch_workspace_bytes(smp, one)
        for tr in (2, 4, 8):
            for npt in (1, 2, 4):
                fixed = U.uqlb_run_opts(U.UQLB_F32, U.UQLB_F32, 0, 0, tr, npt, 0, 0, 0, U.UQLB_SCHEME_ONE_STEP)
                assert U.uqlb_batch_workspace_bytes(smp, fixed) <= one_b
    finally:
        U.uqlb_destroy(ctx)


_C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
_WQ = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
_CLASS = np.array([0, 1, 1, 1, 1, 2, 2, 2, 2])


def _class_max_of_equilibrium(r):
    """Largest |g_i| per velocity class of the shifted equilibrium of an oracle state (u, v, rho)."""
    drho = r.rho - 1.0
    usq = r.u * r.u + r.v * r.v
    out = np.zeros(3)
    fluid = r.rho != 0
    for i in range(9):
        cu = _C[i, 0] * r.u + _C[i, 1] * r.v
        g = _WQ[i] * (drho + r.rho * (3 * cu + 4.5 * cu * cu - 1.5 * usq))
        out[_CLASS[i]] = max(out[_CLASS[i]], np.abs(g[fluid]).max())
    return out


def test_fixed_point_quanta_bound_the_populations():
    """The 16-bit fixed-point storage covers +-32767 quanta per velocity class.  The quanta come
    from a bound on |g_i|; the equilibrium populations of the oracle's states must stay inside that
    range with headroom: the initial Taylor-Green fields at the corners of the 4-D workload's input
    box and the Sec. 8.3 perturbed field keep the bound's margin of 1.5 (less FP32 rounding of the
    quanta), and the channel's states during and after the start-up ramp (halfway and Bouzidi
    obstacle, face and interpolated inlet/outlet, +-20 % inflow) stay below 0.8 of the range."""
    cases = []
    for u0 in (0.008, 0.012):
        for z2 in (-0.1, 0.1):
            for z3 in (-0.1, 0.1):
                cases.append(W.tgv(64, 0, nu=0.04, u0=u0, amp2=z2 * u0, amp3=z3 * u0))
    p = U.uqlb_unit_converter(64, 1.6 / 64, 40.0 * 64)
    ul = p["u_lattice"]
    for zs in ((0.025, -0.025, 0.025, -0.025), (0.0, 0.01, -0.02, 0.025)):
        cases.append(W.SampleSpec(W.TGV_PERTURBED, 63, 63, 0, 0.01, ul, u_ref=ul, pert=tuple(z * ul for z in zs)))
    from tests.helpers import oracle_case
    for spec in cases:
        q = U.uqlb_fx16_quanta(sample_struct(spec))
        r = olbm.run([oracle_case(spec)])[0]
        used = _class_max_of_equilibrium(r) / (32767 * q)
        assert np.all(used <= 1 / 1.45), (spec, used)
        # not loose by more than twice the margin for the moving populations, which carry the velocity
        # (the rest population's bound adds the density and kinetic terms at their separate maxima)
        assert np.all(used[1:] >= 1 / 3.0) and used[0] >= 1 / 6.0, (spec, used)
    # a Taylor-Green field on a non-square lattice is not divergence-free: its acoustic waves move the
    # density far beyond the square lattice's bound; the states over 400 steps stay inside the range
    for nx, ny in ((128, 64), (64, 8), (96, 40)):
        for steps in (20, 100, 400):
            spec = replace(W.tgv(nx, steps, nu=0.03, amp2=0.0005), ny=ny)
            q = U.uqlb_fx16_quanta(sample_struct(spec))
            used = _class_max_of_equilibrium(olbm.run([oracle_case(spec)])[0]) / (32767 * q)
            assert np.all(used < 0.8), (nx, ny, steps, used)
    for u in (0.032, 0.048):
        for bc, io in (("halfway", "face"), ("bouzidi", "interpolated")):
            for steps in (300, 900, 3000):
                spec = W.channel(6, u_mean=u, steps=steps, steady_tol=0.0, bc=bc, inout=io)
                q = U.uqlb_fx16_quanta(sample_struct(spec))
                used = _class_max_of_equilibrium(olbm.run([oracle_case(spec)])[0]) / (32767 * q)
                assert np.all(used < 0.8), (u, bc, io, steps, used)
