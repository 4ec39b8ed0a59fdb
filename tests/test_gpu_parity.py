"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element on the
same seeded inputs.  Tolerances are the stated error budget of each storage format against the
FP64 oracle (relative L2): FP64 1e-12, FP32 1e-5, FP16/BF16 1e-3."""
import math
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lbm as olbm  # noqa: E402
from oracle import uq as ouq  # noqa: E402
from paper_2508_13867_gb300 import uqlb as U  # noqa: E402
from paper_2508_13867_gb300 import workloads as W  # noqa: E402
from paper_2508_13867_gb300.ensemble import Ensemble, sample_struct  # noqa: E402
from tests.helpers import oracle_case, oracle_row, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 1e-3, "bf16": 1e-3, "fx16": 1e-3}

# IEEE BF16 keeps 8 significant bits: every store rounds g by up to 2^-8 of itself (stochastic
# rounding) and the velocity is a sum of six such populations, so a single rounding of the
# initial state already costs ~8e-4 of the field; after a few hundred steps the per-sample field
# error is ~3e-3 to 1e-2 (measured), above the 1e-3 budget.  These cases stay asserted at the
# budget and are expected to fail until a BF16 run meets it; the fixed-point format FX16 is the
# 16-bit storage that does.
BF16_MISS = pytest.mark.xfail(strict=True, reason="IEEE BF16 storage misses the 1e-3 budget (8 significant bits)")


def _storages(*names):
    return [pytest.param(n, marks=BF16_MISS) if n == "bf16" else n for n in names]


@pytest.fixture(scope="module")
def ens():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2508_13867_gb300 import build

    build.build()
    e = Ensemble(0)
    yield e
    e.close()


def _run(ens, specs, storage, qoi_every=0, series=False, tile_rows=0, chunk=0, npt=0, scheme="auto",
         strip=(0, 0, 0)):
    res = ens.run_batch([sample_struct(s) for s in specs], storage=storage,
                        fields_dtype="f64" if storage == "f64" else "f32", qoi_every=qoi_every, series=series,
                        tile_rows=tile_rows, nodes_per_thread=npt, chunk_steps=chunk,
                        fields=len({(s.nx, s.ny) for s in specs}) == 1, scheme=scheme, strip=strip)
    torch.cuda.synchronize()
    return {k: v.double().cpu().numpy() for k, v in res.items()}


def _tgv_specs(n, steps, nus=(0.02, 0.037, 0.06), modes=True):
    out = []
    for i, nu in enumerate(nus):
        a2 = (0.07 - 0.05 * i) * 0.01 if modes else 0.0
        a3 = (-0.04 + 0.03 * i) * 0.01 if modes else 0.0
        out.append(W.tgv(n, steps, nu=nu, u0=0.01 * (0.9 + 0.1 * i), amp2=a2, amp3=a3))
    return out


@pytest.mark.parametrize("n,steps", [(64, 100), (70, 101), (33, 1), (40, 0)])
def test_tgv_f64_fields_energy_and_invariants(ens, n, steps):
    specs = _tgv_specs(n, steps)
    g = _run(ens, specs, "f64", qoi_every=10, series=True)
    ref = olbm.run([oracle_case(s, qoi_every=10) for s in specs])
    for i, r in enumerate(ref):
        assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL["f64"]
        assert abs(g["qoi"][i, U.UQLB_QOI_K] - r.k_final) < 1e-12 * abs(r.k_final)
        assert abs(g["qoi"][i, U.UQLB_QOI_MASS] - r.mass) < 1e-12 * r.mass
        assert abs(g["qoi"][i, U.UQLB_QOI_MOMX] - r.mom_x) < 1e-12 * r.mass
        assert abs(g["qoi"][i, U.UQLB_QOI_MOMY] - r.mom_y) < 1e-12 * r.mass
        assert g["qoi"][i, U.UQLB_QOI_STEPS] == steps and g["qoi"][i, U.UQLB_QOI_STATUS] == 0
        ns = steps // 10 + 1
        assert np.allclose(g["series"][i, :ns], r.series[:ns], rtol=1e-12, atol=0)


@pytest.mark.parametrize("scheme", ["auto", "one_step", "two_step_tiles", "three_step_strips"])
@pytest.mark.parametrize("storage", _storages("f32", "f16", "bf16", "fx16"))
def test_tgv_reduced_precision_storage(ens, storage, scheme):
    """Per-sample velocity fields and K(T) against the oracle within the storage's budget (96 x 96,
    300 steps, three samples), on the row strips (auto), the one-step and the two-step tile kernels."""
    specs = _tgv_specs(96, 300)
    g = _run(ens, specs, storage, scheme=scheme)
    ref = olbm.run([oracle_case(s) for s in specs])
    for i, r in enumerate(ref):
        err = rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1])
        print(f"storage {storage} {scheme} sample {i}: fields {err:.3e}")
        assert err < TOL[storage], (storage, scheme, err)
        assert abs(g["qoi"][i, U.UQLB_QOI_K] - r.k_final) < TOL[storage] * r.k_final, (storage, scheme)
        assert g["qoi"][i, U.UQLB_QOI_STATUS] == 0


@pytest.mark.parametrize("storage,rounding", [("f32", "auto"), ("f16", "auto"), ("f16", "nearest"),
                                              pytest.param("bf16", "auto", marks=BF16_MISS),
                                              pytest.param("bf16", "nearest", marks=BF16_MISS),
                                              ("fx16", "auto"), ("fx16", "nearest")])
def test_reduced_precision_ensemble_statistics(ens, storage, rounding):
    """Mean and standard deviation of the velocity fields over 64 seeded MC samples of the 4-D
    Taylor-Green set-up (64 x 64, 300 steps) against the same statistics of the oracle, within the
    storage's budget.  16-bit storage rounds stochastically by default ("auto") or to nearest even.
    The storage noise e of one sample moves the N-sample std by about e / (sigma sqrt N) (sigma the
    spread of the samples, ~0.12 of the field here); 64 samples is the oracle subset of the 512 x 512
    Monte Carlo workload."""
    e = Ensemble(0)
    w = W.tgv512_mc4d(n=64, steps=300, n_mc=64)
    e.setup(w)
    smp = e.ensemble_samples(w)
    res = e.run_batch(smp, storage=storage, fields_dtype="f32", rounding=rounding)
    mean, var = e.stats(res["fields"], ddof=1)
    torch.cuda.synchronize()
    specs = [W.SampleSpec(W.TGV, 64, 64, 300, s.nu, s.u0, s.amp2, s.amp3) for s in smp]
    mref = np.stack([oracle_row(r) for r in olbm.run([oracle_case(s) for s in specs])])
    mu_r, var_r = ouq.mc_mean_var(mref, ddof=1)
    m_err = rel_l2(mean.cpu().numpy()[:-1], mu_r[:-1])
    s_err = rel_l2(np.sqrt(var.cpu().numpy()[:-1]), np.sqrt(var_r[:-1]))
    f = res["fields"].double().cpu().numpy()
    worst = max(rel_l2(f[i, :-1], mref[i, :-1]) for i in range(len(smp)))
    print(f"precision {storage}/{rounding}: mean {m_err:.3e} std {s_err:.3e} worst sample {worst:.3e}")
    tol = TOL[storage]
    assert m_err < tol and s_err < tol and worst < tol, (storage, rounding, m_err, s_err, worst)
    e.close()


GEOMETRIES = [("f32", tr, n) for tr in (2, 4, 8) for n in (1, 2, 4)] + [("f64", 8, 1), ("f64", 4, 1), ("f64", 4, 2),
                                                                         ("bf16", 2, 4), ("f16", 8, 4)]


@pytest.mark.parametrize("storage,tr,npt", GEOMETRIES)
def test_tile_shapes_and_chunks_agree(ens, storage, tr, npt):
    """Tile shape and graph chunk change the launch geometry and the grouping of the QoI partial
    sums, not the per-node arithmetic: results agree to round-off (ragged 50 x 50 lattices)."""
    specs = _tgv_specs(50, 31)
    a = _run(ens, specs, storage, qoi_every=5, series=True, scheme="one_step")
    b = _run(ens, specs, storage, qoi_every=5, series=True, tile_rows=tr, npt=npt, chunk=6, scheme="one_step")
    tol = 1e-14 if storage == "f64" else 1e-6
    assert rel_l2(b["fields"], a["fields"]) < tol
    assert np.allclose(b["series"], a["series"], rtol=tol, atol=0)


def test_mixed_batch_geometries_agree(ens):
    specs = [W.tgv(40, 21, nu=0.03), _cyl(4, 21, u_mean=0.04)]
    a = _run(ens, specs, "f64", qoi_every=7, series=True)
    b = _run(ens, specs, "f64", qoi_every=7, series=True, tile_rows=4, npt=1, chunk=4)
    assert np.allclose(b["qoi"], a["qoi"], rtol=1e-13, atol=1e-15)


def _cyl(nd, steps, **kw):
    """Coarse channel for parity runs: Re = 5 keeps tau well above 1/2 at 4..6 nodes per diameter."""
    return W.channel(nd, steps=steps, steady_tol=kw.pop("steady_tol", 0.0), re=kw.pop("re", 5.0), **kw)


@pytest.mark.parametrize("steps", [800, 801])
def test_channel_obstacle_f64_fields_and_forces(ens, steps):
    specs = [_cyl(5, steps, u_mean=0.036), _cyl(5, steps, u_mean=0.044)]
    g = _run(ens, specs, "f64", qoi_every=50, series=True)
    ref = olbm.run([oracle_case(s, qoi_every=50) for s in specs])
    for i, r in enumerate(ref):
        assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL["f64"]
        assert abs(g["qoi"][i, U.UQLB_QOI_CD] - r.cd) < 1e-11 * abs(r.cd)
        assert abs(g["qoi"][i, U.UQLB_QOI_CL] - r.cl) < 1e-11 * abs(r.cd)
        assert abs(g["qoi"][i, U.UQLB_QOI_MASS] - r.mass) < 1e-12 * r.mass
        ns = steps // 50
        assert np.allclose(g["series"][i, :ns], r.series[:ns], rtol=1e-11, atol=1e-14)
        assert np.allclose(g["series_cl"][i, :ns], r.series_cl[:ns], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("steps", [600, 601])
def test_bouzidi_obstacle_matches_oracle(ens, steps):
    """Bouzidi interpolated bounce-back on the obstacle (Sec. 8.1): fields, the C_D / C_L series
    written by the between-step force kernel and the final forces against the oracle, for odd and
    even step counts (both AA parities of the last step).  FP32 forces carry 1e-4: the momentum
    sum cancels terms ~10x larger than the force."""
    specs = [_cyl(5, steps, u_mean=0.036, bc="bouzidi"), _cyl(5, steps, u_mean=0.044, bc="bouzidi")]
    ref = olbm.run([oracle_case(s, qoi_every=50) for s in specs])
    ns = steps // 50
    for storage, tol_f in (("f64", 1e-11), ("f32", 1e-4)):
        g = _run(ens, specs, storage, qoi_every=50, series=True)
        for i, r in enumerate(ref):
            assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL[storage], storage
            assert abs(g["qoi"][i, U.UQLB_QOI_CD] - r.cd) < tol_f * abs(r.cd), storage
            assert abs(g["qoi"][i, U.UQLB_QOI_CL] - r.cl) < tol_f * abs(r.cd), storage
            assert np.allclose(g["series"][i, :ns], r.series[:ns], rtol=tol_f, atol=0), storage
            assert np.allclose(g["series_cl"][i, :ns], r.series_cl[:ns], rtol=0, atol=tol_f * abs(r.cd)), storage


def test_bouzidi_steady_state_stops_with_the_oracle_in_a_mixed_batch(ens):
    """The force kernel runs between steps, so a Bouzidi sample stops at the same step as the
    oracle; halfway and TGV samples in the same batch are unaffected."""
    specs = [_cyl(4, 20000, u_mean=0.04, steady_tol=1e-6, bc="bouzidi"),
             _cyl(4, 20000, u_mean=0.036, steady_tol=1e-6), W.tgv(40, 300, nu=0.03)]
    res = ens.run_batch([sample_struct(s) for s in specs], storage="f64", fields_dtype="f64", qoi_every=100,
                        series=True, fields=False)
    torch.cuda.synchronize()
    q = res["qoi"].cpu().numpy()
    ref = olbm.run([oracle_case(s, qoi_every=100) for s in specs])
    for i in (0, 1):
        assert ref[i].steps_run < 20000
        assert q[i, U.UQLB_QOI_STEPS] == ref[i].steps_run
        assert abs(q[i, U.UQLB_QOI_CD] - ref[i].cd) < 1e-10 * abs(ref[i].cd)
        assert abs(q[i, U.UQLB_QOI_MASS] - ref[i].mass) < 1e-12 * ref[i].mass
    assert abs(q[2, U.UQLB_QOI_K] - ref[2].k_final) < 1e-12 * ref[2].k_final


@pytest.mark.parametrize("steps", [600, 601])
def test_interpolated_inlet_outlet_matches_oracle(ens, steps):
    """Interpolated inlet/outlet on the end columns (Sec. 8.1): the boundary kernel between steps
    forms the end columns' state, the step and the finalize read it.  Fields, forces and the C_D
    series against the oracle at both parities of the last step, with the halfway and with the
    Bouzidi obstacle, FP64 and FP32."""
    specs = [_cyl(5, steps, u_mean=0.036, inout="interpolated"),
             _cyl(5, steps, u_mean=0.044, bc="bouzidi", inout="interpolated")]
    ref = olbm.run([oracle_case(s, qoi_every=50) for s in specs])
    ns = steps // 50
    for storage, tol_f in (("f64", 1e-11), ("f32", 1e-4)):
        g = _run(ens, specs, storage, qoi_every=50, series=True)
        for i, r in enumerate(ref):
            assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL[storage], (storage, i)
            assert abs(g["qoi"][i, U.UQLB_QOI_CD] - r.cd) < tol_f * abs(r.cd), (storage, i)
            assert abs(g["qoi"][i, U.UQLB_QOI_MASS] - r.mass) < 10 * TOL[storage] * r.mass, (storage, i)
            assert np.allclose(g["series"][i, :ns], r.series[:ns], rtol=tol_f, atol=0), (storage, i)


def test_interpolated_inlet_outlet_steady_stop_and_resume(ens):
    """A sample with the interpolated inlet/outlet stops at the oracle's steady-state step, and a
    run resumed at an odd step continues it bit for bit (the boundary buffer carries the end
    columns' state across the two calls)."""
    specs = [_cyl(4, 20000, u_mean=0.04, steady_tol=1e-6, inout="interpolated")]
    g = _run(ens, specs, "f64", qoi_every=100, series=True)
    r = olbm.run([oracle_case(specs[0], qoi_every=100)])[0]
    assert r.steps_run < 20000
    assert g["qoi"][0, U.UQLB_QOI_STEPS] == r.steps_run
    assert abs(g["qoi"][0, U.UQLB_QOI_CD] - r.cd) < 1e-10 * abs(r.cd)
    specs = [_cyl(4, 90, u_mean=0.04, inout="interpolated"), _cyl(4, 90, u_mean=0.04, bc="bouzidi", inout="interpolated")]
    whole = _run(ens, specs, "f64", qoi_every=10, series=True)
    first = [sample_struct(s) for s in specs]
    for s in first:
        s.steps = 37
    ens.run_batch(first, storage="f64", fields_dtype="f64", fields=False)
    res = ens.run_batch([sample_struct(s) for s in specs], storage="f64", fields_dtype="f64", fields=True,
                        start_step=37)
    torch.cuda.synchronize()
    assert np.array_equal(res["fields"].cpu().numpy(), whole["fields"])


def test_channel_without_obstacle_and_f32(ens):
    specs = [W.channel(6, steps=600, obstacle=False, steady_tol=0.0, re=5.0), _cyl(6, 600)]
    for storage in ("f64", "f32"):
        g = _run(ens, specs, storage)
        ref = olbm.run([oracle_case(s) for s in specs])
        for i, r in enumerate(ref):
            assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL[storage], storage


def test_channel_steady_state_stops_with_the_oracle(ens):
    specs = [_cyl(4, 20000, u_mean=0.04, steady_tol=1e-6), _cyl(4, 20000, u_mean=0.036, steady_tol=1e-6)]
    g = _run(ens, specs, "f64", qoi_every=100, series=True)
    ref = olbm.run([oracle_case(s, qoi_every=100) for s in specs])
    for i, r in enumerate(ref):
        assert r.steps_run < 20000
        assert g["qoi"][i, U.UQLB_QOI_STEPS] == r.steps_run
        assert abs(g["qoi"][i, U.UQLB_QOI_CD] - r.cd) < 1e-10 * abs(r.cd)
        assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < 1e-11


def test_uneven_batch_sizes_steps_and_kinds(ens):
    specs = [W.tgv(32, 57, nu=0.03), W.tgv(64, 20, nu=0.05, amp2=0.0007), W.tgv(48, 90, nu=0.021),
             _cyl(4, 130, u_mean=0.04), W.tgv(96, 3, nu=0.06)]
    for storage in ("f64", "f32"):
        g = _run(ens, specs, storage)
        ref = olbm.run([oracle_case(s) for s in specs])
        for i, r in enumerate(ref):
            assert g["qoi"][i, U.UQLB_QOI_STEPS] == specs[i].steps
            if specs[i].kind == W.TGV:
                assert abs(g["qoi"][i, U.UQLB_QOI_K] - r.k_final) < TOL[storage] * r.k_final
            else:
                assert abs(g["qoi"][i, U.UQLB_QOI_CD] - r.cd) < 100 * TOL[storage] * abs(r.cd)
            assert abs(g["qoi"][i, U.UQLB_QOI_MASS] - r.mass) < TOL[storage] * r.mass


def test_plain_f64_path_matches_oracle(ens):
    specs = _tgv_specs(40, 77) + [_cyl(4, 210, u_mean=0.04)]
    for group in (specs[:3], specs[3:]):
        res = ens.run_plain_f64([sample_struct(s) for s in group], qoi_every=7, series=True)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in res.items()}
        ref = olbm.run([oracle_case(s, qoi_every=7) for s in group])
        for i, r in enumerate(ref):
            assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL["f64"]
            assert abs(g["qoi"][i, U.UQLB_QOI_MASS] - r.mass) < 1e-12 * r.mass
            if group[i].kind == W.TGV:
                ns = group[i].steps // 7 + 1
                assert np.allclose(g["series"][i, :ns], r.series[:ns], rtol=1e-12, atol=0)
            else:
                assert abs(g["qoi"][i, U.UQLB_QOI_CD] - r.cd) < 1e-11 * abs(r.cd)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_projection_and_gpc_stats_match_oracle(ens, dtype):
    e = Ensemble(0)
    e.set_inputs(W.TGV4D_BOUNDS)
    e.init_gpc(4, 5)
    _, xi, a = ouq.tensor_grid([5] * 4, W.TGV4D_BOUNDS)
    m = W.random_fields(625, 1037, seed=21, dtype=np.float64 if dtype == "f64" else np.float32)
    mt = torch.from_numpy(m).cuda()
    c = e.project(mt)
    mean, var = e.stats(c)
    torch.cuda.synchronize()
    c_ref = ouq.gpc_coefficients(ouq.multi_indices(4, 4), xi, a, m.astype(np.float64))
    mean_ref, var_ref = ouq.gpc_mean_var(c_ref)
    assert np.abs(c.cpu().numpy() - c_ref).max() < 1e-13 * np.abs(c_ref).max()
    assert rel_l2(mean.cpu().numpy(), mean_ref) < 1e-14
    assert rel_l2(var.cpu().numpy(), var_ref) < 1e-12
    e.close()


@pytest.mark.parametrize("dims,pts,order,basis,n_fields,dtype", [
    (1, 5, 4, "total", 1037, "f64"),
    (2, 3, 2, "total", 777, "f32"),
    (2, 4, 3, "tensor", 513, "f64"),
    (3, 2, 1, "total", 300, "f32"),
    (3, 16, 2, "total", 129, "f64"),
    (4, 5, 4, "total", 1037, "f32"),
    (4, 3, 2, "tensor", 65, "f32"),
])
def test_sum_factorized_projection_matches_the_oracle_and_the_dense_contraction(ens, dims, pts, order, basis,
                                                                                n_fields, dtype):
    """Projection on a tensor Gauss-Legendre grid taken one input at a time (Eq. coef_discrete with a
    product weight), against the oracle's dense W M and the library's dense contraction (a block of
    all samples); ragged field counts that leave a partial block of threads."""
    bounds = [(0.5 + q, 1.5 + 2 * q) for q in range(dims)]
    e = Ensemble(0)
    e.set_inputs(bounds)
    e.init_gpc(order, pts, basis=U.UQLB_BASIS_TENSOR if basis == "tensor" else U.UQLB_BASIS_TOTAL)
    _, xi, a = ouq.tensor_grid([pts] * dims, bounds)
    m = W.random_fields(pts ** dims, n_fields, seed=7 + dims, dtype=np.float64 if dtype == "f64" else np.float32)
    mt = torch.from_numpy(m).cuda()
    c_sf = e.project(mt)
    assert U.uqlb_last_projection(e.ctx) == 1
    c_dense = e.project_block(mt, 0)  # the dense contraction over the whole sample set
    torch.cuda.synchronize()
    c_ref = ouq.gpc_coefficients(ouq.multi_indices(dims, order, basis), xi, a, m.astype(np.float64))
    scale = np.abs(c_ref).max()
    assert np.abs(c_sf.cpu().numpy() - c_ref).max() < 1e-13 * scale
    assert np.abs(c_sf.cpu().numpy() - c_dense.cpu().numpy()).max() < 1e-13 * scale
    e.close()


def test_projection_outside_the_sum_factorization_stays_dense(ens):
    """Smolyak points and tensor grids of more than 16 points per input take the dense contraction with
    either workspace."""
    for pts, quad in ((3, U.UQLB_QUAD_CLENSHAW_CURTIS_SMOLYAK), (17, U.UQLB_QUAD_GAUSS_LEGENDRE_TENSOR)):
        e = Ensemble(0)
        bounds = W.TGV4D_BOUNDS if pts == 3 else [(0.0, 1.0)]
        e.set_inputs(bounds)
        e.init_gpc(2, pts, quad=quad)
        xi, a = ouq.smolyak_cc(4, 3) if pts == 3 else ouq.tensor_grid([17], bounds)[1:]
        m = W.random_fields(len(a), 300, seed=5)
        assert U.uqlb_project_workspace_bytes(e.ctx, 300) == U.uqlb_post_workspace_bytes(e.ctx)
        c = e.project(torch.from_numpy(m).cuda())
        assert U.uqlb_last_projection(e.ctx) == 0
        torch.cuda.synchronize()
        c_ref = ouq.gpc_coefficients(ouq.multi_indices(len(bounds), 2), xi, a, m)
        assert np.abs(c.cpu().numpy() - c_ref).max() < 1e-13 * np.abs(c_ref).max()
        e.close()


def test_mc_stats_match_numpy(ens):
    e = Ensemble(0)
    e.set_inputs([(0.0, 1.0)])
    e.init_mc(777, 5)
    m = W.random_fields(777, 513, seed=3)
    mt = torch.from_numpy(m).cuda()
    for ddof in (0, 1):
        mean, var = e.stats(mt, ddof=ddof)
        torch.cuda.synchronize()
        mr, vr = ouq.mc_mean_var(m, ddof=ddof)
        assert rel_l2(mean.cpu().numpy(), mr) < 1e-14 and rel_l2(var.cpu().numpy(), vr) < 1e-12
    e.close()


def test_full_small_pipeline_through_host_buffers(ens):
    """The plain small case end to end (5 GL samples, 64 x 64, 1000 steps, FP64) in one C call."""
    w = W.tgv64_gpc()
    e = Ensemble(0)
    e.setup(w)
    mean, var, coeffs, qoi = e.run_uq_host(w, fields_dtype="f64", coeffs=True, qoi=True)
    z, xi, a = ouq.tensor_grid([5], w.bounds)
    ref = olbm.run([oracle_case(W.tgv(64, 1000, nu=float(nu))) for nu in z[:, 0]])
    mref = np.stack([oracle_row(r) for r in ref])
    c_ref = ouq.gpc_coefficients(ouq.multi_indices(1, 4), xi, a, mref)
    mean_ref, var_ref = ouq.gpc_mean_var(c_ref)
    assert rel_l2(mean, mean_ref) < 1e-12
    assert rel_l2(var, var_ref) < 1e-10
    assert rel_l2(coeffs, c_ref) < 1e-12
    # the kinetic-energy statistics against the closed form of the analytic decay (Sec. 8.2)
    k = 2 * math.pi / 64
    ek = ouq.tgv_mean_k_uniform_nu(0.02, 0.06, k, 1000.0)
    assert abs(mean[-1] - ek) / ek < 5e-3
    e.close()


def test_full_size_tgv256_sampled_against_oracle(ens):
    """The 4-D workload at its full size and in the benchmark's launch configuration (625 samples,
    256 x 256, 2000 steps, FP32 storage): sampled samples against the oracle, invariants for all."""
    w = W.tgv256_gpc4d()
    e = Ensemble(0)
    e.setup(w)
    smp = e.ensemble_samples(w)
    res = e.run_batch(smp, storage="f32", fields_dtype="f32")
    c = e.project(res["fields"])
    mean, var = e.stats(c)
    torch.cuda.synchronize()
    q = res["qoi"].cpu().numpy()
    n2 = 256 * 256
    assert np.all(q[:, U.UQLB_QOI_STATUS] == 0)
    assert np.all(np.abs(q[:, U.UQLB_QOI_MASS] - n2) < 1e-5 * n2)
    assert np.all((q[:, U.UQLB_QOI_K] > 0) & (q[:, U.UQLB_QOI_K] < 1.6))
    picks = [0, 312, 624]
    specs = [W.SampleSpec(W.TGV, 256, 256, 2000, smp[i].nu, smp[i].u0, smp[i].amp2, smp[i].amp3) for i in picks]
    ref = olbm.run([oracle_case(s) for s in specs])
    fields = res["fields"]
    for j, i in enumerate(picks):
        row = fields[i].double().cpu().numpy()
        assert rel_l2(row[:-1], oracle_row(ref[j])[:-1]) < TOL["f32"]
        assert abs(row[-1] - ref[j].k_final) < TOL["f32"] * ref[j].k_final
    assert np.all(np.isfinite(var.cpu().numpy())) and float(mean[-1]) > 0
    e.close()


def test_smolyak_and_qmc_ensembles_match_oracle(ens):
    """Sparse-grid collocation (Clenshaw-Curtis Smolyak, level 2: 41 samples, order 2) and Halton
    QMC (24 points) on the 4-D set-up at 32 x 32, 60 steps, FP64: statistics against the oracle."""
    w = W.tgv_smolyak4d(n=32, steps=60, level=2, order=2, storage="f64")
    e = Ensemble(0)
    e.setup(w)
    smp = e.ensemble_samples(w)
    assert len(smp) == 41
    res = e.run_batch(smp, storage="f64", fields_dtype="f64")
    mean, var = e.stats(e.project(res["fields"]))
    torch.cuda.synchronize()
    xi, a = ouq.smolyak_cc(4, 2)
    z = np.column_stack([ouq.map_uniform(xi[:, k], *w.bounds[k]) for k in range(4)])
    specs = [W.tgv(32, 60, nu=r[0], u0=r[1], amp2=r[2] * r[1], amp3=r[3] * r[1]) for r in z]
    mref = np.stack([oracle_row(r) for r in olbm.run([oracle_case(s) for s in specs])])
    mr, vr = ouq.gpc_mean_var(ouq.gpc_coefficients(ouq.multi_indices(4, 2), xi, a, mref))
    assert rel_l2(mean.cpu().numpy(), mr) < 1e-12 and rel_l2(var.cpu().numpy(), vr) < 1e-10
    e.close()

    q = Ensemble(0)
    wq = W.Workload("qmc", W.tgv(32, 60), W.TGV4D_BOUNDS, W.TGV4D_PARAMS, "qmc", n_mc=24)
    q.setup(wq)
    smp = q.ensemble_samples(wq)
    res = q.run_batch(smp, storage="f64", fields_dtype="f64")
    mean, var = q.stats(res["fields"], ddof=1)
    torch.cuda.synchronize()
    u = ouq.halton(24, 4)
    zq = np.column_stack([lo + (hi - lo) * u[:, k] for k, (lo, hi) in enumerate(W.TGV4D_BOUNDS)])
    specs = [W.tgv(32, 60, nu=r[0], u0=r[1], amp2=r[2] * r[1], amp3=r[3] * r[1]) for r in zq]
    mref = np.stack([oracle_row(r) for r in olbm.run([oracle_case(s) for s in specs])])
    mr, vr = ouq.mc_mean_var(mref, ddof=1)
    assert rel_l2(mean.cpu().numpy(), mr) < 1e-12 and rel_l2(var.cpu().numpy(), vr) < 1e-10
    q.close()


def test_stochastic_rounding_is_reproducible_and_unbiased(ens):
    """Stochastic 16-bit rounding is seeded by (sample, node, step): two runs agree bit for bit.
    On a fine lattice over many steps (where nearest rounding stagnates) it stays closer to the
    oracle than nearest-even rounding, with a rounding at every step (one-step scheme; the
    two-step scheme rounds every other step)."""
    specs = [W.tgv(128, 600, nu=0.03, u0=0.01)]
    ref = olbm.run([oracle_case(s) for s in specs])[0]
    for st in ("f16", "bf16", "fx16"):
        def run(r):
            return ens.run_batch([sample_struct(s) for s in specs], storage=st, rounding=r, scheme="one_step")
        a, b, n = run("stochastic"), run("stochastic"), run("nearest")
        torch.cuda.synchronize()
        fa, fb, fn = (x["fields"][0].double().cpu().numpy() for x in (a, b, n))
        assert np.array_equal(fa, fb), st
        e_sr = rel_l2(fa[:-1], oracle_row(ref)[:-1])
        e_rn = rel_l2(fn[:-1], oracle_row(ref)[:-1])
        print(f"{st}: stochastic {e_sr:.3e} nearest {e_rn:.3e}")
        if st == "fx16":
            # 15 bits over the class's range: both roundings stay well inside the budget here
            assert e_sr < 0.5 * TOL[st] and e_rn < 0.5 * TOL[st], (st, e_sr, e_rn)
        else:
            assert e_sr < e_rn, (st, e_sr, e_rn)


def _paper4d_specs(n, steps, pert_sets):
    p = U.uqlb_unit_converter(n, 1.6 / n, 40.0 * n)
    nu = (p["tau"] - 0.5) / 3.0
    return [W.SampleSpec(W.TGV_PERTURBED, n - 1, n - 1, steps, nu, p["u_lattice"], u_ref=p["u_lattice"],
                         pert=tuple(z * p["u_lattice"] for z in zs)) for zs in pert_sets]


def _oracle_pert(spec, qoi_every=0):
    return olbm.Case(olbm.TGV_PERTURBED, spec.nx, spec.ny, spec.steps, spec.nu, spec.u0, u_ref=spec.u_ref,
                     qoi_every=qoi_every, pert=spec.pert)


def test_paper_perturbed_tgv_matches_oracle(ens):
    """Sec. 8.3 set-up at n = 32 (31 x 31 lattice, Table parameters Ma = 0.05, Re = 1280), four
    amplitudes per sample, FP64 and FP32 storage against the oracle."""
    specs = _paper4d_specs(32, 400, [(0.02, -0.01, 0.015, -0.025), (-0.025, 0.0, 0.01, 0.02), (0, 0, 0, 0)])
    ref = olbm.run([_oracle_pert(s, qoi_every=50) for s in specs])
    for storage in ("f64", "f32"):
        g = _run(ens, specs, storage, qoi_every=50, series=True)
        for i, r in enumerate(ref):
            assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL[storage], storage
            assert np.allclose(g["series"][i, :9], r.series[:9], rtol=10 * TOL[storage], atol=0), storage


@pytest.mark.parametrize("split", [37, 50])
def test_resume_continues_the_run_exactly(ens, split):
    """A run of `split` steps resumed to 100 steps equals a single 100-step run bit for bit
    (odd and even split points; the workspace carries the state)."""
    specs = _tgv_specs(40, 100) + [_cyl(4, 100, u_mean=0.04), _cyl(4, 100, u_mean=0.04, bc="bouzidi")]
    whole = _run(ens, specs, "f64", qoi_every=10, series=True)
    first = [sample_struct(s) for s in specs]
    for s in first:
        s.steps = split
    ens.run_batch(first, storage="f64", fields_dtype="f64", fields=False)
    res = ens.run_batch([sample_struct(s) for s in specs], storage="f64", fields_dtype="f64", fields=False,
                        start_step=split)
    torch.cuda.synchronize()
    q = res["qoi"].cpu().numpy()
    assert np.array_equal(q, whole["qoi"])


def test_w1_of_speed_distributions_matches_exact_within_bin_width(ens):
    """GPU W1 between the |u| distributions of two ensembles (n = 16 and n = 32 of the Sec. 8.3
    set-up) against the oracle's exact W1 of the same fields, within the stated bin-width bound."""
    pert_sets = [(0.02, -0.01, 0.015, -0.025), (-0.025, 0.0, 0.01, 0.02), (0.01, 0.01, -0.02, 0.0)]
    a_specs = _paper4d_specs(16, 200, pert_sets)
    b_specs = _paper4d_specs(32, 800, pert_sets)
    ga = ens.run_batch([sample_struct(s) for s in a_specs], storage="f64", fields_dtype="f64")
    gb = ens.run_batch([sample_struct(s) for s in b_specs], storage="f64", fields_dtype="f64")
    fa, fb = ga["fields"].clone(), gb["fields"].clone()
    for bins in (1 << 10, 1 << 20):
        w1, bound, nonfinite = ens.w1_speed(fa, 15 * 15, fb, 31 * 31, bins=bins)
        assert nonfinite == (0, 0)
        ra = olbm.run([_oracle_pert(s) for s in a_specs])
        rb = olbm.run([_oracle_pert(s) for s in b_specs])
        sa = np.concatenate([np.hypot(r.u, r.v).ravel() for r in ra])
        sb = np.concatenate([np.hypot(r.u, r.v).ravel() for r in rb])
        exact = ouq.wasserstein1(sa, sb)
        assert abs(w1 - exact) <= bound + 1e-12, (bins, w1, exact, bound)
        assert bound <= max(sa.max(), sb.max()) / bins * (1 + 1e-9)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_persistent_mode_matches_graph_mode(ens, storage):
    """One cooperative launch per chunk with the ticket work queue gives the same results as one
    launch per step: per-node arithmetic and per-tile reduction order are the same."""
    specs = _tgv_specs(50, 77) + [W.tgv(32, 40, nu=0.05)]
    a = _run(ens, specs, storage, qoi_every=7, series=True, scheme="one_step")
    res = ens.run_batch([sample_struct(s) for s in specs], storage=storage,
                        fields_dtype="f64" if storage == "f64" else "f32", qoi_every=7, series=True,
                        fields=False, mode="persistent", chunk_steps=16)
    torch.cuda.synchronize()
    assert np.array_equal(res["qoi"].cpu().numpy(), a["qoi"])
    assert np.array_equal(res["series"].cpu().numpy(), a["series"], equal_nan=True)


def test_persistent_mode_mixed_batch_and_steady_state(ens):
    specs = [W.tgv(40, 150, nu=0.03), _cyl(4, 20000, u_mean=0.04, steady_tol=1e-6)]
    a = _run(ens, specs, "f64", qoi_every=100, series=True)
    res = ens.run_batch([sample_struct(s) for s in specs], storage="f64", fields_dtype="f64", qoi_every=100,
                        series=True, fields=False, mode="persistent", chunk_steps=512)
    torch.cuda.synchronize()
    assert np.array_equal(res["qoi"].cpu().numpy(), a["qoi"])
    ref = olbm.run([oracle_case(specs[1], qoi_every=100)])[0]
    assert res["qoi"][1, U.UQLB_QOI_STEPS].item() == ref.steps_run


def test_bounded_barrier_wait_reports_timeout_and_context_survives(ens):
    """Failure detection without a fault: the test hook withholds one block's barrier arrival, the
    other blocks' bounded wait (2 s) runs out, every sample reports UQLB_ERR_TIMEOUT and the
    loop-time query returns it; the same context then runs normally."""
    specs = _tgv_specs(48, 30)
    res = ens.run_batch([sample_struct(s) for s in specs], storage="f32", fields=False,
                        mode="persistent_test_timeout", chunk_steps=8)
    torch.cuda.synchronize()
    assert np.all(res["qoi"][:, U.UQLB_QOI_STATUS].cpu().numpy() == U.UQLB_ERR_TIMEOUT)
    with pytest.raises(U.UqlbError) as e:
        U.uqlb_last_loop_time(ens.ctx)
    assert e.value.status == U.UQLB_ERR_TIMEOUT
    g = _run(ens, specs, "f64")
    ref = olbm.run([oracle_case(s) for s in specs])
    for i, r in enumerate(ref):
        assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL["f64"]
        assert g["qoi"][i, U.UQLB_QOI_STATUS] == 0


def test_w1_leaves_out_and_counts_non_finite_speeds(ens):
    a = torch.tensor([[0.1, 0.2, float("nan"), 0.0, 0.0, 0.0]], dtype=torch.float64, device="cuda")
    b = torch.tensor([[0.3, 0.0, 0.0, 0.0]], dtype=torch.float64, device="cuda")
    w1, bound, nonfinite = ens.w1_speed(a, 3, b, 2, bins=1 << 16)
    assert nonfinite == (1, 0)
    assert abs(w1 - ouq.wasserstein1([0.1, 0.2], [0.3, 0.0])) <= bound + 1e-15


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_two_step_scheme_equals_one_step_scheme(ens, storage):
    """The two-step scheme applies the same per-node formulas as the one-step scheme (in FP32 it
    collides pairs of nodes with packed instructions in a fixed operation order), so results
    agree to round-off; K is summed over the nodes in another order.  The total momentum of the
    Taylor-Green field is zero, so its round-off (~1e-7 on a mass of 1600 in FP32) is compared in
    absolute terms.  Uneven step counts (odd totals end on a one-step launch), ragged lattices
    smaller than a tile, K at every step and at a stride of 7, every two-step geometry."""
    ftol = 1e-13 if storage == "f64" else 1e-6
    qatol = 1e-12 if storage == "f64" else 1e-6
    geoms = [(4, 2), (8, 1), (8, 2)] if storage == "f64" else [(4, 4), (8, 2), (8, 4), (16, 2), (16, 4)]
    for qe in (1, 7):
        specs = [W.tgv(40, 61, nu=0.03, amp2=0.0005), W.tgv(40, 30, nu=0.05), W.tgv(40, 1, nu=0.02),
                 W.tgv(40, 0, nu=0.04)]
        ref = _run(ens, specs, storage, qoi_every=qe, series=True, scheme="one_step")
        for tr, npt in geoms:
            g = _run(ens, specs, storage, qoi_every=qe, series=True, scheme="two_step_tiles", tile_rows=tr, npt=npt)
            assert rel_l2(g["fields"][:, :-1], ref["fields"][:, :-1]) < ftol, (qe, tr, npt)
            assert np.allclose(g["series"], ref["series"], rtol=10 * ftol, atol=0, equal_nan=True), (qe, tr, npt)
            assert np.allclose(g["qoi"], ref["qoi"], rtol=10 * ftol, atol=qatol), (qe, tr, npt)
    small = [W.tgv(5, 9, nu=0.03, amp2=0.0004), W.tgv(5, 12, nu=0.05)]
    a = _run(ens, small, storage, scheme="one_step")
    b = _run(ens, small, storage, scheme="two_step_tiles")
    assert rel_l2(b["fields"][:, :-1], a["fields"][:, :-1]) < ftol


def _strip_specs(n, ny):
    return [replace(W.tgv(n, 61, nu=0.03, amp2=0.0005), ny=ny), replace(W.tgv(n, 30, nu=0.05), ny=ny),
            replace(W.tgv(n, 1, nu=0.02), ny=ny), replace(W.tgv(n, 0, nu=0.04), ny=ny)]


def _close(a, b, tol=1e-6, what=""):
    assert rel_l2(a["fields"][:, :-1], b["fields"][:, :-1]) < tol, what
    # K passes close to zero in the degenerate 2- and 3-row lattices: round-off relative to the series
    scale = np.nanmax(np.abs(b["series"])) if np.isfinite(b["series"]).any() else 0.0
    assert np.allclose(a["series"], b["series"], rtol=10 * tol, atol=tol * scale, equal_nan=True), what
    # the total momentum is zero; its FP32 round-off grows with the node count (~1e-6 at 1600 nodes)
    nodes = (b["fields"].shape[1] - 1) // 2
    assert np.allclose(a["qoi"], b["qoi"], rtol=10 * tol, atol=tol * max(1.0, nodes / 1600)), what


def test_two_step_strips_match_the_tiles_and_the_one_step_scheme(ens):
    """The row-strip two-step kernel applies the same per-node formulas (every node in packed
    pairs), so FP32 results agree with the one-step scheme and the tile kernel to round-off.
    Widths 64 and 128, odd widths (31, 97: the last pair is a lone node) and an even width that
    leaves threads past the row (40); heights equal to the width, ragged (37) and degenerate (2, 3
    rows, where the rows above and below a node coincide); step counts that end on a single-step
    launch (61, 1) or stop at once (0); K at every step and at a stride of 7."""
    for n in (64, 128, 31, 97, 40):
        for ny in (n, 37, 2, 3):
            specs = _strip_specs(n, ny)
            for qe in (1, 7):
                ref = _run(ens, specs, "f32", qoi_every=qe, series=True, scheme="one_step")
                st = _run(ens, specs, "f32", qoi_every=qe, series=True, scheme="two_step_strips")
                assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_TWO_STEP_STRIPS
                ti = _run(ens, specs, "f32", qoi_every=qe, series=True, scheme="two_step_tiles")
                assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_TWO_STEP_TILES
                _close(st, ref, what=(n, ny, qe, "one-step"))
                _close(st, ti, what=(n, ny, qe, "tiles"))


@pytest.mark.parametrize("storage,nx", [("f32", 1600), ("fx16", 2048), pytest.param("bf16", 2048, marks=BF16_MISS),
                                        ("f32", 64 * 13)])
def test_two_step_strips_at_the_widest_rows(ens, storage, nx):
    """The widest rows the strips take (FP32 1600: ring and staging fill 230 KB of shared memory in
    one block of 800 threads; 16-bit 2048: 1024 threads) and an odd multiple of 64, on thin
    lattices: fields and the K series against the oracle within the storage's budget.  The
    fixed-point storage sizes its range for the square lattice's divergence-free Taylor-Green field
    and for flows that the lattice resolves; its case runs on the square 2048 x 2048 lattice."""
    ny = nx if storage == "fx16" else 6
    specs = [replace(W.tgv(nx, 9, nu=0.03, amp2=0.0005), ny=ny), replace(W.tgv(nx, 8, nu=0.05), ny=ny)]
    st = _run(ens, specs, storage, qoi_every=1, series=True, scheme="two_step_strips")
    assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_TWO_STEP_STRIPS
    ref = olbm.run([oracle_case(s, qoi_every=1) for s in specs])
    tol = TOL[storage]
    for i, r in enumerate(ref):
        assert st["qoi"][i, U.UQLB_QOI_STATUS] == 0, (storage, nx, i)
        assert rel_l2(st["fields"][i, :-1], oracle_row(r)[:-1]) < tol, (storage, nx, i)
        ns = specs[i].steps + 1
        assert np.allclose(st["series"][i, :ns], r.series[:ns], rtol=tol, atol=0), (storage, nx, i)


def test_two_step_strips_split_samples_across_blocks(ens):
    """Many samples of mixed heights and step counts in one batch: each block's row range crosses
    samples and each sample's rows are spread over several blocks, whose K partial sums the last
    block adds in row order.  K series and final QoIs against the one-step scheme; a second run
    reproduces the first bit for bit (fixed-order reduction)."""
    specs = []
    for i in range(40):
        ny = (128, 37, 64, 3, 101)[i % 5]
        specs.append(replace(W.tgv(128, 20 + 3 * (i % 7), nu=0.02 + 0.001 * i, amp2=0.0003), ny=ny))
    ref = _run(ens, specs, "f32", qoi_every=1, series=True, scheme="one_step")
    a = _run(ens, specs, "f32", qoi_every=1, series=True, scheme="two_step")
    assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_TWO_STEP_STRIPS
    b = _run(ens, specs, "f32", qoi_every=1, series=True, scheme="two_step")
    assert np.allclose(a["series"], ref["series"], rtol=1e-5, atol=0, equal_nan=True)
    assert np.allclose(a["qoi"], ref["qoi"], rtol=1e-5, atol=1e-6)
    assert np.array_equal(a["series"], b["series"], equal_nan=True)
    assert np.array_equal(a["qoi"], b["qoi"], equal_nan=True)


@pytest.mark.parametrize("first,second", [("two_step_strips", "two_step_strips"), ("two_step_tiles", "two_step_strips"),
                                          ("two_step_strips", "two_step_tiles")])
@pytest.mark.parametrize("split", [38, 51])
def test_two_step_strips_resume_continues_the_run(ens, first, second, split):
    """Strips and tiles leave the same lattice layout, so either continues a run of the other; a
    strip run stopped and resumed on strips at an even split equals the uninterrupted run bit for
    bit, other combinations to FP32 round-off."""
    specs = _tgv_specs(64, 100) + [W.tgv(64, 71, nu=0.04)]
    whole = _run(ens, specs, "f32", qoi_every=10, series=True, scheme="two_step_strips")
    head = [sample_struct(s) for s in specs]
    for s in head:
        s.steps = min(split, s.steps)
    ens.run_batch(head, storage="f32", fields=False, scheme=first)
    res = ens.run_batch([sample_struct(s) for s in specs], storage="f32", fields=True, start_step=split,
                        scheme=second)
    torch.cuda.synchronize()
    got = res["fields"].double().cpu().numpy()[:, :-1]
    if split % 2 == 0 and first == second:
        assert np.array_equal(got, whole["fields"][:, :-1])
    else:
        assert rel_l2(got, whole["fields"][:, :-1]) < 1e-6


def _grouped_specs():
    return [W.tgv(64, 61, nu=0.03, amp2=0.0005), _cyl(4, 130, u_mean=0.04), W.tgv(128, 40, nu=0.05),
            W.tgv(40, 33, nu=0.02), W.tgv(64, 20, nu=0.045), _cyl(5, 77, u_mean=0.035), W.tgv(96, 1, nu=0.06)]


def test_grouped_batch_matches_the_single_one_step_batch(ens):
    """A batch of unlike samples under the auto scheme runs as groups of like samples, one after
    another in slices of one workspace: channel samples on clusters, each periodic width on the row
    strips (64 and 128 fill their blocks, 40 and 96 leave threads past the row).  Every output row
    stays the caller's.  Against the same batch run as one one-step batch the channel rows' final
    state is equal bit for bit (mass, momentum and steps from the same fields; C_D and C_L sum the
    same link forces in another order, FP32 round-off) and the periodic rows agree to FP32
    round-off."""
    specs = _grouped_specs()
    a = _run(ens, specs, "f32", qoi_every=7, series=True)
    assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_GROUPED
    b = _run(ens, specs, "f32", qoi_every=7, series=True, scheme="one_step")
    assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_ONE_STEP
    exact = [U.UQLB_QOI_MASS, U.UQLB_QOI_MOMX, U.UQLB_QOI_STEPS, U.UQLB_QOI_STATUS]
    for i, sp in enumerate(specs):
        if sp.kind == W.CHANNEL:
            assert np.array_equal(a["qoi"][i, exact], b["qoi"][i, exact], equal_nan=True), i
            # C_D sums some twenty FP32 link forces of size ~0.1 scaled by 2 / (U^2 D) ~ 300 at this
            # resolution: FP32 round-off of the sum is a few 1e-5 in C_D units, large against the C_D
            # of the first steps
            assert np.allclose(a["qoi"][i], b["qoi"][i], rtol=1e-5, atol=2e-4, equal_nan=True), i
            assert np.allclose(a["series"][i], b["series"][i], rtol=1e-5, atol=2e-4, equal_nan=True), i
        else:
            assert a["qoi"][i, U.UQLB_QOI_STEPS] == sp.steps
            assert np.allclose(a["qoi"][i], b["qoi"][i], rtol=1e-5, atol=1e-5, equal_nan=True), i
            assert np.allclose(a["series"][i], b["series"][i], rtol=1e-5, atol=0, equal_nan=True), i


def test_grouped_batch_autotune(ens):
    """The autotuner tunes each group of a grouped batch on its own and reports the largest
    group's choice; the tuned run then agrees with the untuned one to round-off (only the tile
    order of the sums can change)."""
    specs = _grouped_specs()
    smp = [sample_struct(s) for s in specs]
    a = _run(ens, specs, "f32", qoi_every=7, series=True)
    tuned = ens.autotune(smp, storage="f32", trial_steps=4)
    assert tuned["tile_rows"] > 0 and tuned["nodes_per_thread"] > 0 and len(tuned["tried"]) >= 1
    b = _run(ens, specs, "f32", qoi_every=7, series=True)
    assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_GROUPED
    assert np.allclose(a["qoi"], b["qoi"], rtol=1e-6, atol=1e-5, equal_nan=True)
    assert np.allclose(a["series"], b["series"], rtol=1e-6, atol=0, equal_nan=True)


@pytest.mark.parametrize("scheme", ["one_step", "two_step_strips", "auto"])
def test_resume_when_the_step_order_changes(ens, scheme):
    """A resumed run presents each sample with its new step total, which can reorder the table
    that is sorted by step count (here the first sample runs fewer steps than the second, but both
    stop together at the split).  Lattice regions and the state that outlives a run are kept by
    the sample's position in the caller's list, so each sample continues its own state: equal bit
    for bit to the uninterrupted run at an even split, for one batch, strips and a grouped batch."""
    if scheme == "auto":
        specs = [W.tgv(64, 41, nu=0.03), _cyl(4, 60, u_mean=0.04), W.tgv(64, 61, nu=0.05), W.tgv(128, 50, nu=0.04),
                 _cyl(4, 90, u_mean=0.035)]
    else:
        specs = [W.tgv(64, 41, nu=0.03, amp2=0.0004), W.tgv(64, 61, nu=0.05), W.tgv(64, 50, nu=0.04)]
    uniform = len({(sp.nx, sp.ny) for sp in specs}) == 1
    split = 30
    whole = _run(ens, specs, "f32", scheme=scheme)
    head = [sample_struct(sp) for sp in specs]
    for h in head:
        h.steps = min(split, h.steps)
    ens.run_batch(head, storage="f32", fields=False, scheme=scheme)
    res = ens.run_batch([sample_struct(sp) for sp in specs], storage="f32", fields=uniform, start_step=split,
                        scheme=scheme)
    torch.cuda.synchronize()
    got = {k: v.double().cpu().numpy() for k, v in res.items()}
    assert np.array_equal(got["qoi"], whole["qoi"], equal_nan=True)
    if uniform:
        assert np.array_equal(got["fields"], whole["fields"])


@pytest.mark.parametrize("split", [37, 50])
def test_two_step_resume_continues_the_run(ens, split):
    """A two-step run stopped after `split` steps and resumed equals the uninterrupted run: bit
    for bit at an even split, to FP32 round-off at an odd one (the step before the split then
    runs on the single-step path, whose scalar operation order differs from the packed pairs)."""
    specs = _tgv_specs(40, 100) + [W.tgv(40, 71, nu=0.04)]
    whole = _run(ens, specs, "f32", qoi_every=10, series=True, scheme="two_step_tiles")
    first = [sample_struct(s) for s in specs]
    for s in first:
        s.steps = min(split, s.steps)
    ens.run_batch(first, storage="f32", fields=False, scheme="two_step_tiles")
    res = ens.run_batch([sample_struct(s) for s in specs], storage="f32", fields=True, start_step=split,
                        scheme="two_step_tiles")
    torch.cuda.synchronize()
    got = res["fields"].double().cpu().numpy()[:, :-1]
    if split % 2 == 0:
        assert np.array_equal(got, whole["fields"][:, :-1])
    else:
        assert rel_l2(got, whole["fields"][:, :-1]) < 1e-6


@pytest.mark.parametrize("storage", _storages("f16", "bf16", "fx16"))
def test_two_step_strips_16_bit_nearest_rounding(ens, storage):
    """Round-to-nearest 16-bit stores on the row strips (pairs of 16-bit values per store where the
    pair is aligned) round every value as the tile kernel's scalar stores do: the two kernels agree
    within half the 16-bit budget (their FP32 collisions differ by round-off, which now and then
    flips a 16-bit rounding), and both stay within the budget of the oracle; a swapped or mis-scaled
    pair would miss the oracle by orders of magnitude."""
    specs = _tgv_specs(64, 300)
    ref = olbm.run([oracle_case(s) for s in specs])
    run = {}
    for scheme in ("two_step_strips", "two_step_tiles"):
        res = ens.run_batch([sample_struct(s) for s in specs], storage=storage, fields_dtype="f32", rounding="nearest",
                            scheme=scheme)
        torch.cuda.synchronize()
        run[scheme] = res["fields"].double().cpu().numpy()
    assert rel_l2(run["two_step_strips"][:, :-1], run["two_step_tiles"][:, :-1]) < 0.5 * TOL[storage]
    for i, r in enumerate(ref):
        for scheme, m in run.items():
            assert rel_l2(m[i, :-1], oracle_row(r)[:-1]) < TOL[storage], (scheme, storage)


@pytest.mark.parametrize("scheme", ["two_step_tiles", "two_step_strips", "three_step_strips"])
@pytest.mark.parametrize("storage", _storages("f16", "bf16", "fx16"))
def test_two_step_16_bit_storage_against_the_oracle(ens, storage, scheme):
    """16-bit storage on the two-step scheme keeps the intermediate step in FP32 shared memory, so
    it rounds half as often; fields stay within the one-step scheme's budget of the oracle (both
    two-step kernels, stochastic rounding)."""
    specs = _tgv_specs(64, 300)
    ref = olbm.run([oracle_case(s) for s in specs])
    g = _run(ens, specs, storage, scheme=scheme)
    one = _run(ens, specs, storage, scheme="one_step")
    for i, r in enumerate(ref):
        e2 = rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1])
        e1 = rel_l2(one["fields"][i, :-1], oracle_row(r)[:-1])
        assert e2 < TOL[storage], (storage, e2)
        assert e2 < 1.5 * e1 + 1e-6, (storage, e2, e1)


@pytest.mark.parametrize("scheme", ["two_step_strips", "three_step_strips"])
@pytest.mark.parametrize("n", [31, 97, 40, 64, 256, 832, 1024])
def test_strip_kernel_edge_geometries_against_the_oracle(ens, n, scheme):
    """The row strips (FP32, two and three steps per launch) against the oracle directly, at the
    geometries whose index arithmetic differs: odd widths (31, 97: the last pair is a lone node whose
    partner is dropped), a width that leaves threads past the row (40), full blocks (64, 256 and 1024,
    which the three-step strips run on their compile-time-width kernel) and an odd multiple of 64
    (832, on the runtime-width kernel); heights equal to the width, ragged (37) and degenerate (3, 2: the rows above
    and below a node coincide); step counts whose last launch runs one step (61, 1), two (62) or three
    (60) or that stop at once (0); K at every step and at a stride of 7.  The Taylor-Green field on 2 and 3 rows is a mode
    near the lattice's Nyquist wavenumber that decays by a factor of 2 to 3 per step (2600x in 9
    steps on 2 rows, measured), so the FP32 round-off of its start, ~1e-7 of it, soon exceeds 1e-5
    of what is left; those run 3, 2 and 1 steps (a launch of each length)."""
    heights = (37, 3, 2) if n > 128 else (n, 37, 3, 2)
    want = {"two_step_strips": U.UQLB_SCHEME_TWO_STEP_STRIPS, "three_step_strips": U.UQLB_SCHEME_THREE_STEP_STRIPS}
    for ny in heights:
        counts = (61, 62, 60) if ny > 3 else (3, 2, 3)
        specs = [replace(W.tgv(n, counts[0], nu=0.03, amp2=0.0005), ny=ny),
                 replace(W.tgv(n, counts[1], nu=0.05, amp3=-0.0004), ny=ny),
                 replace(W.tgv(n, counts[2], nu=0.037, amp2=-0.0003, amp3=0.0002), ny=ny),
                 replace(W.tgv(n, 1, nu=0.02), ny=ny), replace(W.tgv(n, 0, nu=0.04), ny=ny)]
        for qe in (1, 7):
            g = _run(ens, specs, "f32", qoi_every=qe, series=True, scheme=scheme)
            assert U.uqlb_last_run_geometry(ens.ctx)[0] == want[scheme]
            ref = olbm.run([oracle_case(s, qoi_every=qe) for s in specs])
            for i, r in enumerate(ref):
                what = (n, ny, qe, specs[i].steps)
                assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL["f32"], what
                ns = specs[i].steps // qe + 1
                # K passes close to zero on the 2- and 3-row lattices: compare relative to the series
                scale = np.abs(r.series[:ns]).max()
                assert np.allclose(g["series"][i, :ns], r.series[:ns], rtol=TOL["f32"], atol=TOL["f32"] * scale), what
                assert abs(g["qoi"][i, U.UQLB_QOI_K] - r.k_final) <= TOL["f32"] * max(abs(r.k_final), scale), what
                assert abs(g["qoi"][i, U.UQLB_QOI_MASS] - r.mass) < TOL["f32"] * r.mass, what
                assert g["qoi"][i, U.UQLB_QOI_STEPS] == specs[i].steps, what


F16_CHANNEL_MISS = pytest.mark.xfail(
    strict=True, reason="IEEE FP16 storage misses the 1e-3 budget on the channel's C_D (3.5e-3 measured): the "
                        "momentum-exchange sum cancels populations ~10x larger than the force at 11 significant bits")


@pytest.mark.parametrize("storage", ["fx16", pytest.param("f16", marks=F16_CHANNEL_MISS),
                                     pytest.param("bf16", marks=BF16_MISS)])
def test_channel_16_bit_storage_against_the_oracle(ens, storage):
    """16-bit population storage on the channel (one-step kernel): the staircase cylinder with the
    face inlet/outlet, the empty channel, and the Bouzidi cylinder with the interpolated
    inlet/outlet; velocity fields and C_D against the oracle within the 16-bit budget."""
    specs = [_cyl(5, 600), W.channel(5, steps=600, obstacle=False, steady_tol=0.0, re=5.0),
             _cyl(5, 601, u_mean=0.044, bc="bouzidi", inout="interpolated")]
    g = _run(ens, specs, storage)
    ref = olbm.run([oracle_case(s) for s in specs])
    for i, r in enumerate(ref):
        err = rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1])
        print(f"channel {storage} sample {i}: fields {err:.3e} C_D {g['qoi'][i, U.UQLB_QOI_CD]:.6f} vs {r.cd:.6f}")
        assert g["qoi"][i, U.UQLB_QOI_STATUS] == 0, (storage, i)
        assert err < TOL[storage], (storage, i, err)
        if specs[i].cyl_r > 0:
            assert abs(g["qoi"][i, U.UQLB_QOI_CD] - r.cd) < TOL[storage] * abs(r.cd), (storage, i)



def test_fixed_point_storage_reports_a_blown_up_sample(ens):
    """A sample that leaves the fixed-point range saturates instead of turning non-finite; the
    finalize counts the saturated values and reports the sample unstable, as FP32 storage reports
    the non-finite one.  The Sec. 8.3 set-up at n = 8 (7 x 7 lattice, tau - 1/2 = 1.2e-3) blows up
    under BGK by t = 100 (965 steps)."""
    pert_sets = [(0.02, -0.01, 0.015, -0.025), (-0.025, 0.0, 0.01, 0.02), (0.01, 0.01, -0.02, 0.0)]
    specs = _paper4d_specs(8, 965, pert_sets) + [W.tgv(40, 200, nu=0.03)]
    f32 = _run(ens, specs, "f32")
    fx = _run(ens, specs, "fx16")
    bad32 = f32["qoi"][:, U.UQLB_QOI_STATUS] == U.UQLB_ERR_UNSTABLE
    badfx = fx["qoi"][:, U.UQLB_QOI_STATUS] == U.UQLB_ERR_UNSTABLE
    assert bad32[:3].any() and not bad32[3]
    assert np.all(badfx[bad32]) and not badfx[3], (bad32, badfx)


@pytest.mark.parametrize("scheme,split", [("one_step", 37), ("one_step", 50), ("two_step_strips", 50),
                                          ("two_step_tiles", 50)])
def test_fixed_point_resume_continues_the_run_exactly(ens, scheme, split):
    """Fixed-point storage holds the state exactly (integers and per-sample quanta), so a run
    stopped after `split` steps and resumed equals the uninterrupted run bit for bit."""
    specs = _tgv_specs(64, 100) + [W.tgv(64, 71, nu=0.04)]
    whole = _run(ens, specs, "fx16", qoi_every=10, series=True, scheme=scheme)
    head = [sample_struct(s) for s in specs]
    for s in head:
        s.steps = min(split, s.steps)
    ens.run_batch(head, storage="fx16", fields=False, scheme=scheme)
    res = ens.run_batch([sample_struct(s) for s in specs], storage="fx16", fields=True, start_step=split,
                        scheme=scheme)
    torch.cuda.synchronize()
    assert np.array_equal(res["fields"].double().cpu().numpy(), whole["fields"])


def test_sample_blocks_project_and_merge_to_the_full_statistics(ens):
    """The sharded statistics path on one GPU: the partial coefficients of sample blocks
    (uqlb_project_block) sum to uqlb_project's and to the oracle's coefficients; block moments
    (uqlb_block_moments) merged in block order by Chan's update give the Monte Carlo mean and
    variance of the whole set."""
    from paper_2508_13867_gb300 import shard

    e = Ensemble(0)
    e.set_inputs(W.TGV4D_BOUNDS)
    e.init_gpc(4, 5)
    _, xi, a = ouq.tensor_grid([5] * 4, W.TGV4D_BOUNDS)
    m = W.random_fields(625, 1037, seed=21)
    mt = torch.from_numpy(m).cuda()
    c_ref = ouq.gpc_coefficients(ouq.multi_indices(4, 4), xi, a, m)
    full = e.project(mt).clone()
    for world in (2, 3):
        total = torch.zeros_like(full)
        for lo, hi in shard.partition(np.ones(625), world):
            total += e.project_block(mt[lo:hi], lo)
        torch.cuda.synchronize()
        assert np.abs(total.cpu().numpy() - c_ref).max() < 1e-13 * np.abs(c_ref).max(), world
        assert np.abs(total.cpu().numpy() - full.cpu().numpy()).max() < 1e-13 * np.abs(c_ref).max(), world
    e.close()
    e = Ensemble(0)
    e.set_inputs([(0.0, 1.0)])
    e.init_mc(777, 5)
    m = W.random_fields(777, 513, seed=3)
    mt = torch.from_numpy(m).cuda()
    parts = [e.block_moments(mt[lo:hi]) for lo, hi in shard.partition(np.ones(777), 3)]
    n, mean, m2 = shard.chan_merge(parts)
    torch.cuda.synchronize()
    mr, vr = ouq.mc_mean_var(m, ddof=1)
    assert n == 777
    assert rel_l2(mean.cpu().numpy(), mr) < 1e-14 and rel_l2((m2 / (n - 1)).cpu().numpy(), vr) < 1e-12
    e.close()


def test_sharded_pass_on_one_gpu_equals_the_unsharded_pass(ens):
    """Two ranks' blocks of the 4-D workload (3^4 samples, 32 x 32, 40 steps, FP32) run one after
    the other through shard.run_block; their partial coefficients summed (the all-reduce of a
    two-GPU run) give the unsharded pass's statistics."""
    from paper_2508_13867_gb300 import shard

    w = W.tgv256_gpc4d(n=32, steps=40, pts=3)
    e = Ensemble(0)
    e.setup(w)
    smp = e.ensemble_samples(w)
    r = e.run_batch(smp, storage="f32", fields_dtype="f32")
    mean_ref, var_ref = e.stats(e.project(r["fields"]))
    parts = [shard.run_block(e, w, rank, 2)["coeffs"].clone() for rank in range(2)]
    mean, var = e.stats(parts[0] + parts[1])
    torch.cuda.synchronize()
    assert rel_l2(mean.cpu().numpy(), mean_ref.cpu().numpy()) < 1e-13
    assert rel_l2(var.cpu().numpy(), var_ref.cpu().numpy()) < 1e-12
    e.close()


@pytest.mark.parametrize("storage,nx,ny", [("f32", 1280, 6), ("fx16", 1600, 1600), ("f32", 64 * 13, 9)])
def test_three_step_strips_at_the_widest_rows(ens, storage, nx, ny):
    """The widest rows the three-step strips take (FP32 1280: two rings and the staging fill 230 KB of
    shared memory in one block of 640 threads; 16-bit 1600) and an odd multiple of 64: fields and the K
    series against the oracle within the storage's budget (the fixed-point case on a square lattice)."""
    specs = [replace(W.tgv(nx, 9, nu=0.03, amp2=0.0005), ny=ny), replace(W.tgv(nx, 8, nu=0.05), ny=ny)]
    st = _run(ens, specs, storage, qoi_every=1, series=True, scheme="three_step_strips")
    assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_THREE_STEP_STRIPS
    ref = olbm.run([oracle_case(s, qoi_every=1) for s in specs])
    tol = TOL[storage]
    for i, r in enumerate(ref):
        assert st["qoi"][i, U.UQLB_QOI_STATUS] == 0, (storage, nx, i)
        assert rel_l2(st["fields"][i, :-1], oracle_row(r)[:-1]) < tol, (storage, nx, i)
        ns = specs[i].steps + 1
        assert np.allclose(st["series"][i, :ns], r.series[:ns], rtol=tol, atol=0), (storage, nx, i)


def test_three_step_strips_equal_the_two_step_strips_bit_for_bit(ens):
    """With FP32 storage the three-step strips apply the same packed collisions to the same node pairs
    as the two-step strips, and FP32 rows pass through shared memory and HBM unrounded: fields are
    equal bit for bit whatever the grouping of steps into launches (step counts ending on launches of
    one, two and three steps; ragged and degenerate heights; odd width).  K sums the same values with
    the blocks split differently, so it agrees to FP64 round-off."""
    for n, ny in ((64, 64), (97, 37), (40, 3), (128, 2)):
        specs = [replace(W.tgv(n, 61, nu=0.03, amp2=0.0005), ny=ny), replace(W.tgv(n, 62, nu=0.05), ny=ny),
                 replace(W.tgv(n, 60, nu=0.04, amp3=0.0003), ny=ny), replace(W.tgv(n, 1, nu=0.02), ny=ny)]
        a = _run(ens, specs, "f32", qoi_every=5, series=True, scheme="two_step_strips")
        b = _run(ens, specs, "f32", qoi_every=5, series=True, scheme="three_step_strips")
        assert np.array_equal(a["fields"][:, :-1], b["fields"][:, :-1]), (n, ny)
        assert np.allclose(a["series"], b["series"], rtol=1e-12, atol=0, equal_nan=True), (n, ny)


@pytest.mark.parametrize("storage,n,ny", [("f32", 256, 40), ("f16", 128, 77), ("bf16", 512, 20), ("fx16", 64, 64),
                                          ("f32", 200, 31)])
def test_three_step_strip_launch_shapes_agree(ens, storage, n, ny):
    """The launch shape of the three-step strips (resident blocks per SM, so the rows each block takes;
    the staged or direct load of the phase-A rows; the shared-memory share) changes which block updates
    a row and how its values reach the registers, not the arithmetic of a node, and the stochastic
    rounding draws its bits from the node, step and sample: fields are equal bit for bit across shapes,
    the K series (summed per block) to FP64 round-off; the default shape against the oracle within the
    storage's budget (BF16, whose budget misses are asserted elsewhere, on the shapes only).  Width 200
    has no fixed-width kernel (staging option 0 only)."""
    specs = [replace(W.tgv(n, 20, nu=0.03, amp2=0.0005), ny=ny), replace(W.tgv(n, 19, nu=0.05), ny=ny),
             replace(W.tgv(n, 21, nu=0.04, amp3=0.0003), ny=ny)]
    if storage == "fx16":
        specs = [replace(s, ny=n) for s in specs]
    ref = _run(ens, specs, storage, qoi_every=4, series=True, scheme="three_step_strips")
    stages = (1, 2, 3) if n in (64, 128, 256, 512, 1024) else (0,)
    for bps, kb in ((1, 0), (2, 228), (3, 100), (16, 0)):
        for stage in stages:
            got = _run(ens, specs, storage, qoi_every=4, series=True, scheme="three_step_strips",
                       strip=(bps, stage, kb))
            assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_THREE_STEP_STRIPS
            assert np.array_equal(got["fields"][:, :-1], ref["fields"][:, :-1]), (bps, stage, kb)
            assert np.allclose(got["series"], ref["series"], rtol=1e-12, atol=0, equal_nan=True), (bps, stage, kb)
    if storage == "bf16":
        return
    oracle = olbm.run([oracle_case(s, qoi_every=4) for s in specs])
    for i, r in enumerate(oracle):
        assert rel_l2(ref["fields"][i, :-1], oracle_row(r)[:-1]) < TOL[storage], (storage, i)


def test_autotune_tunes_the_three_step_strips(ens):
    """On a batch that runs on the three-step strips the autotuner times staging option x blocks per SM
    x shared-memory share (the tile geometry stays at its default), keeps the fastest, and the next run
    of that batch shape uses it: its fields equal an explicit run with the chosen shape, and the
    oracle's within the FP32 budget."""
    specs = [W.tgv(256, 30, nu=0.03 + 0.002 * k, amp2=0.0004) for k in range(12)]
    smp = [sample_struct(s) for s in specs]
    res = ens.autotune(smp, storage="f32", trial_steps=12)
    cands = res["candidates"]
    assert len(cands) >= 4 and 0 <= res["chosen"] < len(cands)
    configs = {8, 16, 32, 64, 100, 132, 164, 196, 228}
    for c in cands:
        assert c["scheme"] == U.UQLB_SCHEME_THREE_STEP_STRIPS
        assert c["strip_stage"] in (1, 2, 3) and c["strip_blocks_per_sm"] >= 1 and c["strip_smem_kb"] in configs
        assert c["ms_per_step"] > 0
    assert {c["strip_stage"] for c in cands} == {1, 2, 3}
    for stage in (1, 2, 3):
        # the most blocks per SM of each staging option is tried at the largest share too
        most = max(c["strip_blocks_per_sm"] for c in cands if c["strip_stage"] == stage)
        assert any(c["strip_stage"] == stage and c["strip_blocks_per_sm"] == most and c["strip_smem_kb"] == 228
                   for c in cands), stage
    best = cands[res["chosen"]]
    assert best["ms_per_step"] == min(c["ms_per_step"] for c in cands)
    assert len(res["tried"]) == min(len(cands), 16)
    tuned = _run(ens, specs, "f32", qoi_every=5, series=True)
    assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_THREE_STEP_STRIPS
    shape = (best["strip_blocks_per_sm"], best["strip_stage"], best["strip_smem_kb"])
    explicit = _run(ens, specs, "f32", qoi_every=5, series=True, strip=shape)
    assert np.array_equal(tuned["fields"], explicit["fields"])
    oracle = olbm.run([oracle_case(s, qoi_every=5) for s in specs[:3]])
    for i, r in enumerate(oracle):
        assert rel_l2(tuned["fields"][i, :-1], oracle_row(r)[:-1]) < TOL["f32"], i


@pytest.mark.parametrize("first,second", [("three_step_strips", "three_step_strips"),
                                          ("two_step_strips", "three_step_strips"),
                                          ("three_step_strips", "two_step_strips")])
@pytest.mark.parametrize("split", [38, 51, 60])
def test_three_step_strips_resume_continues_the_run(ens, first, second, split):
    """A run stopped after `split` steps and resumed (on either strip kernel) equals the uninterrupted
    three-step run bit for bit with FP32 storage: the launches group the steps differently, the
    per-node arithmetic is the same."""
    specs = _tgv_specs(64, 100) + [W.tgv(64, 71, nu=0.04)]
    whole = _run(ens, specs, "f32", qoi_every=10, series=True, scheme="three_step_strips")
    head = [sample_struct(s) for s in specs]
    for s in head:
        s.steps = min(split, s.steps)
    ens.run_batch(head, storage="f32", fields=False, scheme=first)
    res = ens.run_batch([sample_struct(s) for s in specs], storage="f32", fields=True, start_step=split,
                        scheme=second)
    torch.cuda.synchronize()
    assert np.array_equal(res["fields"].double().cpu().numpy()[:, :-1], whole["fields"][:, :-1])


@pytest.mark.parametrize("steps", [600, 601])
def test_cluster_scheme_matches_the_oracle_and_the_one_step_scheme(ens, steps):
    """Channel samples held on chip by one thread-block cluster each (the staircase cylinder with the
    face inlet/outlet, and the empty channel), FP32: fields, C_D, C_L and the C_D series against the
    oracle; the per-node arithmetic is that of the one-step kernel (push form instead of the in-place
    AA order), so the fields equal the one-step scheme's bit for bit."""
    specs = [_cyl(5, steps, u_mean=0.036), _cyl(5, steps, u_mean=0.044),
             W.channel(5, steps=steps, obstacle=False, steady_tol=0.0, re=5.0)]
    ref = olbm.run([oracle_case(s, qoi_every=50) for s in specs])
    g = _run(ens, specs, "f32", qoi_every=50, series=True, scheme="cluster")
    assert U.uqlb_last_run_geometry(ens.ctx)[0] == U.UQLB_SCHEME_CLUSTER
    one = _run(ens, specs, "f32", qoi_every=50, series=True, scheme="one_step")
    ns = steps // 50
    for i, r in enumerate(ref):
        assert g["qoi"][i, U.UQLB_QOI_STATUS] == 0 and g["qoi"][i, U.UQLB_QOI_STEPS] == steps
        assert rel_l2(g["fields"][i, :-1], oracle_row(r)[:-1]) < TOL["f32"], i
        assert abs(g["qoi"][i, U.UQLB_QOI_MASS] - r.mass) < 10 * TOL["f32"] * r.mass, i
        if specs[i].cyl_r > 0:
            assert abs(g["qoi"][i, U.UQLB_QOI_CD] - r.cd) < 1e-4 * abs(r.cd), i
            assert abs(g["qoi"][i, U.UQLB_QOI_CL] - r.cl) < 1e-4 * abs(r.cd), i
            assert np.allclose(g["series"][i, :ns], r.series[:ns], rtol=1e-4, atol=0), i
    assert np.array_equal(g["fields"][:, :-1], one["fields"][:, :-1])


def test_cluster_scheme_uneven_sizes_and_16_bit_storage(ens):
    """Samples of different sizes in one cluster launch (every block holds the widest sample's slab
    width; narrower samples leave blocks idle) with FX16 storage against the oracle at the 16-bit
    budget, and FP32 against the one-step scheme bit for bit."""
    specs = [_cyl(4, 301, u_mean=0.04), _cyl(6, 301, u_mean=0.038), _cyl(5, 301, u_mean=0.042)]
    ref = olbm.run([oracle_case(s) for s in specs])
    g = _run(ens, specs, "fx16", scheme="cluster")
    for i, r in enumerate(ref):
        assert g["qoi"][i, U.UQLB_QOI_STATUS] == 0
        assert abs(g["qoi"][i, U.UQLB_QOI_CD] - r.cd) < TOL["fx16"] * abs(r.cd), i
        assert abs(g["qoi"][i, U.UQLB_QOI_MASS] - r.mass) < TOL["fx16"] * r.mass, i
    a = _run(ens, specs, "f32", scheme="cluster")
    b = _run(ens, specs, "f32", scheme="one_step")
    assert np.array_equal(a["qoi"][:, [U.UQLB_QOI_MASS, U.UQLB_QOI_MOMX, U.UQLB_QOI_STEPS]],
                          b["qoi"][:, [U.UQLB_QOI_MASS, U.UQLB_QOI_MOMX, U.UQLB_QOI_STEPS]])


def test_cluster_scheme_steady_stop_and_resume(ens):
    """A cluster run stops each sample at the first check where its own C_D series meets the
    steady-state test (|C_D(s) - C_D(s - 100)| < tol |C_D(s)|), and the state it leaves is the state
    at that step: a run of exactly that many steps without the test gives the same QoIs.  The series
    agrees with the one-step scheme's to FP32 round-off (the states are equal bit for bit; C_D sums
    the same link forces in another order, so near the threshold the two schemes' FP32 checks can
    fall on different sides of it).  A run resumed at an odd step continues the state bit for bit."""
    tol = 1e-6
    specs = [_cyl(4, 20000, u_mean=0.04, steady_tol=tol), _cyl(4, 20000, u_mean=0.036, steady_tol=tol)]
    g = _run(ens, specs, "f32", qoi_every=100, series=True, scheme="cluster")
    one = _run(ens, specs, "f32", qoi_every=100, series=True, scheme="one_step")
    for i in range(len(specs)):
        stop = int(g["qoi"][i, U.UQLB_QOI_STEPS])
        assert stop < 20000, i
        cd = g["series"][i, : stop // 100]
        rel = np.abs(np.diff(cd)) / np.abs(cd[1:])
        assert rel[-1] < tol and np.all(rel[:-1] >= tol), i
        n = min(stop, int(one["qoi"][i, U.UQLB_QOI_STEPS])) // 100
        assert np.allclose(cd[:n], one["series"][i, :n], rtol=1e-5, atol=0), i
        exact = replace(specs[i], steps=stop, steady_tol=0.0)
        e = _run(ens, [exact], "f32", scheme="cluster")
        assert np.array_equal(e["qoi"][0, :U.UQLB_QOI_STATUS], g["qoi"][i, :U.UQLB_QOI_STATUS]), i
    specs = [_cyl(4, 90, u_mean=0.04), _cyl(5, 90, u_mean=0.04)]
    whole = _run(ens, specs, "f32", qoi_every=10, series=True, scheme="cluster")
    head = [sample_struct(s) for s in specs]
    for s in head:
        s.steps = 37
    ens.run_batch(head, storage="f32", fields=False, scheme="cluster")
    res = ens.run_batch([sample_struct(s) for s in specs], storage="f32", fields=False, start_step=37, scheme="cluster")
    torch.cuda.synchronize()
    assert np.array_equal(res["qoi"].cpu().numpy(), whole["qoi"])
