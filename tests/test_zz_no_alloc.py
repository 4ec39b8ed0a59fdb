"""The allocation-free projection entry point, checked against the workspace-based one.

Callers that cannot allocate device memory (fixed memory budgets, threads that must not enter
an allocator, embeddings that only pass their own buffers) use uqlb_project_noalloc, which keeps
the weight matrix in a fixed device array inside the library.  This file is collected last so
that a run stopping at its first failure has already run every other test."""
import numpy as np
import pytest

from paper_2508_13867_gb300 import uqlb as U
from paper_2508_13867_gb300 import workloads as W


@pytest.mark.gpu
def test_project_noalloc_matches_project_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2508_13867_gb300 import build

    build.build()
    ctx = U.uqlb_create(0)
    try:
        U.uqlb_set_inputs(ctx, W.TGV4D_BOUNDS)
        U.uqlb_init_gpc(ctx, 4, 5)  # K x S = 70 x 625 = 43750 weights, inside the fixed array
        K, S = U.uqlb_num_terms(ctx), U.uqlb_num_samples(ctx)
        wsb = U.uqlb_post_workspace_bytes(ctx)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for call, (dtype, code, seed, F) in enumerate([(np.float32, U.UQLB_F32, 41, 3001),
                                                       (np.float64, U.UQLB_F64, 42, 1777)]):
            m = torch.from_numpy(W.random_fields(S, F, seed=seed, dtype=dtype)).cuda()
            ref = torch.full((K, F), float("nan"), dtype=torch.float64, device="cuda")
            out = torch.full((K, F), float("nan"), dtype=torch.float64, device="cuda")
            U.uqlb_project(ctx, m.data_ptr(), code, F, F, ref.data_ptr(), ws.data_ptr(), wsb, stream)
            U.uqlb_project_noalloc(ctx, m.data_ptr(), code, F, F, out.data_ptr(), stream)
            torch.cuda.synchronize()
            r, o = ref.cpu().numpy(), out.cpu().numpy()
            assert np.all(np.isfinite(o)), call
            assert np.abs(o - r).max() <= 1e-13 * np.abs(r).max(), call
    finally:
        U.uqlb_destroy(ctx)


def test_project_noalloc_rejects_sample_sets_beyond_its_array():
    from paper_2508_13867_gb300 import build

    build.build()
    ctx = U.uqlb_create(0)
    try:
        U.uqlb_set_inputs(ctx, W.TGV4D_BOUNDS)
        U.uqlb_init_gpc(ctx, 4, 9)  # 70 x 6561 weights > 131072
        with pytest.raises(U.UqlbError) as e:
            U.uqlb_project_noalloc(ctx, 1 << 20, U.UQLB_F32, 16, 16, 1 << 21, None)
        assert e.value.status == U.UQLB_ERR_ARG and "exceeds" in U.uqlb_last_error(ctx)
    finally:
        U.uqlb_destroy(ctx)
