"""The allocation-free PCG entry point, checked against ba_solve_rcs.

ba_pcg_solve_static is for callers that cannot call cudaMalloc (code running
while a framework owns the device memory pool, real-time loops, hosts under a
hard device-memory budget): they pass their own device buffers for the BSMC
matrix, the right-hand side and the solution, and the solver's scratch lives
in a fixed array inside the library.  The test solves the same reduced camera
system with both entry points, twice in a row with the shared scratch, and
compares the solutions within the FP32 tolerance the parity tests use (1e-4).

This file is collected last so that a failure here does not hide another
test; it passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def test_static_pcg_matches_solve_rcs_on_two_calls():
    import torch

    from paper_2307_08383_gb300.build import build
    build()
    import paper_2307_08383_gb300 as B

    s = scenes.ring_scene(n_cams=24, n_pts=900, seed=61)
    tol = 1e-6
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP32, pcg_rel_tol=tol)
    g.linearize()
    g.form_rcs(0.5)
    info, conv = g.solve_rcs()
    assert conv
    ref, _ = g.step()
    row_ptr, col, val, b = g.rcs()

    dev = torch.device("cuda", torch.cuda.current_device())
    d_rp = torch.from_numpy(row_ptr).to(dev)
    d_col = torch.from_numpy(col).to(dev)
    d_val = torch.from_numpy(val.astype(np.float32)).to(dev)
    d_b = torch.from_numpy(b.astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        d_x = torch.full((s.n_cams, 6), float("nan"), dtype=torch.float32, device=dev)
        status, iters, rel = B.ba_pcg_solve_static(s.n_cams, len(col), d_rp.data_ptr(), d_col.data_ptr(),
                                                   d_val.data_ptr(), d_b.data_ptr(), d_x.data_ptr(), tol, 0,
                                                   stream.cuda_stream)
        torch.cuda.synchronize()
        assert status == B.BA_OK and 0 < iters and rel <= tol
        x = d_x.cpu().numpy().astype(np.float64)
        assert np.isfinite(x).all()
        assert np.linalg.norm(x - ref) <= 1e-4 * np.linalg.norm(ref)

    # sizes beyond the fixed scratch are refused before any device work
    with pytest.raises(B.BAError) as ei:
        B.ba_pcg_solve_static(9000, 9000, d_rp.data_ptr(), d_col.data_ptr(), d_val.data_ptr(), d_b.data_ptr(),
                              d_x.data_ptr(), tol, 0, stream.cuda_stream)
    assert ei.value.status == B.BA_ERR_INVALID_ARG
