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


def _raw_static_solve(B, n, row_ptr, col, val, b, stream):
    """Calls the entry point through ctypes directly, so that the iteration
    count is seen also when the status is an error."""
    import ctypes

    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    d = [torch.from_numpy(a).to(dev) for a in (row_ptr, col, val.astype(np.float32), b.astype(np.float32))]
    d_x = torch.zeros((n, 6), dtype=torch.float32, device=dev)
    it = ctypes.c_int32(-1)
    rel = ctypes.c_double(-1.0)
    st = B.lib().ba_pcg_solve_static(n, len(col), d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                                     d[3].data_ptr(), d_x.data_ptr(), 1e-6, 0, stream.cuda_stream,
                                     ctypes.byref(it), ctypes.byref(rel))
    torch.cuda.synchronize()
    return st, it.value


def test_static_pcg_stops_before_iterating_on_bad_input():
    """An indefinite diagonal block gives BA_ERR_NOT_SPD, and a matrix passed
    with both triangles gives BA_ERR_INVALID_ARG, each after zero iterations."""
    import torch

    from paper_2307_08383_gb300.build import build
    build()
    import paper_2307_08383_gb300 as B

    s = scenes.ring_scene(n_cams=10, n_pts=300, seed=62)
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP32, pcg_rel_tol=1e-6)
    g.linearize()
    g.form_rcs(0.1)
    row_ptr, col, val, b = g.rcs()
    stream = torch.cuda.current_stream()
    bad = val.copy()
    bad[row_ptr[4]] = -np.eye(6)  # camera 4's diagonal block: negative definite
    st, it = _raw_static_solve(B, s.n_cams, row_ptr, col, bad, b, stream)
    assert st == B.BA_ERR_NOT_SPD and it == 0
    # both triangles: every row also lists its lower blocks (columns below the row)
    n = s.n_cams
    rows = [[] for _ in range(n)]
    for i in range(n):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            rows[i].append((int(col[k]), val[k]))
            if col[k] != i:
                rows[col[k]].append((i, val[k].T))
    full_ptr = np.zeros(n + 1, np.int32)
    full_col, full_val = [], []
    for i in range(n):
        rows[i].sort(key=lambda t: (t[0] != i, t[0]))  # diagonal first, then by column
        full_ptr[i + 1] = full_ptr[i] + len(rows[i])
        full_col += [c for c, _ in rows[i]]
        full_val += [v for _, v in rows[i]]
    st, it = _raw_static_solve(B, n, full_ptr, np.array(full_col, np.int32), np.array(full_val), b, stream)
    assert st == B.BA_ERR_INVALID_ARG and it == 0
    # the shared scratch is usable again right after the refused calls
    st, it = _raw_static_solve(B, n, row_ptr, col, val, b, stream)
    assert st == B.BA_OK and it > 0
