"""Solves of a reduced camera system given directly (ba_problem_create_rcs):
FP64 block-Jacobi PCG against the oracle, and the mixed-precision solve (FP32
inner PCG on the demoted S, FP64 refinement with the FP64 S) reaching a true
FP64 residual of 1e-8."""
import numpy as np
import pytest

import oracle as O
import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sys64():
    import torch
    from paper_2307_08383_gb300.build import build
    build()
    import paper_2307_08383_gb300 as B
    # the system comes from the oracle (Eq. 4 at the initial state, lambda = 1e-3)
    s = scenes.aerial_small(n_along=16, n_across=10, pts_per_cam=100, seed=91)
    pb = O.Problem(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt, s.obs_uv)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, b = pb.rcs(e, Jc, Jp, 1e-3)
    return B, (A.row_ptr, A.col, A.val, np.asarray(b))


def test_rcs_problem_fp64_matches_oracle_pcg(sys64):
    B, (row_ptr, col, val, b) = sys64
    g = B.Problem.from_rcs(row_ptr, col, val, b, precision=B.BA_FP64, pcg_rel_tol=1e-10)
    info, conv = g.solve_rcs()
    dxc, _ = g.step()
    A = O.BSMC(row_ptr, col, val)
    res = O.pcg(A, b.reshape(-1), O.block_jacobi(A), 1e-10)
    assert conv and abs(info["pcg_iters"] - res.iters) <= 1
    assert np.linalg.norm(dxc.reshape(-1) - res.y) <= 1e-7 * np.linalg.norm(res.y)
    # the RCS round-trips
    rp2, col2, val2, b2 = g.rcs()
    assert np.array_equal(rp2, row_ptr) and np.array_equal(col2, col) and np.array_equal(val2, val)


def test_mixed_precision_solve_true_fp64_residual(sys64):
    B, (row_ptr, col, val, b) = sys64
    g = B.Problem.from_rcs(row_ptr, col, val, b, precision=B.BA_FP64, solve_precision=B.BA_FP32,
                           pcg_rel_tol=1e-8, inner_rel_tol=1e-4)
    info, conv = g.solve_rcs()
    assert conv and info["refine_steps"] >= 2
    dxc, _ = g.step()
    A = O.BSMC(row_ptr, col, val)
    r = b.reshape(-1) - O.bsmc_spmv(A, dxc.reshape(-1))
    assert np.linalg.norm(r) <= 1.5e-8 * np.linalg.norm(b)
    assert info["rcs_rel_resid"] <= 1e-8
    # the residual the refinement judges by (double-float products on the GPU)
    # is the FP64 one: it agrees with the host's to far below the tolerance
    true_rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert abs(info["rcs_rel_resid"] - true_rel) <= 1e-3 * true_rel + 1e-13
    # the state machine: LM calls are refused on an RCS-only problem
    with pytest.raises(B.BAError) as ei:
        g.linearize()
    assert ei.value.status == B.BA_ERR_STATE
