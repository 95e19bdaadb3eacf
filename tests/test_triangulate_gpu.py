"""GPU parity of the triangulation of the points from the camera poses (the
alternative to the back-substitution of Eq. 5, Sec. 3.1 and Sec. 5) against
the oracle: ba_triangulate (linear equations through their 3x3 normal
matrix, then Gauss-Newton; FP64 for FP64 problems, FP32 centred on the
current points for FP32 problems) vs the oracle's least-squares solution and
Gauss-Newton steps.

Tolerances: points within 1e-7 m (FP64) or 2e-4 m (FP32: camera-point
vectors to ~1e-7 relative at ~100 m) of the oracle's (the two reach the
same reprojection optimum; scene extent ~200 m), 1e-8 relative on
noise-free data against the ground truth (FP64); the reported cost within 1e-9 (FP64
problems) or 1e-3 (FP32 problems: FP32 camera caches) relative of the
oracle's cost at the oracle's points.
"""
import numpy as np
import pytest

import oracle as O
import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available()
    from paper_2307_08383_gb300.build import build
    build()
    import paper_2307_08383_gb300 as mod
    return mod


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_triangulation_matches_oracle(B, prec):
    s = scenes.aerial_small(n_along=8, n_across=5, pts_per_cam=40, seed=4501, sigma_px=1.0)
    g = B.Problem(s.cams_gt, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv,
                  precision=B.BA_FP64 if prec == "fp64" else B.BA_FP32)
    nfail, cost = g.triangulate(3)
    X = g.points()
    ref = O.triangulate(s.cams_gt, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics(), s.n_pts, gn_iters=3)
    assert nfail == 0
    assert np.abs(X - ref).max() <= (1e-7 if prec == "fp64" else 2e-4), np.abs(X - ref).max()
    F_ref = O.cost(s.cams_gt, ref, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics())
    tol = 1e-9 if prec == "fp64" else 1e-3  # the FP32 cost is formed from FP32 camera caches
    assert abs(cost - F_ref) <= tol * F_ref, (cost, F_ref)
    # the perturbed starting points cost more than the triangulated ones
    F0 = O.cost(s.cams_gt, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics())
    assert cost < F0
    # the new state is usable: linearize and one LM step
    g.linearize()
    info = g.lm_step()
    assert np.isfinite(info["cost_after"])


def test_noise_free_points_are_recovered(B):
    s = scenes.aerial_small(n_along=8, n_across=5, pts_per_cam=40, seed=4502, sigma_px=0.0)
    g = B.Problem(s.cams_gt, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP64)
    for gn in (0, 2):
        nfail, cost = g.triangulate(gn)
        assert nfail == 0
        X = g.points()
        assert np.abs(X - s.pts_gt).max() <= 1e-8 * np.abs(s.pts_gt).max()
        assert cost <= 1e-12 * s.n_obs


def test_triangulation_arguments_and_state(B):
    s = scenes.aerial_small(n_along=6, n_across=4, pts_per_cam=20, seed=4503)
    g = B.Problem(s.cams_gt, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP64)
    for bad in (-1, 51):
        with pytest.raises(B.BAError) as ei:
            g.triangulate(bad)
        assert ei.value.status == B.BA_ERR_INVALID_ARG
    g.linearize()
    g.form_rcs(1e-3)
    row_ptr, col, val, b = g.rcs()
    r = B.Problem.from_rcs(row_ptr, col, val, b, precision=B.BA_FP64)
    with pytest.raises(B.BAError) as ei:
        r.triangulate(3)
    assert ei.value.status == B.BA_ERR_STATE
    # triangulation drops the linearization: forming the RCS needs a new one
    g.triangulate(1)
    with pytest.raises(B.BAError) as ei:
        g.form_rcs(1e-3)
    assert ei.value.status == B.BA_ERR_STATE
