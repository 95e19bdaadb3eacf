"""The change-form trial cost against the oracle's update, in FP64 (no GPU).

Near convergence the library forms the trial cost as F plus its change, with
the change of every residual written from the step itself: the pose update of
the camera frame, R <- Exp(dw) R and t <- Exp(dw) t + dt, with X <- X + dX,
moves the camera-frame point by

    dX_cam = (Exp(dw) - I)(X_cam + R dX) + R dX + dt,

and the residual by de = f (dx z - x dz) / (z (z + dz)).  These tests write
that expression out in FP64 numpy and check it against the oracle's own
update (apply_update) and residuals, for small steps and for a large one, so
that a wrong sign, a transposed rotation or a dropped term in the formula
shows up here, apart from the CUDA path.
"""
import numpy as np
import pytest

import oracle as O
import scenes


def _residual_change(s, cams, pts, dxc, dxp, intr):
    oc, op = s.obs_cam, s.obs_pt
    Xc, _, R = O.camera_points(cams, pts, oc, op)
    RdX = np.einsum("mij,mj->mi", R, dxp[op])
    v = Xc + RdX
    dw, dt = dxc[oc, :3], dxc[oc, 3:]
    th = np.linalg.norm(dw, axis=1)
    small = th < 1e-8
    ths = np.where(small, 1.0, th)
    a = np.where(small, 1.0 - th ** 2 / 6.0, np.sin(ths) / ths)
    b = np.where(small, 0.5 - th ** 2 / 24.0, 2.0 * np.sin(0.5 * ths) ** 2 / ths ** 2)
    c1 = np.cross(dw, v)
    c2 = np.cross(dw, c1)
    dXc = a[:, None] * c1 + b[:, None] * c2 + RdX + dt
    z, z1 = Xc[:, 2], Xc[:, 2] + dXc[:, 2]
    du = intr.f * (dXc[:, 0] * z - Xc[:, 0] * dXc[:, 2]) / (z * z1)
    dv = intr.f * (dXc[:, 1] * z - Xc[:, 1] * dXc[:, 2]) / (z * z1)
    return np.stack([du, dv], 1)


@pytest.mark.parametrize("scale", [1e-6, 1e-3, 3e-2])
def test_residual_change_equals_the_oracle_update(scale):
    s = scenes.aerial_small(n_along=6, n_across=4, pts_per_cam=60, seed=61)
    intr = O.Intrinsics()
    rng = np.random.default_rng(7)
    dxc = np.concatenate([rng.normal(0, scale, (s.n_cams, 3)), rng.normal(0, 10 * scale, (s.n_cams, 3))], 1)
    dxp = rng.normal(0, 10 * scale, (s.n_pts, 3))
    e0, _ = O.residuals(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, intr)
    cams1, pts1 = O.apply_update(s.cams0, s.pts0, dxc, dxp)
    e1, _ = O.residuals(cams1, pts1, s.obs_cam, s.obs_pt, s.obs_uv, intr)
    de = _residual_change(s, s.cams0, s.pts0, dxc, dxp, intr)
    # the change itself, to FP64 rounding of the pixel coordinates
    err = np.abs((e1 - e0) - de).max()
    assert err <= 1e-9 * max(np.abs(e1 - e0).max(), 1e-3), (scale, err, np.abs(e1 - e0).max())
    # and the cost change formed from it: sum de (2 e + de) / 2
    dF = 0.5 * np.sum(de * (2.0 * e0 + de))
    dF_ref = 0.5 * (np.sum(e1 * e1) - np.sum(e0 * e0))
    assert abs(dF - dF_ref) <= 1e-7 * abs(dF_ref) + 1e-9, (scale, dF, dF_ref)


def test_exp_coefficient_half_angle_form():
    """b = (1 - cos th) / th^2 written as 2 sin^2(th / 2) / th^2 (no
    cancellation for small th) equals Rodrigues' coefficient."""
    th = np.array([1e-7, 1e-4, 1e-2, 0.3, 1.0, 2.5])
    b_half = 2.0 * np.sin(0.5 * th) ** 2 / th ** 2
    b_ref = (1.0 - np.cos(th)) / th ** 2
    big = th > 1e-3
    assert np.allclose(b_half[big], b_ref[big], rtol=1e-12)
    assert np.allclose(b_half[~big], 0.5 - th[~big] ** 2 / 24.0, rtol=1e-9)
