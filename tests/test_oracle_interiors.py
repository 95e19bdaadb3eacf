"""Pins of the interior-parameter / variable-block-size oracle against things
other than itself: a hand-computed projection, finite differences, the
6-unknown oracle it must reduce to, dense brute-force Schur complements,
dense products and solves, and hand byte counts."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
import oracle.interiors as I
import scenes


def _sorted(s):
    order = O.sort_observations(s.obs_cam, s.obs_pt)
    return s.obs_cam[order].astype(np.int64), s.obs_pt[order].astype(np.int64), s.obs_uv[order]


def _project(cams, intr, pts, oc, op):
    """Projection with scipy rotations and the distortion written out."""
    Rm = Rotation.from_rotvec(cams[:, :3]).as_matrix()
    Xc = np.einsum("mij,mj->mi", Rm[oc], pts[op]) + cams[oc, 3:]
    f, cx, cy, k1, k2 = intr[oc].T
    xh, yh = Xc[:, 0] / Xc[:, 2], Xc[:, 1] / Xc[:, 2]
    r2 = xh ** 2 + yh ** 2
    d = 1 + k1 * r2 + k2 * r2 ** 2
    return np.stack([f * d * xh + cx, f * d * yh + cy], 1)


def _retract(cams, intr, pts, dx, cdim):
    """Camera-frame pose update, additive interiors (for the cameras that
    carry them) and points, on one stacked vector."""
    n = len(cams)
    off = np.concatenate([[0], np.cumsum(cdim)])
    dxc = np.stack([dx[off[i]:off[i] + 6] for i in range(n)])
    dR = Rotation.from_rotvec(dxc[:, :3])
    R = dR * Rotation.from_rotvec(cams[:, :3])
    c2 = np.concatenate([R.as_rotvec(), dR.apply(cams[:, 3:]) + dxc[:, 3:]], 1)
    k2 = intr.copy()
    for i in range(n):
        if cdim[i] == 11:
            k2[i] += dx[off[i] + 6:off[i] + 11]
    return c2, k2, pts + dx[off[-1]:].reshape(-1, 3)


def _dense_j(e, Jc, Jp, oc, op, cdim, P):
    n = len(cdim)
    off = np.concatenate([[0], np.cumsum(cdim)])
    J = np.zeros((2 * len(e), off[-1] + 3 * P))
    for a in range(len(e)):
        i, k = oc[a], op[a]
        J[2 * a:2 * a + 2, off[i]:off[i + 1]] = Jc[a][:, :cdim[i]]
        J[2 * a:2 * a + 2, off[-1] + 3 * k:off[-1] + 3 * k + 3] = Jp[a]
    return J, off[-1]


def _dense_schur(J, e, c, lam):
    """Eq. 1 built densely, then its dense Schur complement (Eq. 4)."""
    H = J.T @ J
    H = H + lam * np.diag(np.clip(np.diag(H), 1e-6, 1e32))
    g = -J.T @ e
    U, W, V = H[:c, :c], H[:c, c:], H[c:, c:]
    Vi = np.linalg.inv(V)
    return U - W @ Vi @ W.T, g[:c] - W @ Vi @ g[c:]


def test_distorted_projection_hand_case():
    # X_cam = (0.2, -0.1, 1): xh = 0.2, yh = -0.1, r2 = 0.05;
    # k1 = -0.2, k2 = 0.04: d = 1 - 0.01 + 0.0001 = 0.9901;
    # f = 1000, (cx, cy) = (500, 500): u = 698.02, v = 400.99
    cams = np.zeros((1, 6))
    intr = np.array([[1000.0, 500.0, 500.0, -0.2, 0.04]])
    pts = np.array([[0.2, -0.1, 1.0]])
    e = I.residuals_intr(cams, intr, pts, np.array([0]), np.array([0]), np.zeros((1, 2)))
    np.testing.assert_allclose(e[0], [698.02, 400.99], rtol=0, atol=1e-9)
    # the pinhole when k1 = k2 = 0
    s = scenes.tiny_scene(seed=8)
    pin = np.tile([O.Intrinsics.f, O.Intrinsics.cx, O.Intrinsics.cy, 0.0, 0.0], (s.n_cams, 1))
    a = I.residuals_intr(s.cams0, pin, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv)
    b, _ = O.residuals(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics())
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-9)


def test_interior_jacobians_match_finite_differences():
    s = scenes.tiny_scene(n_cams=4, n_pts=12, seed=31)
    intr = scenes.interiors0(s.n_cams, seed=3, k_sd=0.05)
    cdim = np.full(s.n_cams, 11)
    oc, op, uv = _sorted(s)
    e, Jc, Jp = I.jacobians_intr(s.cams0, intr, s.pts0, oc, op, uv)
    J, c = _dense_j(e, Jc, Jp, oc, op, cdim, s.n_pts)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for k in range(J.shape[1]):
        d = np.zeros(J.shape[1])
        d[k] = h
        cp, kp, pp = _retract(s.cams0, intr, s.pts0, d, cdim)
        cm, km, pm = _retract(s.cams0, intr, s.pts0, -d, cdim)
        Jfd[:, k] = ((_project(cp, kp, pp, oc, op) - _project(cm, km, pm, oc, op)) / (2 * h)).reshape(-1)
    assert np.abs(J - Jfd).max() <= 1e-6 * np.abs(Jfd).max()
    np.testing.assert_allclose(e, _project(s.cams0, intr, s.pts0, oc, op) - uv, atol=1e-9)


def test_six_unknowns_reduce_to_the_pinhole_rcs():
    """Fixed pinhole interiors and c_i = 6 give the 6-unknown oracle's RCS;
    with c_i = 11 the exterior sub-blocks of S and b are still that RCS."""
    s = scenes.tiny_scene(n_cams=6, n_pts=40, seed=32, sigma_px=2.0)
    lam = 1e-3
    pb = O.Problem(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt, s.obs_uv)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A6, b6 = pb.rcs(e, Jc, Jp, lam)
    D6 = O.bsmc_to_dense(A6)
    pin = np.tile([O.Intrinsics.f, O.Intrinsics.cx, O.Intrinsics.cy, 0.0, 0.0], (s.n_cams, 1))
    A, b = I.scene_rcs_vb(s, pin, np.full(s.n_cams, 6), lam)
    assert np.abs(I.vbsmc_to_dense(A) - D6).max() <= 1e-12 * np.abs(D6).max()
    assert np.abs(b - b6.reshape(-1)).max() <= 1e-12 * np.abs(b6).max()
    A11, b11 = I.scene_rcs_vb(s, pin, np.full(s.n_cams, 11), lam)
    ext = np.concatenate([np.arange(11 * i, 11 * i + 6) for i in range(s.n_cams)])
    D11 = I.vbsmc_to_dense(A11)
    assert np.abs(D11[np.ix_(ext, ext)] - D6).max() <= 1e-12 * np.abs(D6).max()
    assert np.abs(b11[ext] - b6.reshape(-1)).max() <= 1e-12 * np.abs(b6).max()


@pytest.mark.parametrize("seed,frac,lam", [(33, 0.5, 1e-4), (34, 1.0, 0.1), (35, 0.0, 1e-2)])
def test_variable_rcs_equals_dense_schur(seed, frac, lam):
    s = scenes.tiny_scene(n_cams=6, n_pts=40, seed=seed, sigma_px=2.0)
    intr = scenes.interiors0(s.n_cams, seed=seed, k_sd=0.05)
    cdim = scenes.block_sizes(s.n_cams, frac, seed=seed)
    A, b = I.scene_rcs_vb(s, intr, cdim, lam)
    oc, op, uv = _sorted(s)
    e, Jc, Jp = I.jacobians_intr(s.cams0, intr, s.pts0, oc, op, uv)
    J, c = _dense_j(e, Jc, Jp, oc, op, cdim, s.n_pts)
    Sd, bd = _dense_schur(J, e.reshape(-1), c, lam)
    D = I.vbsmc_to_dense(A)
    assert np.abs(D - Sd).max() <= 1e-12 * np.abs(Sd).max()
    assert np.abs(b - bd).max() <= 1e-12 * np.abs(bd).max()
    assert np.linalg.eigvalsh(0.5 * (D + D.T)).min() > 0


def test_variable_rcs_equals_dense_schur_of_fd_jacobian():
    """Independent of the analytic Jacobian: J by finite differences."""
    s = scenes.tiny_scene(n_cams=4, n_pts=15, seed=36, sigma_px=2.0)
    intr = scenes.interiors0(s.n_cams, seed=36, k_sd=0.05)
    cdim = np.array([11, 6, 11, 6])
    lam = 1e-2
    oc, op, uv = _sorted(s)
    N = int(cdim.sum()) + 3 * s.n_pts
    h = 1e-6
    Jfd = np.zeros((2 * len(oc), N))
    for k in range(N):
        d = np.zeros(N)
        d[k] = h
        cp, kp, pp = _retract(s.cams0, intr, s.pts0, d, cdim)
        cm, km, pm = _retract(s.cams0, intr, s.pts0, -d, cdim)
        Jfd[:, k] = ((_project(cp, kp, pp, oc, op) - _project(cm, km, pm, oc, op)) / (2 * h)).reshape(-1)
    e = (_project(s.cams0, intr, s.pts0, oc, op) - uv).reshape(-1)
    Sd, bd = _dense_schur(Jfd, e, int(cdim.sum()), lam)
    A, b = I.scene_rcs_vb(s, intr, cdim, lam)
    assert np.abs(I.vbsmc_to_dense(A) - Sd).max() <= 1e-6 * np.abs(Sd).max()
    assert np.abs(b - bd).max() <= 1e-6 * np.abs(bd).max()


def test_variable_bsmc_product_and_pcg_against_dense():
    s = scenes.tiny_scene(n_cams=8, n_pts=60, seed=37, sigma_px=1.0)
    intr = scenes.interiors0(s.n_cams, seed=37)
    cdim = scenes.block_sizes(s.n_cams, 0.5, seed=37)
    A, b = I.scene_rcs_vb(s, intr, cdim, 1e-3)
    D = I.vbsmc_to_dense(A)
    x = np.random.default_rng(0).standard_normal(len(b))
    np.testing.assert_allclose(I.vbsmc_spmv(A, x), D @ x, rtol=0, atol=1e-12 * np.abs(D).max() * np.abs(x).max())
    r = I.vb_pcg(A, b, 1e-12)
    y = np.linalg.solve(D, b)
    assert np.linalg.norm(r.y - y) <= 1e-8 * np.linalg.norm(y)
    # block-Jacobi on a block-diagonal matrix: exact after one iteration
    Ad = I.VBSMC(np.arange(A.n + 1, dtype=np.int32), np.arange(A.n, dtype=np.int32), A.cdim,
                 [A.val[A.row_ptr[i]] for i in range(A.n)])
    assert I.vb_pcg(Ad, b, 1e-12).iters == 1


def test_variable_bsmc_bytes():
    # hand count: c = (6, 11), blocks (0,0), (0,1), (1,1): 36 + 66 + 121 values
    A = I.VBSMC(np.array([0, 2, 3]), np.array([0, 1, 1]), np.array([6, 11]),
                [np.zeros((6, 6)), np.zeros((6, 11)), np.zeros((11, 11))])
    assert I.vbsmc_bytes(A) == (36 + 66 + 121) * 8 + 3 * 3 * 4 + 2 * 4
    # uniform c: Eq. 9 at the matrix's block density alpha = (2 nnzb - n) / n^2
    s = scenes.tiny_scene(n_cams=8, n_pts=60, seed=38)
    rp, col = O.bsmc_pattern(s.obs_cam, s.obs_pt, s.n_cams, s.n_pts)
    n = s.n_cams
    U = I.VBSMC(rp, col, np.full(n, 11), [np.zeros((11, 11))] * len(col))
    alpha = (2 * len(col) - n) / n ** 2
    assert I.vbsmc_bytes(U) == pytest.approx(O.bsmc_bytes(alpha, n, 11), rel=1e-12)


# ------------------------------------------------ interiors shared by the images of a physical camera

def _retract_shared(cams, intr_phys, pts, dx, phys):
    """Camera-frame pose update per image, additive interiors per physical
    camera (every image of it moves with them), additive points."""
    n, K = len(cams), len(intr_phys)
    dxc = dx[:6 * n].reshape(n, 6)
    dR = Rotation.from_rotvec(dxc[:, :3])
    R = dR * Rotation.from_rotvec(cams[:, :3])
    c2 = np.concatenate([R.as_rotvec(), dR.apply(cams[:, 3:]) + dxc[:, 3:]], 1)
    k2 = intr_phys + dx[6 * n:6 * n + 5 * K].reshape(K, 5)
    return c2, k2[phys], pts + dx[6 * n + 5 * K:].reshape(-1, 3)


def _dense_j_shared(e, Jc, Jp, oc, op, phys, K, P):
    n = len(phys)
    J = np.zeros((2 * len(e), 6 * n + 5 * K + 3 * P))
    for a in range(len(e)):
        i, k = oc[a], op[a]
        J[2 * a:2 * a + 2, 6 * i:6 * i + 6] = Jc[a][:, :6]
        J[2 * a:2 * a + 2, 6 * n + 5 * phys[i]:6 * n + 5 * phys[i] + 5] = Jc[a][:, 6:11]
        J[2 * a:2 * a + 2, 6 * n + 5 * K + 3 * k:6 * n + 5 * K + 3 * k + 3] = Jp[a]
    return J, 6 * n + 5 * K


@pytest.mark.parametrize("seed,phys,lam", [(41, [0, 0, 1, 1, 0, 1], 1e-3), (42, [2, 0, 1, 2, 0, 1], 0.1),
                                           (43, [0, 0, 0, 0, 0, 0], 1e-4)])
def test_shared_interiors_rcs_equals_dense_schur(seed, phys, lam):
    s = scenes.tiny_scene(n_cams=6, n_pts=40, seed=seed, sigma_px=2.0)
    phys = np.array(phys)
    K = phys.max() + 1
    intr = scenes.interiors0(K, seed=seed, k_sd=0.05)
    A, b = I.scene_rcs_shared(s, intr, phys, lam)
    assert list(A.cdim) == [6] * s.n_cams + [5] * K
    oc, op, uv = _sorted(s)
    e, Jc, Jp = I.jacobians_intr(s.cams0, intr[phys], s.pts0, oc, op, uv)
    J, c = _dense_j_shared(e, Jc, Jp, oc, op, phys, K, s.n_pts)
    Sd, bd = _dense_schur(J, e.reshape(-1), c, lam)
    D = I.vbsmc_to_dense(A)
    assert np.abs(D - Sd).max() <= 1e-12 * np.abs(Sd).max()
    assert np.abs(b - bd).max() <= 1e-12 * np.abs(bd).max()
    r = I.vb_pcg(A, b, 1e-12)
    y = np.linalg.solve(D, b)
    assert np.linalg.norm(r.y - y) <= 1e-7 * np.linalg.norm(y)


def test_shared_interiors_rcs_equals_dense_schur_of_fd_jacobian():
    """Independent of the analytic Jacobian: shared interiors moved together."""
    s = scenes.tiny_scene(n_cams=4, n_pts=15, seed=44, sigma_px=2.0)
    phys = np.array([0, 1, 0, 1])
    intr = scenes.interiors0(2, seed=44, k_sd=0.05)
    lam = 1e-2
    oc, op, uv = _sorted(s)
    N = 6 * s.n_cams + 5 * 2 + 3 * s.n_pts
    h = 1e-6
    Jfd = np.zeros((2 * len(oc), N))
    for k in range(N):
        d = np.zeros(N)
        d[k] = h
        cp, kp, pp = _retract_shared(s.cams0, intr, s.pts0, d, phys)
        cm, km, pm = _retract_shared(s.cams0, intr, s.pts0, -d, phys)
        Jfd[:, k] = ((_project(cp, kp, pp, oc, op) - _project(cm, km, pm, oc, op)) / (2 * h)).reshape(-1)
    e = (_project(s.cams0, intr[phys], s.pts0, oc, op) - uv).reshape(-1)
    Sd, bd = _dense_schur(Jfd, e, 6 * s.n_cams + 10, lam)
    A, b = I.scene_rcs_shared(s, intr, phys, lam)
    assert np.abs(I.vbsmc_to_dense(A) - Sd).max() <= 1e-6 * np.abs(Sd).max()
    assert np.abs(b - bd).max() <= 1e-6 * np.abs(bd).max()


def test_one_physical_camera_per_image_is_the_per_image_rcs():
    """With a physical camera per image the shared layout is the c_i = 11
    layout with its unknowns reordered (exteriors first, then interiors)."""
    s = scenes.tiny_scene(n_cams=5, n_pts=30, seed=45, sigma_px=1.0)
    n = s.n_cams
    intr = scenes.interiors0(n, seed=45, k_sd=0.05)
    A, b = I.scene_rcs_shared(s, intr, np.arange(n), 1e-3)
    A11, b11 = I.scene_rcs_vb(s, intr, np.full(n, 11), 1e-3)
    perm = np.concatenate([np.arange(11 * i, 11 * i + 6) for i in range(n)] +
                          [np.arange(11 * i + 6, 11 * i + 11) for i in range(n)])
    D11 = I.vbsmc_to_dense(A11)
    D = I.vbsmc_to_dense(A)
    assert np.abs(D - D11[np.ix_(perm, perm)]).max() <= 1e-12 * np.abs(D11).max()
    assert np.abs(b - b11[perm]).max() <= 1e-12 * np.abs(b11).max()


# ------------------------------------------------ Eq. 5 and the LM iteration with interiors

def test_schur_step_equals_the_dense_normal_equations():
    """The variable-size RCS, PCG and Eq. 5 give the solution of Eq. 1 built
    densely (camera, interior and point unknowns together)."""
    s = scenes.tiny_scene(n_cams=6, n_pts=40, seed=46, sigma_px=2.0)
    intr = scenes.interiors0(s.n_cams, seed=46, k_sd=0.05)
    cdim = np.array([11, 6, 11, 6, 11, 11])
    lam = 1e-2
    oc, op, uv = _sorted(s)
    e, Jc, Jp = I.jacobians_intr(s.cams0, intr, s.pts0, oc, op, uv)
    A, b = I.rcs_vb(e, Jc, Jp, oc, op, cdim, s.n_pts, lam)
    dxc = I.vb_pcg(A, b, 1e-13).y
    dxp = I.back_substitute_vb(e, Jc, Jp, oc, op, cdim, s.n_pts, lam, dxc)
    J, c = _dense_j(e, Jc, Jp, oc, op, cdim, s.n_pts)
    H = J.T @ J
    H = H + lam * np.diag(np.clip(np.diag(H), 1e-6, 1e32))
    dx = np.linalg.solve(H, -J.T @ e.reshape(-1))
    assert np.linalg.norm(dxc - dx[:c]) <= 1e-8 * np.linalg.norm(dx[:c])
    assert np.linalg.norm(dxp.reshape(-1) - dx[c:]) <= 1e-8 * np.linalg.norm(dx[c:])


def test_lm_with_interiors_recovers_a_noise_free_scene():
    """Noise-free observations made with the plain pinhole; poses, points and
    the interiors of the self-calibrating cameras start perturbed.  Accepted
    steps lower the cost, and LM drives it to rounding level."""
    s = scenes.tiny_scene(n_cams=6, n_pts=60, seed=47, sigma_px=0.0, track=(3, 5))
    n = s.n_cams
    cdim = np.array([11, 6, 11, 6, 11, 6])
    pin = np.tile([O.Intrinsics.f, O.Intrinsics.cx, O.Intrinsics.cy, 0.0, 0.0], (n, 1))
    intr0 = pin.copy()
    intr0[cdim == 11] = scenes.interiors0(n, seed=47, f_sd=0.002, c_sd=0.5, k_sd=0.002)[cdim == 11]
    oc, op, uv = _sorted(s)
    st = I.LMStateVB(s.cams0.copy(), intr0, s.pts0.copy())
    F_start = I.cost_intr(st.cams, st.intr, st.pts, oc, op, uv)
    last = F_start
    for _ in range(30):
        st, ok, F0, F1, _ = I.lm_step_vb(st, oc, op, uv, cdim, s.n_pts)
        if ok:
            assert F1 < F0
        last = F1
    assert last <= 1e-12 * F_start, (F_start, last)
    # the fixed cameras kept the pinhole they were given
    assert np.array_equal(st.intr[cdim == 6], pin[cdim == 6])
