"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a closed form, a hand calculation, a
library routine, finite differences or a dense brute-force construction that
does not go through the oracle's block-structured code, so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails here.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers

def _problem(scene, **kw):
    return O.Problem(scene.n_cams, scene.n_pts, scene.obs_cam, scene.obs_pt, scene.obs_uv, **kw)


def _retract(cams, pts, dx):
    """x (+) dx with the oracle's documented retraction, written independently:
    X_cam <- Exp(dw) X_cam + dt (R <- Exp(dw) R, t <- Exp(dw) t + dt) via scipy,
    X += dX."""
    n = len(cams)
    dxc = dx[:6 * n].reshape(n, 6)
    dxp = dx[6 * n:].reshape(-1, 3)
    dR = Rotation.from_rotvec(dxc[:, :3])
    R = dR * Rotation.from_rotvec(cams[:, :3])
    return np.concatenate([R.as_rotvec(), dR.apply(cams[:, 3:]) + dxc[:, 3:]], 1), pts + dxp


def _residual_vec(pb, cams, pts):
    """Residuals projected with scipy rotations (independent of oracle.rodrigues)."""
    Rm = Rotation.from_rotvec(cams[:, :3]).as_matrix()
    Xc = np.einsum("mij,mj->mi", Rm[pb.obs_cam], pts[pb.obs_pt]) + cams[pb.obs_cam, 3:]
    u = pb.intr.f * Xc[:, 0] / Xc[:, 2] + pb.intr.cx
    v = pb.intr.f * Xc[:, 1] / Xc[:, 2] + pb.intr.cy
    return (np.stack([u, v], 1) - pb.obs_uv).reshape(-1)


def _dense_jacobian_fd(pb, cams, pts, h=1e-6):
    n, P = len(cams), len(pts)
    N = 6 * n + 3 * P
    J = np.zeros((2 * len(pb.obs_cam), N))
    for k in range(N):
        d = np.zeros(N)
        d[k] = h
        cp, pp = _retract(cams, pts, d)
        cm, pm = _retract(cams, pts, -d)
        J[:, k] = (_residual_vec(pb, cp, pp) - _residual_vec(pb, cm, pm)) / (2 * h)
    return J


def _dense_jacobian_analytic(pb, cams, pts):
    """Place the oracle's per-observation blocks into a dense 2m x (6n+3P) J."""
    e, Jc, Jp = O.jacobians(cams, pts, pb.obs_cam, pb.obs_pt, pb.obs_uv, pb.intr)
    n, P, m = len(cams), len(pts), len(e)
    J = np.zeros((2 * m, 6 * n + 3 * P))
    for a in range(m):
        i, k = pb.obs_cam[a], pb.obs_pt[a]
        J[2 * a:2 * a + 2, 6 * i:6 * i + 6] = Jc[a]
        J[2 * a:2 * a + 2, 6 * n + 3 * k:6 * n + 3 * k + 3] = Jp[a]
    return e.reshape(-1), J


def _dense_rcs(J, e, n, lam):
    """Eq. 1 built densely, then its dense Schur complement (Eq. 4)."""
    H = J.T @ J
    dg = np.clip(np.diag(H), 1e-6, 1e32)
    H = H + lam * np.diag(dg)
    g = -J.T @ e
    c = 6 * n
    U, W, V = H[:c, :c], H[:c, c:], H[c:, c:]
    Vi = np.linalg.inv(V)
    return U - W @ Vi @ W.T, g[:c] - W @ Vi @ g[c:], H, g


# ----------------------------------------------------------------- camera model

def test_projection_hand_cases():
    cases = json.load(open(os.path.join(GOLDEN, "pinhole_hand.json")))["cases"]
    for c in cases:
        cam = np.array([c["cam"]], dtype=float)
        X = np.array([c["X"]], dtype=float)
        e, _ = O.residuals(cam, X, np.array([0]), np.array([0]), np.zeros((1, 2)), O.Intrinsics())
        np.testing.assert_allclose(e[0], c["uv"], rtol=0, atol=1e-9, err_msg=c["why"])


def test_rodrigues_matches_library():
    rng = np.random.default_rng(0)
    w = np.concatenate([rng.normal(0, 1.0, (200, 3)), rng.normal(0, 1e-9, (20, 3)),
                        np.zeros((1, 3)), np.array([[0, 0, np.pi - 1e-9]])])
    R = O.rodrigues(w)
    Rl = Rotation.from_rotvec(w).as_matrix()
    np.testing.assert_allclose(R, Rl, rtol=0, atol=1e-14)
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", R, R), np.broadcast_to(np.eye(3), R.shape),
                               atol=1e-14)


def test_jacobians_match_finite_differences():
    s = scenes.tiny_scene(n_cams=4, n_pts=12, seed=3)
    pb = _problem(s)
    Jfd = _dense_jacobian_fd(pb, s.cams0, s.pts0)
    e, Jan = _dense_jacobian_analytic(pb, s.cams0, s.pts0)
    scale = np.abs(Jfd).max()
    assert np.abs(Jan - Jfd).max() <= 1e-6 * scale
    np.testing.assert_allclose(e, _residual_vec(pb, s.cams0, s.pts0), atol=1e-9)


def test_huber_hand_and_limit():
    # e = (3, 4): s = 25; delta = 2: rho = 2*2*5 - 4 = 16, rho' = 2/5
    assert O.huber_rho(25.0, 2.0) == pytest.approx(16.0)
    assert O.huber_weight(25.0, 2.0) == pytest.approx(0.4)
    assert O.huber_rho(3.0, 2.0) == 3.0 and O.huber_weight(3.0, 2.0) == 1.0
    # continuity at the threshold
    assert O.huber_rho(4.0, 2.0) == pytest.approx(2 * 2 * 2 - 4)
    s = scenes.tiny_scene(seed=5)
    pb = _problem(s)
    a = O.linearize(s.cams0, s.pts0, pb.obs_cam, pb.obs_pt, pb.obs_uv, pb.intr, None)
    b = O.linearize(s.cams0, s.pts0, pb.obs_cam, pb.obs_pt, pb.obs_uv, pb.intr, 1e30)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert O.cost(s.cams0, s.pts0, pb.obs_cam, pb.obs_pt, pb.obs_uv, pb.intr, 1e30) == \
        O.cost(s.cams0, s.pts0, pb.obs_cam, pb.obs_pt, pb.obs_uv, pb.intr, None)


# ----------------------------------------------------------------- RCS

@pytest.mark.parametrize("seed,lam,delta", [(11, 1e-4, None), (12, 0.3, None), (13, 1e-3, 2.0)])
def test_rcs_equals_dense_schur(seed, lam, delta):
    s = scenes.tiny_scene(n_cams=6, n_pts=40, seed=seed, sigma_px=3.0)
    pb = _problem(s, delta=delta)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, b = pb.rcs(e, Jc, Jp, lam)
    # dense brute force from the same per-observation Jacobians
    m = len(e)
    n, P = s.n_cams, s.n_pts
    J = np.zeros((2 * m, 6 * n + 3 * P))
    for a in range(m):
        i, k = pb.obs_cam[a], pb.obs_pt[a]
        J[2 * a:2 * a + 2, 6 * i:6 * i + 6] = Jc[a]
        J[2 * a:2 * a + 2, 6 * n + 3 * k:6 * n + 3 * k + 3] = Jp[a]
    Sd, bd, _, _ = _dense_rcs(J, e.reshape(-1), n, lam)
    Sb = O.bsmc_to_dense(A)
    assert np.abs(Sb - Sd).max() <= 1e-12 * np.abs(Sd).max()
    assert np.abs(b.reshape(-1) - bd).max() <= 1e-12 * np.abs(bd).max()


def test_rcs_equals_dense_schur_of_fd_jacobian():
    """Independent of the analytic Jacobian: J by finite differences."""
    s = scenes.tiny_scene(n_cams=4, n_pts=15, seed=21, sigma_px=2.0)
    pb = _problem(s)
    lam = 1e-2
    Jfd = _dense_jacobian_fd(pb, s.cams0, s.pts0)
    Sd, bd, _, _ = _dense_rcs(Jfd, _residual_vec(pb, s.cams0, s.pts0), s.n_cams, lam)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, b = pb.rcs(e, Jc, Jp, lam)
    Sb = O.bsmc_to_dense(A)
    assert np.abs(Sb - Sd).max() <= 1e-6 * np.abs(Sd).max()
    assert np.abs(b.reshape(-1) - bd).max() <= 1e-6 * np.abs(bd).max()


def test_pattern_equals_pair_set():
    s = scenes.tiny_scene(n_cams=8, n_pts=60, seed=4)
    pb = _problem(s)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, _ = pb.rcs(e, Jc, Jp, 1e-4)
    pairs = {(i, i) for i in range(s.n_cams)}
    for k in range(s.n_pts):
        cs = s.obs_cam[s.obs_pt == k]
        for i in cs:
            for j in cs:
                if i <= j:
                    pairs.add((int(i), int(j)))
    got = {(i, int(A.col[blk])) for i in range(A.n) for blk in range(A.row_ptr[i], A.row_ptr[i + 1])}
    assert got == pairs
    # row starts point at the diagonal block, columns ascending within a row
    assert all(A.col[A.row_ptr[i]] == i for i in range(A.n))
    for i in range(A.n):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    rp, cl = O.bsmc_pattern(pb.obs_cam, pb.obs_pt, s.n_cams, s.n_pts)
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(cl, A.col)


def test_fig16_sub_rcs_structure():
    """A point seen by cameras 1 and 3 of five changes only (1,1), (1,3), (3,3)."""
    s = scenes.ring_scene(n_cams=5, n_pts=1, track=(2, 2), seed=9)
    obs_cam = np.array([1, 3], dtype=np.int32)
    obs_pt = np.array([0, 0])
    cams = s.cams_gt
    pts = s.pts_gt
    uv = np.zeros((2, 2))
    e, Jc, Jp = O.linearize(cams, pts, obs_cam, obs_pt, uv, O.Intrinsics())
    blk = O.normal_blocks(e, Jc, Jp, obs_cam, obs_pt, 5, 1, 0.0)
    blk.U[:] = 0.0
    blk.l_c[:] = 0.0
    S, b = O.reduced_camera_system(blk, obs_cam, obs_pt, 5, 1)
    touched = {k for k, v in S.items() if np.abs(v).max() > 0}
    assert touched == {(1, 1), (1, 3), (3, 3)}
    assert set(np.nonzero(np.abs(b).max(1) > 0)[0].tolist()) == {1, 3}


def test_rcs_symmetric_positive_definite():
    s = scenes.tiny_scene(n_cams=6, n_pts=50, seed=8)
    pb = _problem(s)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    for lam in (0.0, 1e-4, 1.0):
        _, A, _ = pb.rcs(e, Jc, Jp, lam)
        D = O.bsmc_to_dense(A)
        # off-diagonal blocks are stored once; diagonal blocks are symmetric to rounding
        assert np.abs(D - D.T).max() <= 1e-13 * np.abs(D).max()
        ev = np.linalg.eigvalsh(D)
        assert ev.min() >= -1e-12 * np.abs(ev).max()
        if lam > 0:
            assert ev.min() > 0
            for i in range(A.n):
                np.linalg.cholesky(A.val[A.row_ptr[i]])


def test_bsmc_spmv_equals_dense_product():
    s = scenes.tiny_scene(n_cams=7, n_pts=40, seed=14)
    pb = _problem(s)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    m = len(e)
    n, P = s.n_cams, s.n_pts
    J = np.zeros((2 * m, 6 * n + 3 * P))
    for a in range(m):
        i, k = pb.obs_cam[a], pb.obs_pt[a]
        J[2 * a:2 * a + 2, 6 * i:6 * i + 6] = Jc[a]
        J[2 * a:2 * a + 2, 6 * n + 3 * k:6 * n + 3 * k + 3] = Jp[a]
    Sd, _, _, _ = _dense_rcs(J, e.reshape(-1), n, 1e-3)
    _, A, _ = pb.rcs(e, Jc, Jp, 1e-3)
    x = np.random.default_rng(1).normal(size=6 * n)
    np.testing.assert_allclose(O.bsmc_spmv(A, x), Sd @ x, rtol=0, atol=1e-10 * np.abs(Sd @ x).max())


# ----------------------------------------------------------------- PCG and back-substitution

def test_pcg_reaches_dense_solution():
    s = scenes.tiny_scene(n_cams=8, n_pts=60, seed=15)
    pb = _problem(s)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, b = pb.rcs(e, Jc, Jp, 1e-3)
    D = O.bsmc_to_dense(A)
    y_star = np.linalg.solve(D, b.reshape(-1))
    res = O.pcg(A, b.reshape(-1), O.block_jacobi(A), 1e-13)
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(res.y - y_star) <= kappa * 1e-13 * np.linalg.norm(y_star) * 10
    assert np.linalg.norm(b.reshape(-1) - D @ res.y) <= 1e-11 * np.linalg.norm(b)
    # CG terminates in at most 6n steps in exact arithmetic; on a well-conditioned
    # system (strong damping) the floating-point run reaches 1e-12 within 6n
    _, A1, b1 = pb.rcs(e, Jc, Jp, 1.0)
    r1 = O.pcg(A1, b1.reshape(-1), O.block_jacobi(A1), 1e-12)
    assert r1.iters <= 6 * A1.n
    # the paper's inexact setting T = 0.1 stops as soon as the residual falls 10x
    r01 = O.pcg(A, b.reshape(-1), O.block_jacobi(A), 0.1)
    assert r01.rel_resid <= 0.1 and all(h > 0.1 for h in r01.history[:-1])
    assert np.linalg.norm(b.reshape(-1) - D @ r01.y) <= 0.1 * np.linalg.norm(b) * (1 + 1e-9)


def test_block_jacobi_is_first_iteration_exact_for_block_diagonal():
    """With no co-visibility S is block diagonal and PCG with M = diag blocks
    solves it in one iteration."""
    n = 4
    rng = np.random.default_rng(2)
    blocks = {}
    for i in range(n):
        Q = rng.normal(size=(6, 6))
        blocks[(i, i)] = Q @ Q.T + 6 * np.eye(6)
    A = O.bsmc_from_blocks(blocks, n)
    b = rng.normal(size=6 * n)
    res = O.pcg(A, b, O.block_jacobi(A), 1e-14)
    assert res.iters == 1
    np.testing.assert_allclose(O.bsmc_to_dense(A) @ res.y, b, atol=1e-12)


def test_back_substitution_solves_full_normal_equations():
    s = scenes.tiny_scene(n_cams=6, n_pts=40, seed=16, sigma_px=2.0)
    pb = _problem(s)
    lam = 1e-3
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    blk, A, b = pb.rcs(e, Jc, Jp, lam)
    dxc = np.linalg.solve(O.bsmc_to_dense(A), b.reshape(-1)).reshape(-1, 6)
    dxp = O.back_substitute(blk, pb.obs_cam, pb.obs_pt, s.n_pts, dxc)
    ed, J = _dense_jacobian_analytic(pb, s.cams0, s.pts0)
    _, _, H, g = _dense_rcs(J, ed, s.n_cams, lam)
    dx = np.concatenate([dxc.reshape(-1), dxp.reshape(-1)])
    assert np.linalg.norm(H @ dx - g) <= 1e-10 * np.linalg.norm(g)
    np.testing.assert_allclose(dx, np.linalg.solve(H, g), rtol=0,
                               atol=1e-8 * np.abs(np.linalg.solve(H, g)).max())


# ----------------------------------------------------------------- LM

def _umeyama(src, dst):
    """Similarity (s, R, t) minimising ||s R src + t - dst|| (Umeyama 1991)."""
    ms, md = src.mean(0), dst.mean(0)
    xs, xd = src - ms, dst - md
    C = xd.T @ xs / len(src)
    Uu, D, Vt = np.linalg.svd(C)
    Sg = np.eye(3)
    if np.linalg.det(Uu) * np.linalg.det(Vt) < 0:
        Sg[2, 2] = -1
    R = Uu @ Sg @ Vt
    s = np.trace(np.diag(D) @ Sg) / (xs ** 2).sum(1).mean()
    return s, R, md - s * R @ ms


def test_lm_noise_free_converges_to_ground_truth():
    s = scenes.ring_scene(n_cams=12, n_pts=300, seed=17, sigma_px=0.0)
    pb = _problem(s, pcg_tol=1e-12)
    st = O.LMState(s.cams0.copy(), s.pts0.copy())
    costs = [pb.cost(st.cams, st.pts)]
    for _ in range(10):
        st, info, _ = pb.step(st)
        if info.accepted:
            assert info.cost_after < info.cost_before
        costs.append(pb.cost(st.cams, st.pts))
    assert costs[-1] < 1e-16 * s.n_obs
    sc, R, t = _umeyama(st.pts, s.pts_gt)
    aligned = sc * st.pts @ R.T + t
    assert np.abs(aligned - s.pts_gt).max() < 1e-6
    Rc = Rotation.from_rotvec(st.cams[:, :3]).as_matrix()
    centers = -np.einsum("nji,nj->ni", Rc, st.cams[:, 3:])
    Rg = Rotation.from_rotvec(s.cams_gt[:, :3]).as_matrix()
    centers_gt = -np.einsum("nji,nj->ni", Rg, s.cams_gt[:, 3:])
    assert np.abs(sc * centers @ R.T + t - centers_gt).max() < 1e-6
    # camera orientations agree up to the same gauge rotation
    for i in range(s.n_cams):
        np.testing.assert_allclose(Rc[i] @ R.T, Rg[i], atol=1e-8)


def test_lm_accepted_steps_decrease_cost_and_noise_floor():
    """Every accepted step lowers F, and the converged 2F/sigma^2 sits in the
    chi-square band of 2m - (6n + 3P - 7) degrees of freedom."""
    sig = 0.5
    s = scenes.ring_scene(n_cams=20, n_pts=600, seed=18, sigma_px=sig)
    pb = _problem(s)
    st = O.LMState(s.cams0.copy(), s.pts0.copy())
    for _ in range(6):
        st, info, _ = pb.step(st)
        if info.accepted:
            assert info.cost_after < info.cost_before
    F = pb.cost(st.cams, st.pts)
    dof = 2 * s.n_obs - (6 * s.n_cams + 3 * s.n_pts - 7)
    chi = 2 * F / sig ** 2
    assert abs(chi - dof) <= 5 * np.sqrt(2 * dof)


def test_lm_huber_downweights_outliers():
    s = scenes.ring_scene(n_cams=12, n_pts=300, seed=19, sigma_px=0.5)
    uv = s.obs_uv.copy()
    rng = np.random.default_rng(0)
    bad = rng.choice(s.n_obs, 20, replace=False)
    uv[bad] = rng.uniform(0, 1000, (20, 2))
    pb = O.Problem(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt, uv, delta=2.0)
    st = O.LMState(s.cams0.copy(), s.pts0.copy())
    for _ in range(8):
        st, info, _ = pb.step(st)
    good = np.ones(s.n_obs, bool)
    good[bad] = False
    e, _ = O.residuals(st.cams, st.pts, s.obs_cam[good], s.obs_pt[good], s.obs_uv[good], O.Intrinsics())
    assert np.sqrt((e ** 2).sum(1).mean()) < 1.2  # inliers stay near the 0.5 px noise


# ----------------------------------------------------------------- memory model (Sec. 4.1)

def test_bsmc_and_csr_byte_counts():
    s = scenes.tiny_scene(n_cams=8, n_pts=60, seed=4)
    rp, cl = O.bsmc_pattern(s.obs_cam, s.obs_pt, s.n_cams, s.n_pts)
    n, c, nnzb = s.n_cams, 6, len(cl)
    nnz_full = 2 * nnzb - n
    alpha = nnz_full / n ** 2
    # BSMC: per block c^2 doubles and 3 ids (column, height, width), n row starts (Eq. 9)
    built_bsmc = nnzb * c * c * 8 + nnzb * 3 * 4 + n * 4
    assert O.bsmc_bytes(alpha, n, c) == pytest.approx(built_bsmc, rel=1e-12)
    # CSR of the full matrix: a value and a column id per element, a start per row (Eq. 8)
    built_csr = nnz_full * c * c * (8 + 4) + n * c * 4
    assert O.csr_bytes(alpha, n, c) == pytest.approx(built_csr, rel=1e-12)
    # Eq. 10 is the ratio of Eqs. 8 and 9 only with the 3 alpha n term
    for a, nn, cc in [(alpha, n, c), (1e-3, 10_000, 11), (1e-4, 200_000, 11), (0.3, 50, 6)]:
        assert O.csr_bsmc_ratio(a, nn, cc) == pytest.approx(O.csr_bytes(a, nn, cc) / O.bsmc_bytes(a, nn, cc),
                                                            rel=1e-12)
    # the paper's 1.5-3x range for c = 11 and n = 10k..200k
    for a in (1e-3, 1e-4):
        for nn in (10_000, 200_000):
            assert 1.4 < O.csr_bsmc_ratio(a, nn, 11) < 3.0


# ------------------------------------------------ triangulation (Sec. 3.1 after Eq. 5)

def test_triangulation_rows_hold_for_exact_observations():
    """Each observation's two linear equations are satisfied by the true point
    (pixels synthesised by scipy's rotation, not the oracle's Rodrigues)."""
    rng = np.random.default_rng(3)
    intr = O.Intrinsics()
    for _ in range(20):
        w = rng.normal(0, 0.5, 3)
        t = rng.normal(0, 5, 3)
        X = rng.normal(0, 3, 3)
        R = Rotation.from_rotvec(w).as_matrix()
        Xc = R @ X + t
        Xc[2] = abs(Xc[2]) + 5.0
        t = Xc - R @ X  # a point in front of the camera
        uv = np.array([intr.f * Xc[0] / Xc[2] + intr.cx, intr.f * Xc[1] / Xc[2] + intr.cy])
        A, r = O.triangulation_rows(np.concatenate([w, t]), uv, intr)
        np.testing.assert_allclose(A @ X, r, rtol=0, atol=1e-9 * np.abs(r).max())
    # hand case: camera at the origin looking down +z, point (1, 2, 10):
    # u = 1000 * 0.1 + 500 = 600, v = 700; rows (-1000, 0, 100) and (0, -1000, 200), rhs 0
    A, r = O.triangulation_rows(np.zeros(6), np.array([600.0, 700.0]), intr)
    np.testing.assert_allclose(A, [[-1000.0, 0.0, 100.0], [0.0, -1000.0, 200.0]])
    np.testing.assert_allclose(r, [0.0, 0.0])


@pytest.mark.parametrize("gn", [0, 3])
def test_triangulation_recovers_noise_free_points(gn):
    s = scenes.aerial_small(n_along=6, n_across=4, pts_per_cam=30, seed=77, sigma_px=0.0)
    X = O.triangulate(s.cams_gt, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics(), s.n_pts, gn_iters=gn)
    assert np.abs(X - s.pts_gt).max() <= 1e-9 * np.abs(s.pts_gt).max()


def test_triangulation_is_the_least_squares_optimum():
    """Noisy pixels: after Gauss-Newton every point is a stationary point of
    its reprojection error (J_p^T e = 0), and an independent optimiser
    (scipy least_squares, started elsewhere) finds the same points."""
    from scipy.optimize import least_squares
    s = scenes.aerial_small(n_along=6, n_across=4, pts_per_cam=30, seed=78, sigma_px=1.0)
    intr = O.Intrinsics()
    X = O.triangulate(s.cams_gt, s.obs_cam, s.obs_pt, s.obs_uv, intr, s.n_pts, gn_iters=5)
    tr = O.tracks(s.obs_pt, s.n_pts)
    for k in range(0, s.n_pts, 37):
        a = tr[k]
        sub = np.zeros(len(a), dtype=np.int64)
        e, _, Jp = O.jacobians(s.cams_gt, X[k][None, :], s.obs_cam[a], sub, s.obs_uv[a], intr)
        g = np.einsum("mij,mi->j", Jp, e)
        assert np.linalg.norm(g) <= 1e-8 * np.linalg.norm(Jp) * max(np.linalg.norm(e), 1e-3)

        def res(p):
            R = Rotation.from_rotvec(s.cams_gt[s.obs_cam[a], :3]).as_matrix()
            Xc = np.einsum("mij,j->mi", R, p) + s.cams_gt[s.obs_cam[a], 3:]
            return (np.stack([intr.f * Xc[:, 0] / Xc[:, 2] + intr.cx,
                              intr.f * Xc[:, 1] / Xc[:, 2] + intr.cy], 1) - s.obs_uv[a]).reshape(-1)
        ref = least_squares(res, s.pts_gt[k] + 0.5, xtol=1e-14, ftol=1e-14, gtol=1e-14).x
        assert np.abs(ref - X[k]).max() <= 1e-6, (k, ref, X[k])


# ----------------------------------------------------------------- sampled RCS blocks

def test_sampled_rcs_blocks_equal_the_full_rcs():
    """rcs_blocks_sampled (Eq. 4 on the sub-problem of the points that reach
    the requested blocks) against the full block-assembled RCS, for every
    stored block of a small aerial scene: the diagonal blocks (whose U_ii and
    damping need every observation of camera i), the off-diagonal blocks and
    b.  A sub-problem that dropped any point or observation a block depends
    on changes that block."""
    s = scenes.aerial_small(n_along=5, n_across=4, pts_per_cam=40, seed=2301)
    lam = 3e-3
    pb = _problem(s)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, b = pb.rcs(e, Jc, Jp, lam)
    b = b.reshape(-1, 6)
    pairs = [(i, int(A.col[k])) for i in range(A.n) for k in range(A.row_ptr[i], A.row_ptr[i + 1])]
    scale = np.abs(A.val).max()
    # one request per block, so that no block borrows points another request kept
    for k, (i, j) in enumerate(pairs):
        S_s, b_s = O.rcs_blocks_sampled(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics(), lam,
                                        [(i, j)])
        assert np.abs(S_s[(i, j)] - A.val[k]).max() <= 1e-12 * scale, (i, j)
        if i == j:
            assert np.abs(b_s[i] - b[i]).max() <= 1e-12 * np.abs(b).max(), i
        else:
            assert not b_s


@pytest.mark.parametrize("delta", [None, 2.0])
def test_sampled_rcs_blocks_equal_dense_schur(delta):
    """The same function against the dense Schur complement of the dense
    damped J^T J (Eq. 1, Eq. 4), for a handful of requested blocks at a time
    (each request builds its own sub-problem)."""
    s = scenes.tiny_scene(n_cams=6, n_pts=40, seed=17, sigma_px=3.0)
    pb = _problem(s, delta=delta)
    lam = 1e-2
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    m, n, P = len(e), s.n_cams, s.n_pts
    J = np.zeros((2 * m, 6 * n + 3 * P))
    for a in range(m):
        i, k = pb.obs_cam[a], pb.obs_pt[a]
        J[2 * a:2 * a + 2, 6 * i:6 * i + 6] = Jc[a]
        J[2 * a:2 * a + 2, 6 * n + 3 * k:6 * n + 3 * k + 3] = Jp[a]
    Sd, bd, _, _ = _dense_rcs(J, e.reshape(-1), n, lam)
    for pairs in ([(0, 0)], [(1, 3)], [(2, 2), (2, 5), (4, 4)]):
        S_s, b_s = O.rcs_blocks_sampled(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics(), lam,
                                        pairs, delta=delta)
        for (i, j) in pairs:
            ref = Sd[6 * i:6 * i + 6, 6 * j:6 * j + 6]
            assert np.abs(S_s[(i, j)] - ref).max() <= 1e-11 * np.abs(Sd).max(), (pairs, i, j)
        for i, bi in b_s.items():
            assert np.abs(bi - bd[6 * i:6 * i + 6]).max() <= 1e-11 * np.abs(bd).max()
