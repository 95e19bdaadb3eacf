"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (per-block relative Frobenius error of S, denominators guarded
against cancellation by 1e-3 sqrt(||S_ii|| ||S_jj||)):
  FP64 mode <= 1e-10, FP32 mode <= 1e-4; the BSMC pattern is bit-exact;
  LM: final cost within 1e-6 relative of the oracle after the same iterations,
  in FP64 and in FP32 mode (FP32 runs measured on a GB300 stay within 5e-7:
  near the minimum F is flat, so FP32 errors in the steps move it at second
  order only).
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


def _oracle(s, delta=None, tol=1e-10):
    return O.Problem(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt, s.obs_uv, delta=delta, pcg_tol=tol)


def _gpu(B, s, cams=None, pts=None, **kw):
    cams = s.cams0 if cams is None else cams
    pts = s.pts0 if pts is None else pts
    return B.Problem(cams, pts, s.obs_cam, s.obs_pt, s.obs_uv, **kw)


def _host_residual(row_ptr, col, val, b, x):
    """b - S x for the BSMC arrays the GPU solved, with plain numpy (a check
    of the solve on its own system, not an oracle comparison)."""
    n = len(row_ptr) - 1
    D = np.zeros((6 * n, 6 * n))
    for i in range(n):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            j = col[k]
            D[6 * i:6 * i + 6, 6 * j:6 * j + 6] = val[k]
            D[6 * j:6 * j + 6, 6 * i:6 * i + 6] = val[k].T
    return b.reshape(-1) - D @ x


def block_errors(row_ptr, col, val, ref_val):
    n = len(row_ptr) - 1
    dnorm = np.array([np.linalg.norm(ref_val[row_ptr[i]]) for i in range(n)])
    errs = np.empty(len(col))
    for i in range(n):
        for blk in range(row_ptr[i], row_ptr[i + 1]):
            j = col[blk]
            den = max(np.linalg.norm(ref_val[blk]), 1e-3 * np.sqrt(dnorm[i] * dnorm[j]))
            errs[blk] = np.linalg.norm(val[blk] - ref_val[blk]) / den
    return errs


# ----------------------------------------------------------------------------- K1

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("huber", [False, True])
def test_linearize_parity(B, prec, huber):
    s = scenes.shuffled(scenes.ring_scene(n_cams=12, n_pts=400, seed=31, sigma_px=2.0), 3)
    delta = 2.0 if huber else None
    kw = dict(precision=B.BA_FP64 if prec == "fp64" else B.BA_FP32)
    if huber:
        kw.update(robust=B.BA_LOSS_HUBER, huber_delta=2.0)
    g = _gpu(B, s, **kw)
    F = g.linearize()
    e, Jc, Jp = g.linearization()
    er, Jcr, Jpr = O.linearize(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics(), delta)
    Fr = O.cost(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics(), delta)
    if prec == "fp64":
        tj, te, tf = 1e-12, 1e-9, 1e-12
    else:
        # FP32: Jacobian entries to ~1e-6; a Huber weight sqrt(delta/||e||) carries
        # the ~1e-4 px FP32 residual error into the weighted rows (~2.5e-5 relative)
        tj, te, tf = (1e-4 if huber else 2e-6), 2e-3, 1e-5
    keep = np.ones(len(e), bool)
    if huber:
        # rows whose squared residual is within rounding of delta^2 may be weighted on one side only
        e_raw, _ = O.residuals(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics())
        keep = np.abs((e_raw ** 2).sum(1) - 4.0) > 1e-3
        assert keep.mean() > 0.99
    assert np.abs(Jc - Jcr)[keep].max() <= tj * np.abs(Jcr).max()
    assert np.abs(Jp - Jpr)[keep].max() <= tj * np.abs(Jpr).max()
    assert np.abs(e - er)[keep].max() <= te  # px
    assert abs(F - Fr) <= tf * Fr


# ----------------------------------------------------------------------------- K2-K4

def _rcs_case(B, s, prec, lam, delta=None, **kw):
    gk = dict(precision=B.BA_FP64 if prec == "fp64" else B.BA_FP32, **kw)
    if delta is not None:
        gk.update(robust=B.BA_LOSS_HUBER, huber_delta=delta)
    g = _gpu(B, s, **gk)
    g.linearize()
    g.form_rcs(lam)
    row_ptr, col, val, b = g.rcs()
    pb = _oracle(s, delta)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, bref = pb.rcs(e, Jc, Jp, lam)
    return g, (row_ptr, col, val, b), (A, bref)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
@pytest.mark.parametrize("variant", ["ring", "shuffled", "small_groups", "huber", "strong_damping", "aerial"])
def test_rcs_parity(B, prec, tol, variant):
    lam, delta, kw = 1e-4, None, {}
    s = scenes.ring_scene(n_cams=16, n_pts=500, seed=41, sigma_px=1.0)
    if variant == "shuffled":
        s = scenes.shuffled(s, 9)
    elif variant == "small_groups":
        kw["group_max_obs"] = 40
    elif variant == "huber":
        delta = 2.0
        s = scenes.ring_scene(n_cams=16, n_pts=500, seed=42, sigma_px=3.0)
    elif variant == "strong_damping":
        lam = 3.0
    elif variant == "aerial":
        s = scenes.aerial_small(n_along=10, n_across=6, pts_per_cam=120, seed=43)
    g, (row_ptr, col, val, b), (A, bref) = _rcs_case(B, s, prec, lam, delta, **kw)
    assert np.array_equal(row_ptr, A.row_ptr) and np.array_equal(col, A.col)
    errs = block_errors(row_ptr, col, val, A.val)
    assert errs.max() <= tol, (errs.max(), np.argmax(errs))
    bt = 1e-10 if prec == "fp64" else 2e-3
    assert np.abs(b - bref).max() <= bt * np.abs(bref).max()
    st = g.stats()
    assert st["nnzb"] == len(A.col) and st["n_partials"] >= st["nnzb"]
    if variant == "small_groups":
        assert st["n_groups"] > 20


def test_ill_conditioned_points_refactor_in_fp64(B):
    """Points seen along two nearly parallel rays (twin cameras 2 cm apart at
    30 m, lambda = 1e-7) have damped 3x3 blocks V_k with kappa~ ~ 1e5-1e6.  In
    FP32 mode those V_k are re-factored in FP64 (kappa~ > 1e4); the stats
    counter shows it fired for them, and the blocks they form - the twin
    cameras' diagonal blocks and each twin pair's off-diagonal block, made of
    those points alone - match the FP64 oracle within the FP32 bar (1e-4).
    An FP32 factor of V_k instead leaves a relative error of ~1e-3 per point
    at these kappa~ (an FP32 emulation of the factor on the host measures a
    median of 1.6e-3)."""
    s = scenes.short_baseline_scene(baseline=0.02, seed=1201)
    lam = 1e-7
    g, (row_ptr, col, val, b), (A, bref) = _rcs_case(B, s, "fp32", lam)
    assert np.array_equal(row_ptr, A.row_ptr) and np.array_equal(col, A.col)
    # kappa~ of every damped V_k from the oracle's Jacobians
    pb = _oracle(s)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    V = np.zeros((s.n_pts, 3, 3))
    np.add.at(V, pb.obs_pt, np.einsum("mri,mrj->mij", Jp, Jp))
    d = np.clip(np.einsum("kii->ki", V), 1e-6, 1e32)
    V[:, [0, 1, 2], [0, 1, 2]] += lam * d
    kap = np.linalg.norm(V, axis=(1, 2)) * np.linalg.norm(np.linalg.inv(V), axis=(1, 2))
    n64 = g.stats()["n_v_fp64"]
    assert (kap > 2e4).sum() <= n64 <= (kap > 5e3).sum(), (n64, (kap > 1e4).sum())
    assert n64 >= 150  # the 3 x 60 twin points, give or take the threshold
    errs = block_errors(row_ptr, col, val, A.val)
    twin_blocks = []
    for t, h in s.meta["twin_of"].items():
        for (i, j) in ((h, h), (t, t), (min(h, t), max(h, t))):
            twin_blocks.append(row_ptr[i] + int(np.searchsorted(col[row_ptr[i]:row_ptr[i + 1]], j)))
    assert errs[twin_blocks].max() <= 1e-4, errs[twin_blocks]
    assert errs.max() <= 1e-4, (errs.max(), np.argmax(errs))
    # FP64 mode never takes the branch
    g64, _, _ = _rcs_case(B, s, "fp64", lam)
    assert g64.stats()["n_v_fp64"] == 0


def test_rcs_is_deterministic(B):
    s = scenes.ring_scene(n_cams=16, n_pts=600, seed=44)
    g = _gpu(B, s, precision=B.BA_FP32)
    g.linearize()
    g.form_rcs(1e-3)
    v1 = g.rcs()[2]
    g.form_rcs(1e-3)
    v2 = g.rcs()[2]
    assert np.array_equal(v1, v2)


def test_minimal_problem(B):
    """Two cameras, three points each seen by both."""
    s = scenes.ring_scene(n_cams=2, n_pts=3, track=(2, 2), seed=45, sigma_px=0.5)
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-4)):
        g, (row_ptr, col, val, b), (A, bref) = _rcs_case(B, s, prec, 1e-2)
        assert list(col) == [0, 1, 1]
        assert block_errors(row_ptr, col, val, A.val).max() <= tol


def test_long_tracks(B):
    """Tracks of 40 cameras (the longest track of the large workload)."""
    s = scenes.ring_scene(n_cams=48, n_pts=60, track=(36, 40), seed=46)
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-4)):
        g, (row_ptr, col, val, b), (A, bref) = _rcs_case(B, s, prec, 1e-3)
        assert np.array_equal(col, A.col)
        assert block_errors(row_ptr, col, val, A.val).max() <= tol


# ----------------------------------------------------------------------------- PCG, Eq. 5

def test_solve_and_back_substitute_fp64(B):
    s = scenes.ring_scene(n_cams=20, n_pts=800, seed=51, sigma_px=1.0)
    lam = 1e-3
    g = _gpu(B, s, precision=B.BA_FP64, pcg_rel_tol=1e-10)
    g.linearize()
    g.form_rcs(lam)
    info, conv = g.solve_rcs()
    assert conv
    g.back_substitute()
    dxc, dxp = g.step()
    pb = _oracle(s)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    blk, A, b = pb.rcs(e, Jc, Jp, lam)
    res = pb.solve(A, b)
    assert abs(info["pcg_iters"] - res.iters) <= 1, (info["pcg_iters"], res.iters)
    assert np.linalg.norm(dxc.reshape(-1) - res.y) <= 1e-7 * np.linalg.norm(res.y)
    assert info["rcs_rel_resid"] <= 1e-9
    # Eq. 5 from the GPU's own dx_c isolates the back-substitution kernel
    dxp_ref = O.back_substitute(blk, pb.obs_cam, pb.obs_pt, s.n_pts, dxc)
    assert np.abs(dxp - dxp_ref).max() <= 1e-10 * np.abs(dxp_ref).max()


def test_solve_fp32_refinement_reaches_tight_tolerance(B):
    s = scenes.aerial_small(n_along=12, n_across=6, pts_per_cam=150, seed=52)
    g = _gpu(B, s, precision=B.BA_FP32, pcg_rel_tol=1e-8, inner_rel_tol=1e-4)
    g.linearize()
    g.form_rcs(1e-4)
    info, conv = g.solve_rcs()
    assert conv and info["rcs_rel_resid"] <= 1e-8 and info["refine_steps"] >= 2
    # true FP64 residual of the GPU's own system, recomputed on the host
    row_ptr, col, val, b = g.rcs()
    dxc, _ = g.step()
    r = _host_residual(row_ptr, col, val, b, dxc.reshape(-1).astype(np.float32).astype(np.float64))
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(b)


def test_paper_tolerance_stops_early(B):
    s = scenes.ring_scene(n_cams=20, n_pts=800, seed=53)
    g = _gpu(B, s, precision=B.BA_FP64, pcg_rel_tol=0.1)
    g.linearize()
    g.form_rcs(1e-4)
    info, conv = g.solve_rcs()
    pb = _oracle(s, tol=0.1)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, b = pb.rcs(e, Jc, Jp, 1e-4)
    res = pb.solve(A, b)
    assert conv and info["pcg_iters"] == res.iters


def test_fp32_paper_tolerance_follows_oracle(B):
    """FP32 split CG in FP64 refinement at the paper's T = 0.1: one sweep, and
    the PCG stops where the FP64 oracle's block-Jacobi PCG stops (within one
    iteration: the two stop tests see the same residual in two precisions)."""
    s = scenes.aerial_small(n_along=12, n_across=8, pts_per_cam=150, seed=57)
    pb = _oracle(s, tol=0.1)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    for lam in (1e-4, 1e-6):
        g = _gpu(B, s, precision=B.BA_FP32, pcg_rel_tol=0.1)
        g.linearize()
        g.form_rcs(lam)
        info, conv = g.solve_rcs()
        _, A, b = pb.rcs(e, Jc, Jp, lam)
        res = pb.solve(A, b)
        assert conv and info["refine_steps"] == 1 and info["rcs_rel_resid"] <= 0.1
        assert abs(info["pcg_iters"] - res.iters) <= 1, (lam, info["pcg_iters"], res.iters)
        g.close()


# ----------------------------------------------------------------------------- LM

def test_lm_trajectory_fp64_ring50(B):
    """The tiny FP64 workload: 50 cameras, 2,000 points, 10 LM iterations, PCG to 1e-10."""
    s = scenes.ring_scene(seed=1001)
    g = _gpu(B, s, precision=B.BA_FP64, pcg_rel_tol=1e-10)
    pb = _oracle(s, tol=1e-10)
    st = O.LMState(s.cams0.copy(), s.pts0.copy())
    for it in range(10):
        info = g.lm_step()
        st, ref, _ = pb.step(st)
        assert abs(info["cost_before"] - ref.cost_before) <= 1e-6 * ref.cost_before
        significant = ref.predicted > 1e-9 * ref.cost_before
        if significant:
            assert info["accepted"] == int(ref.accepted), (it, info["rho"], ref.rho)
            assert abs(info["cost_trial"] - (ref.cost_after if ref.accepted else info["cost_trial"])) <= \
                1e-6 * ref.cost_before
    _, _, F = g.lm_state()
    Fr = pb.cost(st.cams, st.pts)
    assert abs(F - Fr) <= 1e-6 * Fr, (F, Fr)
    cams = g.cameras()
    pts = g.points()
    assert np.abs(pts - st.pts).max() < 1e-5
    assert np.abs(cams - st.cams).max() < 1e-6


def test_lm_fp32_aerial_against_fp64_oracle(B):
    s = scenes.aerial_small(n_along=10, n_across=6, pts_per_cam=100, seed=54)
    g = _gpu(B, s, precision=B.BA_FP32, pcg_rel_tol=1e-6)
    pb = _oracle(s, tol=1e-6)
    st = O.LMState(s.cams0.copy(), s.pts0.copy())
    for _ in range(5):
        info = g.lm_step()
        st, ref, _ = pb.step(st)
        if ref.predicted > 1e-6 * ref.cost_before:
            assert info["accepted"] == int(ref.accepted)
    _, _, F = g.lm_state()
    Fr = pb.cost(st.cams, st.pts)
    assert abs(F - Fr) <= 1e-6 * Fr, (F, Fr)


@pytest.mark.parametrize("huber", [False, True])
def test_fp32_cost_is_the_fp64_cost(B, huber):
    """FP32 mode evaluates F with double-float residuals against the FP64
    observations: at the initial state it is the oracle's FP64 cost to 1e-12
    (FP32 residuals were ~1e-8 off, more than an LM step changes F near
    convergence).  A trial cost is either evaluated whole (to 1e-12) or, once
    steps change F by less than 1e-3 of it, as F plus the change formed from
    the step (to 1e-6 of the change)."""
    s = scenes.aerial_small(n_along=10, n_across=6, pts_per_cam=100, seed=58, outlier_frac=0.01 if huber else 0.0)
    kw = dict(robust=B.BA_LOSS_HUBER, huber_delta=2.0) if huber else {}
    g = _gpu(B, s, precision=B.BA_FP32, pcg_rel_tol=1e-6, **kw)
    pb = _oracle(s, delta=2.0 if huber else None)
    F0 = pb.cost(s.cams0, s.pts0)
    assert abs(g.lm_state()[2] - F0) <= 1e-12 * F0, (g.lm_state()[2], F0)
    n_small = 0
    for _ in range(12):
        info = g.lm_step()
        if info["accepted"]:
            Fr = pb.cost(g.cameras(), g.points())
            change = abs(info["cost_before"] - Fr)
            assert abs(info["cost_trial"] - Fr) <= 1e-12 * Fr + 1e-6 * change, (info["cost_trial"], Fr, change)
            n_small += change < 1e-3 * Fr
            if n_small >= 2:
                break
    assert n_small >= 2


def test_lm_fp32_follows_the_oracle_at_the_paper_tolerance(B):
    """FP32 LM at T = 0.1 against the FP64 oracle's LM at T = 0.1, step by
    step, while a step's predicted decrease is above 1e-7 of F (below that
    the FP32 gradient is rounding): the same accept/reject decisions where the
    oracle's gain ratio is not within 0.05 of the 1e-3 threshold, and PCG
    iterations within one; the costs after every step within 1e-6."""
    s = scenes.aerial_small(n_along=12, n_across=8, pts_per_cam=150, seed=59)
    g = _gpu(B, s, precision=B.BA_FP32, pcg_rel_tol=0.1)
    pb = _oracle(s, tol=0.1)
    st = O.LMState(s.cams0.copy(), s.pts0.copy())
    for k in range(8):
        info = g.lm_step()
        st, ref, _ = pb.step(st)
        if ref.predicted > 1e-7 * ref.cost_before:
            if abs(ref.rho - 1e-3) > 0.05:
                assert info["accepted"] == int(ref.accepted), (k, info, ref)
            assert abs(info["pcg_iters"] - ref.pcg_iters) <= 1, (k, info["pcg_iters"], ref.pcg_iters)
        F = g.lm_state()[2]
        Fr = pb.cost(st.cams, st.pts)
        assert abs(F - Fr) <= 1e-6 * Fr, (k, F, Fr)


def test_lm_huber_fp32(B):
    s = scenes.aerial_small(n_along=10, n_across=6, pts_per_cam=100, seed=55, outlier_frac=0.01)
    g = _gpu(B, s, precision=B.BA_FP32, pcg_rel_tol=1e-6, robust=B.BA_LOSS_HUBER, huber_delta=2.0)
    pb = _oracle(s, delta=2.0, tol=1e-6)
    st = O.LMState(s.cams0.copy(), s.pts0.copy())
    for _ in range(4):
        info = g.lm_step()
        st, ref, _ = pb.step(st)
    _, _, F = g.lm_state()
    Fr = pb.cost(st.cams, st.pts)
    assert abs(F - Fr) <= 1e-6 * Fr, (F, Fr)


def test_blocks_scene_huber_outliers_parity(B):
    """The large workload's features at a reduced size: overlapping aerial blocks,
    tracks of 2 + Geom (mean 6, max 40), 1% outlier observations, Huber (2 px), FP32.
    The RCS block by block and three LM iterations against the FP64 oracle."""
    s = scenes.blocks_scene(n_blocks_x=2, n_blocks_y=2, block_side=8, n_pts=6000, seed=3101)
    assert s.n_obs / s.n_pts > 4.5
    g = _gpu(B, s, precision=B.BA_FP32, robust=B.BA_LOSS_HUBER, huber_delta=2.0, pcg_rel_tol=1e-6)
    lam0, _, _ = g.lm_state()
    g.linearize()
    g.form_rcs(lam0)
    row_ptr, col, val, b = g.rcs()
    pb = _oracle(s, delta=2.0, tol=1e-6)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, bref = pb.rcs(e, Jc, Jp, lam0)
    assert np.array_equal(row_ptr, A.row_ptr) and np.array_equal(col, A.col)
    assert block_errors(row_ptr, col, val, A.val).max() <= 1e-4
    bref = bref.reshape(-1, 6)
    assert np.linalg.norm(b - bref) <= 1e-4 * np.linalg.norm(bref)
    g.set_state(s.cams0, s.pts0, lam0, 2.0)
    st = O.LMState(s.cams0.copy(), s.pts0.copy())
    for _ in range(3):
        info = g.lm_step()
        st, ref, _ = pb.step(st)
        if ref.predicted > 1e-6 * ref.cost_before:
            assert info["accepted"] == int(ref.accepted)
    _, _, F = g.lm_state()
    Fr = pb.cost(st.cams, st.pts)
    assert abs(F - Fr) <= 1e-6 * Fr, (F, Fr)


def test_state_errors(B):
    s = scenes.ring_scene(n_cams=6, n_pts=50, seed=56)
    g = _gpu(B, s)
    with pytest.raises(B.BAError) as ei:
        g.form_rcs(1e-3)
    assert ei.value.status == B.BA_ERR_STATE
    g.linearize()
    with pytest.raises(B.BAError) as ei:
        g.back_substitute()
    assert ei.value.status == B.BA_ERR_STATE
    with pytest.raises(B.BAError):
        g.form_rcs(-1.0)


def test_set_state_roundtrip(B):
    s = scenes.ring_scene(n_cams=8, n_pts=100, seed=57)
    g = _gpu(B, s)
    g.set_state(s.cams_gt, s.pts_gt, 1e-2, 4.0)
    assert np.array_equal(g.cameras(), s.cams_gt) and np.array_equal(g.points(), s.pts_gt)
    lam, nu, F = g.lm_state()
    assert lam == 1e-2 and nu == 4.0
    assert abs(F - O.cost(s.cams_gt, s.pts_gt, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics())) <= 1e-9 * F


def test_set_state_rejects_non_finite_points_and_keeps_the_state(B):
    """The point upload is checked on the device before the state changes;
    the step (dx_p) comes back in the caller's point order."""
    s = scenes.shuffled(scenes.ring_scene(n_cams=8, n_pts=120, seed=58), 5)
    g = _gpu(B, s, precision=B.BA_FP64, pcg_rel_tol=1e-10)
    bad = s.pts_gt.copy()
    bad[17, 1] = np.nan
    with pytest.raises(B.BAError) as ei:
        g.set_state(s.cams_gt, bad, 1e-2, 4.0)
    assert ei.value.status == B.BA_ERR_NONFINITE
    assert np.array_equal(g.points(), s.pts0)
    # dx_p in caller order: Eq. 5 from the oracle with the GPU's own dx_c
    g.linearize()
    g.form_rcs(1e-3)
    g.solve_rcs()
    g.back_substitute()
    dxc, dxp = g.step()
    pb = _oracle(s)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    blk, A, b = pb.rcs(e, Jc, Jp, 1e-3)
    ref = O.back_substitute(blk, pb.obs_cam, pb.obs_pt, s.n_pts, dxc)
    assert np.abs(dxp - ref).max() <= 1e-10 * np.abs(ref).max()


# ----------------------------------------------------------------------------- full size

@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4)])
def test_aerial5k_full_size_sampled_blocks(B, prec, tol):
    """The aerial workload at full size (5,000 cameras, 1M points) in the
    launch configuration the benchmark uses; sampled blocks against the oracle."""
    s = scenes.aerial_scene(seed=2001)
    g = _gpu(B, s, precision=B.BA_FP32, pcg_rel_tol=0.1)
    lam = 1e-4
    g.linearize()
    g.form_rcs(lam)
    row_ptr, col, val, b = g.rcs()
    # pattern: brute-force set of camera pairs over all tracks (vectorised)
    order = np.lexsort((s.obs_cam, s.obs_pt))
    oc, op = s.obs_cam[order].astype(np.int64), s.obs_pt[order]
    starts = np.searchsorted(op, np.arange(s.n_pts + 1))
    L = np.diff(starts)
    keys = [np.arange(s.n_cams, dtype=np.int64) * (s.n_cams + 1)]
    for dx in range(1, L.max()):
        a = np.nonzero(L > dx)[0]
        for off in range(0, L.max() - dx):
            sel = a[L[a] > off + dx]
            if len(sel) == 0:
                break
            keys.append(oc[starts[sel] + off] * s.n_cams + oc[starts[sel] + off + dx])
    keys = np.unique(np.concatenate(keys))
    got = np.repeat(np.arange(s.n_cams, dtype=np.int64), np.diff(row_ptr)) * s.n_cams + col
    assert np.array_equal(np.sort(got), keys)
    rng = np.random.default_rng(0)
    rows = rng.choice(s.n_cams, 5, replace=False)
    pairs = [(int(i), int(i)) for i in rows]
    for i in rows:
        nb = row_ptr[i + 1] - row_ptr[i]
        if nb > 1:
            pairs.append((int(i), int(col[row_ptr[i] + 1 + rng.integers(0, nb - 1)])))
    S_ref, b_ref = O.rcs_blocks_sampled(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, O.Intrinsics(), lam, pairs)
    for (i, j) in pairs:
        blk = row_ptr[i] + np.searchsorted(col[row_ptr[i]:row_ptr[i + 1]], j)
        assert col[blk] == j
        guard = 1e-3 * np.sqrt(np.linalg.norm(val[row_ptr[i]]) * np.linalg.norm(val[row_ptr[j]]))
        den = max(np.linalg.norm(S_ref[(i, j)]), guard)
        assert np.linalg.norm(val[blk] - S_ref[(i, j)]) / den <= tol, (i, j)
    for i, bi in b_ref.items():
        assert np.abs(b[i] - bi).max() <= 2e-3 * np.abs(bi).max()
    info = g.lm_step()
    assert info["accepted"] == 1 and info["cost_trial"] < info["cost_before"]
    assert info["rcs_rel_resid"] <= 0.1
    # the cost at full size: before the step and at the state it moved to
    # (double-float residuals in FP32 mode: the FP64 value to ~1e-12)
    pb = _oracle(s)
    F0 = pb.cost(s.cams0, s.pts0)
    assert abs(info["cost_before"] - F0) <= 1e-10 * F0, (info["cost_before"], F0)
    _, _, F1 = g.lm_state()
    Fr = pb.cost(g.cameras(), g.points())
    assert abs(F1 - Fr) <= 1e-10 * Fr, (F1, Fr)
