"""The split-preconditioned CG of FP32 solves against the Sec. 3.2
recurrence: CG on G^T S G with M^-1 = G G^T takes the iterates of
block-Jacobi PCG in exact arithmetic, so its iteration counts match the FP64
oracle's PCG on the same system, its solutions reach the same true residual,
and FP64 solves (always the standard recurrence) ignore the option."""
import numpy as np
import pytest

import oracle as O
import oracle.precond_net as N
import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_08383_gb300.build import build
    build()
    import paper_2307_08383_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def scene():
    return scenes.aerial_small(n_along=12, n_across=6, pts_per_cam=150, seed=52)


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


def _solve(B, s, lam, **kw):
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, **kw)
    g.linearize()
    g.form_rcs(lam)
    info, conv = g.solve_rcs()
    dxc, _ = g.step()
    rcs = g.rcs()
    g.close()
    return info, conv, dxc, rcs


@pytest.fixture(scope="module")
def oracle_rcs(scene):
    """The oracle's RCS of the scene at the initial state, lambda = 1e-4."""
    s = scene
    pb = O.Problem(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt, s.obs_uv)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, b = pb.rcs(e, Jc, Jp, 1e-4)
    return A, np.asarray(b)


@pytest.mark.parametrize("tol", [1e-1, 1e-3])
def test_split_iterations_follow_block_jacobi_pcg(B, oracle_rcs, tol):
    """One inner sweep (tol above inner_rel_tol): the sweep runs to
    max(inner_rel_tol, tol), and its iteration count equals the FP64
    oracle's block-Jacobi PCG to that tolerance.  The system is the oracle's;
    the GPU solves it in FP32 (split CG) inside its FP64 refinement."""
    A, b = oracle_rcs
    g = B.Problem.from_rcs(A.row_ptr, A.col, A.val, b, precision=B.BA_FP64, solve_precision=B.BA_FP32,
                           pcg_rel_tol=tol, pcg_variant=B.BA_PCG_SPLIT)
    info, conv = g.solve_rcs()
    dxc, _ = g.step()
    g.close()
    assert conv and info["refine_steps"] == 1
    ref = O.pcg(A, b.reshape(-1), O.block_jacobi(A), max(1e-4, tol))
    assert abs(info["pcg_iters"] - ref.iters) <= 1, (info["pcg_iters"], ref.iters)
    # same iterate up to FP32 rounding: compare with the oracle's y
    assert np.linalg.norm(dxc.reshape(-1) - ref.y) <= 2e-3 * np.linalg.norm(ref.y)


def test_split_and_standard_reach_the_same_tight_residual(B, scene):
    out = {}
    for name, v in (("standard", B.BA_PCG_STANDARD), ("split", B.BA_PCG_SPLIT)):
        info, conv, dxc, (row_ptr, col, val, b) = _solve(B, scene, 1e-4, precision=B.BA_FP32, pcg_rel_tol=1e-8,
                                                         pcg_variant=v)
        r = _host_residual(row_ptr, col, val, b, dxc.reshape(-1).astype(np.float64))
        assert conv and info["rcs_rel_resid"] <= 1e-8
        assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(b)
        out[name] = (info, dxc)
    # the unpreconditioned residual norm of CG is not monotone, so the loose
    # last refinement sweep stops wherever it first dips below its target:
    # totals of two roundings of the same method differ by a few tens
    it_s, it_p = out["standard"][0]["pcg_iters"], out["split"][0]["pcg_iters"]
    print({"standard": it_s, "split": it_p})
    assert it_p <= 1.5 * it_s + 10 and it_s <= 1.5 * it_p + 10, (it_s, it_p)
    # both solve the same system to 1e-8: they differ by up to kappa(S) * 1e-8
    # relative, so compare them through S (FP32 storage of dx_c adds ~1e-7)
    d_s, d_p = out["standard"][1].reshape(-1), out["split"][1].reshape(-1)
    assert np.linalg.norm(_host_residual(row_ptr, col, val, np.zeros_like(b), d_s - d_p)) <= 2e-6 * np.linalg.norm(b)


def test_fp64_solves_ignore_the_variant(B, scene):
    a = _solve(B, scene, 1e-4, precision=B.BA_FP64, pcg_rel_tol=1e-10, pcg_variant=B.BA_PCG_STANDARD)
    b = _solve(B, scene, 1e-4, precision=B.BA_FP64, pcg_rel_tol=1e-10, pcg_variant=B.BA_PCG_SPLIT)
    assert a[0]["pcg_iters"] == b[0]["pcg_iters"]
    assert np.array_equal(a[2], b[2])


def test_split_with_a_learned_preconditioner(B, scene):
    """A learned (non block-Jacobi) M^-1 enters the split system through its
    own Cholesky factor: iterations match the standard recurrence's."""
    rng = np.random.default_rng(4)
    Wt = N.init_weights(4)
    Wt["Wo"] = N.bf16_round(rng.normal(0, 0.2, Wt["Wo"].shape))
    Wt["bo"] = rng.normal(0, 0.2, Wt["bo"].shape)
    net = B.PrecondNet(params=B.pack_params(Wt))
    its = {}
    for name, v in (("standard", B.BA_PCG_STANDARD), ("split", B.BA_PCG_SPLIT)):
        s = scene
        g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP32, pcg_rel_tol=1e-3,
                      pcg_variant=v)
        g.linearize()
        g.form_rcs(1e-4)
        B.ba_set_precond_net(g, net)
        info, conv = g.solve_rcs()
        B.ba_set_precond_net(g, None)
        g.close()
        assert conv and info["used_fallback"] == 0
        its[name] = info["pcg_iters"]
    assert abs(its["standard"] - its["split"]) <= 2, its
    net.close()


def test_implicit_fp64_follows_block_jacobi_pcg(B, scene, oracle_rcs):
    """The implicit variant (S d from the stored J: U d + lambda clamp(diag U) d
    - W V^-1 W^T d, Sec. 4's matrix-free alternative to storing S) in the
    Sec. 3.2 recurrence: its iteration count equals the FP64 oracle's
    block-Jacobi PCG on the oracle's own RCS, and its solution is the
    oracle's iterate up to rounding."""
    A, b = oracle_rcs
    tol = 1e-3
    info, conv, dxc, _ = _solve(B, scene, 1e-4, precision=B.BA_FP64, pcg_rel_tol=tol,
                                pcg_variant=B.BA_PCG_IMPLICIT)
    ref = O.pcg(A, b.reshape(-1), O.block_jacobi(A), tol)
    assert conv
    assert abs(info["pcg_iters"] - ref.iters) <= 1, (info["pcg_iters"], ref.iters)
    assert np.linalg.norm(dxc.reshape(-1) - ref.y) <= 1e-6 * np.linalg.norm(ref.y)


def test_implicit_matches_the_stored_operator(B, scene):
    """FP64: the implicit and the stored-S recurrences take the same number of
    iterations to a tight tolerance and agree to its level; an FP32 inner
    solve asked for is ignored (the operator reads J in the problem's
    precision), bit for bit; LM steps follow the same costs."""
    a = _solve(B, scene, 1e-4, precision=B.BA_FP64, pcg_rel_tol=1e-10, pcg_variant=B.BA_PCG_STANDARD)
    b = _solve(B, scene, 1e-4, precision=B.BA_FP64, pcg_rel_tol=1e-10, pcg_variant=B.BA_PCG_IMPLICIT)
    c = _solve(B, scene, 1e-4, precision=B.BA_FP64, pcg_rel_tol=1e-10, pcg_variant=B.BA_PCG_IMPLICIT,
               solve_precision=B.BA_FP32)
    assert a[1] and b[1]
    # two roundings of the same operator: over ~100 iterations to 1e-10 CG's
    # finite-precision paths drift apart by a few iterations
    it_a, it_b = a[0]["pcg_iters"], b[0]["pcg_iters"]
    assert abs(it_a - it_b) <= 0.1 * it_a + 2, (it_a, it_b)
    assert b[0]["rcs_rel_resid"] <= 1e-9
    # both solve the same system to 1e-10: compare them through S
    row_ptr, col, val, rhs = a[3]
    dd = _host_residual(row_ptr, col, val, np.zeros_like(rhs), a[2].reshape(-1) - b[2].reshape(-1))
    assert np.linalg.norm(dd) <= 3e-10 * np.linalg.norm(rhs)
    assert np.array_equal(b[2], c[2]) and c[0]["refine_steps"] == 0
    s = scene
    costs = {}
    for name, v in (("standard", B.BA_PCG_STANDARD), ("implicit", B.BA_PCG_IMPLICIT)):
        g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP64, pcg_rel_tol=1e-6,
                      pcg_variant=v)
        costs[name] = [g.lm_step()["cost_after"] for _ in range(3)]
        g.close()
    assert np.allclose(costs["standard"], costs["implicit"], rtol=1e-8, atol=0), costs


def test_implicit_fp32_reaches_a_tight_residual(B, scene):
    """FP32: the implicit inner PCG inside the FP64 refinement reaches the
    same true residual as the stored-S variants."""
    info, conv, dxc, (row_ptr, col, val, b) = _solve(B, scene, 1e-4, precision=B.BA_FP32, pcg_rel_tol=1e-8,
                                                     pcg_variant=B.BA_PCG_IMPLICIT)
    r = _host_residual(row_ptr, col, val, b, dxc.reshape(-1).astype(np.float64))
    assert conv and info["rcs_rel_resid"] <= 1e-8
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(b)


def test_implicit_needs_a_linearization(B, oracle_rcs):
    A, b = oracle_rcs
    with pytest.raises(B.BAError) as ei:
        B.Problem.from_rcs(A.row_ptr, A.col, A.val, b, precision=B.BA_FP64, pcg_variant=B.BA_PCG_IMPLICIT)
    assert ei.value.status == B.BA_ERR_INVALID_ARG


def test_standard_fp32_reading_each_block_once(B):
    """FP32 systems whose stored blocks exceed 64 MB run the Sec. 3.2
    recurrence with the product that reads each stored block once (transposed
    products added with reductions).  On an RCS-only system with the pattern
    of 15,000 aerial cameras (about 110 MB of FP32 blocks, seeded SPD values)
    its iteration count stays within 2 % of the FP64 solve's (deterministic
    two-sided product) at the same tolerance, and the FP64 refinement takes
    both to the same true residual."""
    s = scenes.blocks_scene(n_blocks_x=3, n_blocks_y=2, block_side=50, n_pts=1_500_000, seed=3301)
    row_ptr, col = B.ba_symbolic_pattern(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt)
    del s
    n = len(row_ptr) - 1
    assert len(col) * 36 * 4 > 64 << 20
    val, _ = scenes.random_block_spd(row_ptr, col, np.full(n, 6, dtype=np.int32), seed=3302)
    val = val.reshape(-1, 36)
    b = np.random.default_rng(3303).standard_normal(6 * n)
    # inner FP32 PCG to 1e-6 with one refinement sweep; the FP64 solve to the same tolerance
    g32 = B.Problem.from_rcs(row_ptr, col, val, b, precision=B.BA_FP32, pcg_variant=B.BA_PCG_STANDARD,
                             pcg_rel_tol=1e-6, inner_rel_tol=1e-6, refine_max=1)
    i32, _ = g32.solve_rcs()
    g64 = B.Problem.from_rcs(row_ptr, col, val, b, precision=B.BA_FP64, pcg_rel_tol=1e-6)
    i64, conv = g64.solve_rcs()
    assert conv
    assert abs(i32["pcg_iters"] - i64["pcg_iters"]) <= max(2, 0.02 * i64["pcg_iters"]), (i32, i64)
    x32, _ = g32.step()
    x64, _ = g64.step()
    assert np.linalg.norm(x32 - x64) <= 1e-4 * np.linalg.norm(x64)
    # with refinement the FP32 solve reaches a tight true residual
    g = B.Problem.from_rcs(row_ptr, col, val, b, precision=B.BA_FP32, pcg_variant=B.BA_PCG_STANDARD,
                           pcg_rel_tol=1e-9, inner_rel_tol=1e-4)
    info, conv = g.solve_rcs()
    assert conv and info["rcs_rel_resid"] <= 1e-9
    for h in (g32, g64, g):
        h.close()
