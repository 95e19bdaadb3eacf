"""Pins of the learned-preconditioner oracle against things other than itself:
finite differences, the closed form at zero output (block-Jacobi), SPD-ness,
adjointness of the aggregation, BF16 rounding against torch, and PCG with the
zero-output preconditioner against block-Jacobi PCG."""
import numpy as np
import pytest

import oracle as O
import oracle.precond_net as N
import scenes


@pytest.fixture(scope="module")
def inst():
    s = scenes.aerial_small(n_along=6, n_across=4, pts_per_cam=60, seed=71)
    pb = O.Problem(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt, s.obs_uv)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, b = pb.rcs(e, Jc, Jp, 1e-3)
    diag, src, dst, w = N.graph_from_bsmc(A.row_ptr, A.col, A.val)
    return A, b, diag, src, dst, w


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(size=1000) * 10.0 ** np.random.default_rng(1).integers(-5, 5, 1000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(N.bf16_round(x), ref)


def test_zero_output_is_block_jacobi(inst):
    A, b, diag, src, dst, w = inst
    Minv, _, _ = N.precond_blocks(diag, np.zeros((len(diag), N.NOUT)))
    np.testing.assert_allclose(Minv, np.linalg.inv(diag), rtol=1e-10, atol=1e-12 * np.abs(np.linalg.inv(diag)).max())


def test_preconditioner_is_spd_for_any_output(inst):
    A, b, diag, src, dst, w = inst
    o = np.random.default_rng(3).normal(0, 5.0, (len(diag), N.NOUT))
    Minv, _, _ = N.precond_blocks(diag, o)
    for M in Minv:
        assert np.allclose(M, M.T, rtol=1e-12, atol=1e-12 * np.abs(M).max())
        assert np.linalg.eigvalsh(M).min() > 0


def test_aggregation_adjoint(inst):
    A, b, diag, src, dst, w = inst
    n = len(diag)
    rng = np.random.default_rng(4)
    h, g = rng.normal(size=(n, 7)), rng.normal(size=(n, 7))
    lhs = np.sum(N.aggregate(h, src, dst, w, n) * g)
    rhs = np.sum(h * N.aggregate_T(g, src, dst, w, n))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_gradients_match_finite_differences(inst):
    A, b, diag, src, dst, w = inst
    n = len(diag)
    Wt = N.init_weights(5)
    rng = np.random.default_rng(6)
    Wt["Wo"] = rng.normal(0, 0.05, Wt["Wo"].shape)
    Wt["bo"] = rng.normal(0, 0.05, Wt["bo"].shape)
    Wt["b1"] = rng.normal(0, 0.1, Wt["b1"].shape)
    Wt["b2"] = rng.normal(0, 0.1, Wt["b2"].shape)
    Wp = N.probes(n, 3, 7)
    Up = N.apply_S_blocks(A.row_ptr, A.col, A.val, Wp)
    Sap = lambda Z: N.apply_S_blocks(A.row_ptr, A.col, A.val, Z)
    loss, g = N.loss_and_grad(Wt, diag, src, dst, w, Wp, Up, Sap)
    assert 0.0 <= loss <= 1.0
    h = 1e-5
    for name in ("W1", "b1", "W2", "b2", "Wo", "bo"):
        flat = Wt[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for k in idx:
            old = flat[k]
            flat[k] = old + h
            lp, _ = N.loss_and_grad(Wt, diag, src, dst, w, Wp, Up, Sap)
            flat[k] = old - h
            lm, _ = N.loss_and_grad(Wt, diag, src, dst, w, Wp, Up, Sap)
            flat[k] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[k]
            assert abs(fd - an) <= 1e-4 * max(abs(fd), 1e-6), (name, k, fd, an)


def _dense(A):
    return O.bsmc_to_dense(A)


def test_energy_loss_is_the_optimal_richardson_error(inst):
    """Brute force on the dense S: the loss equals min over alpha of
    sum_p ||w_p - alpha M^-1 S w_p||_S^2 / sum_p ||w_p||_S^2, the minimum found
    by a scalar search rather than the closed form."""
    from scipy.optimize import minimize_scalar
    A, b, diag, src, dst, w = inst
    n = len(diag)
    Wt = N.init_weights(11)
    rng = np.random.default_rng(12)
    Wt["Wo"] = rng.normal(0, 0.3, Wt["Wo"].shape)
    Wt["bo"] = rng.normal(0, 0.3, Wt["bo"].shape)
    Wp = N.probes(n, 3, 13)
    Up = N.apply_S_blocks(A.row_ptr, A.col, A.val, Wp)
    Sap = lambda Z: N.apply_S_blocks(A.row_ptr, A.col, A.val, Z)
    loss, _ = N.loss_and_grad(Wt, diag, src, dst, w, Wp, Up, Sap)
    S = _dense(A)
    o, _ = N.forward(Wt, N.node_features(diag, src, dst, w), src, dst, w)
    Minv, _, _ = N.precond_blocks(diag, o)
    Md = np.zeros_like(S)
    for i in range(n):
        Md[6 * i:6 * i + 6, 6 * i:6 * i + 6] = Minv[i]
    Wd = Wp.reshape(6 * n, -1)
    E = lambda al: sum(float(r @ S @ r) for r in (Wd - al * Md @ S @ Wd).T)
    den = sum(float(c @ S @ c) for c in Wd.T)
    best = minimize_scalar(E, bracket=(0.0, 1.0), tol=1e-12)
    assert abs(loss - best.fun / den) <= 1e-7 * max(loss, 1e-3)
    assert 0.0 < loss < 1.0


def test_energy_loss_is_zero_on_a_block_diagonal_system(inst):
    """With the off-diagonal blocks dropped, S is its own block diagonal and
    block-Jacobi (zero output) is S^-1: the optimal Richardson step is exact."""
    A, b, diag, src, dst, w = inst
    n = len(diag)
    rp = np.arange(n + 1)
    col = np.arange(n)
    Wt = N.init_weights(14)
    Wp = N.probes(n, 2, 9)
    Up = N.apply_S_blocks(rp, col, diag, Wp)
    Sap = lambda Z: N.apply_S_blocks(rp, col, diag, Z)
    loss, g = N.loss_and_grad(Wt, diag, src, dst, w, Wp, Up, Sap)
    assert abs(loss) < 1e-12
    # a minimum: the gradient of the output layer vanishes there
    assert np.abs(g["bo"]).max() < 1e-9 and np.abs(g["Wo"]).max() < 1e-9


def test_energy_loss_is_invariant_to_a_common_scale(inst):
    """Equal diagonal outputs s scale every M_i^-1 by exp(2 a s); the optimal
    step absorbs it, so the loss is unchanged."""
    A, b, diag, src, dst, w = inst
    n = len(diag)
    Wp = N.probes(n, 2, 15)
    Up = N.apply_S_blocks(A.row_ptr, A.col, A.val, Wp)
    Sap = lambda Z: N.apply_S_blocks(A.row_ptr, A.col, A.val, Z)
    W0 = N.init_weights(16)
    W1 = N.init_weights(16)
    W1["bo"] = np.array([3.0 if k == l else 0.0 for k, l in N.TRI])
    l0, _ = N.loss_and_grad(W0, diag, src, dst, w, Wp, Up, Sap)
    l1, _ = N.loss_and_grad(W1, diag, src, dst, w, Wp, Up, Sap)
    assert abs(l0 - l1) <= 1e-10 * l0


def test_zero_output_pcg_matches_block_jacobi(inst):
    A, b, diag, src, dst, w = inst
    Minv, _, _ = N.precond_blocks(diag, np.zeros((len(diag), N.NOUT)))
    r1 = O.pcg(A, b.reshape(-1), Minv, 1e-8)
    r2 = O.pcg(A, b.reshape(-1), O.block_jacobi(A), 1e-8)
    assert r1.iters == r2.iters
    # the two inverses differ by rounding (Cholesky vs LU); the iterates agree to kappa * eps
    assert np.linalg.norm(r1.y - r2.y) <= 1e-7 * np.linalg.norm(r2.y)
