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
    loss, g = N.loss_and_grad(Wt, diag, src, dst, w, Wp, Up)
    # the loss is O(1e3): central differences with h = 1e-4 sit between truncation
    # and rounding error (1e-8 relative agreement at smooth points)
    h = 1e-4
    for name in ("W1", "b1", "W2", "b2", "Wo", "bo"):
        flat = Wt[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for k in idx:
            old = flat[k]
            flat[k] = old + h
            lp, _ = N.loss_and_grad(Wt, diag, src, dst, w, Wp, Up)
            flat[k] = old - h
            lm, _ = N.loss_and_grad(Wt, diag, src, dst, w, Wp, Up)
            flat[k] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[k]
            assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-3), (name, k, fd, an)


def test_zero_output_pcg_matches_block_jacobi(inst):
    A, b, diag, src, dst, w = inst
    Minv, _, _ = N.precond_blocks(diag, np.zeros((len(diag), N.NOUT)))
    r1 = O.pcg(A, b.reshape(-1), Minv, 1e-8)
    r2 = O.pcg(A, b.reshape(-1), O.block_jacobi(A), 1e-8)
    assert r1.iters == r2.iters
    # the two inverses differ by rounding (Cholesky vs LU); the iterates agree to kappa * eps
    assert np.linalg.norm(r1.y - r2.y) <= 1e-7 * np.linalg.norm(r2.y)
