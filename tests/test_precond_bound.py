"""How much any block-diagonal preconditioner could gain over block-Jacobi on
an aerial-shaped reduced camera system: the free 6x6 blocks of
M^-1 = L^-T T T^T L^-1 (T lower triangular per camera, the learned
correction's family) are optimised directly for the condition number
kappa(M^-1 S) from the block-Jacobi start, with eigenvector gradients of the
extreme eigenvalues of G^T S G (G = blockdiag(L_i^-T T_i)).

The result bounds what the learned correction can reach on these systems: the
optimum stays within a small factor of block-Jacobi (a block-diagonal
scaling is within a factor of the number of blocks per row of the best one),
and PCG iterations barely move."""
import numpy as np
import pytest

import oracle as O
import oracle.precond_net as N
import scenes


def _kappa_and_grad(o, S, Li, n):
    T = N.tri_from_out(o.reshape(n, N.NOUT))
    G = np.swapaxes(Li, 1, 2) @ T
    Gd = np.zeros_like(S)
    for i in range(n):
        Gd[6 * i:6 * i + 6, 6 * i:6 * i + 6] = G[i]
    w, V = np.linalg.eigh(Gd.T @ S @ Gd)
    lo, hi, vl, vh = w[0], w[-1], V[:, 0], V[:, -1]
    # d lambda / d Gd = 2 S Gd v v^T for a simple eigenvalue with unit eigenvector v
    dGd = 2 * (S @ Gd @ np.outer(vh, vh)) / hi - 2 * (S @ Gd @ np.outer(vl, vl)) / lo
    dT = Li @ np.stack([dGd[6 * i:6 * i + 6, 6 * i:6 * i + 6] for i in range(n)])
    do = np.zeros((n, N.NOUT))
    for q, (k, l) in enumerate(N.TRI):
        do[:, q] = dT[:, k, l] * (N.OUT_SCALE * T[:, k, k] if k == l else N.OUT_SCALE)
    return np.log(hi / lo), do.reshape(-1), G


def test_block_diagonal_optimum_is_close_to_block_jacobi():
    so = pytest.importorskip("scipy.optimize")
    s = scenes.aerial_small(n_along=8, n_across=4, pts_per_cam=200, seed=5)
    pb = O.Problem(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt, s.obs_uv)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, b = pb.rcs(e, Jc, Jp, 1e-4)
    S = O.bsmc_to_dense(A)
    n = len(A.row_ptr) - 1
    diag = np.stack([A.val[A.row_ptr[i]] for i in range(n)])
    Li = np.linalg.inv(np.linalg.cholesky(diag))
    f = lambda o: _kappa_and_grad(o, S, Li, n)[:2]
    o0 = np.zeros(n * N.NOUT)
    # the gradient is right: central differences on its largest coordinates
    k0, g0 = f(o0 + 0.01 * np.random.default_rng(1).normal(size=o0.size))
    x = 0.01 * np.random.default_rng(1).normal(size=o0.size)
    for j in np.argsort(-np.abs(g0))[:4]:
        h = np.zeros_like(x)
        h[j] = 1e-6
        fd = (f(x + h)[0] - f(x - h)[0]) / 2e-6
        assert abs(fd - g0[j]) <= 1e-4 * abs(fd)
    log_k_bj = f(o0)[0]
    r = so.minimize(f, o0, jac=True, method="L-BFGS-B", options={"maxiter": 150})
    assert r.fun <= log_k_bj + 1e-12
    ratio = np.exp(log_k_bj - r.fun)
    G = _kappa_and_grad(r.x, S, Li, n)[2]
    it_bj = O.pcg(A, b.reshape(-1), O.block_jacobi(A), 1e-8, max_iters=20000).iters
    it_opt = O.pcg(A, b.reshape(-1), G @ np.swapaxes(G, 1, 2), 1e-8, max_iters=20000).iters
    print(f"kappa(block-Jacobi) / kappa(optimum) = {ratio:.3f}; PCG iterations {it_bj} -> {it_opt}")
    assert ratio < 1.5
    assert it_opt >= 0.9 * it_bj
