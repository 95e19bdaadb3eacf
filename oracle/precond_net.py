"""FP64 CPU oracle of the learned block-Jacobi correction (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the library.

The paper preconditions PCG with the block diagonal of the RCS (Sec. 3.2).
The learned correction (not in the paper) keeps that structure and changes
each diagonal block's inverse:

    S_ii = L_i L_i^T (Cholesky),  M_i^-1 = L_i^-T T_i T_i^T L_i^-1,

with T_i lower triangular, T_kk = exp(a o_kk), T_kl = a o_kl (k > l),
a = OUT_SCALE, so M^-1 is SPD for any network output o and equals plain
block-Jacobi when o = 0.

The network is two message-passing layers on the camera co-visibility graph
(nodes: cameras; edges: the off-diagonal BSMC blocks, both directions, weight
w_ij = ||S_ij||_F / sqrt(||S_ii||_F ||S_jj||_F)):

    m_i = sum_j w_ij h_j / max(deg_i, 1)
    h'_i = relu([h_i | m_i] W + b)          (W: 2K x 64)

then o_i = h2_i W_o + b_o (64 -> 21).  Layer 1 reads 24 node features, so its
input is [x_i | m_i] of width 48.  Weights are rounded to BF16 on both sides
(the GPU keeps BF16 weights); all arithmetic here is FP64.

Training loss: the energy-norm error left by one preconditioned Richardson
step with the optimal step length, on probe vectors W (columns w_p):

    u_p = S w_p,  z_p = M^-1 u_p,  a = sum_p z_p^T u_p,  c = sum_p z_p^T S z_p,
    e = sum_p w_p^T u_p,  loss = 1 - a^2 / (c e)  in [0, 1],

i.e. min_alpha sum_p ||w_p - alpha M^-1 S w_p||_S^2 / sum_p ||w_p||_S^2: small
when M^-1 acts like S^-1 in the S-norm on the probes.  It is invariant to a
common scale of M^-1 and sees the off-diagonal blocks through S z_p.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
NFEAT = 24
NOUT = 21
OUT_SCALE = 0.1
# lower-triangle order of the 21 outputs: (k, l), k >= l, row by row
TRI = [(k, l) for k in range(6) for l in range(k + 1)]


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def init_weights(seed=0):
    """Layer shapes: W1 (48, 64), b1 (64), W2 (128, 64), b2 (64), Wo (64, 21), bo (21).
    The output layer starts at zero (plain block-Jacobi)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / (2 * NFEAT)), (2 * NFEAT, HIDDEN))
    W2 = rng.normal(0, np.sqrt(2.0 / (2 * HIDDEN)), (2 * HIDDEN, HIDDEN))
    return {"W1": bf16_round(W1), "b1": np.zeros(HIDDEN), "W2": bf16_round(W2), "b2": np.zeros(HIDDEN),
            "Wo": np.zeros((HIDDEN, NOUT)), "bo": np.zeros(NOUT)}


def graph_from_bsmc(row_ptr, col, val):
    """Edges (i, j, w_ij) in both directions and the diagonal blocks."""
    n = len(row_ptr) - 1
    diag = np.stack([val[row_ptr[i]] for i in range(n)])
    dn = np.linalg.norm(diag.reshape(n, -1), axis=1)
    src, dst, w = [], [], []
    for i in range(n):
        for b in range(row_ptr[i] + 1, row_ptr[i + 1]):
            j = col[b]
            wij = np.linalg.norm(val[b]) / np.sqrt(dn[i] * dn[j])
            src += [i, j]
            dst += [j, i]
            w += [wij, wij]
    return diag, np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64), np.array(w)


def node_features(diag, src, dst, w):
    """24 features per camera: the 15 off-diagonal correlations of S_ii, the 6
    log-diagonals centred by their mean over cameras, log(1 + degree), the
    summed edge weight, and a constant 1."""
    n = len(diag)
    d = np.einsum("nkk->nk", diag)
    s = 1.0 / np.sqrt(d)
    corr = diag * s[:, :, None] * s[:, None, :]
    iu = np.triu_indices(6, 1)
    ld = np.log(d)
    ld = ld - ld.mean(axis=0, keepdims=True)
    deg = np.bincount(dst, minlength=n).astype(float)
    wsum = np.bincount(dst, weights=w, minlength=n)
    return np.concatenate([corr[:, iu[0], iu[1]], ld, np.log1p(deg)[:, None], wsum[:, None], np.ones((n, 1))], 1)


def aggregate(h, src, dst, w, n):
    """m_i = sum_{(j -> i)} w_ij h_j / max(deg_i, 1)."""
    deg = np.maximum(np.bincount(dst, minlength=n), 1).astype(float)
    m = np.zeros((n, h.shape[1]))
    np.add.at(m, dst, w[:, None] * h[src])
    return m / deg[:, None]


def aggregate_T(g, src, dst, w, n):
    """Adjoint of aggregate: dh_j += sum_{(j -> i)} w_ij g_i / max(deg_i, 1)."""
    deg = np.maximum(np.bincount(dst, minlength=n), 1).astype(float)
    gs = g / deg[:, None]
    out = np.zeros_like(g)
    np.add.at(out, src, w[:, None] * gs[dst])
    return out


def forward(Wt, x, src, dst, w):
    n = len(x)
    a1 = np.concatenate([x, aggregate(x, src, dst, w, n)], 1)
    z1 = a1 @ Wt["W1"] + Wt["b1"]
    h1 = np.maximum(z1, 0)
    a2 = np.concatenate([h1, aggregate(h1, src, dst, w, n)], 1)
    z2 = a2 @ Wt["W2"] + Wt["b2"]
    h2 = np.maximum(z2, 0)
    o = h2 @ Wt["Wo"] + Wt["bo"]
    return o, (a1, z1, h1, a2, z2, h2)


def tri_from_out(o):
    """T (n, 6, 6) lower triangular from the 21 outputs."""
    n = len(o)
    T = np.zeros((n, 6, 6))
    for q, (k, l) in enumerate(TRI):
        T[:, k, l] = np.exp(OUT_SCALE * o[:, q]) if k == l else OUT_SCALE * o[:, q]
    return T


def precond_blocks(diag, o):
    """M_i^-1 = L_i^-T T_i T_i^T L_i^-1 for every camera."""
    L = np.linalg.cholesky(diag)
    Li = np.linalg.inv(L)
    G = np.swapaxes(Li, 1, 2) @ tri_from_out(o)
    return G @ np.swapaxes(G, 1, 2), G, Li


def loss_and_grad(Wt, diag, src, dst, w, Wp, Up, Sapply):
    """Energy loss and its gradient w.r.t. every weight.

    Wp, Up: (n, 6, k) probes and S @ probes per camera block; Sapply(Z) = S Z."""
    x = node_features(diag, src, dst, w)
    n = len(x)
    o, (a1, z1, h1, a2, z2, h2) = forward(Wt, x, src, dst, w)
    Minv, G, Li = precond_blocks(diag, o)
    Z = Minv @ Up
    V = Sapply(Z)
    a = float(np.sum(Z * Up))
    c = float(np.sum(Z * V))
    e = float(np.sum(Wp * Up))
    loss = 1.0 - a * a / (c * e)
    # d loss / d Z = (2a/(ce)) ((a/c) V - U); Z = Minv U -> dMinv = dZ U^T
    dZ = (2.0 * a / (c * e)) * ((a / c) * V - Up)
    dM = dZ @ np.swapaxes(Up, 1, 2)
    # Minv = G G^T -> dG = (dM + dM^T) G;  G = Li^T T -> dT = Li dG (lower part used)
    dG = (dM + np.swapaxes(dM, 1, 2)) @ G
    dT = Li @ dG
    T = tri_from_out(o)
    do = np.zeros_like(o)
    for q, (k, l) in enumerate(TRI):
        do[:, q] = dT[:, k, l] * (OUT_SCALE * T[:, k, k] if k == l else OUT_SCALE)
    g = {"Wo": h2.T @ do, "bo": do.sum(0)}
    dh2 = do @ Wt["Wo"].T
    dz2 = dh2 * (z2 > 0)
    g["W2"] = a2.T @ dz2
    g["b2"] = dz2.sum(0)
    da2 = dz2 @ Wt["W2"].T
    dh1 = da2[:, :HIDDEN] + aggregate_T(da2[:, HIDDEN:], src, dst, w, n)
    dz1 = dh1 * (z1 > 0)
    g["W1"] = a1.T @ dz1
    g["b1"] = dz1.sum(0)
    return loss, g


def probes(n, k, seed):
    """Rademacher probe vectors (n, 6, k)."""
    rng = np.random.default_rng(seed)
    return rng.choice([-1.0, 1.0], size=(n, 6, k))


def apply_S_blocks(row_ptr, col, val, Wp):
    """U = S W for probe blocks W (n, 6, k) from the upper-triangle BSMC (Fig. 13)."""
    n = len(row_ptr) - 1
    U = np.zeros_like(Wp)
    for i in range(n):
        for b in range(row_ptr[i], row_ptr[i + 1]):
            j = col[b]
            U[i] += val[b] @ Wp[j]
            if j != i:
                U[j] += val[b].T @ Wp[i]
    return U
