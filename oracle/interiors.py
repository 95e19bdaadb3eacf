"""FP64 CPU oracle for interior parameters and variable block sizes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The CUDA
library never calls it and shares no code with it.

Sec. 4: block (i, j) of the reduced camera system has c_i x c_j entries, c_i
being the number of unknowns of camera i, and BSMC stores each upper block with
its position and its size (Fig. 4); the memory analysis of Sec. 4.1 (Eqs. 8-10)
takes c = 11, six exterior and five interior unknowns per camera.  This module
extends the 6-unknown oracle (``ba_oracle``) to cameras that also estimate
their interiors, so that the RCS has blocks of mixed sizes:

* the camera model with five interiors, its residuals and Jacobians (Eq. 1's e
  and J);
* Eq. 3 and Eq. 4 with per-camera block sizes: U_i is c_i x c_i, W_ik is
  c_i x 3, the RCS block (i, j) is c_i x c_j;
* BSMC with per-block sizes (Sec. 4, Fig. 4), its product (Sec. 6.2, Fig. 13),
  its block-Jacobi preconditioner (Sec. 3.2) and its bytes (Eq. 9 with a
  height and width per block);
* the PCG of Sec. 3.2 on it (``ba_oracle.pcg`` with these products);
* interiors shared by the images of one physical camera: a block row of five
  unknowns per physical camera beside the images' six-unknown rows;
* the back-substitution of Eq. 5 and one LM iteration with interiors (the
  gain ratio and damping schedule of ``ba_oracle.Problem.step``).

Readings of what the paper leaves open:

* the five interiors are the focal length f, the principal point (cx, cy) and
  two radial distortion coefficients k1, k2 acting on the normalised image
  coordinates: with xh = x/z, yh = y/z, r2 = xh^2 + yh^2 and
  d = 1 + k1 r2 + k2 r2^2, the projection is u = f d xh + cx, v = f d yh + cy;
* every camera has interiors of its own; a camera whose interiors are held
  fixed has c_i = 6 unknowns, a self-calibrating one c_i = 11, its five
  interior unknowns after the six exterior ones; interiors update additively;
  where several images share a physical camera, its interiors are one block of
  five unknowns of their own (``rcs_shared``);
* damping, as for six unknowns: lambda times diag(J^T J) clamped to
  [1e-6, 1e32], on every unknown.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .ba_oracle import DAMP_MAX, DAMP_MIN, apply_update, camera_points, hat, pcg, sort_observations, tracks

N_EXT = 6
N_INT = 5
C_MAX = N_EXT + N_INT


# ----------------------------------------------------------------------------
# camera model with interiors (Eq. 1: e and J)
# ----------------------------------------------------------------------------

def residuals_intr(cams, intr, pts, obs_cam, obs_pt, obs_uv):
    """e = pi(X_cam; f, cx, cy, k1, k2) - u_obs.  ``intr`` is (n, 5)."""
    Xc, _, _ = camera_points(cams, pts, obs_cam, obs_pt)
    k = intr[obs_cam]
    xh, yh = Xc[:, 0] / Xc[:, 2], Xc[:, 1] / Xc[:, 2]
    r2 = xh * xh + yh * yh
    d = 1.0 + k[:, 3] * r2 + k[:, 4] * r2 * r2
    return np.stack([k[:, 0] * d * xh + k[:, 1], k[:, 0] * d * yh + k[:, 2]], 1) - obs_uv


def jacobians_intr(cams, intr, pts, obs_cam, obs_pt, obs_uv):
    """Residuals and analytic Jacobians per observation.

    J_c (m, 2, 11): de/d[d_omega, dt] (camera-frame pose update, as in
    ``ba_oracle.jacobians``) then de/d[f, cx, cy, k1, k2]; J_p (m, 2, 3).
    With g = 2 (k1 + 2 k2 r2), the image-plane Jacobian is
    D = f [[d + g xh^2, g xh yh], [g xh yh, d + g yh^2]], and
    d(xh, yh)/dX_cam = [[1/z, 0, -xh/z], [0, 1/z, -yh/z]]."""
    Xc, _, R = camera_points(cams, pts, obs_cam, obs_pt)
    k = intr[obs_cam]
    f, k1, k2 = k[:, 0], k[:, 3], k[:, 4]
    z = Xc[:, 2]
    xh, yh = Xc[:, 0] / z, Xc[:, 1] / z
    r2 = xh * xh + yh * yh
    d = 1.0 + k1 * r2 + k2 * r2 * r2
    g = 2.0 * (k1 + 2.0 * k2 * r2)
    m = len(z)
    e = np.stack([f * d * xh + k[:, 1], f * d * yh + k[:, 2]], 1) - obs_uv
    D = np.empty((m, 2, 2))
    D[:, 0, 0] = f * (d + g * xh * xh)
    D[:, 0, 1] = f * g * xh * yh
    D[:, 1, 0] = D[:, 0, 1]
    D[:, 1, 1] = f * (d + g * yh * yh)
    Nz = np.zeros((m, 2, 3))
    Nz[:, 0, 0] = 1.0 / z
    Nz[:, 0, 2] = -xh / z
    Nz[:, 1, 1] = 1.0 / z
    Nz[:, 1, 2] = -yh / z
    A = D @ Nz
    Jc = np.zeros((m, 2, C_MAX))
    Jc[:, :, 0:3] = A @ (-hat(Xc))
    Jc[:, :, 3:6] = A
    Jc[:, 0, 6] = d * xh
    Jc[:, 1, 6] = d * yh
    Jc[:, 0, 7] = 1.0
    Jc[:, 1, 8] = 1.0
    Jc[:, 0, 9] = f * xh * r2
    Jc[:, 1, 9] = f * yh * r2
    Jc[:, 0, 10] = f * xh * r2 * r2
    Jc[:, 1, 10] = f * yh * r2 * r2
    Jp = A @ R
    return e, Jc, Jp


# ----------------------------------------------------------------------------
# variable-size BSMC (Sec. 4, Fig. 4)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class VBSMC:
    row_ptr: np.ndarray  # (n+1,) int32 start of each block row
    col: np.ndarray      # (nnzb,) int32 column id of each block
    cdim: np.ndarray     # (n,) int32 unknowns of each camera (block height / width)
    val: list            # nnzb arrays, block k of row i and column j is (cdim[i], cdim[j])

    @property
    def n(self):
        return len(self.row_ptr) - 1

    @property
    def nnzb(self):
        return len(self.col)

    def offsets(self):
        """First vector entry of every camera: (n+1,)."""
        return np.concatenate([[0], np.cumsum(self.cdim)]).astype(np.int64)


def vbsmc_from_blocks(S: dict, cdim) -> VBSMC:
    """Upper-triangle blocks, row by row, columns ascending (diagonal first)."""
    n = len(cdim)
    keys = sorted(S.keys())
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for (i, _j) in keys:
        row_ptr[i + 1] += 1
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    col = np.array([j for (_i, j) in keys], dtype=np.int32)
    return VBSMC(row_ptr, col, np.asarray(cdim, dtype=np.int32), [S[k] for k in keys])


def vbsmc_spmv(A: VBSMC, x: np.ndarray) -> np.ndarray:
    """y = S x from the upper triangle: S_ij x_j into y_i and, off the
    diagonal, S_ij^T x_i into y_j (Fig. 13), with per-camera slices."""
    off = A.offsets()
    y = np.zeros_like(x)
    row = 0
    for blk in range(A.nnzb):
        while blk >= A.row_ptr[row + 1]:
            row += 1
        j = A.col[blk]
        B = A.val[blk]
        y[off[row]:off[row + 1]] += B @ x[off[j]:off[j + 1]]
        if j != row:
            y[off[j]:off[j + 1]] += B.T @ x[off[row]:off[row + 1]]
    return y


def vbsmc_to_dense(A: VBSMC) -> np.ndarray:
    off = A.offsets()
    D = np.zeros((off[-1], off[-1]))
    for i in range(A.n):
        for blk in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col[blk]
            D[off[i]:off[i + 1], off[j]:off[j + 1]] = A.val[blk]
            if j != i:
                D[off[j]:off[j + 1], off[i]:off[i + 1]] = A.val[blk].T
    return D


def vb_block_jacobi(A: VBSMC):
    """M^-1 per camera: the inverse of its diagonal block (the first of its row)."""
    return [np.linalg.inv(A.val[A.row_ptr[i]]) for i in range(A.n)]


def vb_precond(A: VBSMC, Minv):
    off = A.offsets()

    def apply(v):
        out = np.empty_like(v)
        for i in range(A.n):
            out[off[i]:off[i + 1]] = Minv[i] @ v[off[i]:off[i + 1]]
        return out
    return apply


def vb_pcg(A: VBSMC, b, tol, max_iters=None):
    """Block-Jacobi PCG of Sec. 3.2 on the variable-size system."""
    if max_iters is None:
        max_iters = max(1000, 6 * A.n)
    return pcg(A, b, None, tol, max_iters, spmv=lambda v: vbsmc_spmv(A, v),
               precond=vb_precond(A, vb_block_jacobi(A)))


def vbsmc_bytes(A: VBSMC, val_bytes=8, id_bytes=4):
    """Eq. 9 with the block sizes of this matrix: the values of every upper
    block (c_i c_j each), three ids per block (column, height, width) and one
    row start per camera."""
    vals = sum(int(A.cdim[i]) * int(A.cdim[j]) for i in range(A.n)
               for j in A.col[A.row_ptr[i]:A.row_ptr[i + 1]])
    return vals * val_bytes + A.nnzb * 3 * id_bytes + A.n * id_bytes


# ----------------------------------------------------------------------------
# Eq. 3 and Eq. 4 with per-camera block sizes
# ----------------------------------------------------------------------------

def _damp(v):
    return np.clip(v, DAMP_MIN, DAMP_MAX)


def rcs_vb(e, Jc, Jp, obs_cam, obs_pt, cdim, P, lam):
    """The RCS with c_i unknowns per camera (the first c_i columns of its J_c).

    U_i = sum J_c^T J_c + lam clamp(diag) (c_i x c_i), V_k likewise (3 x 3),
    W_a = J_c^T J_p (c_i x 3), l_c = -J_c^T e, l_p = -J_p^T e (Eq. 3); then
    S = U - W V^-1 W^T and b = l_c - W V^-1 l_p point by point (Eq. 4, Sec. 5),
    upper blocks only.  Observations must be sorted by (point, camera).
    Returns (VBSMC, b as one vector in camera order)."""
    cdim = np.asarray(cdim, dtype=np.int32)
    n = len(cdim)
    U = [np.zeros((c, c)) for c in cdim]
    lc = [np.zeros(c) for c in cdim]
    V = np.zeros((P, 3, 3))
    lp = np.zeros((P, 3))
    W = []
    for a in range(len(e)):
        i, k = obs_cam[a], obs_pt[a]
        Ja = Jc[a][:, :cdim[i]]
        U[i] += Ja.T @ Ja
        lc[i] -= Ja.T @ e[a]
        V[k] += Jp[a].T @ Jp[a]
        lp[k] -= Jp[a].T @ e[a]
        W.append(Ja.T @ Jp[a])
    for i in range(n):
        U[i] = U[i] + lam * np.diag(_damp(np.diag(U[i])))
    for k in range(P):
        V[k] = V[k] + lam * np.diag(_damp(np.diag(V[k])))
    S = {(i, i): U[i].copy() for i in range(n)}
    b = [x.copy() for x in lc]
    for k, tr in enumerate(tracks(obs_pt, P)):
        Vinv = np.linalg.inv(V[k])
        for a in tr:
            Ya = W[a] @ Vinv
            b[obs_cam[a]] = b[obs_cam[a]] - Ya @ lp[k]
            for bb in tr:
                i, j = obs_cam[a], obs_cam[bb]
                if i > j:
                    continue
                S.setdefault((i, j), np.zeros((cdim[i], cdim[j])))
                S[(i, j)] = S[(i, j)] - Ya @ W[bb].T
    return vbsmc_from_blocks(S, cdim), np.concatenate(b)


def scene_rcs_vb(scene, intr, cdim, lam):
    """The variable-size RCS of a scene at its initial state with interiors
    ``intr`` (n, 5) and block sizes ``cdim`` (6 or 11 per camera)."""
    order = sort_observations(scene.obs_cam, scene.obs_pt)
    oc, op, uv = scene.obs_cam[order], scene.obs_pt[order], scene.obs_uv[order]
    e, Jc, Jp = jacobians_intr(scene.cams0, intr, scene.pts0, oc, op, uv)
    return rcs_vb(e, Jc, Jp, oc, op, cdim, scene.n_pts, lam)


# ----------------------------------------------------------------------------
# interiors shared by the images of one physical camera
# ----------------------------------------------------------------------------

def rcs_shared(e, Jc, Jp, obs_cam, obs_pt, phys, K, P, lam):
    """The RCS when the images of a physical camera share one set of
    interiors: images 0..n-1 keep their six exterior unknowns (block size 6),
    and physical camera q becomes block n + q with the five interior unknowns
    (block size 5), coupled to every image phys maps to it.

    Per observation a of image i, the exterior columns of J_c go to block i
    and the interior columns to block n + phys[i].  Eq. 3 per block:
    U = sum J_s^T J_t over the slots s, t of each observation (which couples
    image i and its physical camera even without a point), damped on the
    diagonal; l_c = -sum J_s^T e.  Eq. 4 per point k: with W_beta the sum of
    J_s^T J_p over the point's slots in block beta, S(beta, gamma) -=
    W_beta V_k^-1 W_gamma^T and b_beta -= W_beta V_k^-1 l_p,k for the blocks
    beta <= gamma the point touches.  Observations must be sorted by
    (point, camera).  Returns (VBSMC, b)."""
    n = len(phys)
    cdim = np.array([N_EXT] * n + [N_INT] * K, dtype=np.int32)

    def slots(a):
        i = obs_cam[a]
        return ((i, Jc[a][:, :N_EXT]), (n + phys[i], Jc[a][:, N_EXT:C_MAX]))

    S = {}
    lc = [np.zeros(c) for c in cdim]
    V = np.zeros((P, 3, 3))
    lp = np.zeros((P, 3))
    for a in range(len(e)):
        sl = slots(a)
        for (bs, Js) in sl:
            lc[bs] -= Js.T @ e[a]
            for (bt, Jt) in sl:
                if bs <= bt:
                    S.setdefault((bs, bt), np.zeros((cdim[bs], cdim[bt])))
                    S[(bs, bt)] = S[(bs, bt)] + Js.T @ Jt
        k = obs_pt[a]
        V[k] += Jp[a].T @ Jp[a]
        lp[k] -= Jp[a].T @ e[a]
    for beta in range(n + K):
        D = S[(beta, beta)]
        S[(beta, beta)] = D + lam * np.diag(_damp(np.diag(D)))
    for k in range(P):
        V[k] = V[k] + lam * np.diag(_damp(np.diag(V[k])))
    b = [x.copy() for x in lc]
    for k, tr in enumerate(tracks(obs_pt, P)):
        Vinv = np.linalg.inv(V[k])
        W = {}
        for a in tr:
            for (bs, Js) in slots(a):
                W[bs] = W.get(bs, np.zeros((cdim[bs], 3))) + Js.T @ Jp[a]
        for beta, Wb in W.items():
            b[beta] = b[beta] - Wb @ Vinv @ lp[k]
            for gamma, Wg in W.items():
                if beta <= gamma:
                    S.setdefault((beta, gamma), np.zeros((cdim[beta], cdim[gamma])))
                    S[(beta, gamma)] = S[(beta, gamma)] - Wb @ Vinv @ Wg.T
    return vbsmc_from_blocks(S, cdim), np.concatenate(b)


def scene_rcs_shared(scene, intr_phys, phys, lam):
    """The shared-interior RCS of a scene at its initial state: ``intr_phys``
    (K, 5) are the physical cameras' interiors, ``phys`` (n,) maps each image
    to its physical camera."""
    order = sort_observations(scene.obs_cam, scene.obs_pt)
    oc, op, uv = scene.obs_cam[order], scene.obs_pt[order], scene.obs_uv[order]
    phys = np.asarray(phys)
    e, Jc, Jp = jacobians_intr(scene.cams0, intr_phys[phys], scene.pts0, oc, op, uv)
    return rcs_shared(e, Jc, Jp, oc, op, phys, len(intr_phys), scene.n_pts, lam)


# ----------------------------------------------------------------------------
# Eq. 5 and one LM iteration with per-camera interiors
# ----------------------------------------------------------------------------

def back_substitute_vb(e, Jc, Jp, obs_cam, obs_pt, cdim, P, lam, dxc):
    """Eq. 5 with c_i unknowns per camera: V_k dx_p,k = l_p,k - sum_a
    W_a^T dx_c,cam(a), W_a = J_c,a^T J_p,a over the camera's c_i columns.
    ``dxc`` is one vector in camera order; returns (P, 3)."""
    off = np.concatenate([[0], np.cumsum(cdim)])
    V = np.zeros((P, 3, 3))
    rhs = np.zeros((P, 3))
    for a in range(len(e)):
        i, k = obs_cam[a], obs_pt[a]
        Ja = Jc[a][:, :cdim[i]]
        V[k] += Jp[a].T @ Jp[a]
        rhs[k] -= Jp[a].T @ e[a] + (Ja.T @ Jp[a]).T @ dxc[off[i]:off[i + 1]]
    for k in range(P):
        V[k] = V[k] + lam * np.diag(_damp(np.diag(V[k])))
    return np.linalg.solve(V, rhs[..., None])[..., 0]


@dataclasses.dataclass
class LMStateVB:
    cams: np.ndarray
    intr: np.ndarray
    pts: np.ndarray
    lam: float = 1e-4
    nu: float = 2.0


def cost_intr(cams, intr, pts, obs_cam, obs_pt, obs_uv):
    e = residuals_intr(cams, intr, pts, obs_cam, obs_pt, obs_uv)
    return 0.5 * float(np.sum(e * e))


def lm_step_vb(st: LMStateVB, obs_cam, obs_pt, obs_uv, cdim, P, tol=1e-10):
    """One LM iteration with interiors: linearize, the variable-size RCS,
    block-Jacobi PCG, Eq. 5, the update (the pose as in ``apply_update``,
    interiors and points additively), the gain ratio against the model
    decrease 1/2 (||e||^2 - ||e + J dx||^2) and Nielsen's damping rule.
    Observations sorted by (point, camera).  Returns (new state, accepted,
    cost before, cost after, (dxc, dxp))."""
    cdim = np.asarray(cdim)
    off = np.concatenate([[0], np.cumsum(cdim)])
    F0 = cost_intr(st.cams, st.intr, st.pts, obs_cam, obs_pt, obs_uv)
    e, Jc, Jp = jacobians_intr(st.cams, st.intr, st.pts, obs_cam, obs_pt, obs_uv)
    A, b = rcs_vb(e, Jc, Jp, obs_cam, obs_pt, cdim, P, st.lam)
    dxc = vb_pcg(A, b, tol).y
    dxp = back_substitute_vb(e, Jc, Jp, obs_cam, obs_pt, cdim, P, st.lam, dxc)
    n = len(cdim)
    ext = np.stack([dxc[off[i]:off[i] + N_EXT] for i in range(n)])
    cams1, pts1 = apply_update(st.cams, st.pts, ext, dxp)
    intr1 = st.intr.copy()
    for i in range(n):
        if cdim[i] == C_MAX:
            intr1[i] += dxc[off[i] + N_EXT:off[i + 1]]
    F1 = cost_intr(cams1, intr1, pts1, obs_cam, obs_pt, obs_uv)
    Jd = np.stack([Jc[a][:, :cdim[obs_cam[a]]] @ dxc[off[obs_cam[a]]:off[obs_cam[a] + 1]] for a in range(len(e))])
    Jd = Jd + np.einsum("mij,mj->mi", Jp, dxp[obs_pt])
    pred = 0.5 * float(np.sum(e * e) - np.sum((e + Jd) ** 2))
    rho = (F0 - F1) / pred if pred > 0 else -np.inf
    ok = bool(pred > 0 and rho > 1e-3 and np.isfinite(F1))
    if ok:
        new = LMStateVB(cams1, intr1, pts1, st.lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), 2.0)
    else:
        new = LMStateVB(st.cams, st.intr, st.pts, st.lam * st.nu, st.nu * 2.0)
    return new, ok, F0, (F1 if ok else F0), (dxc, dxp)
