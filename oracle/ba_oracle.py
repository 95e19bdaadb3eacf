"""FP64 CPU oracle for exact Levenberg-Marquardt bundle adjustment.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The CUDA
library never calls it and shares no code with it.

Plain, slow, obviously-correct float64 numpy, written from the paper
(arXiv 2307.08383, "Distributed bundle adjustment with block-based sparse
matrix compression for super large scale datasets"):

* Sec. 3.1, Eq. 1: the damped normal equations (J^T J + lambda D^T D) dx = -J^T e.
* Sec. 3.1, Eq. 3: the camera / point partition U, V, W, l_c, l_p.
* Sec. 3.1, Eq. 4: the reduced camera system (RCS) S = U - W V^-1 W^T,
  b = l_c - W V^-1 l_p, formed point by point (Sec. 5, Fig. 16).
* Sec. 3.1, Eq. 5: back-substitution V dx_p = l_p - W^T dx_c.
* Sec. 3.2, Eqs. 6-7: block-Jacobi PCG on R y = b.
* Sec. 4 (Fig. 4, Eq. 9): BSMC storage - upper-triangle non-zero blocks,
  per-block column ids, per-row start, diagonal block first in each row.
* Sec. 6.2 (Fig. 13): the BSMC matrix-vector product.
* Sec. 3.1 (after Eq. 5) and Sec. 5: the points may instead be triangulated
  from the camera poses; the method is not given (a reading below).

Readings of what the paper leaves open:

* camera model: pinhole, +z forward, focal f, principal point (cx, cy), no
  distortion; cameras are [omega(3), t(3)] with X_cam = R(omega) X + t;
* update: the pose is perturbed in the camera frame, X_cam <- Exp(d_omega) X_cam + dt,
  i.e. R <- Exp(d_omega) R, t <- Exp(d_omega) t + dt; points X <- X + dX;
* damping: D^T D = diag(J^T J) with every entry clamped to [1e-6, 1e32];
* PCG: M = the diagonal blocks of S; stop when ||r_k|| / ||r_0|| <= T (the
  printed ratio is inverted, which would never stop);
* LM schedule: Nielsen's rule (lambda0 = 1e-4; accept iff rho > 1e-3 with a
  positive predicted decrease; lambda *= max(1/3, 1 - (2 rho - 1)^3), nu = 2;
  on reject lambda *= nu, nu *= 2);
* robust loss (not in the paper): Huber on the squared norm s = ||e||^2,
  rho(s) = s for s <= delta^2 else 2 delta sqrt(s) - delta^2, applied by
  scaling e and J with sqrt(rho'(s)) (first-order IRLS);
* triangulation: per point, the linear least-squares intersection of its
  observations (each gives two equations linear in X from the pinhole model
  with the depth multiplied out), then Gauss-Newton steps on the point's
  plain reprojection error.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.spatial.transform import Rotation

DAMP_MIN = 1e-6
DAMP_MAX = 1e32


# ----------------------------------------------------------------------------
# camera model (Sec. 3.1: e is the vector of reprojection errors)
# ----------------------------------------------------------------------------

def hat(w: np.ndarray) -> np.ndarray:
    """Skew matrices [w]x of shape (..., 3, 3) so that hat(w) @ v = w x v."""
    w = np.asarray(w, dtype=np.float64)
    z = np.zeros(w.shape[:-1])
    return np.stack([np.stack([z, -w[..., 2], w[..., 1]], -1),
                     np.stack([w[..., 2], z, -w[..., 0]], -1),
                     np.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def rodrigues(w: np.ndarray) -> np.ndarray:
    """R = Exp(w) = I + sin(th)/th [w]x + (1 - cos(th))/th^2 [w]x^2 (Rodrigues).

    For th < 1e-8 the second-order Taylor expansion is used.
    """
    w = np.asarray(w, dtype=np.float64)
    th = np.linalg.norm(w, axis=-1)
    K = hat(w)
    K2 = K @ K
    small = th < 1e-8
    ths = np.where(small, 1.0, th)
    a = np.where(small, 1.0 - th ** 2 / 6.0, np.sin(ths) / ths)
    b = np.where(small, 0.5 - th ** 2 / 24.0, (1.0 - np.cos(ths)) / ths ** 2)
    return np.eye(3) + a[..., None, None] * K + b[..., None, None] * K2


def so3_log(R: np.ndarray) -> np.ndarray:
    """Angle-axis of a rotation matrix (library routine)."""
    return Rotation.from_matrix(R).as_rotvec()


@dataclasses.dataclass
class Intrinsics:
    f: float = 1000.0
    cx: float = 500.0
    cy: float = 500.0


def camera_points(cams, pts, obs_cam, obs_pt):
    """X_cam = R(omega_c) X_k + t_c for every observation."""
    R = rodrigues(cams[obs_cam, :3])
    X = pts[obs_pt]
    RX = np.einsum("mij,mj->mi", R, X)
    return RX + cams[obs_cam, 3:], RX, R


def residuals(cams, pts, obs_cam, obs_pt, obs_uv, intr: Intrinsics):
    """e = pi(X_cam) - u_obs, pi = (f x/z + cx, f y/z + cy); returns (e, z)."""
    Xc, _, _ = camera_points(cams, pts, obs_cam, obs_pt)
    u = intr.f * Xc[:, 0] / Xc[:, 2] + intr.cx
    v = intr.f * Xc[:, 1] / Xc[:, 2] + intr.cy
    return np.stack([u, v], 1) - obs_uv, Xc[:, 2]


def jacobians(cams, pts, obs_cam, obs_pt, obs_uv, intr: Intrinsics):
    """Residuals and analytic Jacobians per observation.

    J_c = de/d[d_omega, dt] (m, 2, 6), J_p = de/dX (m, 2, 3), using
    dX_cam/d(d_omega) = -[X_cam]x, dX_cam/d(dt) = I (camera-frame update),
    dX_cam/dX = R, and dpi/dX_cam = [[f/z, 0, -f x/z^2], [0, f/z, -f y/z^2]].
    """
    Xc, _, R = camera_points(cams, pts, obs_cam, obs_pt)
    x, y, z = Xc[:, 0], Xc[:, 1], Xc[:, 2]
    e = np.stack([intr.f * x / z + intr.cx, intr.f * y / z + intr.cy], 1) - obs_uv
    m = len(x)
    A = np.zeros((m, 2, 3))
    A[:, 0, 0] = intr.f / z
    A[:, 0, 2] = -intr.f * x / z ** 2
    A[:, 1, 1] = intr.f / z
    A[:, 1, 2] = -intr.f * y / z ** 2
    Jc = np.concatenate([A @ (-hat(Xc)), A], axis=2)
    Jp = A @ R
    return e, Jc, Jp


def huber_rho(s, delta):
    """rho(s) on the squared norm s: s if s <= delta^2 else 2 delta sqrt(s) - delta^2."""
    s = np.asarray(s, dtype=np.float64)
    if delta is None or not np.isfinite(delta):
        return s
    return np.where(s <= delta * delta, s, 2.0 * delta * np.sqrt(s) - delta * delta)


def huber_weight(s, delta):
    """rho'(s): 1 if s <= delta^2 else delta / sqrt(s)."""
    s = np.asarray(s, dtype=np.float64)
    if delta is None or not np.isfinite(delta):
        return np.ones_like(s)
    return np.where(s <= delta * delta, 1.0, delta / np.sqrt(np.maximum(s, 1e-300)))


def cost(cams, pts, obs_cam, obs_pt, obs_uv, intr, delta=None):
    """F = 1/2 sum_i rho(||e_i||^2)."""
    e, _ = residuals(cams, pts, obs_cam, obs_pt, obs_uv, intr)
    return 0.5 * float(np.sum(huber_rho(np.sum(e * e, 1), delta)))


def linearize(cams, pts, obs_cam, obs_pt, obs_uv, intr, delta=None):
    """Weighted residuals and Jacobians: sqrt(rho'(s)) e, sqrt(rho'(s)) J."""
    e, Jc, Jp = jacobians(cams, pts, obs_cam, obs_pt, obs_uv, intr)
    sw = np.sqrt(huber_weight(np.sum(e * e, 1), delta))
    return e * sw[:, None], Jc * sw[:, None, None], Jp * sw[:, None, None]


# ----------------------------------------------------------------------------
# Eq. 3 blocks and Eq. 4 reduced camera system, point by point (Sec. 5)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Blocks:
    U: np.ndarray      # (n, 6, 6) damped J_c^T J_c per camera
    V: np.ndarray      # (P, 3, 3) damped J_p^T J_p per point
    W: np.ndarray      # (m, 6, 3) J_c^T J_p per observation (block (cam, pt))
    l_c: np.ndarray    # (n, 6)  -J_c^T e
    l_p: np.ndarray    # (P, 3)  -J_p^T e


def damp(diag):
    return np.clip(diag, DAMP_MIN, DAMP_MAX)


def normal_blocks(e, Jc, Jp, obs_cam, obs_pt, n, P, lam) -> Blocks:
    """U = J_c^T J_c + lam D_c^T D_c, V = J_p^T J_p + lam D_p^T D_p, W = J_c^T J_p,
    l_c = -J_c^T e, l_p = -J_p^T e (Eq. 3), with D^T D = clamp(diag(J^T J))."""
    U = np.zeros((n, 6, 6))
    V = np.zeros((P, 3, 3))
    np.add.at(U, obs_cam, np.einsum("mai,maj->mij", Jc, Jc))
    np.add.at(V, obs_pt, np.einsum("mai,maj->mij", Jp, Jp))
    W = np.einsum("mai,maj->mij", Jc, Jp)
    l_c = np.zeros((n, 6))
    l_p = np.zeros((P, 3))
    np.add.at(l_c, obs_cam, -np.einsum("mai,ma->mi", Jc, e))
    np.add.at(l_p, obs_pt, -np.einsum("mai,ma->mi", Jp, e))
    for k in range(6):
        U[:, k, k] += lam * damp(U[:, k, k])
    for k in range(3):
        V[:, k, k] += lam * damp(V[:, k, k])
    return Blocks(U, V, W, l_c, l_p)


def tracks(obs_pt, P):
    """Observation indices of every point, each track ordered by camera id
    (the caller passes observations already sorted by (point, camera))."""
    order = np.argsort(obs_pt, kind="stable")
    starts = np.searchsorted(obs_pt[order], np.arange(P + 1))
    return [order[starts[k]:starts[k + 1]] for k in range(P)]


def sort_observations(obs_cam, obs_pt):
    """Permutation that sorts observations by (point, camera)."""
    return np.lexsort((obs_cam, obs_pt))


def reduced_camera_system(blk: Blocks, obs_cam, obs_pt, n, P):
    """Eq. 4, S = U - W V^-1 W^T and b = l_c - W V^-1 l_p, formed point by point.

    For each point k (Sec. 5 step 1) the sub-RCS is -W_ak V_k^-1 W_bk^T on the
    block (cam_a, cam_b) of every pair of its observations, and -W_ak V_k^-1 l_pk
    on b; the sub-RCSs are summed (step 2).  Only blocks with cam_a <= cam_b are
    kept (BSMC stores the upper triangle).  Returns ({(i, j): 6x6}, b).
    """
    S = {(i, i): blk.U[i].copy() for i in range(n)}
    b = blk.l_c.copy()
    for k, tr in enumerate(tracks(obs_pt, P)):
        Vinv = np.linalg.inv(blk.V[k])
        for a in tr:
            Ya = blk.W[a] @ Vinv
            b[obs_cam[a]] -= Ya @ blk.l_p[k]
            for bb in tr:
                i, j = obs_cam[a], obs_cam[bb]
                if i > j:
                    continue
                S.setdefault((i, j), np.zeros((6, 6)))
                S[(i, j)] = S[(i, j)] - Ya @ blk.W[bb].T
    return S, b


def back_substitute(blk: Blocks, obs_cam, obs_pt, P, dxc):
    """Eq. 5: V dx_p = l_p - W^T dx_c, point by point."""
    rhs = blk.l_p.copy()
    np.add.at(rhs, obs_pt, -np.einsum("mij,mi->mj", blk.W, dxc[obs_cam]))
    return np.linalg.solve(blk.V, rhs[..., None])[..., 0]


# ----------------------------------------------------------------------------
# BSMC (Sec. 4, Fig. 4) and its matrix-vector product (Sec. 6.2, Fig. 13)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class BSMC:
    row_ptr: np.ndarray  # (n+1,) int32 start of each block row
    col: np.ndarray      # (nnzb,) int32 column id of each block
    val: np.ndarray      # (nnzb, 6, 6) float64 block values

    @property
    def n(self):
        return len(self.row_ptr) - 1

    @property
    def nnzb(self):
        return len(self.col)


def bsmc_from_blocks(S: dict, n: int) -> BSMC:
    """Upper-triangle blocks, row by row, columns ascending (diagonal first)."""
    keys = sorted(S.keys())
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    for (i, _j) in keys:
        row_ptr[i + 1] += 1
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    col = np.array([j for (_i, j) in keys], dtype=np.int32)
    val = np.stack([S[k] for k in keys]) if keys else np.zeros((0, 6, 6))
    return BSMC(row_ptr, col, val)


def bsmc_pattern(obs_cam, obs_pt, n, P):
    """Structural BSMC pattern: all diagonals plus every (i<j) sharing a point."""
    pairs = {(i, i) for i in range(n)}
    for tr in tracks(obs_pt, P):
        cs = sorted(set(obs_cam[tr].tolist()))
        for x in range(len(cs)):
            for y in range(x + 1, len(cs)):
                pairs.add((cs[x], cs[y]))
    keys = sorted(pairs)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for (i, _j) in keys:
        row_ptr[i + 1] += 1
    return np.cumsum(row_ptr).astype(np.int32), np.array([j for _, j in keys], dtype=np.int32)


def bsmc_spmv(A: BSMC, x: np.ndarray) -> np.ndarray:
    """y = S x from the upper triangle: every block is read once, its row id
    found by counting row starts; it adds S_ij x_j to y_i and, off the
    diagonal, S_ij^T x_i to y_j; the components are summed (Fig. 13)."""
    x = x.reshape(-1, 6)
    y = np.zeros_like(x)
    row = 0
    for blk in range(A.nnzb):
        while blk >= A.row_ptr[row + 1]:
            row += 1
        j = A.col[blk]
        y[row] += A.val[blk] @ x[j]
        if j != row:
            y[j] += A.val[blk].T @ x[row]
    return y.reshape(-1)


def bsmc_to_dense(A: BSMC) -> np.ndarray:
    n = A.n
    D = np.zeros((6 * n, 6 * n))
    for i in range(n):
        for blk in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col[blk]
            D[6 * i:6 * i + 6, 6 * j:6 * j + 6] = A.val[blk]
            if j != i:
                D[6 * j:6 * j + 6, 6 * i:6 * i + 6] = A.val[blk].T
    return D


def block_jacobi(A: BSMC) -> np.ndarray:
    """M^-1: the inverses of the diagonal blocks S_ii (first block of each row)."""
    return np.linalg.inv(A.val[A.row_ptr[:-1]])


# ----------------------------------------------------------------------------
# PCG (Sec. 3.2, Eqs. 6-7)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class PCGResult:
    y: np.ndarray
    iters: int
    rel_resid: float       # ||r_k|| / ||r_0|| of the recurrence
    history: list


def pcg(A: BSMC, b: np.ndarray, Minv: np.ndarray, tol: float, max_iters: int | None = None,
        spmv=None, precond=None) -> PCGResult:
    """Preconditioned CG on R y = b with y_0 = 0:
        r_0 = b, d_0 = M^-1 r_0;
        repeat: alpha = r^T M^-1 r / d^T R d; y += alpha d; r -= alpha R d;
                beta = r+^T M^-1 r+ / r^T M^-1 r; d = M^-1 r+ + beta d
        until ||r_k|| / ||r_0|| <= tol (or max_iters iterations).
    ``spmv`` / ``precond`` replace the products with R and M^-1 (other
    storage, other block sizes)."""
    n = A.n
    if max_iters is None:
        max_iters = max(1000, 6 * n)
    mv = spmv or (lambda v: bsmc_spmv(A, v))
    apply_m = precond or (lambda v: np.einsum("nij,nj->ni", Minv, v.reshape(-1, 6)).reshape(-1))
    y = np.zeros_like(b)
    r = b.copy()
    r0 = np.linalg.norm(r)
    if r0 == 0.0:
        return PCGResult(y, 0, 0.0, [])
    z = apply_m(r)
    d = z.copy()
    rz = r @ z
    hist = []
    k = 0
    while k < max_iters:
        q = mv(d)
        alpha = rz / (d @ q)
        y = y + alpha * d
        r = r - alpha * q
        k += 1
        eta = np.linalg.norm(r) / r0
        hist.append(eta)
        if eta <= tol:
            break
        z = apply_m(r)
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        d = z + beta * d
    return PCGResult(y, k, hist[-1], hist)


# ----------------------------------------------------------------------------
# LM iteration (Eq. 1 with the Schur trick, Fig. 2 pipeline)
# ----------------------------------------------------------------------------

def apply_update(cams, pts, dxc, dxp):
    """R <- Exp(d_omega) R, t <- Exp(d_omega) t + dt, X <- X + dX."""
    dxc = dxc.reshape(-1, 6)
    dR = rodrigues(dxc[:, :3])
    R = dR @ rodrigues(cams[:, :3])
    t = np.einsum("nij,nj->ni", dR, cams[:, 3:]) + dxc[:, 3:]
    new = np.concatenate([so3_log(R), t], 1)
    return new, pts + dxp.reshape(-1, 3)


@dataclasses.dataclass
class LMState:
    cams: np.ndarray
    pts: np.ndarray
    lam: float = 1e-4
    nu: float = 2.0


@dataclasses.dataclass
class StepInfo:
    cost_before: float
    cost_after: float
    rho: float
    lam: float
    accepted: bool
    pcg_iters: int
    pcg_rel: float
    predicted: float


class Problem:
    """An observation set in (point, camera) order plus the solver options."""

    def __init__(self, n_cams, n_pts, obs_cam, obs_pt, obs_uv, intr=None, delta=None,
                 pcg_tol=1e-10, pcg_max_iters=None):
        perm = sort_observations(np.asarray(obs_cam), np.asarray(obs_pt))
        self.perm = perm
        self.obs_cam = np.asarray(obs_cam)[perm].astype(np.int64)
        self.obs_pt = np.asarray(obs_pt)[perm].astype(np.int64)
        self.obs_uv = np.asarray(obs_uv, dtype=np.float64)[perm]
        self.n = int(n_cams)
        self.P = int(n_pts)
        self.intr = intr or Intrinsics()
        self.delta = delta
        self.pcg_tol = pcg_tol
        self.pcg_max_iters = pcg_max_iters

    def cost(self, cams, pts):
        return cost(cams, pts, self.obs_cam, self.obs_pt, self.obs_uv, self.intr, self.delta)

    def linearize(self, cams, pts):
        return linearize(cams, pts, self.obs_cam, self.obs_pt, self.obs_uv, self.intr, self.delta)

    def rcs(self, e, Jc, Jp, lam):
        blk = normal_blocks(e, Jc, Jp, self.obs_cam, self.obs_pt, self.n, self.P, lam)
        S, b = reduced_camera_system(blk, self.obs_cam, self.obs_pt, self.n, self.P)
        return blk, bsmc_from_blocks(S, self.n), b

    def solve(self, A: BSMC, b):
        return pcg(A, b.reshape(-1), block_jacobi(A), self.pcg_tol, self.pcg_max_iters)

    def step(self, st: LMState):
        """One LM iteration: linearize, RCS, PCG, back-substitute, gain ratio."""
        F0 = self.cost(st.cams, st.pts)
        e, Jc, Jp = self.linearize(st.cams, st.pts)
        blk, A, b = self.rcs(e, Jc, Jp, st.lam)
        res = self.solve(A, b)
        dxc = res.y.reshape(-1, 6)
        dxp = back_substitute(blk, self.obs_cam, self.obs_pt, self.P, dxc)
        cams1, pts1 = apply_update(st.cams, st.pts, dxc, dxp)
        F1 = self.cost(cams1, pts1)
        Jd = np.einsum("mij,mj->mi", Jc, dxc[self.obs_cam]) + \
            np.einsum("mij,mj->mi", Jp, dxp[self.obs_pt])
        pred = 0.5 * float(np.sum(e * e) - np.sum((e + Jd) ** 2))
        rho = (F0 - F1) / pred if pred > 0 else -np.inf
        ok = bool(pred > 0 and rho > 1e-3 and np.isfinite(F1))
        lam_used = st.lam
        if ok:
            new = LMState(cams1, pts1, st.lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), 2.0)
        else:
            new = LMState(st.cams, st.pts, st.lam * st.nu, st.nu * 2.0)
        info = StepInfo(F0, F1 if ok else F0, rho, lam_used, ok, res.iters, res.rel_resid, pred)
        return new, info, (dxc, dxp)


def rms_px(cams, pts, obs_cam, obs_pt, obs_uv, intr):
    e, _ = residuals(cams, pts, obs_cam, obs_pt, obs_uv, intr)
    return float(np.sqrt(np.sum(e * e) / len(e)))


# ----------------------------------------------------------------------------
# triangulation from the camera poses (Sec. 3.1 after Eq. 5; Sec. 5)
# ----------------------------------------------------------------------------

def triangulation_rows(cam, uv, intr: Intrinsics):
    """The two equations a X = r of one observation, linear in the point X:
    with X_cam = R X + t, u - cx = f x/z and v - cy = f y/z, multiplying out z
    gives ((u - cx) R_3 - f R_1) . X = f t_1 - (u - cx) t_3 and the same with
    (v, cy, R_2, t_2)."""
    R = rodrigues(cam[:3])
    t = cam[3:]
    du, dv = uv[0] - intr.cx, uv[1] - intr.cy
    A = np.stack([du * R[2] - intr.f * R[0], dv * R[2] - intr.f * R[1]])
    r = np.array([intr.f * t[0] - du * t[2], intr.f * t[1] - dv * t[2]])
    return A, r


def triangulate(cams, obs_cam, obs_pt, obs_uv, intr: Intrinsics, P: int, gn_iters: int = 3):
    """Every point from the cameras: the least-squares solution of its stacked
    linear equations (numpy lstsq), then gn_iters Gauss-Newton steps
    (J_p^T J_p) dX = -J_p^T e on its reprojection error."""
    obs_cam = np.asarray(obs_cam, dtype=np.int64)
    out = np.zeros((P, 3))
    for k, tr in enumerate(tracks(obs_pt, P)):
        rows = [triangulation_rows(cams[obs_cam[a]], obs_uv[a], intr) for a in tr]
        A = np.concatenate([r[0] for r in rows])
        r = np.concatenate([r[1] for r in rows])
        X = np.linalg.lstsq(A, r, rcond=None)[0]
        for _ in range(gn_iters):
            e, _, Jp = jacobians(cams, X[None, :], obs_cam[tr], np.zeros(len(tr), dtype=np.int64), obs_uv[tr], intr)
            Jp = Jp.reshape(-1, 3)
            X = X + np.linalg.solve(Jp.T @ Jp, -Jp.T @ e.reshape(-1))
        out[k] = X
    return out


# ----------------------------------------------------------------------------
# memory model of Sec. 4.1 (Eqs. 8-10)
# ----------------------------------------------------------------------------

def csr_bytes(alpha, n, c, val_bytes=8, id_bytes=4):
    """Eq. 8: Y_C = alpha n^2 c^2 8 + alpha n^2 c^2 4 + n c 4."""
    return alpha * n * n * c * c * val_bytes + alpha * n * n * c * c * id_bytes + n * c * id_bytes


def bsmc_bytes(alpha, n, c, val_bytes=8, id_bytes=4):
    """Eq. 9: Y_B = (alpha n^2 + n)/2 c^2 8 + (alpha n^2 + n)/2 3 4 + n 4."""
    nb = (alpha * n * n + n) / 2.0
    return nb * c * c * val_bytes + nb * 3 * id_bytes + n * id_bytes


def csr_bsmc_ratio(alpha, n, c):
    """Eq. 10 with the denominator term 3 alpha n (printed as 3 alpha):
    Y_C / Y_B = (6 alpha n c^2 + 2c) / (2 alpha n c^2 + 2 c^2 + 3 alpha n + 5)."""
    return (6 * alpha * n * c * c + 2 * c) / (2 * alpha * n * c * c + 2 * c * c + 3 * alpha * n + 5)


# ----------------------------------------------------------------------------
# selected RCS blocks of a large problem (Eq. 4 restricted to the points that
# reach them), for spot checks at sizes where the full oracle is too slow
# ----------------------------------------------------------------------------

def rcs_blocks_sampled(cams, pts, obs_cam, obs_pt, obs_uv, intr, lam, pairs, delta=None):
    """S_ij for each (i <= j) in pairs and b_i for each diagonal pair.

    S_ij only receives terms from points seen by both i and j, and S_ii, b_i
    only from points seen by i (plus U_ii, which needs every observation of
    camera i); so Eq. 3-4 are evaluated on the sub-problem made of all
    observations of those points."""
    obs_cam = np.asarray(obs_cam, dtype=np.int64)
    obs_pt = np.asarray(obs_pt, dtype=np.int64)
    P = len(pts)
    cam_pts = {}
    need = set(i for p in pairs for i in p)
    for c in need:
        cam_pts[c] = set(np.unique(obs_pt[obs_cam == c]).tolist())
    keep = set()
    for (i, j) in pairs:
        keep |= cam_pts[i] if i == j else (cam_pts[i] & cam_pts[j])
    keep = np.array(sorted(keep), dtype=np.int64)
    remap = -np.ones(P, dtype=np.int64)
    remap[keep] = np.arange(len(keep))
    sel = np.nonzero(remap[obs_pt] >= 0)[0]
    sc, sp = obs_cam[sel], remap[obs_pt[sel]]
    order = sort_observations(sc, sp)
    sc, sp, suv = sc[order], sp[order], np.asarray(obs_uv)[sel][order]
    e, Jc, Jp = linearize(cams, pts[keep], sc, sp, suv, intr, delta)
    blk = normal_blocks(e, Jc, Jp, sc, sp, len(cams), len(keep), lam)
    S, b = reduced_camera_system(blk, sc, sp, len(cams), len(keep))
    out = {}
    for (i, j) in pairs:
        out[(i, j)] = S[(i, j)]
    return out, {i: b[i] for (i, j) in pairs if i == j}
