"""Seeded synthetic bundle-adjustment scenes.

This module only makes input data: camera poses, 3-D points, which camera sees
which point, and noisy image observations.  It holds none of the solver's
arithmetic (no residual Jacobians, no normal equations, no Schur complement, no
PCG); both the FP64 oracle and the CUDA library consume what it returns.

Conventions shared with every consumer (the problem statement, Sec. 3.1):

* a camera is 6 numbers ``[omega(3), t(3)]``: an angle-axis rotation ``omega``
  and a translation ``t`` with ``X_cam = R(omega) X + t``;
* a pinhole with focal length ``f`` (px) and principal point ``(cx, cy)`` (px),
  +z in front of the camera, no distortion;
* observations are ``(cam, point, u, v)`` in pixels.

The observations are synthesised from ground truth with rotation matrices built
by a look-at construction and converted to angle-axis with scipy, then Gaussian
pixel noise is added; the initial values handed to the solver are perturbed
ground truth.  For cameras that also estimate interior parameters the module
gives perturbed initial interiors and the number of unknowns per camera; for
storage and solver measurements at sizes no reference can form, it gives
seeded symmetric positive definite values for a block pattern.  Scene shapes follow the paper's workloads (aerial grids, tracks
of a few cameras per point, N(0, sigma^2) px noise, Sec. 7.1).
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

F_PX = 1000.0
C_PX = 500.0
IMG_PX = 1000.0


@dataclasses.dataclass
class Scene:
    """A synthetic scene.  Arrays are host numpy arrays.

    cams_gt, cams0: (n, 6) float64  [omega, t], ground truth and initial value
    pts_gt, pts0:   (P, 3) float64
    obs_cam: (m,) int32, obs_pt: (m,) int64, obs_uv: (m, 2) float64 (noisy px)
    """
    name: str
    cams_gt: np.ndarray
    pts_gt: np.ndarray
    cams0: np.ndarray
    pts0: np.ndarray
    obs_cam: np.ndarray
    obs_pt: np.ndarray
    obs_uv: np.ndarray
    f: float = F_PX
    cx: float = C_PX
    cy: float = C_PX
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_cams(self) -> int:
        return self.cams_gt.shape[0]

    @property
    def n_pts(self) -> int:
        return self.pts_gt.shape[0]

    @property
    def n_obs(self) -> int:
        return self.obs_cam.shape[0]


# --------------------------------------------------------------------------
# geometry helpers for synthesis only (look-at frames, ground-truth pixels)
# --------------------------------------------------------------------------

def _look_at(centers: np.ndarray, targets: np.ndarray, up: np.ndarray) -> np.ndarray:
    """World->camera rotation matrices whose third row looks from center to target."""
    fwd = targets - centers
    fwd /= np.linalg.norm(fwd, axis=1, keepdims=True)
    down = -up[None, :] + (fwd @ up)[:, None] * fwd
    down /= np.linalg.norm(down, axis=1, keepdims=True)
    right = np.cross(down, fwd)
    return np.stack([right, down, fwd], axis=1)  # rows: x, y, z axes


def _nadir(centers: np.ndarray, yaw: np.ndarray) -> np.ndarray:
    c, s = np.cos(yaw), np.sin(yaw)
    z = np.zeros_like(c)
    r1 = np.stack([c, s, z], axis=1)
    r2 = np.stack([s, -c, z], axis=1)
    r3 = np.tile(np.array([0.0, 0.0, -1.0]), (len(c), 1))
    return np.stack([r1, r2, r3], axis=1)


def _pack_cams(Rw2c: np.ndarray, centers: np.ndarray) -> np.ndarray:
    omega = Rotation.from_matrix(Rw2c).as_rotvec()
    t = -np.einsum("nij,nj->ni", Rw2c, centers)
    return np.concatenate([omega, t], axis=1)


def _pixels(Rw2c, centers, cam_idx, X, f, cx, cy):
    """Ground-truth pixel positions of points X seen by cameras cam_idx."""
    Xc = np.einsum("mij,mj->mi", Rw2c[cam_idx], X - centers[cam_idx])
    return np.stack([f * Xc[:, 0] / Xc[:, 2] + cx, f * Xc[:, 1] / Xc[:, 2] + cy], 1), Xc[:, 2]


def _finish(name, Rw2c, centers, pts, obs_cam, obs_pt, rng, sigma_px, rot_sd, t_sd, pt_sd,
            outlier_frac=0.0, meta=None):
    uv, _ = _pixels(Rw2c, centers, obs_cam, pts[obs_pt], F_PX, C_PX, C_PX)
    if sigma_px > 0:
        uv = uv + rng.normal(0.0, sigma_px, uv.shape)
    meta = dict(meta or {})
    if outlier_frac > 0:
        k = int(round(outlier_frac * len(obs_cam)))
        idx = rng.choice(len(obs_cam), size=k, replace=False)
        uv[idx] = rng.uniform(0.0, IMG_PX, (k, 2))
        meta["n_outliers"] = k
    cams_gt = _pack_cams(Rw2c, centers)
    # initial poses: orientation perturbed by a rotation of N(0, rot_sd) rad per
    # axis in the camera frame, camera centre moved by N(0, t_sd) m per axis
    dR = Rotation.from_rotvec(rng.normal(0.0, rot_sd, (len(centers), 3))).as_matrix()
    R0 = np.einsum("nij,njk->nik", dR, Rw2c)
    cams0 = _pack_cams(R0, centers + rng.normal(0.0, t_sd, centers.shape))
    pts0 = pts + rng.normal(0.0, pt_sd, pts.shape)
    meta.setdefault("sigma_px", sigma_px)
    meta["mean_track"] = len(obs_cam) / len(pts)
    return Scene(name, cams_gt, pts.copy(), cams0, pts0, obs_cam.astype(np.int32),
                 obs_pt.astype(np.int64), uv, meta=meta)


def _choose_visible(rng, vis_lists, lo, hi):
    cams, ptid = [], []
    for k, vis in enumerate(vis_lists):
        L = int(rng.integers(lo, hi + 1))
        L = min(L, len(vis))
        pick = np.sort(rng.choice(vis, size=L, replace=False))
        cams.append(pick)
        ptid.append(np.full(L, k))
    return np.concatenate(cams), np.concatenate(ptid)


# --------------------------------------------------------------------------
# ring scene (the tiny FP64 workload and its scaled-down variants)
# --------------------------------------------------------------------------

def ring_scene(n_cams=50, n_pts=2000, track=(3, 8), seed=1001, sigma_px=0.5,
               rot_sd=0.01, t_sd=0.05, pt_sd=0.1, radius=30.0, half=5.0,
               name="ring") -> Scene:
    """Cameras on a horizontal ring looking at the centre of a cube of points.

    n_cams cameras evenly spaced on a circle of ``radius`` m at mid-height,
    n_pts points uniform in [-half, half]^3, each seen by L ~ U{track} cameras
    chosen uniformly among those that image it inside the frame with z > 0.
    """
    rng = np.random.default_rng(seed)
    phi = 2 * np.pi * np.arange(n_cams) / n_cams
    centers = np.stack([radius * np.cos(phi), radius * np.sin(phi), np.zeros(n_cams)], 1)
    Rw2c = _look_at(centers, np.zeros_like(centers), np.array([0.0, 0.0, 1.0]))
    pts = rng.uniform(-half, half, (n_pts, 3))
    # visibility: inside the image with positive depth
    vis = []
    for k in range(n_pts):
        uv, z = _pixels(Rw2c, centers, np.arange(n_cams), np.repeat(pts[k:k + 1], n_cams, 0),
                        F_PX, C_PX, C_PX)
        ok = (z > 0) & (uv[:, 0] >= 0) & (uv[:, 0] < IMG_PX) & (uv[:, 1] >= 0) & (uv[:, 1] < IMG_PX)
        vis.append(np.nonzero(ok)[0])
    lo, hi = track
    lo = min(lo, n_cams)
    hi = min(hi, n_cams)
    obs_cam, obs_pt = _choose_visible(rng, vis, lo, hi)
    return _finish(name, Rw2c, centers, pts, obs_cam, obs_pt, rng, sigma_px, rot_sd, t_sd, pt_sd,
                   meta={"seed": seed, "layout": "ring"})


def short_baseline_scene(n_cams=12, n_pts=400, n_twins=3, baseline=0.05, twin_pts=60, seed=1201,
                         sigma_px=0.5, radius=30.0, half=5.0) -> Scene:
    """A ring scene plus ``n_twins`` twin cameras: each stands ``baseline`` m
    beside a ring camera (along the ring's tangent, same orientation) and
    shares ``twin_pts`` extra points with it alone.  Those points are seen
    along two nearly parallel rays (about baseline / radius rad apart), so the
    depth of each is poorly determined: the ill-conditioned 3x3 point blocks of
    short-baseline image pairs.  Twin cameras are appended after the ring
    cameras; ring camera 2 k + 1 has twin n_cams + k."""
    base = ring_scene(n_cams=n_cams, n_pts=n_pts, seed=seed, sigma_px=0.0, radius=radius, half=half,
                      name="short_baseline")
    rng = np.random.default_rng(seed + 17)
    phi = 2 * np.pi * np.arange(n_cams) / n_cams
    centers = np.stack([radius * np.cos(phi), radius * np.sin(phi), np.zeros(n_cams)], 1)
    Rw2c = _look_at(centers, np.zeros_like(centers), np.array([0.0, 0.0, 1.0]))
    host = 2 * np.arange(n_twins) + 1
    tangent = np.stack([-np.sin(phi[host]), np.cos(phi[host]), np.zeros(n_twins)], 1)
    centers = np.concatenate([centers, centers[host] + baseline * tangent])
    Rw2c = np.concatenate([Rw2c, Rw2c[host]])
    pts, obs_cam, obs_pt = [base.pts_gt], [base.obs_cam], [base.obs_pt]
    P = base.n_pts
    for k in range(n_twins):
        X = rng.uniform(-half, half, (twin_pts, 3))
        pts.append(X)
        ids = P + np.arange(twin_pts)
        obs_cam += [np.full(twin_pts, host[k]), np.full(twin_pts, n_cams + k)]
        obs_pt += [ids, ids]
        P += twin_pts
    pts = np.concatenate(pts)
    obs_cam = np.concatenate(obs_cam)
    obs_pt = np.concatenate(obs_pt)
    return _finish("short_baseline", Rw2c, centers, pts, obs_cam, obs_pt, rng, sigma_px, 0.01, 0.05, 0.1,
                   meta={"seed": seed, "layout": "ring + short-baseline twins", "baseline_m": baseline,
                         "twin_of": {int(n_cams + k): int(host[k]) for k in range(n_twins)}})


def tiny_scene(n_cams=5, n_pts=30, seed=7, sigma_px=0.5, track=(2, 4), **kw) -> Scene:
    """A few cameras and points, small enough for dense brute force."""
    return ring_scene(n_cams=n_cams, n_pts=n_pts, track=track, seed=seed, sigma_px=sigma_px,
                      radius=30.0, name="tiny", **kw)


# --------------------------------------------------------------------------
# aerial grids (the FP32 workloads)
# --------------------------------------------------------------------------

def _terrain(x, y):
    return 10.0 * np.sin(2 * np.pi * x / 500.0) * np.sin(2 * np.pi * y / 500.0)


def _geom_track(rng, size, mean, lo, hi):
    """L = lo + G with G geometric on {0,1,...} of mean (mean - lo); redrawn above hi."""
    p = 1.0 / (mean - lo + 1.0)
    L = lo + rng.geometric(p, size) - 1
    bad = L > hi
    while bad.any():
        L[bad] = lo + rng.geometric(p, bad.sum()) - 1
        bad = L > hi
    return L


def _nearest_tracks(rng, cam_xy, pts_xy, L, chunk=1 << 20):
    """For each point, the L[k] camera centres nearest in xy (sorted by camera id)."""
    tree = cKDTree(cam_xy)
    kmax = int(L.max())
    cams, ptid = [], []
    for s in range(0, len(pts_xy), chunk):
        e = min(s + chunk, len(pts_xy))
        _, nn = tree.query(pts_xy[s:e], k=kmax)
        nn = nn.reshape(e - s, kmax)
        Lc = L[s:e]
        mask = np.arange(kmax)[None, :] < Lc[:, None]
        nn_sorted = np.where(mask, nn, np.iinfo(np.int64).max)
        nn_sorted.sort(axis=1)
        cams.append(nn_sorted[np.arange(kmax)[None, :] < Lc[:, None]])
        ptid.append(np.repeat(np.arange(s, e), Lc))
    return np.concatenate(cams), np.concatenate(ptid)


def aerial_scene(n_along=100, n_across=50, n_pts=1_000_000, along_m=40.0, across_m=70.0,
                 height=100.0, track_mean=5.0, track_max=20, seed=2001, sigma_px=1.0,
                 rot_sd=0.01, t_sd=0.05, pt_sd=0.1, yaw_sd=0.02, outlier_frac=0.0,
                 origin=(0.0, 0.0), name="aerial", track_min=2) -> Scene:
    """Nadir cameras on an n_along x n_across flight grid over sinusoidal terrain.

    Default: 50 x 100 = 5,000 cameras at 100 m (100 m footprint at f = 1000 px),
    40 m along track (60% forward overlap), 70 m across (30% side overlap),
    1M points uniform in xy, track length L = track_min + Geometric (mean 5, min 2, max 20),
    the L cameras being the nearest camera centres in xy (image bounds are not
    enforced: tracks of 20 do not fit a 60/30 overlap).
    """
    rng = np.random.default_rng(seed)
    ix, iy = np.meshgrid(np.arange(n_along), np.arange(n_across), indexing="ij")
    cx = origin[0] + ix.ravel() * along_m
    cy = origin[1] + iy.ravel() * across_m
    centers = np.stack([cx, cy, np.full(cx.shape, height)], 1)
    yaw = rng.normal(0.0, yaw_sd, len(cx))
    Rw2c = _nadir(centers, yaw)
    x = rng.uniform(cx.min(), cx.max(), n_pts)
    y = rng.uniform(cy.min(), cy.max(), n_pts)
    pts = np.stack([x, y, _terrain(x, y)], 1)
    L = _geom_track(rng, n_pts, track_mean, track_min, track_max)
    obs_cam, obs_pt = _nearest_tracks(rng, centers[:, :2], pts[:, :2], L)
    return _finish(name, Rw2c, centers, pts, obs_cam, obs_pt, rng, sigma_px, rot_sd, t_sd, pt_sd,
                   outlier_frac=outlier_frac,
                   meta={"seed": seed, "layout": f"aerial {n_along}x{n_across}",
                         "track_mean_target": track_mean, "track_max": track_max})


def blocks_scene(n_blocks_x=5, n_blocks_y=4, block_side=50, n_pts=10_000_000, overlap=0.2,
                 track_mean=6.0, track_max=40, seed=3001, sigma_px=1.0, outlier_frac=0.01,
                 along_m=40.0, across_m=70.0, height=100.0, name="blocks") -> Scene:
    """Several overlapping aerial blocks (20 blocks of 50 x 50 cameras by default).

    Block origins sit on an n_blocks_x x n_blocks_y layout so that neighbouring
    blocks overlap by ``overlap`` of their extent; points are spread uniformly
    over the union, tracks are L = 2 + Geometric (mean 6, max 40) nearest
    cameras, 1% of observations are replaced by uniform draws in the image.
    """
    rng = np.random.default_rng(seed)
    ext_x = (block_side - 1) * along_m
    ext_y = (block_side - 1) * across_m
    step_x = ext_x * (1 - overlap)
    step_y = ext_y * (1 - overlap)
    ix, iy = np.meshgrid(np.arange(block_side), np.arange(block_side), indexing="ij")
    cs = []
    for bx in range(n_blocks_x):
        for by in range(n_blocks_y):
            cs.append(np.stack([bx * step_x + ix.ravel() * along_m,
                                by * step_y + iy.ravel() * across_m], 1))
    cxy = np.concatenate(cs)
    centers = np.concatenate([cxy, np.full((len(cxy), 1), height)], 1)
    yaw = rng.normal(0.0, 0.02, len(cxy))
    Rw2c = _nadir(centers, yaw)
    x = rng.uniform(cxy[:, 0].min(), cxy[:, 0].max(), n_pts)
    y = rng.uniform(cxy[:, 1].min(), cxy[:, 1].max(), n_pts)
    pts = np.stack([x, y, _terrain(x, y)], 1)
    L = _geom_track(rng, n_pts, track_mean, 2, track_max)
    obs_cam, obs_pt = _nearest_tracks(rng, centers[:, :2], pts[:, :2], L)
    return _finish(name, Rw2c, centers, pts, obs_cam, obs_pt, rng, sigma_px, 0.01, 0.05, 0.1,
                   outlier_frac=outlier_frac,
                   meta={"seed": seed, "layout": f"{n_blocks_x*n_blocks_y} blocks of "
                                                 f"{block_side}x{block_side}",
                         "track_mean_target": track_mean, "track_max": track_max})


def aerial_small(n_along=20, n_across=10, pts_per_cam=200, seed=2101, **kw) -> Scene:
    """The aerial layout scaled down (same density of points per camera)."""
    return aerial_scene(n_along=n_along, n_across=n_across, n_pts=pts_per_cam * n_along * n_across,
                        seed=seed, name="aerial_small", **kw)


def preconditioner_scene(seed: int, n_cams=None, pts_per_cam=200) -> Scene:
    """A training / held-out instance for the learned preconditioner.

    Aerial-shaped, n ~ U[2000, 8000] cameras on a grid of aspect 1:2 and 200
    points per camera; seeds 0-199 train, 200-219 are held out.
    """
    rng = np.random.default_rng(10_000 + seed)
    if n_cams is None:
        n_cams = int(rng.integers(2000, 8001))
    n_across = max(2, int(round(np.sqrt(n_cams / 2))))
    n_along = max(2, int(round(n_cams / n_across)))
    return aerial_scene(n_along=n_along, n_across=n_across, n_pts=pts_per_cam * n_along * n_across,
                        seed=40_000 + seed, name=f"precond{seed}")


CONFIGS = {
    "ring50": lambda: ring_scene(seed=1001),
    "aerial5k": lambda: aerial_scene(seed=2001),
    "blocks50k": lambda: blocks_scene(seed=3001),
}


def shuffled(scene: Scene, seed: int = 0) -> Scene:
    """The same scene with its observation list in random order."""
    rng = np.random.default_rng(seed)
    p = rng.permutation(scene.n_obs)
    return dataclasses.replace(scene, obs_cam=scene.obs_cam[p], obs_pt=scene.obs_pt[p],
                               obs_uv=scene.obs_uv[p])


def capacity_scene(seed=5001, n_along=500, n_across=400, n_pts=40_000_000) -> Scene:
    """The capacity workload: 200,000 nadir cameras on a 400 x 500 flight grid,
    40M points, tracks L = 5 + Geometric (parameter 6.5, redrawn above 9) of
    the nearest cameras: a realised mean of about 6.1, so about 243M
    observations, and about 33 co-visible cameras per camera."""
    return aerial_scene(n_along=n_along, n_across=n_across, n_pts=n_pts, track_mean=6.5, track_max=9,
                        track_min=5, seed=seed, name="capacity")


# ----------------------------------------------------------------------------
# interior parameters and variable block sizes (inputs only)
# ----------------------------------------------------------------------------

def interiors0(n: int, seed: int = 0, f_sd=0.01, c_sd=2.0, k_sd=0.01) -> np.ndarray:
    """Initial interiors [f, cx, cy, k1, k2] per camera, (n, 5): the pinhole the
    observations were made with, perturbed (relative N(0, f_sd) on f,
    N(0, c_sd) px on the principal point, N(0, k_sd) on k1 and k2)."""
    rng = np.random.default_rng(seed)
    k = np.empty((n, 5))
    k[:, 0] = F_PX * (1.0 + rng.normal(0.0, f_sd, n))
    k[:, 1] = C_PX + rng.normal(0.0, c_sd, n)
    k[:, 2] = C_PX + rng.normal(0.0, c_sd, n)
    k[:, 3] = rng.normal(0.0, k_sd, n)
    k[:, 4] = rng.normal(0.0, k_sd, n)
    return k


def block_sizes(n: int, frac_self_cal: float, seed: int = 0) -> np.ndarray:
    """Unknowns per camera: 11 (six exterior + five interior) for a random
    fraction of self-calibrating cameras, 6 for the rest; int32 (n,)."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random(n) < frac_self_cal, 11, 6).astype(np.int32)


def random_block_spd(row_ptr, col, cdim, seed: int = 0, dtype=np.float64):
    """Values for a symmetric positive definite matrix with the given upper
    block pattern (diagonal block first in each row) and block sizes, in one
    packed array (block k row-major, c_i x c_j): off-diagonal blocks N(0, 1);
    each diagonal block G G^T / c + (1 + the sum of the Frobenius norms of its
    row's and column's off-diagonal blocks) I, so that every diagonal block
    dominates its block row (block Gershgorin) and the matrix is SPD.
    Returns (values, block offsets (nnzb + 1,) int64)."""
    rng = np.random.default_rng(seed)
    n = len(cdim)
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    row = np.repeat(np.arange(n), np.diff(row_ptr))
    size = cdim[row].astype(np.int64) * cdim[col].astype(np.int64)
    boff = np.concatenate([[0], np.cumsum(size)])
    val = rng.standard_normal(int(boff[-1]))
    off = row != col
    seg = np.repeat(np.arange(len(col)), size)
    nrm = np.sqrt(np.bincount(seg, weights=val * val, minlength=len(col)))
    dom = np.ones(n)
    np.add.at(dom, row[off], nrm[off])
    np.add.at(dom, col[off], nrm[off])
    for i in range(n):
        k = row_ptr[i]
        c = int(cdim[i])
        G = val[boff[k]:boff[k + 1]].reshape(c, c)
        Dm = G @ G.T / c + dom[i] * np.eye(c)
        val[boff[k]:boff[k + 1]] = Dm.reshape(-1)
    return val.astype(dtype), boff
