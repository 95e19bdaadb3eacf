"""GPU parity of the variable-size BSMC (Sec. 4, Fig. 4: block (i, j) is
c_i x c_j; c = 6 exterior or 11 with five interior unknowns, Sec. 4.1)
against the oracle: the RCS with interiors formed on the device (Eqs. 1, 3, 4),
the product (Sec. 6.2, Fig. 13) and the block-Jacobi PCG (Sec. 3.2) of
ba_vbsmc_* on the oracle's RCS with interiors, and on seeded
SPD systems at the edge sizes (one camera, blocks of 1..16 unknowns, the
5,000-camera aerial pattern with c = 11).

Tolerances: products per component relative to the row's |S||x| - 1e-12
(FP64: the same products summed in another order) and, in FP32 (the oracle
given the FP32-rounded S and x), 1.5 (t + 2) 2^-24 for a component summed
from t products: the worst-case error of a t-term FP32 dot product;
solutions within 1e-8 (FP64, PCG to 1e-12) of the oracle's PCG iterate, iteration counts within one of the oracle's at the same tolerance;
bytes exactly Eq. 9 at the system's block sizes plus the row starts and
block sizes the format also keeps."""
import numpy as np
import pytest

import oracle as O
import oracle.interiors as I
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


def _packed(A):
    return np.concatenate([v.reshape(-1) for v in A.val])


def _from_packed(row_ptr, col, cdim, val):
    rows = np.repeat(np.arange(len(cdim)), np.diff(row_ptr))
    out, o = [], 0
    for k in range(len(col)):
        r, c = cdim[rows[k]], cdim[col[k]]
        out.append(val[o:o + r * c].reshape(r, c))
        o += r * c
    return I.VBSMC(np.asarray(row_ptr, dtype=np.int32), np.asarray(col, dtype=np.int32),
                   np.asarray(cdim, dtype=np.int32), out)


def _fp32_tol(A):
    """1.5 (t_e + 2) 2^-24 per vector entry e, t_e the products its row sums."""
    off = A.offsets()
    t = np.zeros(A.n)
    for i in range(A.n):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col[k]
            t[i] += A.cdim[j]
            if j != i:
                t[j] += A.cdim[i]
    return np.repeat(1.5 * (t + 2) * 2.0 ** -24, np.diff(off))


def vb_block_errors(row_ptr, col, cdim, val, A):
    """Per-block relative Frobenius error of packed values against the oracle's
    blocks, the denominator guarded against cancellation by
    1e-3 sqrt(||S_ii|| ||S_jj||) (as for the six-unknown RCS)."""
    got = _from_packed(row_ptr, col, cdim, val)
    dn = np.array([np.linalg.norm(A.val[A.row_ptr[i]]) for i in range(A.n)])
    errs = np.empty(len(col))
    for i in range(A.n):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col[k]
            den = max(np.linalg.norm(A.val[k]), 1e-3 * np.sqrt(dn[i] * dn[j]))
            errs[k] = np.linalg.norm(got.val[k] - A.val[k]) / den
    return errs


def _abs_product(A, x):
    return I.vbsmc_spmv(I.VBSMC(A.row_ptr, A.col, A.cdim, [np.abs(v) for v in A.val]), np.abs(x))


_SCENE = dict(n_along=8, n_across=5, pts_per_cam=40, seed=4601)


@pytest.fixture(scope="module", params=[0.0, 0.5, 1.0], ids=["c6", "mixed", "c11"])
def interior_case(request):
    s = scenes.aerial_small(**_SCENE)
    intr = scenes.interiors0(s.n_cams, seed=4602)
    cdim = scenes.block_sizes(s.n_cams, request.param, seed=4603)
    A, b = I.scene_rcs_vb(s, intr, cdim, 1e-3)
    return s, intr, cdim, A, b


@pytest.fixture(scope="module")
def interior_system(interior_case):
    return interior_case[3], interior_case[4]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_device_rcs_with_interiors_matches_oracle(B, interior_case, prec):
    """ba_vbsmc_create_interiors (e, J with five interiors; Eq. 3-4 with c_i
    unknowns, formed on the device) against the oracle's RCS of the same
    scene: the same pattern; FP64: values and b within 1e-11 of the largest
    |S| (the same sums in another order); FP32 (Jacobians and formation in
    FP32): the FP32 bar of the six-unknown RCS, 1e-4 per block (relative
    Frobenius, guarded denominators) and 2e-3 of the largest |b|; then the
    solve."""
    s, intr, cdim, A, b = interior_case
    fp64 = prec == "fp64"
    g = B.VBSMC.from_scene(s.cams0, intr, cdim, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, 1e-3,
                           precision=B.BA_FP64 if fp64 else B.BA_FP32)
    row_ptr, col, val, bg = g.system()
    assert np.array_equal(row_ptr, A.row_ptr) and np.array_equal(col, A.col)
    ref = _packed(A)
    scale = np.abs(ref).max()
    bs = np.abs(b).max()
    if fp64:
        assert np.all(np.abs(val - ref) <= 1e-11 * scale), np.abs(val - ref).max() / scale
        assert np.all(np.abs(bg - b) <= 1e-11 * bs), np.abs(bg - b).max() / bs
    else:
        errs = vb_block_errors(row_ptr, col, cdim, val, A)
        assert errs.max() <= 1e-4, errs.max()
        assert np.abs(bg - b).max() <= 2e-3 * bs, np.abs(bg - b).max() / bs
    if fp64:
        x, it, rel, _, _ = g.solve(1e-10)
        y = I.vb_pcg(A, b, 1e-10)
        assert abs(it - y.iters) <= 1
        assert np.linalg.norm(x - y.y) <= 1e-7 * np.linalg.norm(y.y)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_product_matches_oracle(B, interior_system, prec):
    import torch
    A, b = interior_system
    fp64 = prec == "fp64"
    g = B.VBSMC(A.cdim, A.row_ptr, A.col, _packed(A), b, precision=B.BA_FP64 if fp64 else B.BA_FP32)
    x = np.random.default_rng(1).standard_normal(len(b))
    dt = torch.float64 if fp64 else torch.float32
    if not fp64:
        x = x.astype(np.float32).astype(np.float64)
        A = I.VBSMC(A.row_ptr, A.col, A.cdim, [v.astype(np.float32).astype(np.float64) for v in A.val])
    xt = torch.tensor(x, dtype=dt, device="cuda")
    yt = torch.full_like(xt, float("nan"))
    g.spmv(xt, yt)
    torch.cuda.synchronize()
    y = yt.double().cpu().numpy()
    err = np.abs(y - I.vbsmc_spmv(A, x)) / _abs_product(A, x)
    tol = 1e-12 if fp64 else _fp32_tol(A)
    assert np.all(err <= tol), (err / tol).max()
    N, nbytes = g.info()
    assert N == len(b)
    assert nbytes == I.vbsmc_bytes(A, val_bytes=8 if fp64 else 4) + 4 + 4 * A.n
    g.close()


def test_pcg_follows_oracle(B, interior_system):
    A, b = interior_system
    g = B.VBSMC(A.cdim, A.row_ptr, A.col, _packed(A), b, precision=B.BA_FP64)
    for tol in (1e-3, 1e-6):
        x, it, rel, ms, _ = g.solve(tol)
        ref = I.vb_pcg(A, b, tol)
        assert abs(it - ref.iters) <= 1, (tol, it, ref.iters)
        assert rel <= tol and ms > 0
    x, it, rel, _, _ = g.solve(1e-12)
    ref = I.vb_pcg(A, b, 1e-12)
    assert np.linalg.norm(x - ref.y) <= 1e-8 * np.linalg.norm(ref.y)
    # the true residual, from the oracle's product
    assert np.linalg.norm(b - I.vbsmc_spmv(A, x)) <= 1e-10 * np.linalg.norm(b)
    g.close()


def test_fp32_pcg_reaches_its_tolerance(B, interior_system):
    A, b = interior_system
    g = B.VBSMC(A.cdim, A.row_ptr, A.col, _packed(A), b, precision=B.BA_FP32)
    x, it, rel, _, _ = g.solve(1e-4)
    ref = I.vb_pcg(A, b, 1e-4)
    assert rel <= 1e-4
    assert abs(it - ref.iters) <= max(3, 0.2 * ref.iters), (it, ref.iters)
    # the true residual, from the oracle's FP64 product: the FP32 rounding of
    # S moves it little from the recurrence's on these block-scaled systems
    assert np.linalg.norm(b - I.vbsmc_spmv(A, x)) <= 2e-4 * np.linalg.norm(b)
    g.close()


@pytest.mark.parametrize("case", ["one_camera", "sizes_1_to_16", "zero_b"])
def test_edge_systems(B, case):
    import torch
    rng = np.random.default_rng(4604)
    if case == "one_camera":
        cdim = np.array([11], dtype=np.int32)
        row_ptr, col = np.array([0, 1], dtype=np.int32), np.array([0], dtype=np.int32)
    else:
        s = scenes.tiny_scene(n_cams=12, n_pts=80, seed=4605)
        row_ptr, col = O.bsmc_pattern(s.obs_cam, s.obs_pt, s.n_cams, s.n_pts)
        cdim = rng.integers(1, B.BA_VB_CMAX + 1, s.n_cams).astype(np.int32)
        cdim[:2] = (1, B.BA_VB_CMAX)
    val, _ = scenes.random_block_spd(row_ptr, col, cdim, seed=4606)
    b = rng.standard_normal(int(cdim.sum())) if case != "zero_b" else np.zeros(int(cdim.sum()))
    A = _from_packed(row_ptr, col, cdim, val)
    g = B.VBSMC(cdim, row_ptr, col, val, b, precision=B.BA_FP64)
    x = rng.standard_normal(len(b))
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    g.spmv(xt, yt)
    torch.cuda.synchronize()
    err = np.abs(yt.cpu().numpy() - I.vbsmc_spmv(A, x)) / _abs_product(A, x)
    assert err.max() <= 1e-12
    y, it, rel, _, _ = g.solve(1e-12)
    if case == "zero_b":
        assert it == 0 and not np.any(y)
    else:
        ref = I.vb_pcg(A, b, 1e-12)
        assert abs(it - ref.iters) <= 1
        assert np.linalg.norm(y - ref.y) <= 1e-9 * np.linalg.norm(ref.y)
        if case == "one_camera":
            assert it == 1   # block-Jacobi inverts the only block
    g.close()


def test_errors_on_the_device(B):
    # a diagonal block that is not positive definite
    cdim = np.array([6, 11], dtype=np.int32)
    row_ptr, col = np.array([0, 2, 3], dtype=np.int32), np.array([0, 1, 1], dtype=np.int32)
    val, boff = scenes.random_block_spd(row_ptr, col, cdim, seed=4607)
    bad = val.copy()
    bad[boff[2]:boff[3]] *= -1.0
    with pytest.raises(B.BAError) as ei:
        B.VBSMC(cdim, row_ptr, col, bad, np.ones(17), precision=B.BA_FP64)
    assert ei.value.status == B.BA_ERR_NOT_SPD
    # an iteration cap below what the tolerance needs
    s = scenes.tiny_scene(n_cams=12, n_pts=80, seed=4608)
    row_ptr, col = O.bsmc_pattern(s.obs_cam, s.obs_pt, s.n_cams, s.n_pts)
    cdim = np.full(s.n_cams, 11, dtype=np.int32)
    val, _ = scenes.random_block_spd(row_ptr, col, cdim, seed=4609)
    g = B.VBSMC(cdim, row_ptr, col, val, np.ones(11 * s.n_cams), precision=B.BA_FP64)
    x, it, rel, _, st = g.solve(1e-14, max_iters=2, allow=(B.BA_ERR_NO_CONVERGENCE,))
    assert st == B.BA_ERR_NO_CONVERGENCE and it == 2 and rel > 1e-14
    with pytest.raises(B.BAError) as ei:
        g.solve(0.0)
    assert ei.value.status == B.BA_ERR_INVALID_ARG
    g.close()


def test_aerial_pattern_with_interiors(B):
    """The 5,000-camera aerial RCS pattern with c = 11 on every camera (the
    size the product is measured at), seeded SPD values: the whole product
    against the oracle's, and a solve to 1e-8 whose true residual the oracle
    checks."""
    import torch
    s = scenes.aerial_scene()
    g6 = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP32)
    g6.linearize()
    g6.form_rcs(1e-4)
    row_ptr, col, _, _ = g6.rcs()
    g6.close()
    n = len(row_ptr) - 1
    cdim = np.full(n, 11, dtype=np.int32)
    val, _ = scenes.random_block_spd(row_ptr, col, cdim, seed=4610)
    b = np.random.default_rng(4611).standard_normal(11 * n)
    A = _from_packed(row_ptr, col, cdim, val)
    for prec in ("fp64", "fp32"):
        fp64 = prec == "fp64"
        g = B.VBSMC(cdim, row_ptr, col, val, b, precision=B.BA_FP64 if fp64 else B.BA_FP32)
        x = np.random.default_rng(4612).standard_normal(11 * n)
        Ax = A
        if not fp64:
            x = x.astype(np.float32).astype(np.float64)
            Ax = I.VBSMC(A.row_ptr, A.col, A.cdim, [v.astype(np.float32).astype(np.float64) for v in A.val])
        xt = torch.tensor(x, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
        yt = torch.empty_like(xt)
        g.spmv(xt, yt)
        torch.cuda.synchronize()
        err = np.abs(yt.double().cpu().numpy() - I.vbsmc_spmv(Ax, x)) / _abs_product(Ax, x)
        tol = 1e-12 if fp64 else _fp32_tol(Ax)
        assert np.all(err <= tol), (prec, (err / tol).max())
        if fp64:
            y, it, rel, _, _ = g.solve(1e-8)
            assert rel <= 1e-8
            assert np.linalg.norm(b - I.vbsmc_spmv(A, y)) <= 2e-8 * np.linalg.norm(b)
        g.close()


def test_shared_interior_system(B):
    """Interiors shared by the images of a physical camera (three physical
    cameras over 40 images): image rows of 6 unknowns and physical-camera
    rows of 5, the latter coupled to every image they serve.  The oracle's
    system through ba_vbsmc_create: the product against the oracle's, and a
    solve whose true residual the oracle's product checks."""
    import torch
    s = scenes.aerial_small(n_along=8, n_across=5, pts_per_cam=40, seed=4620)
    phys = np.arange(s.n_cams) % 3
    intr = scenes.interiors0(3, seed=4621)
    A, b = I.scene_rcs_shared(s, intr, phys, 1e-3)
    g = B.VBSMC(A.cdim, A.row_ptr, A.col, _packed(A), b, precision=B.BA_FP64)
    x = np.random.default_rng(4622).standard_normal(len(b))
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    g.spmv(xt, yt)
    torch.cuda.synchronize()
    err = np.abs(yt.cpu().numpy() - I.vbsmc_spmv(A, x)) / _abs_product(A, x)
    assert err.max() <= 1e-12
    y, it, rel, _, _ = g.solve(1e-8)
    assert rel <= 1e-8
    assert np.linalg.norm(b - I.vbsmc_spmv(A, y)) <= 1e-6 * np.linalg.norm(b)
    g.close()
