"""GPU parity of y = S x in the three RCS storage formats (Sec. 4, Table 1,
Eqs. 8-10): the library's BSMC, block CSR of the full symmetric matrix,
scalar CSR and the implicit product from the stored linearization (no S),
each through its own kernels via ba_rcs_spmv, against the oracle's product
with the oracle's own S.

Tolerances: per component, relative to the row's |S||x| (the oracle's
product of absolute values): 1e-10 in FP64 mode, 2e-4 in FP32 mode (both
bounded by the per-block error allowed to the RCS itself); BSMC and full
BSR apply the same blocks in the same order, so they agree bit for bit; the
scalar CSR sums in another order (FP32: within 1e-5 of |S||x|).  Bytes: the
arrays each format holds, against Eqs. 8 and 9 of the oracle's memory model.
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


@pytest.fixture(scope="module")
def scene():
    return scenes.aerial_small(n_along=10, n_across=6, pts_per_cam=60, seed=4401)


def _oracle_rcs(s, lam):
    pb = O.Problem(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt, s.obs_uv)
    e, Jc, Jp = pb.linearize(s.cams0, s.pts0)
    _, A, _ = pb.rcs(e, Jc, Jp, lam)
    return A


def _products(B, g, x, dtype):
    import torch
    xt = torch.tensor(x, dtype=dtype, device="cuda")
    out, nbytes = {}, {}
    for name, fmt in (("bsmc", B.BA_FMT_BSMC), ("bsr", B.BA_FMT_BSR_FULL), ("csr", B.BA_FMT_CSR),
                      ("implicit", B.BA_FMT_IMPLICIT), ("bsmc_once", B.BA_FMT_BSMC_ONCE)):
        yt = torch.full_like(xt, float("nan"))
        nbytes[name] = g.rcs_spmv(fmt, xt, yt)
        torch.cuda.synchronize()
        out[name] = yt.double().cpu().numpy()
    return out, nbytes


@pytest.mark.parametrize("prec,tol,tol_csr", [("fp64", 1e-10, 1e-13), ("fp32", 2e-4, 1e-5)])
def test_formats_match_oracle_product(B, scene, prec, tol, tol_csr):
    import torch
    s = scene
    lam = 1e-3
    fp64 = prec == "fp64"
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP64 if fp64 else B.BA_FP32)
    g.linearize()
    g.form_rcs(lam)
    A = _oracle_rcs(s, lam)
    n = s.n_cams
    x = np.random.default_rng(7).standard_normal(6 * n)
    if not fp64:
        x = x.astype(np.float32).astype(np.float64)  # the FP32 path sees exactly these values
    y_ref = O.bsmc_spmv(A, x)
    mag = O.bsmc_spmv(O.BSMC(A.row_ptr, A.col, np.abs(A.val)), np.abs(x))
    out, nbytes = _products(B, g, x, torch.float64 if fp64 else torch.float32)
    for name, y in out.items():
        assert np.all(np.isfinite(y)), name
        err = np.abs(y - y_ref) / mag
        assert err.max() <= tol, (name, err.max())
    assert np.array_equal(out["bsmc"], out["bsr"])
    assert (np.abs(out["csr"] - out["bsmc"]) / mag).max() <= tol_csr
    # the implicit product forms U x - W V^-1 W^T x without S: other rounding
    assert (np.abs(out["implicit"] - out["bsmc"]) / mag).max() <= (1e-12 if fp64 else 5e-5)
    # BSMC read once: the same products, added with reductions in no fixed order
    assert (np.abs(out["bsmc_once"] - out["bsmc"]) / mag).max() <= (1e-13 if fp64 else 1e-5)

    # bytes of each format's arrays, against the memory model of Sec. 4.1
    nnzb = len(A.col)
    E = 2 * nnzb - n                      # non-zero blocks of the full matrix
    esz = 8 if fp64 else 4
    assert nbytes["bsmc"] == nnzb * 36 * esz + nnzb * 4 + (n + 1) * 4
    assert nbytes["bsmc_once"] == nbytes["bsmc"]
    assert nbytes["bsr"] == E * 36 * esz + E * 4 + (n + 1) * 4
    assert nbytes["csr"] == E * 36 * (esz + 4) + (6 * n + 1) * 4
    m, P = s.n_obs, s.n_pts
    assert nbytes["implicit"] == m * (20 + 12) * esz + P * 6 * esz + m * 4 * esz + (m + n + 1) * 4
    alpha = E / n ** 2                    # block density of the full matrix, as in Eq. 8
    # Eq. 8 (scalar CSR) counts n c row starts; the built array has one more
    assert nbytes["csr"] == pytest.approx(O.csr_bytes(alpha, n, 6, val_bytes=esz) + 4, rel=1e-12)
    # Eq. 9 (BSMC) keeps three ids per block (column, height, width); with
    # uniform 6x6 blocks only the column is stored, plus one more row start
    assert nbytes["bsmc"] == pytest.approx(O.bsmc_bytes(alpha, n, 6, val_bytes=esz) - nnzb * 8 + 4, rel=1e-12)


def test_formats_follow_a_new_rcs(B, scene):
    """The full-format copies are rebuilt when S changes (ba_form_rcs with
    another lambda; an RCS formed after an LM step)."""
    import torch
    s = scene
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP64)
    g.linearize()
    g.form_rcs(1e-3)
    x = np.random.default_rng(11).standard_normal(6 * s.n_cams)
    first, _ = _products(B, g, x, torch.float64)
    g.form_rcs(10.0)
    A = _oracle_rcs(s, 10.0)
    second, _ = _products(B, g, x, torch.float64)
    y_ref = O.bsmc_spmv(A, x)
    mag = O.bsmc_spmv(O.BSMC(A.row_ptr, A.col, np.abs(A.val)), np.abs(x))
    for name in ("bsmc", "bsr", "csr", "implicit"):
        assert not np.allclose(second[name], first[name])
        assert (np.abs(second[name] - y_ref) / mag).max() <= 1e-10, name
    # an accepted LM step moves the state (and drops the RCS); the next one
    # formed there is copied afresh
    info = g.lm_step()
    assert info["accepted"]
    with pytest.raises(B.BAError):
        _products(B, g, x, torch.float64)
    g.linearize()
    g.form_rcs(10.0)
    third, _ = _products(B, g, x, torch.float64)
    assert np.array_equal(third["bsmc"], third["bsr"])
    assert not np.array_equal(third["bsr"], second["bsr"])
    assert not np.array_equal(third["implicit"], second["implicit"])


def test_format_argument_and_state_errors(B, scene):
    import torch
    s = scene
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP64)
    x = torch.zeros(6 * s.n_cams, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(B.BAError) as ei:
        g.rcs_spmv(B.BA_FMT_BSMC, x, y)
    assert ei.value.status == B.BA_ERR_STATE
    g.linearize()
    g.form_rcs(1e-3)
    with pytest.raises(B.BAError) as ei:
        g.rcs_spmv(7, x, y)
    assert ei.value.status == B.BA_ERR_INVALID_ARG
    with pytest.raises(B.BAError) as ei:
        B.ba_rcs_spmv(g.h, B.BA_FMT_CSR, 0, y.data_ptr())
    assert ei.value.status == B.BA_ERR_INVALID_ARG
    # an RCS-only problem has no linearization for the implicit product
    row_ptr, col, val, b = g.rcs()
    r = B.Problem.from_rcs(row_ptr, col, val, b, precision=B.BA_FP64)
    r.rcs_spmv(B.BA_FMT_BSMC, x, y)
    with pytest.raises(B.BAError) as ei:
        r.rcs_spmv(B.BA_FMT_IMPLICIT, x, y)
    assert ei.value.status == B.BA_ERR_STATE
