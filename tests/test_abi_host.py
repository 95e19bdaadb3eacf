"""CPU-only tests of the C ABI: the library loads, exports what include/*.h
declares, validates inputs before touching the GPU, and its host-side
symbolic phase (BSMC pattern, Sec. 4) matches the oracle."""
import os
import re

import numpy as np
import pytest

import oracle as O
import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2307_08383_gb300.build import build
    build()
    import paper_2307_08383_gb300 as mod
    mod.lib()
    return mod


def _declared():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(B):
    names = _declared()
    assert len(names) >= 20
    L = B.lib()
    for n in names:
        assert hasattr(L, n), n
    bound = {s[0] for s in B.SIGNATURES}
    assert set(names) == bound


def test_kernel_names(B):
    names = B.ba_kernel_names()
    assert "form_rcs" in names and "pcg_loop" in names and "linearize" in names


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_host_pattern_matches_oracle(B, seed):
    s = scenes.shuffled(scenes.tiny_scene(n_cams=9, n_pts=80, seed=seed), seed)
    rp, cl = B.ba_symbolic_pattern(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt)
    rp2, cl2 = O.bsmc_pattern(s.obs_cam.astype(np.int64), s.obs_pt, s.n_cams, s.n_pts)
    assert np.array_equal(rp, rp2) and np.array_equal(cl, cl2)


def test_host_pattern_aerial(B):
    s = scenes.aerial_small(n_along=12, n_across=6, pts_per_cam=100, seed=5)
    rp, cl = B.ba_symbolic_pattern(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt)
    rp2, cl2 = O.bsmc_pattern(s.obs_cam.astype(np.int64), s.obs_pt, s.n_cams, s.n_pts)
    assert np.array_equal(rp, rp2) and np.array_equal(cl, cl2)


def _create(B, s, **kw):
    o = B.ba_options_default(**kw)
    return B.ba_problem_create(o, s["cams"], s["pts"], s["obs_cam"], s["obs_pt"], s["obs_uv"])


def _valid():
    sc = scenes.tiny_scene(n_cams=4, n_pts=10, seed=3)
    return dict(cams=sc.cams0.copy(), pts=sc.pts0.copy(), obs_cam=sc.obs_cam.copy(), obs_pt=sc.obs_pt.copy(),
                obs_uv=sc.obs_uv.copy())


@pytest.mark.parametrize("case", ["cam_range", "pt_range", "duplicate", "single_obs", "idle_camera", "nan_uv",
                                  "inf_cam", "bad_precision", "bad_delta", "bad_tol", "bad_pcg_variant"])
def test_create_rejects_bad_input_without_gpu(B, case):
    s = _valid()
    kw = {}
    want = B.BA_ERR_INVALID_ARG
    if case == "cam_range":
        s["obs_cam"][3] = 99
    elif case == "pt_range":
        s["obs_pt"][0] = -1
    elif case == "duplicate":
        k = s["obs_pt"][0]
        idx = np.nonzero(s["obs_pt"] == k)[0]
        s["obs_cam"][idx[1]] = s["obs_cam"][idx[0]]
    elif case == "single_obs":
        s["obs_pt"] = np.append(s["obs_pt"], len(s["pts"]))
        s["obs_cam"] = np.append(s["obs_cam"], 0).astype(np.int32)
        s["obs_uv"] = np.vstack([s["obs_uv"], [1.0, 2.0]])
        s["pts"] = np.vstack([s["pts"], [0.0, 0.0, 0.0]])
    elif case == "idle_camera":
        s["cams"] = np.vstack([s["cams"], s["cams"][:1]])
    elif case == "nan_uv":
        s["obs_uv"][2, 1] = np.nan
        want = B.BA_ERR_NONFINITE
    elif case == "inf_cam":
        s["cams"][1, 4] = np.inf
        want = B.BA_ERR_NONFINITE
    elif case == "bad_precision":
        kw["precision"] = 7
    elif case == "bad_delta":
        kw["robust"] = B.BA_LOSS_HUBER
        kw["huber_delta"] = -1.0
    elif case == "bad_tol":
        kw["pcg_rel_tol"] = 0.0
    elif case == "bad_pcg_variant":
        kw["pcg_variant"] = 4
    with pytest.raises(B.BAError) as ei:
        _create(B, s, **kw)
    assert ei.value.status == want


def test_memory_cap_is_checked_before_allocation(B):
    s = _valid()
    with pytest.raises(B.BAError) as ei:
        _create(B, s, device_mem_cap=1024)
    assert ei.value.status == B.BA_ERR_OOM


def test_null_problem_calls_fail_cleanly(B):
    assert B.lib().ba_linearize(None, None) == B.BA_ERR_INVALID_ARG
    assert B.lib().ba_lm_step(None, None) == B.BA_ERR_INVALID_ARG
    assert B.lib().ba_rcs_spmv(None, B.BA_FMT_BSMC, None, None, None) == B.BA_ERR_INVALID_ARG
    assert B.lib().ba_triangulate(None, 3, None, None) == B.BA_ERR_INVALID_ARG
    B.lib().ba_problem_destroy(None)


@pytest.mark.parametrize("case", ["no_diag_first", "descending", "col_range", "row_ptr_end", "nan"])
def test_create_rcs_rejects_malformed_input_without_gpu(B, case):
    row_ptr = np.array([0, 2, 3], np.int32)
    col = np.array([0, 1, 1], np.int32)
    val = np.tile(np.eye(6).reshape(1, 36), (3, 1))
    b = np.ones((2, 6))
    want = B.BA_ERR_INVALID_ARG
    if case == "no_diag_first":
        col = np.array([1, 0, 1], np.int32)
    elif case == "descending":
        row_ptr = np.array([0, 3, 4], np.int32)
        col = np.array([0, 1, 1, 1], np.int32)
        val = np.tile(np.eye(6).reshape(1, 36), (4, 1))
    elif case == "col_range":
        col = np.array([0, 5, 1], np.int32)
    elif case == "row_ptr_end":
        row_ptr = np.array([0, 2, 2], np.int32)
    elif case == "nan":
        val = val.copy()
        val[1, 3] = np.nan
        want = B.BA_ERR_NONFINITE
    o = B.ba_options_default()
    with pytest.raises(B.BAError) as ei:
        B.ba_problem_create_rcs(o, row_ptr, col, val, b)
    assert ei.value.status == want


def _vb_valid():
    cdim = np.array([6, 11, 2], dtype=np.int32)
    row_ptr = np.array([0, 2, 4, 5], dtype=np.int32)
    col = np.array([0, 2, 1, 2, 2], dtype=np.int32)
    val, _ = scenes.random_block_spd(row_ptr, col, cdim, seed=1)
    return dict(cdim=cdim, row_ptr=row_ptr, col=col, val=val, b=np.ones(int(cdim.sum())))


@pytest.mark.parametrize("case", ["c_zero", "c_too_big", "no_diagonal", "unsorted", "col_range", "row_ptr_end",
                                  "nan_val", "inf_b", "bad_precision"])
def test_vbsmc_create_rejects_bad_input_without_gpu(B, case):
    s = _vb_valid()
    kw = {}
    want = B.BA_ERR_INVALID_ARG
    if case == "c_zero":
        s["cdim"][2] = 0
        s["val"] = s["val"][:36 + 11 * 11]       # blocks (0,0), (1,1) keep their sizes
        s["b"] = s["b"][:17]
    elif case == "c_too_big":
        s["cdim"][1] = B.BA_VB_CMAX + 1
        s["val"] = np.ones(36 + 12 + 17 * 17 + 17 * 2 + 4)
        s["b"] = np.ones(6 + 17 + 2)
    elif case == "no_diagonal":
        s["col"][2], s["col"][3] = 2, 1          # row 1 starts with column 2
    elif case == "unsorted":
        s["row_ptr"] = np.array([0, 2, 3, 5], dtype=np.int32)
        s["col"] = np.array([0, 2, 1, 2, 1], dtype=np.int32)
    elif case == "col_range":
        s["col"][1] = 3
    elif case == "row_ptr_end":
        s["row_ptr"][3] = 4
    elif case == "nan_val":
        s["val"][40] = np.nan
        want = B.BA_ERR_NONFINITE
    elif case == "inf_b":
        s["b"][3] = np.inf
        want = B.BA_ERR_NONFINITE
    elif case == "bad_precision":
        kw["precision"] = 3
    with pytest.raises(B.BAError) as ei:
        B.VBSMC(s["cdim"], s["row_ptr"], s["col"], s["val"], s["b"], stream=None, **kw)
    assert ei.value.status == want


@pytest.mark.parametrize("case", ["cdim_7", "neg_lambda", "nan_intr", "cam_range", "single_obs"])
def test_vbsmc_interiors_rejects_bad_input_without_gpu(B, case):
    s = _valid()
    n = len(s["cams"])
    intr = np.tile([1000.0, 500.0, 500.0, 0.0, 0.0], (n, 1))
    cdim = np.full(n, 11, dtype=np.int32)
    lam = 1e-3
    want = B.BA_ERR_INVALID_ARG
    if case == "cdim_7":
        cdim[1] = 7
    elif case == "neg_lambda":
        lam = -1.0
    elif case == "nan_intr":
        intr[2, 3] = np.nan
        want = B.BA_ERR_NONFINITE
    elif case == "cam_range":
        s["obs_cam"][0] = n
    elif case == "single_obs":
        s["obs_pt"] = np.append(s["obs_pt"], len(s["pts"]))
        s["obs_cam"] = np.append(s["obs_cam"], 0).astype(np.int32)
        s["obs_uv"] = np.vstack([s["obs_uv"], [1.0, 2.0]])
        s["pts"] = np.vstack([s["pts"], [0.0, 0.0, 5.0]])
    with pytest.raises(B.BAError) as ei:
        B.VBSMC.from_scene(s["cams"], intr, cdim, s["pts"], s["obs_cam"], s["obs_pt"], s["obs_uv"], lam, stream=None)
    assert ei.value.status == want
