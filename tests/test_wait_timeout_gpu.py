"""The bounded device waits, made to run out on purpose.

Every grid-wide wait in the PCG kernels gives up after a limit of SM clock
cycles, sets an error word and leaves its kernel.  ba_debug_arm_wait_timeout
starts the next PCG launch's all-reduce counters one arrival short (so no CTA
ever sees every arrival) with a wait limit of about a millisecond: no fault,
no trap and no unbounded wait is involved.  The tests check that the status
reaches the host as BA_ERR_TIMEOUT, that the problem is then refused with
BA_ERR_STATE, and that the CUDA context still serves a fresh problem, whose
solve matches an untouched one.
"""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

LIMIT = 2_000_000  # SM cycles, about 1 ms at 2 GHz


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available()
    from paper_2307_08383_gb300.build import build
    build()
    import paper_2307_08383_gb300 as mod
    return mod


def _formed(B, s, **kw):
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, **kw)
    g.linearize()
    g.form_rcs(1e-3)
    return g


@pytest.mark.parametrize("prec,variant", [("fp32", "split"), ("fp32", "standard"), ("fp64", "standard")])
def test_pcg_wait_runs_out_and_reports_timeout(B, prec, variant):
    import torch

    s = scenes.ring_scene(n_cams=16, n_pts=500, seed=71)
    kw = dict(precision=B.BA_FP32 if prec == "fp32" else B.BA_FP64, pcg_rel_tol=1e-6,
              pcg_variant=B.BA_PCG_SPLIT if variant == "split" else B.BA_PCG_STANDARD)
    ref = _formed(B, s, **kw)
    ref.solve_rcs()
    dx_ref, _ = ref.step()

    g = _formed(B, s, **kw)
    g.arm_wait_timeout(LIMIT)
    with pytest.raises(B.BAError) as ei:
        g.solve_rcs()
    assert ei.value.status == B.BA_ERR_TIMEOUT
    # the problem is unusable afterwards, as documented
    with pytest.raises(B.BAError) as ei:
        g.form_rcs(1e-3)
    assert ei.value.status == B.BA_ERR_STATE
    g.close()
    torch.cuda.synchronize()  # the context answers: no kernel is left waiting

    # a fresh problem on the same context solves normally, to the same result
    h = _formed(B, s, **kw)
    info, conv = h.solve_rcs()
    assert conv
    dx, _ = h.step()
    assert np.array_equal(dx, dx_ref)
    h.close()


def test_arming_is_validated(B):
    s = scenes.ring_scene(n_cams=6, n_pts=60, seed=72)
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv)
    for bad in (0, -5, 10 ** 10):
        with pytest.raises(B.BAError) as ei:
            g.arm_wait_timeout(bad)
        assert ei.value.status == B.BA_ERR_INVALID_ARG
    g.close()


def test_profile_switch(B):
    """Kernel timers switched on a live problem: none counted while off,
    the launches of a step counted once on; levels outside 0..2 refused."""
    s = scenes.ring_scene(n_cams=6, n_pts=60, seed=73)
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, profile=0)
    g.lm_step()
    assert sum(v[0] for v in g.kernel_times().values()) == 0
    g.set_profile(1)
    g.lm_step()
    assert g.kernel_times()["form_rcs"][0] == 1
    for bad in (-1, 3):
        with pytest.raises(B.BAError) as ei:
            g.set_profile(bad)
        assert ei.value.status == B.BA_ERR_INVALID_ARG
    g.close()
