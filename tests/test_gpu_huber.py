"""The Huber loss option (Sec. 5.1, huber_a) through the C ABI against the oracle, on scenes with gross
outliers so that both branches of the loss are active.  FP64: the cluster systems, steps and costs agree
with the oracle to the FP64 bars of the plain objective (S'_k 1e-8, steps 1e-6, F 1e-8); the accept /
lambda sequence is identical.  Mixed precision: first step 1e-3, robust cost after ten iterations within
0.1 %.  The full-RCS comparator takes the same weights."""
import numpy as np
import pytest

import scenes
from oracle import stba as ostba

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2008_00446_gb300 import stba  # noqa: E402

A = 0.5

from elementwise import blocks, cols, rows  # noqa: E402


def outlier_scene(m=9, n=90, seed=8, clusters=None):
    s = scenes.make_tiny_scene(m=m, n=n, seed=seed, clusters=clusters)
    uv = s.obs_uv.copy()
    rng = np.random.default_rng(seed)
    bad = rng.choice(len(uv), size=max(3, len(uv) // 20), replace=False)
    uv[bad] += rng.normal(0.0, 30.0, size=(len(bad), 2))
    return s, uv


@pytest.mark.parametrize("lam", [1e-4, 0.5])
def test_first_step_fp64(lam):
    cl = np.array([2, 0, 1, 2, 0, 1, 2, 0, 1], np.int32)
    s, uv = outlier_scene(clusters=cl)
    F0 = ostba.robust_cost(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, A)
    opt = ostba.Options(lambda0=lam, huber=A)
    c2, p2, lam2, F2, rec = ostba.lm_iteration(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, cl, lam, F0, opt,
                                               keep=True)
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, cl, precision=stba.STBA_FP64,
                           lambda0=lam, huber_a=A)
    F_dev = stba.stba_cost(ctx)
    assert abs(F_dev - F0) <= 1e-12 * F0
    info = stba.stba_lm_iteration(ctx)
    st = rec["step"]
    for k in range(3):
        S, b = stba.stba_get_cluster_system(ctx, k)
        assert blocks(S, st["S_blocks"][k]) < 1e-8, blocks(S, st["S_blocks"][k])
        assert rows(b, st["b_blocks"][k], 9) < 1e-8, rows(b, st["b_blocks"][k], 9)
    dc, dp = stba.stba_last_step(ctx)
    assert rows(dc, rec["dc"], 9) < 1e-6 and rows(dp, rec["dp"], 3) < 1e-6
    assert info["accepted"] == rec["accepted"]
    assert abs(info["F_after"] - rec["F_after"]) <= 1e-8 * rec["F_after"]


def test_iterations_fp64_and_mixed():
    s = scenes.make_config("c0_ring")
    uv = s.obs_uv.copy()
    rng = np.random.default_rng(1)
    bad = rng.choice(len(uv), size=len(uv) // 50, replace=False)
    uv[bad] += rng.normal(0.0, 30.0, size=(len(bad), 2))
    c, p, lam, F, hist = ostba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, s.clusters, 10,
                                     ostba.Options(huber=A))
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, s.clusters, precision=stba.STBA_FP64,
                           huber_a=A)
    for rec in hist:
        info = stba.stba_lm_iteration(ctx)
        assert info["accepted"] == rec["accepted"]
        assert abs(info["F_after"] - rec["F_after"]) <= 1e-8 * rec["F_after"]
    cams, pts = stba.stba_get_params(ctx)
    assert rows(cams, c, 9) < 1e-8 and rows(pts, p, 3) < 1e-8
    mx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, s.clusters, precision=stba.STBA_MIXED,
                          huber_a=A)
    stba.stba_lm_iteration(mx)
    dc, dp = stba.stba_last_step(mx)
    assert cols(dc, hist[0]["dc"], 9) < 1e-3 and cols(dp, hist[0]["dp"], 3) < 1e-3
    for _ in range(9):
        stba.stba_lm_iteration(mx)
    _, Fm, _ = stba.stba_get_state(mx)
    assert abs(Fm - F) <= 1e-3 * F


def test_full_rcs_comparator_fp64():
    s, uv = outlier_scene(m=8, n=80, seed=5)
    F0 = ostba.robust_cost(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, A)
    c2, p2, lam2, F2, rec = ostba.lm_iteration(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, s.clusters, 1e-4, F0,
                                               ostba.Options(huber=A), method="lm")
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, s.clusters, huber_a=A,
                           linear_solver=stba.STBA_SOLVER_PCG_FULL, pcg_tol=1e-12, pcg_max_iter=1000)
    info = stba.stba_lm_iteration(ctx)
    dc, dp = stba.stba_last_step(ctx)
    assert rows(dc, rec["dc"], 9) < 1e-7 and rows(dp, rec["dp"], 3) < 1e-7
    assert abs(info["F_after"] - rec["F_after"]) <= 1e-7 * rec["F_after"]


def test_adjoint_refuses_the_robust_loss():
    s, uv = outlier_scene(m=6, n=50, seed=7)
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, s.clusters, huber_a=A)
    stba.stba_record(ctx, 2)
    stba.stba_lm_iteration(ctx)
    with pytest.raises(stba.StbaError):
        stba.stba_adjoint(ctx, np.zeros((s.m, 9)))
