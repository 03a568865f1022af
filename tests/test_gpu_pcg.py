"""The full-RCS comparator (STBA_SOLVER_PCG_FULL): plain LM whose camera step solves the full reduced camera
system of all cameras (Eq. 5) by block-Jacobi preconditioned CG, against the oracle's full-RCS LM
(method="lm", a direct solve).  FP64 with pcg_tol = 1e-12: the CG solution equals the direct one up to
the stopping residual amplified by cond(S) (~1e4 after scaling), so steps agree to 1e-7.  Mixed precision
(FP32 Jacobians in the matrix-free products, pcg_tol = 1e-6): ten iterations on the 30-camera ring reach the
oracle's final RMSE within 0.1 %, the bar of the mixed mode."""
import numpy as np
import pytest

import scenes
from oracle import camera as ocam
from oracle import stba as ostba

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2008_00446_gb300 import stba  # noqa: E402

from elementwise import rows  # noqa: E402


@pytest.mark.parametrize("lam", [1e-4, 0.5])
def test_pcg_first_step_fp64_matches_direct_full_rcs(lam):
    s = scenes.make_tiny_scene(m=8, n=80, seed=5)
    F0 = ocam.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
    c2, p2, lam2, F2, rec = ostba.lm_iteration(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, lam,
                                               F0, ostba.Options(lambda0=lam), method="lm")
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, lambda0=lam,
                           linear_solver=stba.STBA_SOLVER_PCG_FULL, pcg_tol=1e-12, pcg_max_iter=1000)
    info = stba.stba_lm_iteration(ctx)
    dc, dp = stba.stba_last_step(ctx)
    assert rows(dc, rec["dc"], 9) < 1e-7, rows(dc, rec["dc"], 9)
    assert rows(dp, rec["dp"], 3) < 1e-7, rows(dp, rec["dp"], 3)
    assert info["accepted"] == rec["accepted"]
    assert 0 < info["linear_iterations"] <= 1000
    assert abs(info["F_after"] - rec["F_after"]) <= 1e-7 * rec["F_after"]
    with pytest.raises(stba.StbaError):
        stba.stba_get_cluster_system(ctx, 0)
    ctx.close()


def test_pcg_lm_mixed_reaches_oracle_rmse_on_ring():
    s = scenes.make_config("c0_ring")
    iters = 10
    co, po, lam, F, hist = ostba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, iters,
                                       method="lm")
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED, linear_solver=stba.STBA_SOLVER_PCG_FULL)
    for _ in range(iters):
        stba.stba_lm_iteration(ctx)
    F_gpu = stba.stba_cost(ctx)
    rm_o, rm_g = np.sqrt(F / (2 * s.q)), np.sqrt(F_gpu / (2 * s.q))
    assert abs(rm_g - rm_o) <= 1e-3 * rm_o, (rm_g, rm_o)
    ctx.close()


def test_pcg_equals_cluster_solver_with_one_cluster_fp64():
    """With a single cluster the method's step is exactly the full-RCS LM step (Sec. 4), so the dense
    cluster solve and the PCG solve of the same system agree."""
    s = scenes.make_tiny_scene(m=7, n=60, seed=6)
    one = np.zeros(s.m, np.int32)
    a = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, one)
    b = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, one,
                         linear_solver=stba.STBA_SOLVER_PCG_FULL, pcg_tol=1e-12, pcg_max_iter=1000)
    stba.stba_lm_iteration(a)
    stba.stba_lm_iteration(b)
    dca, _ = stba.stba_last_step(a)
    dcb, _ = stba.stba_last_step(b)
    assert rows(dcb, dca, 9) < 1e-7
    a.close()
    b.close()


# The method's split system by PCG (STBA_SOLVER_PCG_CLUSTERS): the same STBA step as the cluster
# factorisations, reached by conjugate gradients over the virtual points.  FP64 with pcg_tol = 1e-12: the
# step equals the oracle's STBA step (direct per-cluster solves) to 1e-7, with and without the correction;
# mixed precision: ten iterations on the ring reach the oracle's RMSE within 0.1 %.
@pytest.mark.parametrize("lam", [1e-4, 0.5])
def test_split_pcg_first_step_fp64_matches_the_stba_step(lam):
    cl = np.array([0, 0, 0, 1, 1, 1, 2, 2], np.int32)
    s = scenes.make_tiny_scene(m=8, n=80, seed=5, clusters=cl)
    F0 = ocam.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
    c2, p2, lam2, F2, rec = ostba.lm_iteration(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, cl, lam, F0,
                                               ostba.Options(lambda0=lam))
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, cl, lambda0=lam,
                           linear_solver=stba.STBA_SOLVER_PCG_CLUSTERS, pcg_tol=1e-12, pcg_max_iter=1000)
    info = stba.stba_lm_iteration(ctx)
    assert info["corrected"] == rec["corrected"] == (lam >= 0.1)
    dc, dp = stba.stba_last_step(ctx)
    assert rows(dc, rec["dc"], 9) < 1e-7, rows(dc, rec["dc"], 9)
    assert rows(dp, rec["dp"], 3) < 1e-7, rows(dp, rec["dp"], 3)
    assert info["accepted"] == rec["accepted"]
    assert 0 < info["linear_iterations"] <= 1000
    assert abs(info["F_after"] - rec["F_after"]) <= 1e-7 * rec["F_after"]
    with pytest.raises(stba.StbaError):
        stba.stba_get_cluster_system(ctx, 0)


def test_split_pcg_mixed_reaches_oracle_rmse_on_ring():
    s = scenes.make_config("c0_ring")
    c, p, lam, F, hist = ostba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, 10,
                                     ostba.Options())
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED, linear_solver=stba.STBA_SOLVER_PCG_CLUSTERS)
    for _ in range(10):
        stba.stba_lm_iteration(ctx)
    _, Fg, _ = stba.stba_get_state(ctx)
    assert abs(ostba.rmse(Fg, s.q) - ostba.rmse(F, s.q)) <= 1e-3 * ostba.rmse(F, s.q)
    stba.stba_record(ctx, 1)
    stba.stba_lm_iteration(ctx)
    with pytest.raises(stba.StbaError):
        stba.stba_adjoint(ctx, np.zeros((s.m, 9)))
