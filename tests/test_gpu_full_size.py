"""Oracle parity at the sizes the kernels take in the benchmark, element-wise (tests/elementwise.py).

Scenes:
  - the 500-camera differentiable configuration (50k points, 276k observations, 5 azimuth clusters of 100
    cameras): 900 unknowns per cluster, i.e. 15 factor tiles of 64 in mixed mode and 29 of 32 in FP64, the
    tile counts of the 1000-camera benchmark's clusters;
  - a 4000-camera hemisphere scene with 40 clusters of 100 cameras: every tile step of the factorisation then
    has more CTAs than the GPU holds at once, so each step runs in several waves.
Bars: FP64 mode, steps and parameters 1e-6 per camera / point row, cluster systems 1e-8 per 9 x 9 block and
per camera row of b', F(x + dx) 1e-8; mixed mode, every element of the first step within 1e-3 of its
parameter kind's largest reference value (elementwise.cols) and the RMSE after five
iterations within 0.1 % of the oracle's.  Both lambda = 1e-4 and lambda = 0.5 (the steepest-descent correction, Sec. 4.3)
are compared in FP64.  The mixed-mode bar holds with margin because every FP32 pass that forms V_v and S' takes
the Jacobian rows with each operation rounded on its own (measured <= 1.9e-4 on dc, 3.8e-4 on dp, the same
whether G_o is stored or recomputed)."""
import numpy as np
import pytest

import scenes
from oracle import camera as ocam
from oracle import stba as ostba

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2008_00446_gb300 import stba  # noqa: E402
from elementwise import blocks, cols, rows  # noqa: E402


def many_clusters_scene():
    return scenes.make_hemisphere_scene(m=4000, n=40_000, radius=40.0, half=10.0, lmax=30, max_cluster=100,
                                        seed=77, name="many")


SCENES = {"c3_diff": lambda: scenes.make_config("c3_diff"), "many_clusters": many_clusters_scene}
_cache = {}


def scene(name):
    if name not in _cache:
        _cache[name] = SCENES[name]()
    return _cache[name]


def oracle_first(s, lam):
    F0 = ocam.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
    return ostba.lm_iteration(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, lam, F0,
                              ostba.Options(lambda0=lam), keep=True)


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("lam,cs,pairs", [(1e-4, 0, 0), (0.5, 0, 0), (1e-4, 2, 0), (1e-4, 0, 1)])
def test_first_step_fp64_elementwise(name, lam, cs, pairs):
    # cs: CTAs per thread-block cluster of the cluster solves (0 = the default 8); pairs = 1: the pair pass
    # reads the camera pass's stored G_o instead of recomputing them (the default)
    s = scene(name)
    l = int(s.clusters.max()) + 1
    c2, p2, _, _, rec = oracle_first(s, lam)
    st = rec["step"]
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, precision=stba.STBA_FP64,
                           lambda0=lam, solve_cluster=cs, pair_blocks=pairs)
    info = stba.stba_lm_iteration(ctx)
    assert info["failed_clusters"] == 0
    assert info["corrected"] == rec["corrected"] == (lam >= 0.1)
    errS, errb = [], []
    for k in range(l):
        S, b = stba.stba_get_cluster_system(ctx, k)
        errS.append(blocks(S, st["S_blocks"][k]))
        errb.append(rows(b, st["b_blocks"][k], 9))
    assert max(errS) < 1e-8 and max(errb) < 1e-8, (max(errS), max(errb))
    dc, dp = stba.stba_last_step(ctx)
    e_c, e_p = rows(dc, rec["dc"], 9), rows(dp, rec["dp"], 3)
    print(f"{name} lambda {lam}: S {max(errS):.2e} b {max(errb):.2e} dc {e_c:.2e} dp {e_p:.2e}")
    assert e_c < 1e-6 and e_p < 1e-6, (e_c, e_p)
    assert info["accepted"] == rec["accepted"]
    assert abs(info["F_after"] - rec["F_after"]) <= 1e-8 * rec["F_after"]
    cams, pts = stba.stba_get_params(ctx)
    assert rows(cams, c2, 9) < 1e-8 and rows(pts, p2, 3) < 1e-8
    ctx.close()


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("panel,pairs", [(stba.STBA_FACTOR_PANEL_STACKED, 0), (stba.STBA_FACTOR_PANEL_SPLIT, 0),
                                         (stba.STBA_FACTOR_PANEL_PERSISTENT, 0), (stba.STBA_FACTOR_PANEL_DEFAULT, 1),
                                         (stba.STBA_FACTOR_PANEL_DEFAULT, 2)])
def test_mixed_first_step_elementwise(name, panel, pairs):
    # every panel of the FP32 factor (the default picks one by the number of tiles per step), and both ways of
    # forming the off-diagonal blocks (pairs: 1 = stored G_o, 2 = recomputed, the default; both from the
    # Jacobian rows with strict FP32 rounding)
    s = scene(name)
    _, _, _, _, rec = oracle_first(s, 1e-4)
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED, factor_panel=panel, pair_blocks=pairs)
    info = stba.stba_lm_iteration(ctx)
    assert info["failed_clusters"] == 0
    dc, dp = stba.stba_last_step(ctx)
    e_c, e_p = cols(dc, rec["dc"], 9), cols(dp, rec["dp"], 3)
    print(f"{name} mixed panel {panel} pairs {pairs}: dc {e_c:.2e} dp {e_p:.2e}")
    assert e_c < 1e-3 and e_p < 1e-3, (e_c, e_p)
    assert info["accepted"] == rec["accepted"]
    ctx.close()


@pytest.mark.parametrize("name", list(SCENES))
def test_mixed_fp64_factor_first_step_elementwise(name):
    # FP32 Jacobians and Schur terms, the cluster systems factored in FP64 (option factor_fp64)
    s = scene(name)
    _, _, _, _, rec = oracle_first(s, 1e-4)
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED, factor_fp64=1)
    info = stba.stba_lm_iteration(ctx)
    assert info["failed_clusters"] == 0 and info["boosted_pivots"] == 0
    dc, dp = stba.stba_last_step(ctx)
    e_c, e_p = cols(dc, rec["dc"], 9), cols(dp, rec["dp"], 3)
    print(f"{name} mixed, FP64 factor: dc {e_c:.2e} dp {e_p:.2e}")
    assert e_c < 1e-3 and e_p < 1e-3, (e_c, e_p)
    assert info["accepted"] == rec["accepted"]
    ctx.close()


@pytest.mark.parametrize("pairs", [0, 1])
def test_mixed_rmse_after_five_iterations_c3(pairs):
    s = scene("c3_diff")
    _, _, _, F, hist = ostba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, 5,
                                   ostba.Options())
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED, pair_blocks=pairs)
    for rec in hist:
        info = stba.stba_lm_iteration(ctx)
        assert info["accepted"] == rec["accepted"]
    _, Fg, _ = stba.stba_get_state(ctx)
    rm_o, rm_g = ostba.rmse(F, s.q), ostba.rmse(Fg, s.q)
    print(f"c3 mixed RMSE after 5: device {rm_g:.6f} oracle {rm_o:.6f}")
    assert abs(rm_g - rm_o) <= 1e-3 * rm_o, (rm_g, rm_o)
    ctx.close()
