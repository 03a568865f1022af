"""Many camera clusters at once: a tile step of the factorisation then has more panel CTAs than the GPU
holds at a time, so CTAs of one step run in several waves (the 1000-camera scene fits one wave).  Every
cluster's step is checked against a dense solve of the cluster system the device built (a property that
holds at any size): dc_k = S'_k^-1 b'_k, camera by camera.  (tests/test_gpu_full_size.py compares the same
scene's step with the oracle.)  Tolerances per camera row: FP64 1e-6, the FP64 step bar (measured 6e-8:
both sides are FP64 solves of a system whose gauge directions are damped only by lambda = 1e-4, so the rows
of cameras with small steps carry kappa eps_64 of the large ones); mixed 1e-5 (FP32 factor, one FP64
refinement step: (kappa eps_32)^2 ~ 1e-7 after Jacobi scaling)."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2008_00446_gb300 import stba  # noqa: E402
from elementwise import rows  # noqa: E402


def scene():
    return scenes.make_hemisphere_scene(m=4000, n=40_000, radius=40.0, half=10.0, lmax=30, max_cluster=100,
                                        seed=77, name="many")


@pytest.mark.parametrize("precision,tol,tile,panel", [(stba.STBA_FP64, 1e-6, 0, 0), (stba.STBA_MIXED, 1e-5, 0, 0),
                                                      (stba.STBA_MIXED, 1e-5, 32, 0),
                                                      (stba.STBA_MIXED, 1e-5, 64, stba.STBA_FACTOR_PANEL_PERSISTENT)])
def test_every_cluster_step_solves_its_system(precision, tol, tile, panel):
    s = scene()
    l = int(s.clusters.max()) + 1
    assert l >= 40
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, precision=precision,
                           factor_tile=tile, factor_panel=panel)
    info = stba.stba_lm_iteration(ctx)
    assert info["failed_clusters"] == 0
    dc, _ = stba.stba_last_step(ctx)
    assert np.isfinite(dc).all()
    errs = []
    for k in range(l):
        S, b = stba.stba_get_cluster_system(ctx, k)
        cams = np.nonzero(s.clusters == k)[0]
        x = np.linalg.solve(S, b)
        errs.append(rows(dc[cams].ravel(), x, 9))
    assert max(errs) < tol, max(errs)
    ctx.close()


@pytest.mark.parametrize("precision", [stba.STBA_FP64, stba.STBA_MIXED])
def test_a_cluster_too_large_for_the_solve_is_refused(precision):
    # the cluster solve holds a cluster's vector in shared memory: one cluster of 4000 cameras (36000
    # unknowns) exceeds it in both precisions and is refused at create, and by stba_set_clusters on a
    # context whose clusters fit; nothing is allocated for the dense systems first
    rng = np.random.default_rng(5)
    m, n = 4000, 4000
    cams = np.zeros((m, 9))
    cams[:, 5] = 10.0                                  # every camera 10 units in front of the points
    cams[:, 6] = 500.0
    pts = rng.uniform(-1.0, 1.0, size=(n, 3))
    oc = np.stack([np.arange(n), (np.arange(n) + 1) % m], axis=1).ravel().astype(np.int32)
    op = np.repeat(np.arange(n), 2).astype(np.int32)
    uv = rng.normal(0.0, 1.0, size=(2 * n, 2))
    with pytest.raises(stba.StbaError, match="shared memory"):
        stba.stba_create(cams, pts, oc, op, uv, np.zeros(m, np.int32), precision=precision)
    ctx = stba.stba_create(cams, pts, oc, op, uv, (np.arange(m) // 100).astype(np.int32), precision=precision)
    F0 = stba.stba_cost(ctx)
    with pytest.raises(stba.StbaError, match="shared memory"):
        stba.stba_set_clusters(ctx, np.zeros(m, np.int32))
    info = stba.stba_lm_iteration(ctx)   # the previous assignment (40 clusters) stays in force
    assert info["failed_clusters"] == 0 and info["F_before"] == F0 and np.isfinite(info["F_after"])


@pytest.mark.parametrize("precision", [stba.STBA_FP64, stba.STBA_MIXED])
def test_two_live_contexts_with_different_cluster_sizes(precision):
    # the largest dynamic shared memory of the panel and solve kernels is a per-function attribute; a context
    # created later with smaller clusters must not lower it below what the earlier one's launches ask for
    s = scenes.make_config("c0_ring")
    big = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, np.zeros(s.m, np.int32),
                           precision=precision)
    t = scenes.make_tiny_scene(m=6, n=50, seed=7)
    small = stba.stba_create(t.cameras, t.points, t.obs_cam, t.obs_pt, t.obs_uv, np.arange(6, dtype=np.int32),
                             precision=precision)
    for _ in range(2):
        ia = stba.stba_lm_iteration(big)
        ib = stba.stba_lm_iteration(small)
        assert ia["failed_clusters"] == 0 and ib["failed_clusters"] == 0
        assert np.isfinite(ia["F_after"]) and np.isfinite(ib["F_after"])
    big.close()
    small.close()
