"""The factorisation tile as a runtime choice and the autotuner that picks it.  Both FP32 tiles give the
mixed-precision bar against the oracle on the 30-camera ring (first step 1e-3, RMSE after ten iterations
within 0.1 %); stba_autotune leaves the parameters, damping and cost as it found them and keeps a tile
whose next iteration agrees with a context created with that tile (to the mixed-mode bar)."""
import numpy as np
import pytest

import scenes
from oracle import stba as ostba

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2008_00446_gb300 import stba  # noqa: E402

from elementwise import cols  # noqa: E402


@pytest.fixture(scope="module")
def ring():
    s = scenes.make_config("c0_ring")
    c, p, lam, F, hist = ostba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, 10,
                                     ostba.Options())
    return s, F, hist


@pytest.mark.parametrize("cand", list(stba.AUTOTUNE_CANDIDATES) + ["solve_cs4", "solve_cs2"])
def test_every_fp32_factorisation_meets_the_mixed_bar(ring, cand):
    s, F, hist = ring
    tile, update, panel = stba.AUTOTUNE_CANDIDATES.get(cand, (64, 2, 1))
    cs = {"solve_cs4": 4, "solve_cs2": 2}.get(cand, 0)
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED, factor_tile=tile, factor_update=update, factor_panel=panel,
                           solve_cluster=cs)
    stba.stba_lm_iteration(ctx)
    dc, dp = stba.stba_last_step(ctx)
    assert cols(dc, hist[0]["dc"], 9) < 1e-3 and cols(dp, hist[0]["dp"], 3) < 1e-3
    for _ in range(9):
        stba.stba_lm_iteration(ctx)
    _, Fg, _ = stba.stba_get_state(ctx)
    assert abs(np.sqrt(Fg) - np.sqrt(F)) <= 1e-3 * np.sqrt(F)


def test_autotune_restores_the_state_and_keeps_a_working_tile(ring):
    s, F, hist = ring
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED)
    stba.stba_lm_iteration(ctx)
    lam0, F0, it0 = stba.stba_get_state(ctx)
    c0, p0 = stba.stba_get_params(ctx)
    kept, ms = stba.stba_autotune(ctx, 3)
    assert kept in stba.AUTOTUNE_CANDIDATES
    tile, update, panel = stba.AUTOTUNE_CANDIDATES[kept]
    assert all(v > 0 for v in ms.values()), ms
    lam1, F1, it1 = stba.stba_get_state(ctx)
    c1, p1 = stba.stba_get_params(ctx)
    assert lam1 == lam0 and F1 == F0 and np.array_equal(c1, c0) and np.array_equal(p1, p0)
    info = stba.stba_lm_iteration(ctx)
    ref = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED, factor_tile=tile, factor_update=update, factor_panel=panel)
    stba.stba_lm_iteration(ref)
    info_ref = stba.stba_lm_iteration(ref)
    assert info["accepted"] == info_ref["accepted"]
    # mixed precision: FP32 sums reach the FP64 accumulators in a run-dependent order, so two runs of the same
    # iteration agree to the mixed-mode bar, not bit for bit
    assert abs(info["F_after"] - info_ref["F_after"]) <= 1e-4 * info_ref["F_after"]
    stba.stba_record(ctx, 2)
    with pytest.raises(stba.StbaError):
        stba.stba_autotune(ctx, 2)
