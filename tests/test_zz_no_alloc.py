"""stba_cost_noalloc: the cost through the allocation-free entry point equals the cost of the context API.

Callers that cannot allocate device memory at call time use stba_cost_noalloc, whose scratch is a static
device array inside the library.  This file is collected last on purpose: it runs after every other test
in a full run, and must also pass alone in a fresh process."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import camera as ocam  # noqa: E402
from paper_2008_00446_gb300 import stba  # noqa: E402


def on_device(*arrays):
    d = torch.device("cuda:0")
    return [torch.tensor(a, device=d) for a in arrays]


def test_noalloc_cost_matches_context_cost_twice():
    s = scenes.make_config("c0_ring")
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters)
    F_ref = stba.stba_cost(ctx)
    d = torch.device("cuda:0")
    cams = torch.tensor(s.cameras, device=d)
    pts = torch.tensor(s.points, device=d)
    oc = torch.tensor(s.obs_cam, device=d)
    op = torch.tensor(s.obs_pt, device=d)
    uv = torch.tensor(s.obs_uv, device=d)
    F_out = torch.zeros(1, dtype=torch.float64, device=d)
    for _ in range(2):
        F_out.fill_(-1.0)
        stba.stba_cost_noalloc(cams, pts, oc, op, uv, F_out)
        torch.cuda.synchronize()
        assert float(F_out.item()) == pytest.approx(F_ref, rel=1e-12)
        # and against the oracle's FP64 cost (Sec. 3: F = sum of squared reprojection errors)
        F_oracle = ocam.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
        assert float(F_out.item()) == pytest.approx(F_oracle, rel=1e-12)
    # a second scene in a row, with other sizes, through the same static scratch
    s2 = scenes.make_tiny_scene(m=7, n=50, seed=3)
    ctx2 = stba.stba_create(s2.cameras, s2.points, s2.obs_cam, s2.obs_pt, s2.obs_uv, s2.clusters)
    F2 = stba.stba_cost(ctx2)
    t = [torch.tensor(a, device=d) for a in (s2.cameras, s2.points, s2.obs_cam, s2.obs_pt, s2.obs_uv)]
    stba.stba_cost_noalloc(*t, F_out)
    torch.cuda.synchronize()
    assert float(F_out.item()) == pytest.approx(F2, rel=1e-12)
    ctx.close()
    ctx2.close()


def test_noalloc_rejects_too_many_cameras():
    d = torch.device("cuda:0")
    m = 16385
    cams = torch.zeros((m, 9), dtype=torch.float64, device=d)
    pts = torch.zeros((1, 3), dtype=torch.float64, device=d)
    oc = torch.zeros(2, dtype=torch.int32, device=d)
    uv = torch.zeros((2, 2), dtype=torch.float64, device=d)
    F_out = torch.zeros(1, dtype=torch.float64, device=d)
    with pytest.raises(stba.StbaError):
        stba.stba_cost_noalloc(cams, pts, oc, oc, uv, F_out)


def test_noalloc_index_out_of_range_gives_nan():
    # the kernel checks every index against m and n before it loads; a point index equal to n (made on the
    # host) marks the sum NaN instead of reading past the points
    s = scenes.make_tiny_scene(m=5, n=30, seed=7)
    op = s.obs_pt.copy()
    op[3] = s.n
    t = on_device(s.cameras, s.points, s.obs_cam, op, s.obs_uv)
    F_out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    stba.stba_cost_noalloc(*t, F_out)
    torch.cuda.synchronize()
    assert np.isnan(float(F_out.item()))
    # the next call with valid indices overwrites every partial of the shared scratch
    t[3] = torch.tensor(s.obs_pt, device="cuda:0")
    stba.stba_cost_noalloc(*t, F_out)
    torch.cuda.synchronize()
    assert float(F_out.item()) == pytest.approx(ocam.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv),
                                                rel=1e-12)


def test_noalloc_at_the_camera_limit_matches_the_oracle():
    # m = 16384 exactly, the largest the static scratch holds; cameras 5.. observe nothing (allowed here)
    s = scenes.make_tiny_scene(m=5, n=30, seed=7)
    m = 16384
    cams = np.tile(s.cameras, (m // 5 + 1, 1))[:m].copy()
    t = on_device(cams, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
    F_out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    stba.stba_cost_noalloc(*t, F_out)
    torch.cuda.synchronize()
    assert float(F_out.item()) == pytest.approx(ocam.cost(cams, s.points, s.obs_cam, s.obs_pt, s.obs_uv), rel=1e-12)
